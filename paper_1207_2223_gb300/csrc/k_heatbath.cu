// Heat bath of the HMC trajectory on the device (paper Sec. 2: momenta drawn
// from a Gaussian at the start of every trajectory; Sec. 3 step 1: the
// pseudofermion field from Gaussian noise, phi = M^dag chi).
//
// Streams and counters of the generator (key = (seed, stream), 32-bit words):
//   momenta   stream 1, counter (site, mu + 4 traj, call k, 0), k = 0..3:
//             p_{2k}, p_{2k+1} of link (site, mu) = the Box-Muller pair of call k
//   chi       stream 2, counter (site, traj, call k, 0), k = 0..11:
//             complex component k of the spinor (k = 3 spin + colour) =
//             (z0 + i z1) sqrt(1/2), density exp(-chi^dag chi)
//   Metropolis stream 3, counter (traj, 0, 0, 0): u = uniform53 of words 0, 1
#include "lq_internal.h"
#include "lq_philox.cuh"

namespace lq {

namespace {

constexpr int kBS = 256;
constexpr uint32_t kStreamMomenta = 1, kStreamChi = 2, kStreamMetropolis = 3;

// One thread per link (site, mu): 8 su(3) coefficients into the SoA momenta
// [32][V] (component mu * 8 + a) and, when canon != null, the canonical [V][4][8].
__global__ void __launch_bounds__(kBS) momenta_kernel(int V, uint32_t seed, uint32_t traj, double* soa,
                                                      double* canon) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= 4 * V) return;
  const int s = l >> 2, mu = l & 3;
  const uint32_t c1 = (uint32_t)mu + 4u * traj;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const rng::Words w = rng::philox4x32_10((uint32_t)s, c1, (uint32_t)k, 0u, seed, kStreamMomenta);
    double z0, z1;
    rng::gaussian_pair(w, &z0, &z1);
    const int a = mu * 8 + 2 * k;
    if (soa) {
      soa[(size_t)a * V + s] = z0;
      soa[(size_t)(a + 1) * V + s] = z1;
    }
    if (canon) {
      canon[(size_t)s * 32 + a] = z0;
      canon[(size_t)s * 32 + a + 1] = z1;
    }
  }
}

// One thread per site: the 12 complex components of chi into the FP64 spinor
// field (double2 [12][V]) and, when canon != null, the canonical [V][4][3] complex.
__global__ void __launch_bounds__(kBS) chi_kernel(int V, uint32_t seed, uint32_t traj, double2* soa, double2* canon) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  for (int k = 0; k < 12; ++k) {
    const rng::Words w = rng::philox4x32_10((uint32_t)s, traj, (uint32_t)k, 0u, seed, kStreamChi);
    double z0, z1;
    rng::gaussian_pair(w, &z0, &z1);
    const double2 v = make_double2(rng::mul(z0, rng::kSqrtHalf), rng::mul(z1, rng::kSqrtHalf));
    if (soa) soa[(size_t)k * V + s] = v;
    if (canon) canon[(size_t)s * 12 + k] = v;
  }
}

__global__ void __launch_bounds__(kBS) philox_kernel(int n, const uint32_t* in, uint32_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t* a = in + (size_t)i * 6;
  const rng::Words w = rng::philox4x32_10(a[0], a[1], a[2], a[3], a[4], a[5]);
  uint32_t* o = out + (size_t)i * 4;
  o[0] = w.x; o[1] = w.y; o[2] = w.z; o[3] = w.w;
}

bool device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

bool heatbath_counters_ok(uint64_t seed, uint64_t traj) { return seed <= 0xFFFFFFFFull && traj < (1ull << 30); }

void launch_heatbath_momenta(const Geom& g, uint64_t seed, uint64_t traj, double* soa, double* canon,
                             cudaStream_t st) {
  momenta_kernel<<<grid_for(4 * g.V, kBS), kBS, 0, st>>>(g.V, (uint32_t)seed, (uint32_t)traj, soa, canon);
}

void launch_heatbath_chi(const Geom& g, uint64_t seed, uint64_t traj, SpinorRef soa, double* canon, cudaStream_t st) {
  chi_kernel<<<grid_for(g.V, kBS), kBS, 0, st>>>(g.V, (uint32_t)seed, (uint32_t)traj,
                                                 static_cast<double2*>(soa.p), reinterpret_cast<double2*>(canon));
}

double metropolis_uniform(uint64_t seed, uint64_t traj) {
  const rng::Words w = rng::philox4x32_10((uint32_t)traj, 0u, 0u, 0u, (uint32_t)seed, kStreamMetropolis);
  return rng::uniform53(w.x, w.y);
}

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_philox4x32_10(lq_ctx* c, const uint32_t* in, uint32_t* out, int n) {
  if (!c) return LQ_ERR_ARG;
  if (n < 0 || (n > 0 && (!in || !out))) {
    c->last_error = "lq_philox4x32_10: bad count or null buffer";
    return LQ_ERR_ARG;
  }
  if (n == 0) return LQ_OK;
  if (!device_ptr(in) || !device_ptr(out)) {
    c->last_error = "lq_philox4x32_10: in and out must be device buffers";
    return LQ_ERR_ARG;
  }
  philox_kernel<<<grid_for(n, kBS), kBS, 0, c->stream>>>(n, in, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->last_error = std::string("lq_philox4x32_10: ") + cudaGetErrorString(e);
    return LQ_ERR_CUDA;
  }
  return LQ_OK;
}
