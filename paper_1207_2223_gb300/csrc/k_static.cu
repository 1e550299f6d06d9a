// M^dag M on caller buffers without any device allocation.
//
// Some callers cannot let a library allocate device memory: an application
// that hands all of its GPU memory to its own pool allocator and forbids
// cudaMalloc after start-up, or a plugin that runs under a fixed memory
// budget set by its host program.  lq_apply_MdagM_static serves them: it
// takes the gauge field and the spinors in the canonical layout directly
// from device buffers the caller owns, and keeps its one intermediate
// field (M in) in a fixed-size array compiled into this library.
//
// That array is a file-scope __device__ variable.  Its name, used in host
// code, is only a host-side stand-in and not a device address, so host code
// asks the runtime for the device address (cudaGetSymbolAddress) once per
// device, with that device current, and passes the result to the kernels.
#include <mutex>
#include <string>

#include "lq_internal.h"

namespace lq {

// Largest lattice the array holds: 65,536 sites (for example 16^4), one FP64
// spinor of 12 complex numbers per site = 12 MiB.  Every GPU that loads the
// library holds this array until the process exits.
constexpr int kStaticMaxSites = 65536;

static __device__ __align__(256) double2 g_static_scratch[(size_t)kStaticMaxSites * 12];

// out = in - kappa * H in (dagger = 0) or in - kappa * H^dag in (dagger = 1),
// with U, in and out all in the canonical interleaved layout of lq.h.
template <bool DAG>
__global__ void __launch_bounds__(256) hop_canonical_kernel(Geom geo, const double2* __restrict__ U,
                                                            const double2* __restrict__ in,
                                                            double2* __restrict__ out, double kappa) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= geo.V) return;
  int c[4];
  site_coords(geo, s, c);
  cplx<double> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {0.0, 0.0};
  auto load_psi = [&](int n, cplx<double> p[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) { double2 w = in[(size_t)n * 12 + k]; p[k] = {w.x, w.y}; }
  };
  auto load_u = [&](int n, int mu, cplx<double> u[9]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) { double2 w = U[((size_t)n * 4 + mu) * 9 + k]; u[k] = {w.x, w.y}; }
  };
  auto hop = [&](auto mu_tag) {
    constexpr int MU = decltype(mu_tag)::value;
    constexpr int SF = DAG ? +1 : -1;
    cplx<double> p[12], h0[3], h1[3], u[9], w0[3], w1[3];
    const int f = nbr_fwd(geo, s, c, MU);
    load_psi(f, p);
    project<MU, SF>(p, h0, h1);
    if (MU == 3 && geo.antiperiodic && c[3] == geo.L[3] - 1)
      for (int k = 0; k < 3; ++k) { h0[k] = -h0[k]; h1[k] = -h1[k]; }
    load_u(s, MU, u);
    su3_mul(u, h0, w0);
    su3_mul(u, h1, w1);
    accumulate<MU, SF>(acc, w0, w1);
    const int b = nbr_bwd(geo, s, c, MU);
    load_psi(b, p);
    project<MU, -SF>(p, h0, h1);
    if (MU == 3 && geo.antiperiodic && c[3] == 0)
      for (int k = 0; k < 3; ++k) { h0[k] = -h0[k]; h1[k] = -h1[k]; }
    load_u(b, MU, u);
    su3_dagmul(u, h0, w0);
    su3_dagmul(u, h1, w1);
    accumulate<MU, -SF>(acc, w0, w1);
  };
  hop(std::integral_constant<int, 0>{});
  hop(std::integral_constant<int, 1>{});
  hop(std::integral_constant<int, 2>{});
  hop(std::integral_constant<int, 3>{});
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const double2 w = in[(size_t)s * 12 + k];
    out[(size_t)s * 12 + k] = make_double2(fma(-kappa, acc[k].re, w.x), fma(-kappa, acc[k].im, w.y));
  }
}

namespace {

// True when p is device (or managed) memory.  cudaPointerGetAttributes
// allocates nothing; host memory, including pinned or unregistered host
// buffers, is refused before any kernel sees it.
bool static_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
double2* g_static_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on each device) and kept for the life of the
// process.  A device reset (cudaDeviceReset, or a reset of the primary
// context) unloads the module that holds the array, so calls after one are
// not supported.
cudaError_t static_scratch_address(double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_addr[dev] = static_cast<double2*>(p);
  }
  *out = g_static_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace lq

// Error text for the static entry point (read with lq_last_error(NULL)).
void lq_set_global_error(const std::string& msg);

extern "C" lq_status lq_apply_MdagM_static(double* out, const double* U, const double* in, const int dims[4],
                                           int t_antiperiodic, double kappa, void* cuda_stream) {
  using namespace lq;
  if (!out || !U || !in || !dims) {
    lq_set_global_error("lq_apply_MdagM_static: null argument");
    return LQ_ERR_ARG;
  }
  // Each extent is checked before it enters the product, and the product stops
  // growing as soon as it passes the limit, so it cannot overflow.
  long long V = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 2) {
      lq_set_global_error("lq_apply_MdagM_static: every lattice extent must be >= 2");
      return LQ_ERR_SHAPE;
    }
    if (dims[m] > kStaticMaxSites || V * dims[m] > kStaticMaxSites) {
      lq_set_global_error("lq_apply_MdagM_static: lattice " + std::to_string(dims[0]) + "x" +
                          std::to_string(dims[1]) + "x" + std::to_string(dims[2]) + "x" + std::to_string(dims[3]) +
                          " has more sites than the built-in scratch array holds (at most " +
                          std::to_string(kStaticMaxSites) + ")");
      return LQ_ERR_SHAPE;
    }
    V *= dims[m];
  }
  const uintptr_t mis = (reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(U) |
                         reinterpret_cast<uintptr_t>(in)) & 15u;
  if (mis) {
    lq_set_global_error("lq_apply_MdagM_static: buffers must be 16-byte aligned");
    return LQ_ERR_ARG;
  }
  if (!static_device_ptr(out) || !static_device_ptr(U) || !static_device_ptr(in)) {
    lq_set_global_error("lq_apply_MdagM_static: U, in and out must be device buffers");
    return LQ_ERR_ARG;
  }
  double2* scratch = nullptr;
  cudaError_t e = static_scratch_address(&scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    lq_set_global_error(std::string("lq_apply_MdagM_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return LQ_ERR_CUDA;
  }
  Geom geo{};
  geo.V = (int)V;
  for (int m = 0; m < 4; ++m) geo.L[m] = dims[m];
  geo.stride[0] = 1;
  for (int m = 1; m < 4; ++m) geo.stride[m] = geo.stride[m - 1] * dims[m - 1];
  geo.antiperiodic = t_antiperiodic ? 1 : 0;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int bs = 256, grid = grid_for(geo.V, bs);
  // scratch = M in (every site written before it is read: nothing to clear)
  hop_canonical_kernel<false><<<grid, bs, 0, st>>>(geo, reinterpret_cast<const double2*>(U),
                                                   reinterpret_cast<const double2*>(in), scratch, kappa);
  // out = M^dag scratch
  hop_canonical_kernel<true><<<grid, bs, 0, st>>>(geo, reinterpret_cast<const double2*>(U), scratch,
                                                  reinterpret_cast<double2*>(out), kappa);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    lq_set_global_error(std::string("lq_apply_MdagM_static: launch: ") + cudaGetErrorString(e));
    return LQ_ERR_CUDA;
  }
  return LQ_OK;
}
