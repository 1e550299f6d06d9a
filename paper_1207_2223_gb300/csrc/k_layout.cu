// Conversions between the canonical interleaved-complex FP64 layout of the
// C interface ([site][mu][3][3] links, [site][spin][colour] spinors) and the
// internal site-major structure-of-arrays formats of lq_device.cuh.
#include "lq_internal.h"

namespace lq {

int resident_grid(const void* kernel, int block) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
  if (sms <= 0) sms = 1;
  if (per_sm <= 0) per_sm = 1;
  return sms * per_sm;
}

size_t spinor_bytes(SStore s, int V) {
  switch (s) {
    case SStore::F64: case SStore::DF64: return (size_t)V * 24 * 8;
    case SStore::F32: return (size_t)V * 24 * 4;
    default: return (size_t)V * 24 * 2;
  }
}
size_t gauge_bytes(GStore g, int V) {
  switch (g) {
    case GStore::F64_18: case GStore::DF64_18: return (size_t)V * 4 * 18 * 8;
    case GStore::F32_18: return (size_t)V * 4 * 18 * 4;
    case GStore::F32_12: return (size_t)V * 4 * 12 * 4;
    default: return (size_t)V * 4 * 12 * 2;
  }
}

// The canonical layouts are read and written in contiguous runs: a block stages the
// canonical records of a tile of sites in shared memory (row padded by one complex entry)
// and the structure-of-arrays side is accessed one component at a time across the tile.
// Coalesced on both sides, which matters most when the canonical buffer is host memory
// accessed in place.
constexpr int kGaugeTile = 64;           // sites per block, 36 complex entries each
constexpr int kSpinTile = 128;           // sites per block, 12 complex entries each

__global__ void __launch_bounds__(256) pack_gauge64_kernel(int V, const double2* __restrict__ canon,
                                                           double2* __restrict__ soa) {
  __shared__ double2 sh[kGaugeTile * 37];
  const int s0 = blockIdx.x * kGaugeTile;
  const int n = min(kGaugeTile, V - s0);
  for (int i = threadIdx.x; i < n * 36; i += blockDim.x) {
    const int sl = i / 36;
    sh[sl * 37 + (i - sl * 36)] = canon[(size_t)s0 * 36 + i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n * 36; i += blockDim.x) {
    const int k = i / n, sl = i - k * n;
    soa[(size_t)k * V + s0 + sl] = sh[sl * 37 + k];
  }
}

__global__ void __launch_bounds__(256) unpack_gauge64_kernel(int V, const double2* __restrict__ soa,
                                                             double2* __restrict__ canon) {
  __shared__ double2 sh[kGaugeTile * 37];
  const int s0 = blockIdx.x * kGaugeTile;
  const int n = min(kGaugeTile, V - s0);
  for (int i = threadIdx.x; i < n * 36; i += blockDim.x) {
    const int k = i / n, sl = i - k * n;
    sh[sl * 37 + k] = soa[(size_t)k * V + s0 + sl];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n * 36; i += blockDim.x) {
    const int sl = i / 36;
    canon[(size_t)s0 * 36 + i] = sh[sl * 37 + (i - sl * 36)];
  }
}

template <GStore G>
__global__ void convert_gauge_kernel(int V, const double2* __restrict__ soa64, void* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  for (int mu = 0; mu < 4; ++mu) {
    double2 u[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) u[c] = soa64[((size_t)mu * 9 + c) * V + s];
    if constexpr (G == GStore::DF64_18) {
      float4* o = static_cast<float4*>(out) + (size_t)mu * 9 * V;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const df64 a(u[c].x), b(u[c].y);
        o[(size_t)c * V + s] = make_float4(a.hi, a.lo, b.hi, b.lo);
      }
    } else if constexpr (G == GStore::I16_12) {
      uint2* o = static_cast<uint2*>(out) + (size_t)mu * 3 * V;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        uint2 w;
        w.x = q16_from2((float)u[2 * k].x * kQ16, (float)u[2 * k].y * kQ16);
        w.y = q16_from2((float)u[2 * k + 1].x * kQ16, (float)u[2 * k + 1].y * kQ16);
        o[(size_t)k * V + s] = w;
      }
    } else if constexpr (G == GStore::F32_18) {
      float2* o = static_cast<float2*>(out) + (size_t)mu * 9 * V;
#pragma unroll
      for (int c = 0; c < 9; ++c) o[(size_t)c * V + s] = make_float2((float)u[c].x, (float)u[c].y);
    } else if constexpr (G == GStore::F32_12) {
      float4* o = static_cast<float4*>(out) + (size_t)mu * 3 * V;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        o[(size_t)k * V + s] = make_float4((float)u[2 * k].x, (float)u[2 * k].y, (float)u[2 * k + 1].x, (float)u[2 * k + 1].y);
    } else {
      using H = typename GaugeTraits<G>::half_t;
      uint2* o = static_cast<uint2*>(out) + (size_t)mu * 3 * V;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        uint2 w;
        w.x = HalfOps<H>::from2((float)u[2 * k].x, (float)u[2 * k].y);
        w.y = HalfOps<H>::from2((float)u[2 * k + 1].x, (float)u[2 * k + 1].y);
        o[(size_t)k * V + s] = w;
      }
    }
  }
}

template <SStore S>
__global__ void __launch_bounds__(kSpinTile) pack_spinor_kernel(int V, const double2* __restrict__ canon,
                                                                SpinorRef out) {
  __shared__ double2 sh[kSpinTile * 13];
  const int s0 = blockIdx.x * kSpinTile;
  const int n = min(kSpinTile, V - s0);
  for (int i = threadIdx.x; i < n * 12; i += blockDim.x) {
    const int sl = i / 12;
    sh[sl * 13 + (i - sl * 12)] = canon[(size_t)s0 * 12 + i];
  }
  __syncthreads();
  const int sl = threadIdx.x;
  if (sl >= n) return;
  cplx<double> v[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) { const double2 w = sh[sl * 13 + c]; v[c] = {w.x, w.y}; }
  store_spinor<S, double>(out, V, s0 + sl, v);
}

template <SStore S>
__global__ void __launch_bounds__(kSpinTile) unpack_spinor_kernel(int V, SpinorRef in, double2* __restrict__ canon) {
  __shared__ double2 sh[kSpinTile * 13];
  const int s0 = blockIdx.x * kSpinTile;
  const int n = min(kSpinTile, V - s0);
  const int sl = threadIdx.x;
  if (sl < n) {
    cplx<double> v[12];
    load_spinor<S, double>(in, V, s0 + sl, v);
#pragma unroll
    for (int c = 0; c < 12; ++c) sh[sl * 13 + c] = make_double2(v[c].re, v[c].im);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n * 12; i += blockDim.x) {
    const int t = i / 12;
    canon[(size_t)s0 * 12 + i] = sh[t * 13 + (i - t * 12)];
  }
}

static constexpr int kBS = 256;

void launch_pack_gauge64(const Geom& g, const double* canon, void* soa, cudaStream_t st) {
  pack_gauge64_kernel<<<grid_for(g.V, kGaugeTile), 256, 0, st>>>(g.V, reinterpret_cast<const double2*>(canon),
                                                                  static_cast<double2*>(soa));
}
void launch_unpack_gauge64(const Geom& g, const void* soa, double* canon, cudaStream_t st) {
  unpack_gauge64_kernel<<<grid_for(g.V, kGaugeTile), 256, 0, st>>>(g.V, static_cast<const double2*>(soa),
                                                                    reinterpret_cast<double2*>(canon));
}
void launch_convert_gauge(const Geom& g, const void* soa64, GStore dst, void* out, cudaStream_t st) {
  const double2* in = static_cast<const double2*>(soa64);
  const int grid = grid_for(g.V, kBS);
  switch (dst) {
    case GStore::F64_18: cudaMemcpyAsync(out, soa64, gauge_bytes(dst, g.V), cudaMemcpyDeviceToDevice, st); break;
    case GStore::F32_18: convert_gauge_kernel<GStore::F32_18><<<grid, kBS, 0, st>>>(g.V, in, out); break;
    case GStore::F32_12: convert_gauge_kernel<GStore::F32_12><<<grid, kBS, 0, st>>>(g.V, in, out); break;
    case GStore::F16_12: convert_gauge_kernel<GStore::F16_12><<<grid, kBS, 0, st>>>(g.V, in, out); break;
    case GStore::BF16_12: convert_gauge_kernel<GStore::BF16_12><<<grid, kBS, 0, st>>>(g.V, in, out); break;
    case GStore::DF64_18: convert_gauge_kernel<GStore::DF64_18><<<grid, kBS, 0, st>>>(g.V, in, out); break;
    case GStore::I16_12: convert_gauge_kernel<GStore::I16_12><<<grid, kBS, 0, st>>>(g.V, in, out); break;
  }
}

// field-to-field format conversion (through FP64 values)
template <SStore A, SStore B>
__global__ void convert_spinor_kernel(int V, SpinorRef in, SpinorRef out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  cplx<double> v[12];
  load_spinor<A, double>(in, V, s, v);
  store_spinor<B, double>(out, V, s, v);
}

void launch_convert_spinor(const Geom& g, SStore a, SpinorRef in, SStore b, SpinorRef out, cudaStream_t st) {
  const int grid = grid_for(g.V, kBS);
  if (a == SStore::F64 && b == SStore::DF64)
    convert_spinor_kernel<SStore::F64, SStore::DF64><<<grid, kBS, 0, st>>>(g.V, in, out);
  else if (a == SStore::DF64 && b == SStore::F64)
    convert_spinor_kernel<SStore::DF64, SStore::F64><<<grid, kBS, 0, st>>>(g.V, in, out);
}
void launch_pack_spinor(const Geom& g, const double* canon, SStore s, SpinorRef out, cudaStream_t st) {
  const int grid = grid_for(g.V, kSpinTile);
  const double2* in = reinterpret_cast<const double2*>(canon);
  switch (s) {
    case SStore::F64: pack_spinor_kernel<SStore::F64><<<grid, kSpinTile, 0, st>>>(g.V, in, out); break;
    case SStore::F32: pack_spinor_kernel<SStore::F32><<<grid, kSpinTile, 0, st>>>(g.V, in, out); break;
    case SStore::F16: pack_spinor_kernel<SStore::F16><<<grid, kSpinTile, 0, st>>>(g.V, in, out); break;
    case SStore::BF16: pack_spinor_kernel<SStore::BF16><<<grid, kSpinTile, 0, st>>>(g.V, in, out); break;
    case SStore::DF64: pack_spinor_kernel<SStore::DF64><<<grid, kSpinTile, 0, st>>>(g.V, in, out); break;
    case SStore::I16: pack_spinor_kernel<SStore::I16><<<grid, kSpinTile, 0, st>>>(g.V, in, out); break;
  }
}
void launch_unpack_spinor(const Geom& g, SStore s, SpinorRef in, double* canon, cudaStream_t st) {
  const int grid = grid_for(g.V, kSpinTile);
  double2* out = reinterpret_cast<double2*>(canon);
  switch (s) {
    case SStore::F64: unpack_spinor_kernel<SStore::F64><<<grid, kSpinTile, 0, st>>>(g.V, in, out); break;
    case SStore::F32: unpack_spinor_kernel<SStore::F32><<<grid, kSpinTile, 0, st>>>(g.V, in, out); break;
    case SStore::F16: unpack_spinor_kernel<SStore::F16><<<grid, kSpinTile, 0, st>>>(g.V, in, out); break;
    case SStore::BF16: unpack_spinor_kernel<SStore::BF16><<<grid, kSpinTile, 0, st>>>(g.V, in, out); break;
    case SStore::DF64: unpack_spinor_kernel<SStore::DF64><<<grid, kSpinTile, 0, st>>>(g.V, in, out); break;
    case SStore::I16: unpack_spinor_kernel<SStore::I16><<<grid, kSpinTile, 0, st>>>(g.V, in, out); break;
  }
}

}  // namespace lq
