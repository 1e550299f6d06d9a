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

__global__ void pack_gauge64_kernel(int V, const double* __restrict__ canon, double2* __restrict__ soa) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const double2* src = reinterpret_cast<const double2*>(canon) + (size_t)s * 36;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
#pragma unroll
    for (int c = 0; c < 9; ++c) soa[((size_t)mu * 9 + c) * V + s] = src[mu * 9 + c];
}

__global__ void unpack_gauge64_kernel(int V, const double2* __restrict__ soa, double* __restrict__ canon) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  double2* dst = reinterpret_cast<double2*>(canon) + (size_t)s * 36;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
#pragma unroll
    for (int c = 0; c < 9; ++c) dst[mu * 9 + c] = soa[((size_t)mu * 9 + c) * V + s];
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
__global__ void pack_spinor_kernel(int V, const double* __restrict__ canon, SpinorRef out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const double2* src = reinterpret_cast<const double2*>(canon) + (size_t)s * 12;
  cplx<double> v[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) { double2 w = src[c]; v[c] = {w.x, w.y}; }
  store_spinor<S, double>(out, V, s, v);
}

template <SStore S>
__global__ void unpack_spinor_kernel(int V, SpinorRef in, double* __restrict__ canon) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  cplx<double> v[12];
  load_spinor<S, double>(in, V, s, v);
  double2* dst = reinterpret_cast<double2*>(canon) + (size_t)s * 12;
#pragma unroll
  for (int c = 0; c < 12; ++c) dst[c] = make_double2(v[c].re, v[c].im);
}

static constexpr int kBS = 256;

void launch_pack_gauge64(const Geom& g, const double* canon, void* soa, cudaStream_t st) {
  pack_gauge64_kernel<<<grid_for(g.V, kBS), kBS, 0, st>>>(g.V, canon, static_cast<double2*>(soa));
}
void launch_unpack_gauge64(const Geom& g, const void* soa, double* canon, cudaStream_t st) {
  unpack_gauge64_kernel<<<grid_for(g.V, kBS), kBS, 0, st>>>(g.V, static_cast<const double2*>(soa), canon);
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
  const int grid = grid_for(g.V, kBS);
  switch (s) {
    case SStore::F64: pack_spinor_kernel<SStore::F64><<<grid, kBS, 0, st>>>(g.V, canon, out); break;
    case SStore::F32: pack_spinor_kernel<SStore::F32><<<grid, kBS, 0, st>>>(g.V, canon, out); break;
    case SStore::F16: pack_spinor_kernel<SStore::F16><<<grid, kBS, 0, st>>>(g.V, canon, out); break;
    case SStore::BF16: pack_spinor_kernel<SStore::BF16><<<grid, kBS, 0, st>>>(g.V, canon, out); break;
    case SStore::DF64: pack_spinor_kernel<SStore::DF64><<<grid, kBS, 0, st>>>(g.V, canon, out); break;
    case SStore::I16: pack_spinor_kernel<SStore::I16><<<grid, kBS, 0, st>>>(g.V, canon, out); break;
  }
}
void launch_unpack_spinor(const Geom& g, SStore s, SpinorRef in, double* canon, cudaStream_t st) {
  const int grid = grid_for(g.V, kBS);
  switch (s) {
    case SStore::F64: unpack_spinor_kernel<SStore::F64><<<grid, kBS, 0, st>>>(g.V, in, canon); break;
    case SStore::F32: unpack_spinor_kernel<SStore::F32><<<grid, kBS, 0, st>>>(g.V, in, canon); break;
    case SStore::F16: unpack_spinor_kernel<SStore::F16><<<grid, kBS, 0, st>>>(g.V, in, canon); break;
    case SStore::BF16: unpack_spinor_kernel<SStore::BF16><<<grid, kBS, 0, st>>>(g.V, in, canon); break;
    case SStore::DF64: unpack_spinor_kernel<SStore::DF64><<<grid, kBS, 0, st>>>(g.V, in, canon); break;
    case SStore::I16: unpack_spinor_kernel<SStore::I16><<<grid, kBS, 0, st>>>(g.V, in, canon); break;
  }
}

}  // namespace lq
