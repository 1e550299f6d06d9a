// Device-side building blocks of the lattice library: complex arithmetic,
// the site-major structure-of-arrays storage formats of gauge links and
// spinors, the Wilson spin projectors, and a deterministic grid reduction.
//
// Storage formats (every array is [chunk][site]: consecutive threads read
// consecutive 8- or 16-byte words, so every load and store is coalesced):
//   spinor F64   double2 [12][V]          complex c = 3*spin + colour
//   spinor F32   float4  [6][V]           chunk k holds complex 2k, 2k+1
//   spinor F16 / BF16  uint4 [3][V] + float norm[V]
//                chunk k holds reals 8k..8k+7 (re, im interleaved) scaled by
//                1/norm, norm = max |real| of the site (0 for a zero site)
//   gauge F64_18 double2 [4][9][V]        U_mu(x) row-major, complex (i,j) = 3i+j
//   gauge F32_18 float2  [4][9][V]
//   gauge F32_12 float4  [4][3][V]        rows 0, 1 only (12 reals)
//   gauge F16_12 / BF16_12  uint2 [4][3][V]  rows 0, 1 only, 4 reals per chunk
//   spinor DF64  float4 [12][V]           (re.hi, re.lo, im.hi, im.lo) double-float
//   gauge DF64_18 float4 [4][9][V]        double-float, 18 reals
//   spinor I16   uint4 [3][V] + float norm[V]: 16-bit fixed point, value = q / 32767 * norm,
//                stored as u = q + 32768
//   gauge I16_12 uint2 [4][3][V]          rows 0, 1 as 16-bit fixed point, value = q / 32767
// Links stored with 12 reals are rebuilt on the fly with
// row 2 = conj(row 0 x row 1), exact for SU(3).  The antiperiodic time
// boundary is applied as a sign on the hop, never folded into links, so
// the reconstruction stays valid.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <type_traits>

#include "lq_df64.cuh"

namespace lq {

template <typename T> struct cplx { T re, im; };

template <typename T> __device__ __forceinline__ cplx<T> mk(T a, T b) { return {a, b}; }
template <typename T> __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __device__ __forceinline__ cplx<T> operator-(cplx<T> a) { return {-a.re, -a.im}; }
template <typename T> __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <typename T> __device__ __forceinline__ cplx<T> cjmul(cplx<T> a, cplx<T> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// acc + a * b
template <typename T> __device__ __forceinline__ cplx<T> cmadd(cplx<T> acc, cplx<T> a, cplx<T> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a) * b
template <typename T> __device__ __forceinline__ cplx<T> cjmadd(cplx<T> acc, cplx<T> a, cplx<T> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
template <typename T> __device__ __forceinline__ cplx<T> times_i(cplx<T> a) { return {-a.im, a.re}; }
template <typename T> __device__ __forceinline__ cplx<T> conjg(cplx<T> a) { return {a.re, -a.im}; }
template <typename T> __device__ __forceinline__ T norm2(cplx<T> a) { return a.re * a.re + a.im * a.im; }

// ---------------------------------------------------------------- formats
enum class SStore : int { F64 = 0, F32 = 1, F16 = 2, BF16 = 3, DF64 = 4, I16 = 5 };
enum class GStore : int { F64_18 = 0, F32_18 = 1, F32_12 = 2, F16_12 = 3, BF16_12 = 4, DF64_18 = 5, I16_12 = 6 };

// 16-bit fixed point, value q / 32767 (times the site norm for spinors),
// stored offset-binary: u = q + 32768 in 16 bits.  A byte permutation builds
// the float bits 0x4B000000 | u, i.e. the float 2^23 + u exactly (floats in
// [2^23, 2^24) are the integers), so decoding is one PRMT and one FADD.
// Encoding rounds x + 2^23 + 32768 to an integer in the same binade and keeps
// the low 16 bits of the two results with one PRMT.
constexpr float kQ16 = 32767.0f;
constexpr float kQ16Inv = 1.0f / 32767.0f;
constexpr float kQ16Bias = 8421376.0f;   // 2^23 + 32768
// The two halves of a word are decoded with one packed FP32x2 add (and scaled
// with one packed multiply): Blackwell issues these as single instructions.
__device__ __forceinline__ float2 q16_to2(uint32_t w) {   // raw q values
  const float2 b = make_float2(__int_as_float((int)__byte_perm(w, 0x4B00u, 0x5410u)),
                               __int_as_float((int)__byte_perm(w, 0x4B00u, 0x5432u)));
  return __fadd2_rn(b, make_float2(-kQ16Bias, -kQ16Bias));
}
__device__ __forceinline__ float2 q16_to2(uint32_t w, float scale) {
  return __fmul2_rn(q16_to2(w), make_float2(scale, scale));
}
__device__ __forceinline__ uint32_t q16_from2(float a, float b) {   // a, b in [-32767, 32767]
  const uint32_t ua = (uint32_t)__float_as_int(a + kQ16Bias);
  const uint32_t ub = (uint32_t)__float_as_int(b + kQ16Bias);
  return __byte_perm(ua, ub, 0x5410u);
}

// Conversions of a double-float to the arithmetic type of a kernel.
template <typename T> __device__ __forceinline__ T from_df(df64 v) { return (T)v; }
template <> __device__ __forceinline__ df64 from_df<df64>(df64 v) { return v; }
template <typename T> __device__ __forceinline__ df64 to_df(T v) { return df64(v); }
template <> __device__ __forceinline__ df64 to_df<df64>(df64 v) { return v; }

struct SpinorRef {           // device view of one spinor field
  void* p;                   // chunk array
  float* norm;               // per-site norm (F16 / BF16 only)
};
struct GaugeRef {
  const void* p;
};

struct Geom {
  int V;
  int L[4];
  int stride[4];             // 1, Lx, Lx*Ly, Lx*Ly*Lz
  int antiperiodic;          // time direction
};

template <typename H> struct HalfOps;
template <> struct HalfOps<__half> {
  static __device__ __forceinline__ float2 to2(uint32_t w) {
    __half2 h = *reinterpret_cast<__half2*>(&w); return __half22float2(h);
  }
  static __device__ __forceinline__ uint32_t from2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b); return *reinterpret_cast<uint32_t*>(&h);
  }
};
template <> struct HalfOps<__nv_bfloat16> {
  static __device__ __forceinline__ float2 to2(uint32_t w) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w); return __bfloat1622float2(h);
  }
  static __device__ __forceinline__ uint32_t from2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b); return *reinterpret_cast<uint32_t*>(&h);
  }
};

template <SStore S> struct SpinorTraits;
template <> struct SpinorTraits<SStore::F64> { using half_t = void; };
template <> struct SpinorTraits<SStore::F32> { using half_t = void; };
template <> struct SpinorTraits<SStore::F16> { using half_t = __half; };
template <> struct SpinorTraits<SStore::BF16> { using half_t = __nv_bfloat16; };
template <> struct SpinorTraits<SStore::DF64> { using half_t = void; };
template <> struct SpinorTraits<SStore::I16> { using half_t = void; };

// ----------------------------------------------------------- spinor I/O
// Load path of a field:
//   1 (true)   read-only for the whole kernel: the non-coherent read-only path
//   0 (false)  a field the kernel also writes (each element by the thread that reads it)
//   2          written by other blocks of the same kernel before a device-wide barrier
//              (persistent kernels): L2 only, never a stale L1 line
template <int RO, typename W> __device__ __forceinline__ W ld(const W* p) {
  if constexpr (RO == 1) return __ldg(p);
  else if constexpr (RO == 2) return __ldcg(p);
  else return *p;
}

template <SStore S, typename T, int RO = 1>
__device__ __forceinline__ void load_spinor(const SpinorRef& f, int V, int s, cplx<T> v[12]) {
  if constexpr (S == SStore::DF64) {
    const float4* p = static_cast<const float4*>(f.p);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      float4 w = ld<RO>(p + (size_t)c * V + s);
      v[c] = {from_df<T>(df64(w.x, w.y)), from_df<T>(df64(w.z, w.w))};
    }
  } else if constexpr (S == SStore::F64) {
    const double2* p = static_cast<const double2*>(f.p);
#pragma unroll
    for (int c = 0; c < 12; ++c) { double2 w = ld<RO>(p + (size_t)c * V + s); v[c] = {(T)w.x, (T)w.y}; }
  } else if constexpr (S == SStore::F32) {
    const float4* p = static_cast<const float4*>(f.p);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float4 w = ld<RO>(p + (size_t)k * V + s);
      v[2 * k] = {(T)w.x, (T)w.y}; v[2 * k + 1] = {(T)w.z, (T)w.w};
    }
  } else if constexpr (S == SStore::I16) {
    const uint4* p = static_cast<const uint4*>(f.p);
    const float sc = ld<RO>(f.norm + s) * kQ16Inv;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 w = ld<RO>(p + (size_t)k * V + s);
      float2 a = q16_to2(w.x, sc), b = q16_to2(w.y, sc), c = q16_to2(w.z, sc), e = q16_to2(w.w, sc);
      v[4 * k + 0] = {(T)a.x, (T)a.y};
      v[4 * k + 1] = {(T)b.x, (T)b.y};
      v[4 * k + 2] = {(T)c.x, (T)c.y};
      v[4 * k + 3] = {(T)e.x, (T)e.y};
    }
  } else {
    using H = typename SpinorTraits<S>::half_t;
    const uint4* p = static_cast<const uint4*>(f.p);
    const float nrm = ld<RO>(f.norm + s);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 w = ld<RO>(p + (size_t)k * V + s);
      float2 a = HalfOps<H>::to2(w.x), b = HalfOps<H>::to2(w.y), c = HalfOps<H>::to2(w.z), d = HalfOps<H>::to2(w.w);
      v[4 * k + 0] = {(T)(a.x * nrm), (T)(a.y * nrm)};
      v[4 * k + 1] = {(T)(b.x * nrm), (T)(b.y * nrm)};
      v[4 * k + 2] = {(T)(c.x * nrm), (T)(c.y * nrm)};
      v[4 * k + 3] = {(T)(d.x * nrm), (T)(d.y * nrm)};
    }
  }
}

// Load without applying the per-site norm of 16-bit formats; returns the
// norm (1 for FP32 / FP64).  The stencil applies it to the projected half
// spinor, half as many multiplications as scaling all 24 reals.
template <SStore S, typename T, int RO = 1>
__device__ __forceinline__ T load_spinor_raw(const SpinorRef& f, int V, int s, cplx<T> v[12]) {
  if constexpr (S == SStore::F64 || S == SStore::F32 || S == SStore::DF64) {
    load_spinor<S, T, RO>(f, V, s, v);
    return (T)1;
  } else if constexpr (S == SStore::I16) {
    const uint4* p = static_cast<const uint4*>(f.p);
    const float nrm = ld<RO>(f.norm + s);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 w = ld<RO>(p + (size_t)k * V + s);
      float2 a = q16_to2(w.x), b = q16_to2(w.y), c = q16_to2(w.z), e = q16_to2(w.w);
      v[4 * k + 0] = {(T)a.x, (T)a.y};
      v[4 * k + 1] = {(T)b.x, (T)b.y};
      v[4 * k + 2] = {(T)c.x, (T)c.y};
      v[4 * k + 3] = {(T)e.x, (T)e.y};
    }
    return (T)(nrm * kQ16Inv);
  } else {
    using H = typename SpinorTraits<S>::half_t;
    const uint4* p = static_cast<const uint4*>(f.p);
    const float nrm = ld<RO>(f.norm + s);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 w = ld<RO>(p + (size_t)k * V + s);
      float2 a = HalfOps<H>::to2(w.x), b = HalfOps<H>::to2(w.y), c = HalfOps<H>::to2(w.z), e = HalfOps<H>::to2(w.w);
      v[4 * k + 0] = {(T)a.x, (T)a.y};
      v[4 * k + 1] = {(T)b.x, (T)b.y};
      v[4 * k + 2] = {(T)c.x, (T)c.y};
      v[4 * k + 3] = {(T)e.x, (T)e.y};
    }
    return (T)nrm;
  }
}

template <SStore S, typename T>
__device__ __forceinline__ void store_spinor(const SpinorRef& f, int V, int s, const cplx<T> v[12]) {
  if constexpr (S == SStore::DF64) {
    float4* p = static_cast<float4*>(f.p);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const df64 a = to_df<T>(v[c].re), b = to_df<T>(v[c].im);
      p[(size_t)c * V + s] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
  } else if constexpr (S == SStore::F64) {
    double2* p = static_cast<double2*>(f.p);
#pragma unroll
    for (int c = 0; c < 12; ++c) p[(size_t)c * V + s] = make_double2((double)v[c].re, (double)v[c].im);
  } else if constexpr (S == SStore::F32) {
    float4* p = static_cast<float4*>(f.p);
#pragma unroll
    for (int k = 0; k < 6; ++k)
      p[(size_t)k * V + s] = make_float4((float)v[2 * k].re, (float)v[2 * k].im, (float)v[2 * k + 1].re, (float)v[2 * k + 1].im);
  } else if constexpr (S == SStore::I16) {
    uint4* p = static_cast<uint4*>(f.p);
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < 12; ++c) m = fmaxf(m, fmaxf(fabsf((float)v[c].re), fabsf((float)v[c].im)));
    const float inv = m > 0.f ? kQ16 / m : 0.f;
    f.norm[s] = m;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 w;
      w.x = q16_from2((float)v[4 * k + 0].re * inv, (float)v[4 * k + 0].im * inv);
      w.y = q16_from2((float)v[4 * k + 1].re * inv, (float)v[4 * k + 1].im * inv);
      w.z = q16_from2((float)v[4 * k + 2].re * inv, (float)v[4 * k + 2].im * inv);
      w.w = q16_from2((float)v[4 * k + 3].re * inv, (float)v[4 * k + 3].im * inv);
      p[(size_t)k * V + s] = w;
    }
  } else {
    using H = typename SpinorTraits<S>::half_t;
    uint4* p = static_cast<uint4*>(f.p);
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < 12; ++c) m = fmaxf(m, fmaxf(fabsf((float)v[c].re), fabsf((float)v[c].im)));
    const float inv = m > 0.f ? 1.0f / m : 0.f;
    f.norm[s] = m;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 w;
      w.x = HalfOps<H>::from2((float)v[4 * k + 0].re * inv, (float)v[4 * k + 0].im * inv);
      w.y = HalfOps<H>::from2((float)v[4 * k + 1].re * inv, (float)v[4 * k + 1].im * inv);
      w.z = HalfOps<H>::from2((float)v[4 * k + 2].re * inv, (float)v[4 * k + 2].im * inv);
      w.w = HalfOps<H>::from2((float)v[4 * k + 3].re * inv, (float)v[4 * k + 3].im * inv);
      p[(size_t)k * V + s] = w;
    }
  }
}

// ------------------------------------------------------------- gauge I/O
template <GStore G> struct GaugeTraits;
template <> struct GaugeTraits<GStore::F64_18> { using half_t = void; };
template <> struct GaugeTraits<GStore::F32_18> { using half_t = void; };
template <> struct GaugeTraits<GStore::F32_12> { using half_t = void; };
template <> struct GaugeTraits<GStore::F16_12> { using half_t = __half; };
template <> struct GaugeTraits<GStore::BF16_12> { using half_t = __nv_bfloat16; };
template <> struct GaugeTraits<GStore::DF64_18> { using half_t = void; };
template <> struct GaugeTraits<GStore::I16_12> { using half_t = void; };

template <typename T>
__device__ __forceinline__ void reconstruct_row2(cplx<T> u[9]) {
  u[6] = conjg(cmul(u[1], u[5]) - cmul(u[2], u[4]));
  u[7] = conjg(cmul(u[2], u[3]) - cmul(u[0], u[5]));
  u[8] = conjg(cmul(u[0], u[4]) - cmul(u[1], u[3]));
}

template <GStore G, typename T>
__device__ __forceinline__ void load_link(const GaugeRef& g, int V, int mu, int s, cplx<T> u[9]) {
  if constexpr (G == GStore::DF64_18) {
    const float4* p = static_cast<const float4*>(g.p) + (size_t)mu * 9 * V;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      float4 w = __ldg(p + (size_t)c * V + s);
      u[c] = {from_df<T>(df64(w.x, w.y)), from_df<T>(df64(w.z, w.w))};
    }
  } else if constexpr (G == GStore::F64_18) {
    const double2* p = static_cast<const double2*>(g.p) + (size_t)mu * 9 * V;
#pragma unroll
    for (int c = 0; c < 9; ++c) { double2 w = __ldg(p + (size_t)c * V + s); u[c] = {(T)w.x, (T)w.y}; }
  } else if constexpr (G == GStore::F32_18) {
    const float2* p = static_cast<const float2*>(g.p) + (size_t)mu * 9 * V;
#pragma unroll
    for (int c = 0; c < 9; ++c) { float2 w = __ldg(p + (size_t)c * V + s); u[c] = {(T)w.x, (T)w.y}; }
  } else if constexpr (G == GStore::I16_12) {
    const uint2* p = static_cast<const uint2*>(g.p) + (size_t)mu * 3 * V;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint2 w = __ldg(p + (size_t)k * V + s);
      float2 a = q16_to2(w.x, kQ16Inv), b = q16_to2(w.y, kQ16Inv);
      u[2 * k] = {(T)a.x, (T)a.y}; u[2 * k + 1] = {(T)b.x, (T)b.y};
    }
    reconstruct_row2(u);
  } else if constexpr (G == GStore::F32_12) {
    const float4* p = static_cast<const float4*>(g.p) + (size_t)mu * 3 * V;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float4 w = __ldg(p + (size_t)k * V + s);
      u[2 * k] = {(T)w.x, (T)w.y}; u[2 * k + 1] = {(T)w.z, (T)w.w};
    }
    reconstruct_row2(u);
  } else {
    using H = typename GaugeTraits<G>::half_t;
    const uint2* p = static_cast<const uint2*>(g.p) + (size_t)mu * 3 * V;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint2 w = __ldg(p + (size_t)k * V + s);
      float2 a = HalfOps<H>::to2(w.x), b = HalfOps<H>::to2(w.y);
      u[2 * k] = {(T)a.x, (T)a.y}; u[2 * k + 1] = {(T)b.x, (T)b.y};
    }
    reconstruct_row2(u);
  }
}

// A 16-bit fixed-point link with every row carrying 32767 U: rows 0, 1 are the
// stored integers and the rebuilt row 2 (32767^2 U) is divided by 32767 once.
// The stencil folds the remaining 1/32767 into the scale of the half spinor,
// which it multiplies anyway, instead of scaling the 12 stored reals.
template <typename T>
__device__ __forceinline__ void load_link_q16(const GaugeRef& g, int V, int mu, int s, cplx<T> u[9]) {
  const uint2* p = static_cast<const uint2*>(g.p) + (size_t)mu * 3 * V;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint2 w = __ldg(p + (size_t)k * V + s);
    float2 a = q16_to2(w.x), b = q16_to2(w.y);
    u[2 * k] = {(T)a.x, (T)a.y}; u[2 * k + 1] = {(T)b.x, (T)b.y};
  }
  reconstruct_row2(u);
#pragma unroll
  for (int c = 6; c < 9; ++c) {
    const float2 r = __fmul2_rn(make_float2((float)u[c].re, (float)u[c].im), make_float2(kQ16Inv, kQ16Inv));
    u[c] = {(T)r.x, (T)r.y};
  }
}

// -x by flipping the sign bit (an integer operation: exact, and off the FP64 pipe for doubles)
__device__ __forceinline__ double flip_sign(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}
__device__ __forceinline__ float flip_sign(float x) { return __int_as_float(__float_as_int(x) ^ (int)0x80000000); }
__device__ __forceinline__ df64 flip_sign(df64 x) { return df64(flip_sign(x.hi), flip_sign(x.lo)); }
template <typename T> __device__ __forceinline__ void negate3(cplx<T> h[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) h[k] = {flip_sign(h[k].re), flip_sign(h[k].im)};
}

// ----------------------------------------------------- spin projection
// Projector (1 + S gamma_mu) in the DeGrand-Rossi basis.  The projected
// spinor has rank 2: components 0, 1 ("h0", "h1") determine 2, 3.
//   mu=x: h0 = p0 + S i p3, h1 = p1 + S i p2, c2 = -S i h1, c3 = -S i h0
//   mu=y: h0 = p0 - S p3,   h1 = p1 + S p2,   c2 =  S h1,   c3 = -S h0
//   mu=z: h0 = p0 + S i p2, h1 = p1 - S i p3, c2 = -S i h0, c3 =  S i h1
//   mu=t: h0 = p0 + S p2,   h1 = p1 + S p3,   c2 =  S h0,   c3 =  S h1
template <int MU, int S, typename T>
__device__ __forceinline__ void project(const cplx<T> p[12], cplx<T> h0[3], cplx<T> h1[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cplx<T> p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
    if constexpr (MU == 0) {
      h0[c] = S > 0 ? p0 + times_i(p3) : p0 - times_i(p3);
      h1[c] = S > 0 ? p1 + times_i(p2) : p1 - times_i(p2);
    } else if constexpr (MU == 1) {
      h0[c] = S > 0 ? p0 - p3 : p0 + p3;
      h1[c] = S > 0 ? p1 + p2 : p1 - p2;
    } else if constexpr (MU == 2) {
      h0[c] = S > 0 ? p0 + times_i(p2) : p0 - times_i(p2);
      h1[c] = S > 0 ? p1 - times_i(p3) : p1 + times_i(p3);
    } else {
      h0[c] = S > 0 ? p0 + p2 : p0 - p2;
      h1[c] = S > 0 ? p1 + p3 : p1 - p3;
    }
  }
}

// INIT: the first contribution of a site sets the accumulator instead of adding to zero
// (the same values; no additions).
template <int MU, int S, typename T, bool INIT = false>
__device__ __forceinline__ void accumulate(cplx<T> acc[12], const cplx<T> w0[3], const cplx<T> w1[3]) {
  if constexpr (INIT) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[c] = w0[c];
      acc[3 + c] = w1[c];
      if constexpr (MU == 0) {
        if (S > 0) { acc[6 + c] = -times_i(w1[c]); acc[9 + c] = -times_i(w0[c]); }
        else       { acc[6 + c] = times_i(w1[c]); acc[9 + c] = times_i(w0[c]); }
      } else if constexpr (MU == 1) {
        if (S > 0) { acc[6 + c] = w1[c]; acc[9 + c] = -w0[c]; }
        else       { acc[6 + c] = -w1[c]; acc[9 + c] = w0[c]; }
      } else if constexpr (MU == 2) {
        if (S > 0) { acc[6 + c] = -times_i(w0[c]); acc[9 + c] = times_i(w1[c]); }
        else       { acc[6 + c] = times_i(w0[c]); acc[9 + c] = -times_i(w1[c]); }
      } else {
        if (S > 0) { acc[6 + c] = w0[c]; acc[9 + c] = w1[c]; }
        else       { acc[6 + c] = -w0[c]; acc[9 + c] = -w1[c]; }
      }
    }
    return;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = acc[c] + w0[c];
    acc[3 + c] = acc[3 + c] + w1[c];
    if constexpr (MU == 0) {
      if (S > 0) { acc[6 + c] = acc[6 + c] - times_i(w1[c]); acc[9 + c] = acc[9 + c] - times_i(w0[c]); }
      else       { acc[6 + c] = acc[6 + c] + times_i(w1[c]); acc[9 + c] = acc[9 + c] + times_i(w0[c]); }
    } else if constexpr (MU == 1) {
      if (S > 0) { acc[6 + c] = acc[6 + c] + w1[c]; acc[9 + c] = acc[9 + c] - w0[c]; }
      else       { acc[6 + c] = acc[6 + c] - w1[c]; acc[9 + c] = acc[9 + c] + w0[c]; }
    } else if constexpr (MU == 2) {
      if (S > 0) { acc[6 + c] = acc[6 + c] - times_i(w0[c]); acc[9 + c] = acc[9 + c] + times_i(w1[c]); }
      else       { acc[6 + c] = acc[6 + c] + times_i(w0[c]); acc[9 + c] = acc[9 + c] - times_i(w1[c]); }
    } else {
      if (S > 0) { acc[6 + c] = acc[6 + c] + w0[c]; acc[9 + c] = acc[9 + c] + w1[c]; }
      else       { acc[6 + c] = acc[6 + c] - w0[c]; acc[9 + c] = acc[9 + c] - w1[c]; }
    }
  }
}

// w = U h   and   w = U^dag h
template <typename T>
__device__ __forceinline__ void su3_mul(const cplx<T> u[9], const cplx<T> h[3], cplx<T> w[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    cplx<T> a = cmul(u[3 * i], h[0]);
    a = cmadd(a, u[3 * i + 1], h[1]);
    w[i] = cmadd(a, u[3 * i + 2], h[2]);
  }
}
template <typename T>
__device__ __forceinline__ void su3_dagmul(const cplx<T> u[9], const cplx<T> h[3], cplx<T> w[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    cplx<T> a = cjmul(u[i], h[0]);
    a = cjmadd(a, u[3 + i], h[1]);
    w[i] = cjmadd(a, u[6 + i], h[2]);
  }
}

// --------------------------------------------------- grid reductions
// Every reducing kernel adds up to NRED doubles per thread.  Each block
// reduces them (warp shuffles, then shared memory) and writes one partial
// per quantity; the last block to finish (atomic ticket) sums the partials
// in a fixed order, so the result does not depend on block scheduling,
// and hands them to a finaliser that runs in one thread.
struct ReduceScratch {
  double* partials;          // [NRED][max_blocks]
  unsigned int* ticket;      // one counter per reduction slot, left at 0
  int max_blocks;
};

template <int NRED>
__device__ __forceinline__ void block_sum(double (&v)[NRED], double* sh /* [NRED][32] */) {
#pragma unroll
  for (int q = 0; q < NRED; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NRED; ++q) sh[q * 32 + warp] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NRED; ++q) {
      double x = lane < nw ? sh[q * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      v[q] = x;               // valid in warp 0
    }
  }
}

// Returns true in thread 0 of the last block, with the grid totals in tot.
template <int NRED>
__device__ bool grid_sum(double (&v)[NRED], const ReduceScratch& rs, double (&tot)[NRED]) {
  __shared__ double sh[NRED * 32];
  __shared__ bool last;
  block_sum<NRED>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NRED; ++q) rs.partials[(size_t)q * rs.max_blocks + blockIdx.x] = v[q];
    __threadfence();
    unsigned int t = atomicAdd(rs.ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double w[NRED];
#pragma unroll
  for (int q = 0; q < NRED; ++q) {
    double x = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      x += __ldcg(rs.partials + (size_t)q * rs.max_blocks + b);
    w[q] = x;
  }
  __syncthreads();
  block_sum<NRED>(w, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NRED; ++q) tot[q] = w[q];
    *rs.ticket = 0u;
    return true;
  }
  return false;
}

// ------------------------------------------------------------ geometry
__device__ __forceinline__ void site_coords(const Geom& g, int s, int c[4]) {
  c[0] = s % g.L[0];
  int r = s / g.L[0];
  c[1] = r % g.L[1];
  r /= g.L[1];
  c[2] = r % g.L[2];
  c[3] = r / g.L[2];
}
__device__ __forceinline__ int nbr_fwd(const Geom& g, int s, const int c[4], int mu) {
  return c[mu] == g.L[mu] - 1 ? s - (g.L[mu] - 1) * g.stride[mu] : s + g.stride[mu];
}
__device__ __forceinline__ int nbr_bwd(const Geom& g, int s, const int c[4], int mu) {
  return c[mu] == 0 ? s + (g.L[mu] - 1) * g.stride[mu] : s - g.stride[mu];
}

}  // namespace lq
