// Two-site packed form of the Wilson stencil for 16-bit fixed-point storage
// (I16 spinors with per-site norms, I16_12 links), selected with
// LQ_OPT_PAIR_SITES.  The operator is the one of lq_dslash.cuh (Eq. 4; Sec. 3
// kernel 1); what differs is the mapping to the hardware.  The one-site
// 16-bit stencil issues ~2100 instructions per site (decoding, rebuilding the
// third link row, the half-spinor algebra) and keeps ~70% of the issue slots
// busy.  Here each thread applies the stencil at two sites, x = (x, y, z, t)
// and x' = (x, y, z, t + L_t/2), and every real of the arithmetic is the pair
// (value at x, value at x') in one register pair, so one packed FP32x2
// instruction (FFMA2 / FADD2 / FMUL2) does the work of two scalar ones.
// Measured on GB300 it issues about a third fewer instructions but runs 8-15% slower:
// a packed instruction holds the FMA pipe for two cycles, so the pipe time
// per site does not change, and the doubled per-thread state lowers the
// resident warps from 16 to 12 per SM.  It is therefore off by default.
//
// x' is x shifted by half the lattice in time, so every neighbour of x' is
// the corresponding neighbour of x shifted by V/2 (mod V); only the signs of
// the antiperiodic time boundary differ (the forward hop of x' crosses it
// when t = L_t/2 - 1, the backward hop of x when t = 0).  Both halves are
// read with the same coalesced pattern: a warp loads 32 consecutive sites in
// each half.  Needs an even L_t.
//
// Scaling: links are used as raw 16-bit integers q (rows 0, 1 carry 32767 U,
// the rebuilt row 2 carries 32767^2 U and is brought to 32767 U on the
// output of U h, or through the input of U^dag h); the factors 1/32767 of
// link and spinor and -kappa are folded into one scale of each half spinor.
#pragma once
#include "lq_dslash.cuh"

namespace lq {
namespace pair {

struct c2 { float2 re, im; };   // a complex number at two sites

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as fma(b, -1, a): one rounding, the same result as a subtraction
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg(float2 a) { return __fmul2_rn(a, f2(-1.f, -1.f)); }
__device__ __forceinline__ c2 cscale(c2 a, float2 s) { return {mul(a.re, s), mul(a.im, s)}; }

// Raw fixed-point values q of the low / high 16-bit halves of one word of
// each site (see q16_to2 in lq_device.cuh for the byte-permutation decode).
__device__ __forceinline__ float2 q_lo(uint32_t w0, uint32_t w1) {
  return add(f2(__int_as_float((int)__byte_perm(w0, 0x4B00u, 0x5410u)),
                __int_as_float((int)__byte_perm(w1, 0x4B00u, 0x5410u))),
             f2(-kQ16Bias, -kQ16Bias));
}
__device__ __forceinline__ float2 q_hi(uint32_t w0, uint32_t w1) {
  return add(f2(__int_as_float((int)__byte_perm(w0, 0x4B00u, 0x5432u)),
                __int_as_float((int)__byte_perm(w1, 0x4B00u, 0x5432u))),
             f2(-kQ16Bias, -kQ16Bias));
}

// The 24 raw reals of an I16 spinor at sites n0, n1 and the two site norms.
// (value = q * norm / 32767.)  RO: the field is read-only in this kernel.
template <bool RO>
__device__ __forceinline__ void load_q(const SpinorRef& f, int V, int n0, int n1, c2 v[12], float2& nrm) {
  const uint4* p = static_cast<const uint4*>(f.p);
  nrm = f2(ld<RO>(f.norm + n0), ld<RO>(f.norm + n1));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint4 a = ld<RO>(p + (size_t)k * V + n0), b = ld<RO>(p + (size_t)k * V + n1);
    v[4 * k + 0] = {q_lo(a.x, b.x), q_hi(a.x, b.x)};
    v[4 * k + 1] = {q_lo(a.y, b.y), q_hi(a.y, b.y)};
    v[4 * k + 2] = {q_lo(a.z, b.z), q_hi(a.z, b.z)};
    v[4 * k + 3] = {q_lo(a.w, b.w), q_hi(a.w, b.w)};
  }
}

// Encode 24 reals per site with a fresh per-site norm (max |real|).  The
// scaled value is rounded to the nearest integer by one fused multiply-add
// into the binade [2^23, 2^24), whose low 16 bits are the stored word.
__device__ __forceinline__ void store_q(const SpinorRef& f, int V, int n0, int n1, const c2 v[12]) {
  float m0 = 0.f, m1 = 0.f;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    m0 = fmaxf(m0, fmaxf(fabsf(v[c].re.x), fabsf(v[c].im.x)));
    m1 = fmaxf(m1, fmaxf(fabsf(v[c].re.y), fabsf(v[c].im.y)));
  }
  const float2 inv = f2(m0 > 0.f ? kQ16 / m0 : 0.f, m1 > 0.f ? kQ16 / m1 : 0.f);
  f.norm[n0] = m0;
  f.norm[n1] = m1;
  uint4* p = static_cast<uint4*>(f.p);
  const float2 bias = f2(kQ16Bias, kQ16Bias);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint32_t a[4], b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 re = fma2(v[4 * k + j].re, inv, bias), im = fma2(v[4 * k + j].im, inv, bias);
      a[j] = __byte_perm(__float_as_uint(re.x), __float_as_uint(im.x), 0x5410u);
      b[j] = __byte_perm(__float_as_uint(re.y), __float_as_uint(im.y), 0x5410u);
    }
    p[(size_t)k * V + n0] = make_uint4(a[0], a[1], a[2], a[3]);
    p[(size_t)k * V + n1] = make_uint4(b[0], b[1], b[2], b[3]);
  }
}

// FP32 spinor (float4 [6][V]) at sites n0, n1 as complex pairs, and back
__device__ __forceinline__ void load_f32(const SpinorRef& f, int V, int n0, int n1, c2 v[12]) {
  const float4* p = static_cast<const float4*>(f.p);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 a = p[(size_t)k * V + n0], b = p[(size_t)k * V + n1];
    v[2 * k] = {f2(a.x, b.x), f2(a.y, b.y)};
    v[2 * k + 1] = {f2(a.z, b.z), f2(a.w, b.w)};
  }
}
__device__ __forceinline__ void store_f32(const SpinorRef& f, int V, int n0, int n1, const c2 v[12]) {
  float4* p = static_cast<float4*>(f.p);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    p[(size_t)k * V + n0] = make_float4(v[2 * k].re.x, v[2 * k].im.x, v[2 * k + 1].re.x, v[2 * k + 1].im.x);
    p[(size_t)k * V + n1] = make_float4(v[2 * k].re.y, v[2 * k].im.y, v[2 * k + 1].re.y, v[2 * k + 1].im.y);
  }
}

// conj(a b - c d)
__device__ __forceinline__ c2 cross_conj(c2 a, c2 b, c2 c, c2 d) {
  const float2 x = fma2(c.im, d.im, mul(a.re, b.re));
  const float2 y = fma2(c.re, d.re, mul(a.im, b.im));
  const float2 z = fma2(a.re, b.im, mul(a.im, b.re));
  const float2 w = fma2(c.re, d.im, mul(c.im, d.re));
  return {sub(x, y), sub(w, z)};
}

// Raw I16_12 link of direction mu at sites n0, n1: rows 0, 1 as stored
// (32767 U), row 2 = conj(row 0 x row 1) in units of 32767^2.
__device__ __forceinline__ void load_link_q(const GaugeRef& g, int V, int mu, int n0, int n1, c2 u[9]) {
  const uint2* p = static_cast<const uint2*>(g.p) + (size_t)mu * 3 * V;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint2 a = __ldg(p + (size_t)k * V + n0), b = __ldg(p + (size_t)k * V + n1);
    u[2 * k] = {q_lo(a.x, b.x), q_hi(a.x, b.x)};
    u[2 * k + 1] = {q_lo(a.y, b.y), q_hi(a.y, b.y)};
  }
  u[6] = cross_conj(u[1], u[5], u[2], u[4]);
  u[7] = cross_conj(u[2], u[3], u[0], u[5]);
  u[8] = cross_conj(u[0], u[4], u[1], u[3]);
}

// a + SG b  and  a + SG i b
template <int SG> __device__ __forceinline__ c2 plus(c2 a, c2 b) {
  if constexpr (SG > 0) return {add(a.re, b.re), add(a.im, b.im)};
  else return {sub(a.re, b.re), sub(a.im, b.im)};
}
template <int SG> __device__ __forceinline__ c2 plus_i(c2 a, c2 b) {
  if constexpr (SG > 0) return {sub(a.re, b.im), add(a.im, b.re)};
  else return {add(a.re, b.im), sub(a.im, b.re)};
}
// the same with a = 0 on the first hop
template <int SG, bool FIRST> __device__ __forceinline__ c2 acc_plus(c2 a, c2 b) {
  if constexpr (!FIRST) return plus<SG>(a, b);
  else if constexpr (SG > 0) return b;
  else return {neg(b.re), neg(b.im)};
}
template <int SG, bool FIRST> __device__ __forceinline__ c2 acc_plus_i(c2 a, c2 b) {
  if constexpr (!FIRST) return plus_i<SG>(a, b);
  else if constexpr (SG > 0) return {neg(b.im), b.re};
  else return {b.im, neg(b.re)};
}

// Projector (1 + S gamma_mu), DeGrand-Rossi basis (table in lq_device.cuh).
template <int MU, int S>
__device__ __forceinline__ void project(const c2 p[12], c2 h0[3], c2 h1[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const c2 p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
    if constexpr (MU == 0) { h0[c] = plus_i<S>(p0, p3); h1[c] = plus_i<S>(p1, p2); }
    else if constexpr (MU == 1) { h0[c] = plus<-S>(p0, p3); h1[c] = plus<S>(p1, p2); }
    else if constexpr (MU == 2) { h0[c] = plus_i<S>(p0, p2); h1[c] = plus_i<-S>(p1, p3); }
    else { h0[c] = plus<S>(p0, p2); h1[c] = plus<S>(p1, p3); }
  }
}

template <int MU, int S, bool FIRST>
__device__ __forceinline__ void accumulate(c2 acc[12], const c2 w0[3], const c2 w1[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = acc_plus<1, FIRST>(acc[c], w0[c]);
    acc[3 + c] = acc_plus<1, FIRST>(acc[3 + c], w1[c]);
    if constexpr (MU == 0) {
      acc[6 + c] = acc_plus_i<-S, FIRST>(acc[6 + c], w1[c]);
      acc[9 + c] = acc_plus_i<-S, FIRST>(acc[9 + c], w0[c]);
    } else if constexpr (MU == 1) {
      acc[6 + c] = acc_plus<S, FIRST>(acc[6 + c], w1[c]);
      acc[9 + c] = acc_plus<-S, FIRST>(acc[9 + c], w0[c]);
    } else if constexpr (MU == 2) {
      acc[6 + c] = acc_plus_i<-S, FIRST>(acc[6 + c], w0[c]);
      acc[9 + c] = acc_plus_i<S, FIRST>(acc[9 + c], w1[c]);
    } else {
      acc[6 + c] = acc_plus<S, FIRST>(acc[6 + c], w0[c]);
      acc[9 + c] = acc_plus<S, FIRST>(acc[9 + c], w1[c]);
    }
  }
}

// w = U h
__device__ __forceinline__ void su3_mul(const c2 u[9], const c2 h[3], c2 w[3]) {
  float2 nh[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) nh[k] = neg(h[k].im);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float2 re = mul(u[3 * i].re, h[0].re), im = mul(u[3 * i].re, h[0].im);
    re = fma2(u[3 * i].im, nh[0], re);
    im = fma2(u[3 * i].im, h[0].re, im);
#pragma unroll
    for (int k = 1; k < 3; ++k) {
      re = fma2(u[3 * i + k].re, h[k].re, re);
      re = fma2(u[3 * i + k].im, nh[k], re);
      im = fma2(u[3 * i + k].re, h[k].im, im);
      im = fma2(u[3 * i + k].im, h[k].re, im);
    }
    w[i] = {re, im};
  }
}
// w = U^dag h:  w_i = sum_k conj(U_ki) h_k
__device__ __forceinline__ void su3_dagmul(const c2 u[9], const c2 h[3], c2 w[3]) {
  float2 nh[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) nh[k] = neg(h[k].re);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float2 re = mul(u[i].re, h[0].re), im = mul(u[i].re, h[0].im);
    re = fma2(u[i].im, h[0].im, re);
    im = fma2(u[i].im, nh[0], im);
#pragma unroll
    for (int k = 1; k < 3; ++k) {
      re = fma2(u[3 * k + i].re, h[k].re, re);
      re = fma2(u[3 * k + i].im, h[k].im, re);
      im = fma2(u[3 * k + i].re, h[k].im, im);
      im = fma2(u[3 * k + i].im, nh[k], im);
    }
    w[i] = {re, im};
  }
}

__device__ __forceinline__ int partner(int n, int half) { return n < half ? n + half : n - half; }

// The two hops of direction MU at the site pair (s, s + V/2); acc += -kappa
// times their contribution (acc = it, on the first hop).  mkq = -kappa/32767^2.
template <int MU, bool DAG, bool FIRST>
__device__ __forceinline__ void hop(const Geom& geo, const GaugeRef& U, const SpinorRef& in, int s, int half,
                                    const int c[4], float mkq, c2 acc[12]) {
  constexpr int SF = DAG ? +1 : -1;   // forward hop uses (1 + SF g_mu)
  const int V = geo.V;
  {
    const int n0 = nbr_fwd(geo, s, c, MU), n1 = partner(n0, half);
    c2 p[12];
    float2 nrm;
    load_q<true>(in, V, n0, n1, p, nrm);
    c2 h0[3], h1[3];
    project<MU, SF>(p, h0, h1);
    float2 sc = mul(nrm, f2(mkq, mkq));
    if (MU == 3 && geo.antiperiodic && c[3] == (geo.L[3] >> 1) - 1) sc.y = -sc.y;
#pragma unroll
    for (int k = 0; k < 3; ++k) { h0[k] = cscale(h0[k], sc); h1[k] = cscale(h1[k], sc); }
    c2 u[9];
    load_link_q(U, V, MU, s, s + half, u);
    c2 w0[3], w1[3];
    su3_mul(u, h0, w0);
    su3_mul(u, h1, w1);
    const float2 r2 = f2(kQ16Inv, kQ16Inv);   // row 2 of the rebuilt link
    w0[2] = cscale(w0[2], r2);
    w1[2] = cscale(w1[2], r2);
    accumulate<MU, SF, FIRST>(acc, w0, w1);
  }
  {
    const int n0 = nbr_bwd(geo, s, c, MU), n1 = partner(n0, half);
    c2 p[12];
    float2 nrm;
    load_q<true>(in, V, n0, n1, p, nrm);
    c2 h0[3], h1[3];
    project<MU, -SF>(p, h0, h1);
    float2 sc = mul(nrm, f2(mkq, mkq));
    if (MU == 3 && geo.antiperiodic && c[3] == 0) sc.x = -sc.x;
    const float2 sc2 = mul(sc, f2(kQ16Inv, kQ16Inv));   // meets row 2 of the link
#pragma unroll
    for (int k = 0; k < 2; ++k) { h0[k] = cscale(h0[k], sc); h1[k] = cscale(h1[k], sc); }
    h0[2] = cscale(h0[2], sc2);
    h1[2] = cscale(h1[2], sc2);
    c2 u[9];
    load_link_q(U, V, MU, n0, n1, u);
    c2 w0[3], w1[3];
    su3_dagmul(u, h0, w0);
    su3_dagmul(u, h1, w1);
    accumulate<MU, -SF, false>(acc, w0, w1);
  }
}

__device__ __forceinline__ double norm2(const c2 v[12]) {
  float2 a = f2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 12; ++k) { a = fma2(v[k].re, v[k].re, a); a = fma2(v[k].im, v[k].im, a); }
  return (double)a.x + (double)a.y;
}

}  // namespace pair

// ~170 registers a thread: three blocks of 128 per SM (faster than one of 256
// with ~230 registers)
#ifndef LQ_PAIR_BLOCK
#define LQ_PAIR_BLOCK 128
#endif
#ifndef LQ_PAIR_MIN_BLOCKS
#define LQ_PAIR_MIN_BLOCKS 3
#endif

// out = M in (or M^dag) at the site pairs (s, s + V/2), s < V/2, handed to
// the epilogue's apply_pair; grid-stride over the pairs like dslash_kernel.
template <bool DAG, class Epi>
__global__ void __launch_bounds__(LQ_PAIR_BLOCK, LQ_PAIR_MIN_BLOCKS)
dslash_pair_kernel(Geom geo, GaugeRef U, SpinorRef in, float kappa, Epi epi, ReduceScratch rs) {
  using namespace pair;
  if (epi.halted()) return;
  double red[Epi::NRED];
#pragma unroll
  for (int q = 0; q < Epi::NRED; ++q) red[q] = 0.0;
  const int half = geo.V >> 1;
  const float mkq = -kappa * kQ16Inv * kQ16Inv;
  const int stride = gridDim.x * blockDim.x;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < half; s += stride) {
    int c[4];
    site_coords(geo, s, c);
    c2 acc[12];
    hop<0, DAG, true>(geo, U, in, s, half, c, mkq, acc);
    hop<1, DAG, false>(geo, U, in, s, half, c, mkq, acc);
    hop<2, DAG, false>(geo, U, in, s, half, c, mkq, acc);
    hop<3, DAG, false>(geo, U, in, s, half, c, mkq, acc);
    {
      c2 q[12];
      float2 nrm;
      load_q<true>(in, geo.V, s, s + half, q, nrm);
      const float2 sc = mul(nrm, f2(kQ16Inv, kQ16Inv));
#pragma unroll
      for (int k = 0; k < 12; ++k) { acc[k].re = fma2(q[k].re, sc, acc[k].re); acc[k].im = fma2(q[k].im, sc, acc[k].im); }
    }
    epi.apply_pair(geo.V, s, s + half, acc, red);
  }
  if constexpr (Epi::REDUCE) {
    double tot[Epi::NRED];
    if (grid_sum<Epi::NRED>(red, rs, tot)) epi.finalize(tot);
  }
}

// ------------------------------------------------- pair epilogues (I16)
struct PairStore : EpiStore<SStore::I16> {             // out = M psi
  __device__ void apply_pair(int V, int n0, int n1, pair::c2 v[12], double (&)[NRED]) const {
    pair::store_q(out, V, n0, n1, v);
  }
};

struct PairCG1 : EpiCG1<SStore::I16> {                 // t = M p, |t|^2
  __device__ void apply_pair(int V, int n0, int n1, pair::c2 v[12], double (&red)[NRED]) const {
    pair::store_q(t, V, n0, n1, v);
    red[0] += pair::norm2(v);
  }
};

// r -= alpha M^dag t, x += alpha p, |r|^2 (x in FP32, r and p 16-bit)
struct PairCG2 : EpiCG2<SStore::I16, SStore::F32, SStore::I16> {
  __device__ void apply_pair(int V, int n0, int n1, pair::c2 v[12], double (&red)[NRED]) const {
    using namespace pair;
    const float a = (float)st->alpha;
    {
      c2 rq[12];
      float2 nr;
      load_q<false>(r, V, n0, n1, rq, nr);
      const float2 sr = mul(nr, f2(kQ16Inv, kQ16Inv)), ma = f2(-a, -a);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        rq[k].re = fma2(rq[k].re, sr, mul(v[k].re, ma));
        rq[k].im = fma2(rq[k].im, sr, mul(v[k].im, ma));
      }
      store_q(r, V, n0, n1, rq);
      red[0] += norm2(rq);
    }
    c2 xv[12], pq[12];
    float2 np;
    load_f32(x, V, n0, n1, xv);
    load_q<true>(p, V, n0, n1, pq, np);
    const float2 sp = mul(np, f2(a * kQ16Inv, a * kQ16Inv));
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      xv[k].re = fma2(pq[k].re, sp, xv[k].re);
      xv[k].im = fma2(pq[k].im, sp, xv[k].im);
    }
    store_f32(x, V, n0, n1, xv);
  }
};

}  // namespace lq
