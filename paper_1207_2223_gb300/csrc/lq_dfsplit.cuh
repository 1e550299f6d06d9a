// Double-float Wilson operator with two threads per site (the operator of
// Sec. 3 kernel 1 in ~48-bit double-float arithmetic on the FP32 pipe, used
// for the intermediate true residuals of mixed-precision CG).
//
// Double-float values double the registers of every quantity, and the long
// dependent chains of the compensated sums need many warps in flight.  The
// work of a site is therefore split between a pair of adjacent lanes by the
// rank-2 structure of the spin projection: with (1 -+ g_mu) in the
// DeGrand-Rossi basis the projected spinor is two colour vectors h0, h1 built
// from spins (0, 3) and (1, 2) for mu = x, y, or (0, 2) and (1, 3) for
// mu = z, t, and U h0 feeds spin 0 and one lower spin, U h1 spin 1 and the
// other.  Lane 0 of the pair computes everything that comes from h0, lane 1
// everything from h1; each accumulates its upper spin and partial sums of
// spins 2 and 3, and one exchange of partial sums at the end completes the
// lower spins (lane 0 keeps spins 0 and 2, lane 1 spins 1 and 3).  Links are
// read one row (U) or one column (U^dag) at a time and each row product is
// added at once, so no thread holds a whole link.  128 registers per thread,
// two blocks of 256 threads per SM: twice the warps of a one-thread-per-site
// double-float stencil (a third block spills).
#pragma once

#include "lq_dslash.cuh"

namespace lq {

constexpr int kDFSplitBlock = 256;
// resident blocks of 256 threads per SM requested from the compiler (register cap)
#ifndef LQ_DFSPLIT_MIN_BLOCKS
#define LQ_DFSPLIT_MIN_BLOCKS 2
#endif

struct DFLower {
  cplx<df64> s2[3], s3[3];
};

__device__ __forceinline__ cplx<df64> ldf(const float4* p, size_t i) {
  const float4 w = __ldg(p + i);
  return {df64(w.x, w.y), df64(w.z, w.w)};
}

// Projected colour component of lane `half` in direction MU with projector sign S
// (+1: 1 + g, -1: 1 - g) from the lane's two spin components pa (spin half) and pb (its
// partner); flip: the hop crosses the antiperiodic time boundary (sign -1).
template <int MU, int S>
__device__ __forceinline__ cplx<df64> df_proj(cplx<df64> pa, cplx<df64> pb, int half, bool flip) {
  // h0 (half 0) / h1 (half 1) of the projector (1 + S g_mu)
  cplx<df64> q;
  if constexpr (MU == 0) q = times_i(pb);                                     // x: p0 + S i p3, p1 + S i p2
  else if constexpr (MU == 1) q = (half == 0) ? -pb : pb;                     // y: p0 - S p3,   p1 + S p2
  else if constexpr (MU == 2) q = (half == 0) ? times_i(pb) : -times_i(pb);   // z: p0 + S i p2, p1 - S i p3
  else q = pb;                                                                // t: p0 + S p2,   p1 + S p3
  cplx<df64> h = (S > 0) ? pa + q : pa - q;
  if (flip) h = -h;
  return h;
}

// U h (FWD, link rows) or U^dag h (columns) for the lane's projected colour vector h, each
// row product added to the lane's upper spin and to its share of the lower spins at once.
// link(e) returns link element e (row-major 3 x 3).
template <int MU, int S, bool FWD, class Link>
__device__ __forceinline__ void df_mul_acc(const cplx<df64> h[3], const Link& link, int half, cplx<df64> up[3],
                                           DFLower& lo) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    cplx<df64> w;
    if constexpr (FWD) {
      w = cmul(link(3 * i), h[0]);
      w = cmadd(w, link(3 * i + 1), h[1]);
      w = cmadd(w, link(3 * i + 2), h[2]);
    } else {
      w = cjmul(link(i), h[0]);
      w = cjmadd(w, link(3 + i), h[1]);
      w = cjmadd(w, link(6 + i), h[2]);
    }
    up[i] = up[i] + w;
    // lower spins (accumulate<MU, S> of the one-thread stencil, restricted to w0 or w1)
    if constexpr (MU == 0) {           // spin 2 += -S i w1, spin 3 += -S i w0
      const cplx<df64> t = (S > 0) ? -times_i(w) : times_i(w);
      if (half == 0) lo.s3[i] = lo.s3[i] + t; else lo.s2[i] = lo.s2[i] + t;
    } else if constexpr (MU == 1) {    // spin 2 += S w1, spin 3 += -S w0
      if (half == 0) lo.s3[i] = (S > 0) ? lo.s3[i] - w : lo.s3[i] + w;
      else lo.s2[i] = (S > 0) ? lo.s2[i] + w : lo.s2[i] - w;
    } else if constexpr (MU == 2) {    // spin 2 += -S i w0, spin 3 += S i w1
      const cplx<df64> t = times_i(w);
      if (half == 0) lo.s2[i] = (S > 0) ? lo.s2[i] - t : lo.s2[i] + t;
      else lo.s3[i] = (S > 0) ? lo.s3[i] + t : lo.s3[i] - t;
    } else {                           // spin 2 += S w0, spin 3 += S w1
      if (half == 0) lo.s2[i] = (S > 0) ? lo.s2[i] + w : lo.s2[i] - w;
      else lo.s3[i] = (S > 0) ? lo.s3[i] + w : lo.s3[i] - w;
    }
  }
}

// One hop of lane `half` in direction MU with projector sign S, loading from global memory.
// FWD: the link U_mu(s) and the spinor at the forward neighbour; otherwise U_mu(n)^dag
// and the spinor at the backward neighbour n.
template <int MU, int S, bool FWD>
__device__ __forceinline__ void df_hop(const float4* psi, const float4* U, int V, int sstride, int n, int link_site,
                                       int half, bool flip, cplx<df64> up[3], DFLower& lo) {
  // spins of this lane: a (upper) and b (the partner in the projection)
  const int a = half;
  const int b = (MU <= 1) ? 3 - half : 2 + half;
  cplx<df64> h[3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    h[c] = df_proj<MU, S>(ldf(psi, (size_t)(3 * a + c) * sstride + n), ldf(psi, (size_t)(3 * b + c) * sstride + n),
                          half, flip);
  const float4* Um = U + (size_t)MU * 9 * V;
  df_mul_acc<MU, S, FWD>(h, [&](int e) { return ldf(Um, (size_t)e * V + link_site); }, half, up, lo);
}

// psi: the field shifted to the column's first element (site n at psi + chunk * sstride + n)
template <int MU, bool DAG>
__device__ __forceinline__ void df_dir(const Geom& geo, const float4* psi, int sstride, const float4* U, int s,
                                       const int c[4], int half, cplx<df64> up[3], DFLower& lo) {
  constexpr int SF = DAG ? +1 : -1;
  const int f = nbr_fwd(geo, s, c, MU);
  df_hop<MU, SF, true>(psi, U, geo.V, sstride, f, s, half, MU == 3 && geo.antiperiodic && c[3] == geo.L[3] - 1, up,
                       lo);
  const int b = nbr_bwd(geo, s, c, MU);
  df_hop<MU, -SF, false>(psi, U, geo.V, sstride, b, b, half, MU == 3 && geo.antiperiodic && c[3] == 0, up, lo);
}

__device__ __forceinline__ df64 shfl_df(df64 v) {
  return df64(__shfl_xor_sync(0xffffffffu, v.hi, 1), __shfl_xor_sync(0xffffffffu, v.lo, 1));
}

// out spins of lane `half`: v[0..2] = spin half, v[3..5] = spin half + 2 (colour fastest).
// Spinor fields are [chunk][element] with chunk stride `sstride` (V for a single lattice, the
// batch's element count for one column of a batch) and the lattice's sites at elements
// off .. off + V - 1; the epilogue gets the element index.
template <bool DAG, class Epi>
__global__ void __launch_bounds__(kDFSplitBlock, LQ_DFSPLIT_MIN_BLOCKS)
    dslash_dfsplit_kernel(Geom geo, const float4* __restrict__ U, const float4* __restrict__ psi_base, int sstride,
                          int off, df64 kappa, Epi epi, ReduceScratch rs) {
  const float4* psi = psi_base + off;
  double red[1] = {0.0};
  const int half = threadIdx.x & 1;
  const int Vr = (geo.V + 15) & ~15;                     // whole warps iterate together
  const int stride = (gridDim.x * blockDim.x) >> 1;
  for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 1; s < Vr; s += stride) {
    const bool active = s < geo.V;
    const int ss = active ? s : 0;
    int c[4];
    site_coords(geo, ss, c);
    cplx<df64> up[3];
    DFLower lo;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      up[i] = {df64(0.f), df64(0.f)};
      lo.s2[i] = up[i];
      lo.s3[i] = up[i];
    }
    df_dir<0, DAG>(geo, psi, sstride, U, ss, c, half, up, lo);
    df_dir<1, DAG>(geo, psi, sstride, U, ss, c, half, up, lo);
    df_dir<2, DAG>(geo, psi, sstride, U, ss, c, half, up, lo);
    df_dir<3, DAG>(geo, psi, sstride, U, ss, c, half, up, lo);
    // lane 0 keeps spin 2 and hands its spin-3 sums to lane 1, and the other way round
    cplx<df64> v[6];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const cplx<df64> give = half == 0 ? lo.s3[i] : lo.s2[i];
      const cplx<df64> mine = half == 0 ? lo.s2[i] : lo.s3[i];
      const cplx<df64> got = {shfl_df(give.re), shfl_df(give.im)};
      v[i] = up[i];
      v[3 + i] = mine + got;
    }
    // M = 1 - kappa H on the lane's two spins
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int comp = (k < 3) ? 3 * half + k : 3 * (half + 2) + (k - 3);
      const cplx<df64> ctr = ldf(psi, (size_t)comp * sstride + ss);
      v[k] = {fma(-kappa, v[k].re, ctr.re), fma(-kappa, v[k].im, ctr.im)};
    }
    epi.apply(sstride, off + ss, half, active, v, red);
  }
  if constexpr (Epi::REDUCE) {
    double tot[1];
    if (grid_sum<1>(red, rs, tot)) epi.finalize(tot);
  }
}

// ------------------------------------------------------------ epilogues
// out = M in, double-float field
struct DFEpiStore {
  static constexpr bool REDUCE = false;
  SpinorRef out;
  __device__ void apply(int V, int s, int half, bool active, const cplx<df64> v[6], double (&)[1]) const {
    if (!active) return;
    float4* p = static_cast<float4*>(out.p);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int comp = (k < 3) ? 3 * half + k : 3 * (half + 2) + (k - 3);
      p[(size_t)comp * V + s] = make_float4(v[k].re.hi, v[k].re.lo, v[k].im.hi, v[k].im.lo);
    }
  }
  __device__ void finalize(double (&)[1]) const {}
};

// |r|^2 of a single solve goes to its state
struct DFFinSolver {
  SolverState* st;
  __device__ void operator()(double rr) const { st->rr_true = rr; }
};

// r = phi - M^dag tmp (double-float), r_lo = r in the inner format, |r|^2 to the
// finaliser; RDF: r is also stored as a double-float field (rdf)
template <SStore SLO, class Fin = DFFinSolver, bool RDF = true>
struct DFEpiResidual {
  static constexpr bool REDUCE = true;
  SpinorRef phi, rdf, rlo;
  Fin fin;
  __device__ void apply(int V, int s, int half, bool active, const cplx<df64> v[6], double (&red)[1]) const {
    const float4* ph = static_cast<const float4*>(phi.p);
    float4* rp = static_cast<float4*>(rdf.p);
    cplx<float> mine[6];
    float a = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int comp = (k < 3) ? 3 * half + k : 3 * (half + 2) + (k - 3);
      const cplx<df64> f = ldf(ph, (size_t)comp * V + s);
      const cplx<df64> r = {f.re - v[k].re, f.im - v[k].im};
      if (RDF && active) rp[(size_t)comp * V + s] = make_float4(r.re.hi, r.re.lo, r.im.hi, r.im.lo);
      mine[k] = {(float)r.re, (float)r.im};
      a = fmaf(mine[k].re, mine[k].re, a);
      a = fmaf(mine[k].im, mine[k].im, a);
    }
    // the inner-format copy needs all 12 components of the site (per-site norm): lane 0 gathers
    cplx<float> full[12];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const cplx<float> o = {__shfl_xor_sync(0xffffffffu, mine[k].re, 1), __shfl_xor_sync(0xffffffffu, mine[k].im, 1)};
      // lane 0 holds spins 0, 2; the partner spins 1, 3
      const int ca = (k < 3) ? k : 6 + (k - 3);        // own components (lane 0 view)
      const int cb = (k < 3) ? 3 + k : 9 + (k - 3);    // partner's components
      full[ca] = mine[k];
      full[cb] = o;
    }
    if (active && half == 0) store_spinor<SLO, float>(rlo, V, s, full);
    if (active) red[0] += (double)a;
  }
  __device__ void finalize(double (&tot)[1]) const { fin(tot[0]); }
};

// ------------------------------------------------------------ prefetching variant
// The same operator with the next hop's operands copied into shared memory by
// asynchronous copies (cp.async, 16 bytes each) while the current hop computes: the
// double-float stencil above waits on memory (few warps, long dependent chains), and the
// copies need no registers.  Per site and stage a slot of 21 float4: the 9 link elements
// (lane 0 copies 0-4, lane 1 5-8; both read all 9), then lane 0's and lane 1's 6 spinor
// components (spins a, b x colours).  Two stages: 128 sites x 2 x 336 B = 84 KB per block
// of 256 threads, two blocks per SM.
constexpr int kDFSlot = 21;
constexpr size_t kDFAsyncSmem = (size_t)(kDFSplitBlock / 2) * 2 * kDFSlot * sizeof(float4);

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ cplx<df64> sdf(const float4& w) { return {df64(w.x, w.y), df64(w.z, w.w)}; }

// Hop H (direction H / 2; forward for even H, backward for odd) of site s: start the copies
// of its operands into `slot` (one commit group per hop).
template <int H>
__device__ __forceinline__ void df_issue(const Geom& geo, const float4* psi, int sstride, const float4* U, int s,
                                         const int c[4], int half, float4* slot) {
  constexpr int MU = H >> 1;
  constexpr bool FWD = (H & 1) == 0;
  const int n = FWD ? nbr_fwd(geo, s, c, MU) : nbr_bwd(geo, s, c, MU);
  const int link_site = FWD ? s : n;
  const float4* Um = U + (size_t)MU * 9 * geo.V + link_site;
  const int e0 = half ? 5 : 0, e1 = half ? 9 : 5;
  for (int e = e0; e < e1; ++e) cp_async16(slot + e, Um + (size_t)e * geo.V);
  const int a = half;
  const int b = (MU <= 1) ? 3 - half : 2 + half;
  float4* sp = slot + 9 + 6 * half;
#pragma unroll
  for (int cc = 0; cc < 3; ++cc) {
    cp_async16(sp + 2 * cc, psi + (size_t)(3 * a + cc) * sstride + n);
    cp_async16(sp + 2 * cc + 1, psi + (size_t)(3 * b + cc) * sstride + n);
  }
  cp_async_commit();
}

// Hop H computed from its operands in `slot`.
template <int H, bool DAG>
__device__ __forceinline__ void df_consume(const Geom& geo, const int c[4], int half, const float4* slot,
                                           cplx<df64> up[3], DFLower& lo) {
  constexpr int MU = H >> 1;
  constexpr bool FWD = (H & 1) == 0;
  constexpr int SF = DAG ? +1 : -1;
  constexpr int S = FWD ? SF : -SF;
  const bool flip = MU == 3 && geo.antiperiodic && (FWD ? c[3] == geo.L[3] - 1 : c[3] == 0);
  const float4* sp = slot + 9 + 6 * half;
  cplx<df64> h[3];
#pragma unroll
  for (int cc = 0; cc < 3; ++cc) h[cc] = df_proj<MU, S>(sdf(sp[2 * cc]), sdf(sp[2 * cc + 1]), half, flip);
  df_mul_acc<MU, S, FWD>(h, [&](int e) { return sdf(slot[e]); }, half, up, lo);
}

// One step of the two-stage pipeline: start hop H + 1 (unless H is the last), wait for
// hop H's copies, compute it; the warp barriers make the partner lane's link copies
// visible and keep a stage from being refilled while the partner still reads it.
template <int H, bool DAG>
__device__ __forceinline__ void df_step(const Geom& geo, const float4* psi, int sstride, const float4* U, int s,
                                        const int c[4], int half, float4* const stage[2], cplx<df64> up[3],
                                        DFLower& lo) {
  if constexpr (H < 7) {
    df_issue<H + 1>(geo, psi, sstride, U, s, c, half, stage[(H + 1) & 1]);
    cp_async_wait<1>();
  } else {
    cp_async_wait<0>();
  }
  __syncwarp();
  df_consume<H, DAG>(geo, c, half, stage[H & 1], up, lo);
  __syncwarp();
}

template <bool DAG, class Epi>
__global__ void __launch_bounds__(kDFSplitBlock, LQ_DFSPLIT_MIN_BLOCKS)
    dslash_dfsplit_async_kernel(Geom geo, const float4* __restrict__ U, const float4* __restrict__ psi_base,
                                int sstride, int off, df64 kappa, Epi epi, ReduceScratch rs) {
  extern __shared__ float4 df_smem[];
  const float4* psi = psi_base + off;
  double red[1] = {0.0};
  const int half = threadIdx.x & 1;
  const int slot = threadIdx.x >> 1;
  float4* const stage[2] = {df_smem + (size_t)slot * kDFSlot,
                            df_smem + (size_t)(kDFSplitBlock / 2 + slot) * kDFSlot};
  const int Vr = (geo.V + 15) & ~15;                     // whole warps iterate together
  const int stride = (gridDim.x * blockDim.x) >> 1;
  for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 1; s < Vr; s += stride) {
    const bool active = s < geo.V;
    const int ss = active ? s : 0;
    int c[4];
    site_coords(geo, ss, c);
    cplx<df64> up[3];
    DFLower lo;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      up[i] = {df64(0.f), df64(0.f)};
      lo.s2[i] = up[i];
      lo.s3[i] = up[i];
    }
    df_issue<0>(geo, psi, sstride, U, ss, c, half, stage[0]);
    df_step<0, DAG>(geo, psi, sstride, U, ss, c, half, stage, up, lo);
    df_step<1, DAG>(geo, psi, sstride, U, ss, c, half, stage, up, lo);
    df_step<2, DAG>(geo, psi, sstride, U, ss, c, half, stage, up, lo);
    df_step<3, DAG>(geo, psi, sstride, U, ss, c, half, stage, up, lo);
    df_step<4, DAG>(geo, psi, sstride, U, ss, c, half, stage, up, lo);
    df_step<5, DAG>(geo, psi, sstride, U, ss, c, half, stage, up, lo);
    df_step<6, DAG>(geo, psi, sstride, U, ss, c, half, stage, up, lo);
    df_step<7, DAG>(geo, psi, sstride, U, ss, c, half, stage, up, lo);
    // lane 0 keeps spin 2 and hands its spin-3 sums to lane 1, and the other way round
    cplx<df64> v[6];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const cplx<df64> give = half == 0 ? lo.s3[i] : lo.s2[i];
      const cplx<df64> mine = half == 0 ? lo.s2[i] : lo.s3[i];
      const cplx<df64> got = {shfl_df(give.re), shfl_df(give.im)};
      v[i] = up[i];
      v[3 + i] = mine + got;
    }
    // M = 1 - kappa H on the lane's two spins
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int comp = (k < 3) ? 3 * half + k : 3 * (half + 2) + (k - 3);
      const cplx<df64> ctr = ldf(psi, (size_t)comp * sstride + ss);
      v[k] = {fma(-kappa, v[k].re, ctr.re), fma(-kappa, v[k].im, ctr.im)};
    }
    epi.apply(sstride, off + ss, half, active, v, red);
  }
  if constexpr (Epi::REDUCE) {
    double tot[1];
    if (grid_sum<1>(red, rs, tot)) epi.finalize(tot);
  }
}

// Resident blocks of the prefetching kernel, its shared memory opted in once.  Internal
// linkage: every translation unit launches its own instance of the kernel and must opt in
// that instance (a cached flag shared across units would leave the others at the default).
template <bool DAG, class Epi>
static int dfsplit_async_wave() {
  static const int wave = [] {
    const void* k = reinterpret_cast<const void*>(&dslash_dfsplit_async_kernel<DAG, Epi>);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDFAsyncSmem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kDFSplitBlock, kDFAsyncSmem);
    return std::max(1, sms) * std::max(1, per_sm);
  }();
  return wave;
}

// sstride < 0: a single lattice (chunk stride V, sites at elements 0 .. V - 1).  prefetch:
// the variant with asynchronous copies of the next hop's operands into shared memory.
template <bool DAG, class Epi>
inline void launch_dslash_dfsplit(const Geom& geo, const void* U, SpinorRef in, double kappa, const Epi& epi,
                                  const ReduceScratch& rs, cudaStream_t stream, int sstride = -1, int off = 0,
                                  bool prefetch = false) {
  const float4* u = static_cast<const float4*>(U);
  const float4* p = static_cast<const float4*>(in.p);
  const int st = sstride < 0 ? geo.V : sstride;
  if (prefetch) {
    const int grid = std::max(1, std::min(grid_for(2 * geo.V, kDFSplitBlock), dfsplit_async_wave<DAG, Epi>()));
    dslash_dfsplit_async_kernel<DAG, Epi><<<grid, kDFSplitBlock, kDFAsyncSmem, stream>>>(geo, u, p, st, off,
                                                                                          df64(kappa), epi, rs);
    return;
  }
  static const int wave =
      resident_grid(reinterpret_cast<const void*>(&dslash_dfsplit_kernel<DAG, Epi>), kDFSplitBlock);
  const int grid = std::max(1, std::min(grid_for(2 * geo.V, kDFSplitBlock), wave));
  dslash_dfsplit_kernel<DAG, Epi><<<grid, kDFSplitBlock, 0, stream>>>(geo, u, p, st, off, df64(kappa), epi, rs);
}

}  // namespace lq
