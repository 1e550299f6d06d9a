// Batched CG on M^dag M (the paper's CG routine, Sec. 3, over a batch of
// systems): descriptors, per-column solver state, epilogues and the
// register-blocked stencil kernel shared by the translation units of the
// batched solver (k_batch.cu drives it; k_batch_*.cu instantiate the
// iteration for each storage format).
#pragma once
#include <algorithm>

#include "lq_internal.h"

namespace lq {

constexpr int kMaxSys = 16;
constexpr int kMaxCols = 64;
constexpr int kMaxWarps = 8;          // warps per block of the batched passes (<= 256 threads)
constexpr int kMaxRB = 4;

struct SysDesc {
  Geom geo;
  const void* gauge_lo;   // inner-format links of the system (SoA, stride V)
  const void* gauge64;    // FP64 links
  const void* gauge_df;   // links as double-float pairs (double-float updates), else null
  double kappa;
  int R;                  // right-hand sides
  int off;                // first element in the batch fields
  int col;                // first reduction column
  int tile0;              // first tile
  int tpg;                // tiles per group of rb right-hand sides: ceil(V / tile)
  const double* phi_in;   // canonical [R][V][4][3] complex (device)
  double* x_out;          // canonical [R][V][4][3] complex (device)
};

struct BatchDesc {
  int nsys, total, ncols, tile, ntiles, rb;
  int site_major;         // tile order inside a system: 1 site tile outer, rhs group inner; 0 group outer
  SysDesc sys[kMaxSys];
};

// Per-column solver scalars (device).
struct BatchState {
  double rr[kMaxCols], rr_prev[kMaxCols], alpha[kMaxCols], beta[kMaxCols], phi2[kMaxCols], rr_true[kMaxCols];
  double rr_ref[kMaxCols];   // |r|^2 right after the column's last reliable update
  int done[kMaxCols];
  int conv_iter[kMaxCols];
  double stop2;            // tol^2
  double delta2;           // reliable update once a column's |r|^2 fell below delta2 * rr_ref
  int iter, iter_since_ru, ru_every, maxiter, halt, breakdown, hist_len;
  int timeout;             // a bounded wait of the persistent iteration gave up
  double* hist;            // [ncols][hist_len] relative iterated residuals
  // device-side solve loop (one graph with conditional nodes): body counts of the
  // current iteration loop and of the update loop (each loop stops at a cap), whether
  // the current update skipped the double-float residual, and how many CG iterations,
  // update cycles, double-float updates and FP64 certifications ran
  int guard_inner, guard_outer, df_last;
  int loops[4];
};

struct BatchReduce {
  double* partials;        // [kMaxCols][max_blocks]
  unsigned int* ticket;
  int max_blocks;
};

__device__ __forceinline__ int system_of_tile(const BatchDesc& bd, int t) {
  int k = 0;
  while (k + 1 < bd.nsys && t >= bd.sys[k + 1].tile0) ++k;
  return k;
}

__device__ __forceinline__ int system_of_element(const BatchDesc& bd, int e) {
  int k = 0;
  while (k + 1 < bd.nsys && e >= bd.sys[k + 1].off) ++k;
  return k;
}

// The (system, first column, site) of this thread in tile t.
struct TileWork {
  int k, r0, s;
};
template <bool ONE = false>
__device__ __forceinline__ TileWork tile_work(const BatchDesc& bd, int t) {
  const int k = ONE ? 0 : system_of_tile(bd, t);
  const SysDesc& sd = bd.sys[k];
  const int rel = t - sd.tile0;
  int g, st;
  if (bd.site_major) {            // the rhs groups of one site tile are consecutive tiles
    const int ng = sd.R / bd.rb;
    st = rel / ng;
    g = rel - st * ng;
  } else {                        // all site tiles of one rhs group, then the next group
    g = rel / sd.tpg;
    st = rel - g * sd.tpg;
  }
  return {k, g * bd.rb, st * bd.tile + (int)threadIdx.x};
}

// Column totals of one pass: warp w sums columns w, w + nwarps, ...; lane l adds blocks
// l, l + 32, ... and the warp adds the lanes in a fixed tree: the same in every block.
__device__ __forceinline__ void column_totals(const double* part, int stride, int ncols, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < ncols; c += nw) {
    double x = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) x += __ldcg(part + (size_t)c * stride + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) out[c] = x;
  }
}

// Column sums of one block (sh_col[ncols]) -> partials; the last block adds
// them up per column (column_totals: a warp per column, fixed order) and calls
// fin(col_totals) in every one of its threads (finalisers spread the columns over
// the threads and vote on block-wide decisions).
template <class Fin>
__device__ void batch_grid_sum(const BatchDesc& bd, double* sh_col, const BatchReduce& br, const Fin& fin) {
  __shared__ bool last;
  __syncthreads();
  for (int c = threadIdx.x; c < bd.ncols; c += blockDim.x)
    br.partials[(size_t)c * br.max_blocks + blockIdx.x] = sh_col[c];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(br.ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double tot[kMaxCols];
  column_totals(br.partials, br.max_blocks, bd.ncols, tot);
  __syncthreads();
  fin(tot);
  if (threadIdx.x == 0) *br.ticket = 0u;
}

// Adds the block's per-thread sums v[0..RB) to columns col0 .. col0 + RB - 1 of
// sh_col (block-uniform call; fixed reduction order).
template <int RB>
__device__ __forceinline__ void flush_columns(double (&v)[RB], int col0, double* sh_red, double* sh_col) {
  block_sum<RB>(v, sh_red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < RB; ++q) sh_col[col0 + q] += v[q];
  }
  __syncthreads();
}

// Adds the warp's per-thread sums v[0..RB) to its slots of columns col0 .. col0 + RB - 1
// (sh_wcol[column * kMaxWarps + warp]): a fixed butterfly over the lanes, no block-wide
// synchronisation (warp-uniform call).
template <int RB>
__device__ __forceinline__ void flush_columns_warp(double (&v)[RB], int col0, double* sh_wcol) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < RB; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh_wcol[(col0 + q) * kMaxWarps + warp] += x;
  }
}

// sh_col[c] = the warps' slots of column c added in warp order (block-wide, synchronises).
__device__ __forceinline__ void gather_columns(int ncols, const double* sh_wcol, double* sh_col) {
  __syncthreads();
  const int nw = blockDim.x >> 5;
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
    double a = 0.0;
    for (int w = 0; w < nw; ++w) a += sh_wcol[c * kMaxWarps + w];
    sh_col[c] = a;
  }
  __syncthreads();
}

// Zeroes the warp slots of every column (block-wide, synchronises).
__device__ __forceinline__ void clear_columns(int ncols, double* sh_wcol) {
  for (int i = threadIdx.x; i < ncols * kMaxWarps; i += blockDim.x) sh_wcol[i] = 0.0;
  __syncthreads();
}

// ------------------------------------------------------------ epilogues
// Each gets the element index e (in the batch fields), its column, the
// result v = M in (or M^dag in) of that element, and returns the value to
// be summed for its column.
struct BEpiStore64 {                        // tmp = M x (FP64)
  SpinorRef out;
  int total;
  __device__ bool halted() const { return false; }
  template <typename T> __device__ double apply(int e, int, const cplx<T> v[12]) const {
    store_spinor<SStore::F64, T>(out, total, e, v);
    return 0.0;
  }
  static constexpr bool REDUCE = false;
  __device__ void finalize_cols(const double*, int) const {}
};

template <SStore S>
struct BEpiCG1 {                             // t = M p, tt = |t|^2, alpha = rr / tt
  SpinorRef t;
  int total;
  BatchState* st;
  static constexpr bool REDUCE = true;
  __device__ bool halted() const { return *(volatile const int*)&st->halt; }
  template <typename T> __device__ double apply(int e, int, const cplx<T> v[12]) const {
    store_spinor<S, T>(t, total, e, v);
    T a = (T)0;
#pragma unroll
    for (int k = 0; k < 12; ++k) { a = fma(v[k].re, v[k].re, a); a = fma(v[k].im, v[k].im, a); }
    return (double)a;
  }
  // every thread of the reducing block: one column per thread
  __device__ void finalize_cols(const double* tot, int ncols) const {
    int bad = 0;
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
      if (st->done[c]) { st->alpha[c] = 0.0; continue; }
      const double tt = tot[c];
      if (!(tt > 0.0) || !isfinite(tt)) { bad = 1; st->alpha[c] = 0.0; }
      else st->alpha[c] = st->rr[c] / tt;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) { st->breakdown = 1; st->halt = 1; }
  }
};

template <SStore S>
struct BEpiCG2 {                             // r -= alpha M^dag t, x += alpha p, rr = |r|^2
  SpinorRef r, x, p;
  int total;
  BatchState* st;
  static constexpr bool REDUCE = true;
  __device__ bool halted() const { return *(volatile const int*)&st->halt; }
  template <typename T> __device__ double apply(int e, int col, const cplx<T> v[12]) const {
    const T alpha = (T)st->alpha[col];
    cplx<T> rv[12], xv[12], pv[12];
    load_spinor<S, T, false>(r, total, e, rv);
    load_spinor<xlo_store(S), T, false>(x, total, e, xv);
    load_spinor<S, T>(p, total, e, pv);
    T a = (T)0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rv[k].re = fma(-alpha, v[k].re, rv[k].re);
      rv[k].im = fma(-alpha, v[k].im, rv[k].im);
      xv[k].re = fma(alpha, pv[k].re, xv[k].re);
      xv[k].im = fma(alpha, pv[k].im, xv[k].im);
      a = fma(rv[k].re, rv[k].re, a);
      a = fma(rv[k].im, rv[k].im, a);
    }
    store_spinor<S, T>(r, total, e, rv);
    store_spinor<xlo_store(S), T>(x, total, e, xv);
    return (double)a;
  }
  // every thread of the reducing block: one column per thread, block-wide votes
  __device__ void finalize_cols(const double* tot, int ncols) const {
    const int it = st->iter;
    int above = 0, trigger = 0, bad = 0;
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
      if (st->hist && it < st->hist_len) st->hist[(size_t)c * st->hist_len + it] = sqrt(tot[c] / st->phi2[c]);
      if (st->done[c]) { st->beta[c] = 0.0; continue; }
      const double rr_new = tot[c];
      if (!isfinite(rr_new)) bad = 1;
      st->beta[c] = rr_new / st->rr[c];
      st->rr_prev[c] = st->rr[c];
      st->rr[c] = rr_new;
      if (rr_new > st->stop2 * st->phi2[c]) above = 1;
      if (rr_new < st->delta2 * st->rr_ref[c]) trigger = 1;      // fell far: reliable update due
    }
    above = __syncthreads_or(above);
    trigger = __syncthreads_or(trigger);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
      const int since = st->iter_since_ru + 1;
      st->iter = it + 1;
      st->iter_since_ru = since;
      if (bad) st->breakdown = 1;
      if (bad || trigger || !above) st->halt = 1;
      if (st->ru_every > 0 && since >= st->ru_every) st->halt = 1;
      if (it + 1 >= st->maxiter) st->halt = 1;
    }
  }
};

// A column's true residual |r|^2 = tot after a reliable update: freeze the column once it
// meets the tolerance (alpha = beta = 0 from then on), reopen a frozen column whose
// residual no longer does (a double-float estimate that the FP64 certification overrules),
// restart the search direction when the recursion drifted far from the true residual.
__device__ __forceinline__ void reliable_update_column(BatchState* st, int c, double tot) {
  st->rr_true[c] = tot;
  if (!isfinite(tot)) { st->breakdown = 1; return; }
  const bool meets = tot <= st->stop2 * st->phi2[c];
  if (st->done[c] && meets) { st->beta[c] = 0.0; return; }
  if (meets) {                                      // converged: freeze the column
    st->done[c] = 1;
    st->conv_iter[c] = st->iter;
    st->beta[c] = 0.0;
    st->alpha[c] = 0.0;
  } else if (st->done[c] || tot > 100.0 * st->rr[c]) {
    // reopened, or the low-precision recursion drifted far below the true
    // residual: the search direction no longer fits it, restart from r
    st->done[c] = 0;
    st->beta[c] = 0.0;
  } else {
    st->beta[c] = tot / st->rr_prev[c];
  }
  st->rr[c] = tot;
  st->rr_ref[c] = tot;
}

template <SStore S>
struct BEpiResidual {                        // r64 = phi - M^dag tmp, r_lo = r64, rr_true = |r64|^2
  SpinorRef phi, r64, rlo;
  int total;
  BatchState* st;
  static constexpr bool REDUCE = true;
  __device__ bool halted() const { return false; }
  template <typename T> __device__ double apply(int e, int, const cplx<T> v[12]) const {
    cplx<double> ph[12], rv[12];
    load_spinor<SStore::F64, double>(phi, total, e, ph);
    double a = 0.0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rv[k] = {ph[k].re - (double)v[k].re, ph[k].im - (double)v[k].im};
      a += rv[k].re * rv[k].re + rv[k].im * rv[k].im;
    }
    store_spinor<SStore::F64, double>(r64, total, e, rv);
    store_spinor<S, double>(rlo, total, e, rv);
    return a;
  }
  // every thread of the reducing block: one column per thread
  __device__ void finalize_cols(const double* tot, int ncols) const {
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) reliable_update_column(st, c, tot[c]);
    if (threadIdx.x == 0) {
      st->iter_since_ru = 0;
      st->halt = 0;
    }
  }
};

// ------------------------------------------------------------ stencil
// Both hops of direction MU at site s for RB right-hand sides: the links
// U_mu(s) and U_mu(s - mu) are loaded and decoded once each and applied to the
// RB neighbour spinors (column r0 + j at element e0 + j V + n).  INIT: the forward hop is
// the site's first contribution and sets acc.
template <int MU, bool DAG, GStore G, SStore SI, typename T, int RB, int LD = 1, bool INIT = false>
__device__ __forceinline__ void batch_hops(const Geom& geo, int total, const GaugeRef& U, const SpinorRef& in, int s,
                                           const int c[4], int e0, cplx<T> (&acc)[RB][12]) {
  constexpr int SF = DAG ? +1 : -1;
  constexpr bool SCALED = SI == SStore::F16 || SI == SStore::BF16 || SI == SStore::I16 || G == GStore::I16_12;
  {
    const int n = nbr_fwd(geo, s, c, MU);
    const bool flip = MU == 3 && geo.antiperiodic && c[3] == geo.L[3] - 1;
    cplx<T> u[9];
    if constexpr (G == GStore::I16_12) load_link_q16<T>(U, geo.V, MU, s, u);
    else load_link<G, T>(U, geo.V, MU, s, u);
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      cplx<T> p[12];
      T sc = load_spinor_raw<SI, T, LD>(in, total, e0 + j * geo.V + n, p);
      cplx<T> h0[3], h1[3];
      project<MU, SF>(p, h0, h1);
      if (flip) sc = -sc;
      if constexpr (G == GStore::I16_12) sc = sc * (T)kQ16Inv;
      if (SCALED || (MU == 3 && geo.antiperiodic)) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { h0[k] = scale_c(sc, h0[k]); h1[k] = scale_c(sc, h1[k]); }
      }
      cplx<T> w0[3], w1[3];
      su3_mul(u, h0, w0);
      su3_mul(u, h1, w1);
      accumulate<MU, SF, T, INIT>(acc[j], w0, w1);
    }
  }
  {
    const int n = nbr_bwd(geo, s, c, MU);
    const bool flip = MU == 3 && geo.antiperiodic && c[3] == 0;
    cplx<T> u[9];
    if constexpr (G == GStore::I16_12) load_link_q16<T>(U, geo.V, MU, n, u);
    else load_link<G, T>(U, geo.V, MU, n, u);
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      cplx<T> p[12];
      T sc = load_spinor_raw<SI, T, LD>(in, total, e0 + j * geo.V + n, p);
      cplx<T> h0[3], h1[3];
      project<MU, -SF>(p, h0, h1);
      if (flip) sc = -sc;
      if constexpr (G == GStore::I16_12) sc = sc * (T)kQ16Inv;
      if (SCALED || (MU == 3 && geo.antiperiodic)) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { h0[k] = scale_c(sc, h0[k]); h1[k] = scale_c(sc, h1[k]); }
      }
      cplx<T> w0[3], w1[3];
      su3_dagmul(u, h0, w0);
      su3_dagmul(u, h1, w1);
      accumulate<MU, -SF>(acc[j], w0, w1);
    }
  }
}

// Register cap: one right-hand side per thread fits two blocks of 256 threads per
// SM (128 registers); more need the larger register budget of one block.
template <typename T, int RB> struct BatchMinBlocks { static constexpr int value = (RB == 1) ? 2 : 1; };
template <int RB> struct BatchMinBlocks<double, RB> { static constexpr int value = 1; };

// One stencil pass over the block's tiles: out = M in (or M^dag in) per right-hand side,
// handed to the epilogue; with Epi::REDUCE every warp adds its per-column sums to its slots
// of sh_wcol (cleared by the caller) whenever the block moves to another rhs group, and
// the pass ends with the block's column sums in sh_col (block-uniform calls: every thread
// of the block runs the same tiles).  ONE: the
// batch holds a single system, whose descriptor is then read at fixed offsets of the
// kernel parameters (no per-access indexed constant loads).
template <typename T, GStore G, SStore SI, bool DAG, int RB, class Epi, int LD = 1, bool ONE = false>
__device__ __forceinline__ void batch_stencil_pass(const BatchDesc& bd, const SpinorRef& in, const Epi& epi,
                                                   int use64, double* sh_wcol, double* sh_col) {
  int cur = -1;                       // first column of the group the sums belong to
  double red[RB];
#pragma unroll
  for (int j = 0; j < RB; ++j) red[j] = 0.0;
  for (int t = blockIdx.x; t < bd.ntiles; t += gridDim.x) {
    const TileWork w = tile_work<ONE>(bd, t);
    const SysDesc& sd = bd.sys[ONE ? 0 : w.k];
    const int col0 = sd.col + w.r0;
    if constexpr (Epi::REDUCE) {
      if (col0 != cur) {            // block-uniform: every thread of the tile has the same columns
        if (cur >= 0) flush_columns_warp<RB>(red, cur, sh_wcol);
        cur = col0;
#pragma unroll
        for (int j = 0; j < RB; ++j) red[j] = 0.0;
      }
    }
    if (w.s < sd.geo.V) {
      const int s = w.s;
      int c[4];
      site_coords(sd.geo, s, c);
      const GaugeRef U{use64 ? sd.gauge64 : sd.gauge_lo};
      const int e0 = sd.off + w.r0 * sd.geo.V;
      cplx<T> acc[RB][12];
      batch_hops<0, DAG, G, SI, T, RB, LD, true>(sd.geo, bd.total, U, in, s, c, e0, acc);
      batch_hops<1, DAG, G, SI, T, RB, LD>(sd.geo, bd.total, U, in, s, c, e0, acc);
      batch_hops<2, DAG, G, SI, T, RB, LD>(sd.geo, bd.total, U, in, s, c, e0, acc);
      batch_hops<3, DAG, G, SI, T, RB, LD>(sd.geo, bd.total, U, in, s, c, e0, acc);
      const T kappa = (T)sd.kappa;
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        const int e = e0 + j * sd.geo.V + s;
        cplx<T> ctr[12];
        load_spinor<SI, T, LD>(in, bd.total, e, ctr);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          acc[j][q].re = fma(-kappa, acc[j][q].re, ctr[q].re);
          acc[j][q].im = fma(-kappa, acc[j][q].im, ctr[q].im);
        }
        red[j] += epi.apply(e, col0 + j, acc[j]);
      }
    }
  }
  if constexpr (Epi::REDUCE) {
    if (cur >= 0) flush_columns_warp<RB>(red, cur, sh_wcol);
    gather_columns(bd.ncols, sh_wcol, sh_col);
  }
}

template <typename T, GStore G, SStore SI, bool DAG, int RB, class Epi, bool ONE = false>
__global__ void __launch_bounds__(256, (BatchMinBlocks<T, RB>::value))
    batch_dslash_kernel(BatchDesc bd, SpinorRef in, Epi epi, BatchReduce br, int use64) {
  if (epi.halted()) return;
  __shared__ double sh_col[kMaxCols];
  __shared__ double sh_wcol[Epi::REDUCE ? kMaxCols * kMaxWarps : 1];
  if constexpr (Epi::REDUCE) clear_columns(bd.ncols, sh_wcol);
  batch_stencil_pass<T, G, SI, DAG, RB, Epi, 1, ONE>(bd, in, epi, use64, sh_wcol, sh_col);
  if constexpr (Epi::REDUCE) {
    auto fin = [&](const double* tot) { epi.finalize_cols(tot, bd.ncols); };
    batch_grid_sum(bd, sh_col, br, fin);
  }
}

// ------------------------------------------------------ persistent iteration
// One cooperative launch runs up to max_iters CG iterations of the batch: the three
// passes with a device-wide barrier after each.  Every block reads the per-block
// column sums of a pass in block order and derives alpha, beta and the halt decision
// itself, so all blocks take the same decision (deterministic, no broadcast needed);
// block 0 writes the solver state back for the host.  Barrier waits are bounded: past
// spin_cycles a block gives up, raises st->timeout and st->halt and returns, and every
// other block then leaves at its next wait.
struct PersistArgs {
  SpinorRef plo, tlo, rlo, xlo;
  BatchState* st;
  double* part;                 // [2][kMaxCols][stride] per-block column sums of passes 1 and 2
  int stride;                   // >= gridDim.x
  unsigned int* bar_count;      // arrivals at the current barrier (0 at launch)
  unsigned int* bar_gen;        // barrier generation
  int bar_extra;                // blocks the barrier also waits for that do not exist (timeout tests)
  int max_iters;
  long long spin_cycles;        // wait limit of one barrier, in SM clock cycles
};

// CG step 2 with alpha from the block's shared memory (persistent iteration).
template <SStore S>
struct PEpiCG2 {
  SpinorRef r, x, p;
  int total;
  const double* alpha;          // [ncols], shared memory
  static constexpr bool REDUCE = true;
  template <typename T> __device__ double apply(int e, int col, const cplx<T> v[12]) const {
    const T al = (T)alpha[col];
    cplx<T> rv[12], xv[12], pv[12];
    load_spinor<S, T, 2>(r, total, e, rv);
    load_spinor<xlo_store(S), T, 2>(x, total, e, xv);
    load_spinor<S, T, 2>(p, total, e, pv);
    T a = (T)0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rv[k].re = fma(-al, v[k].re, rv[k].re);
      rv[k].im = fma(-al, v[k].im, rv[k].im);
      xv[k].re = fma(al, pv[k].re, xv[k].re);
      xv[k].im = fma(al, pv[k].im, xv[k].im);
      a = fma(rv[k].re, rv[k].re, a);
      a = fma(rv[k].im, rv[k].im, a);
    }
    store_spinor<S, T>(r, total, e, rv);
    store_spinor<xlo_store(S), T>(x, total, e, xv);
    return (double)a;
  }
};

// CG step 1 without the halt check (persistent iteration).
template <SStore S>
struct PEpiCG1 {
  SpinorRef t;
  int total;
  static constexpr bool REDUCE = true;
  template <typename T> __device__ double apply(int e, int, const cplx<T> v[12]) const {
    store_spinor<S, T>(t, total, e, v);
    T a = (T)0;
#pragma unroll
    for (int k = 0; k < 12; ++k) { a = fma(v[k].re, v[k].re, a); a = fma(v[k].im, v[k].im, a); }
    return (double)a;
  }
};

// Device-wide barrier with a bounded wait; false when this block gave up (or another did).
__device__ __forceinline__ bool grid_barrier(const PersistArgs& a, unsigned int& gen, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    *s_ok = 1;
    __threadfence();
    const unsigned int target = gridDim.x + (unsigned int)a.bar_extra;
    if (atomicAdd(a.bar_count, 1u) == target - 1) {
      atomicExch(a.bar_count, 0u);
      __threadfence();
      atomicAdd(a.bar_gen, 1u);
    } else {
      const long long t0 = clock64();
      while (atomicAdd(a.bar_gen, 0u) == gen) {
        if (*(volatile int*)&a.st->timeout) { *s_ok = 0; break; }
        if (clock64() - t0 > a.spin_cycles) {
          atomicExch(&a.st->timeout, 1);
          atomicExch(&a.st->halt, 1);
          *s_ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  gen += 1;
  return *s_ok != 0;
}

template <GStore G, SStore S, int RB>
__global__ void __launch_bounds__(256, (BatchMinBlocks<float, RB>::value))
    batch_persistent_kernel(BatchDesc bd, PersistArgs a) {
  __shared__ double sh_col[kMaxCols], sh_wcol[kMaxCols * kMaxWarps];
  __shared__ double s_rr[kMaxCols], s_alpha[kMaxCols], s_beta[kMaxCols], s_tot[kMaxCols];
  __shared__ int s_ok, s_gen;
  BatchState* st = a.st;
  if (*(volatile int*)&st->halt) return;
  if (threadIdx.x == 0) s_gen = (int)atomicAdd(a.bar_gen, 0u);
  for (int c = threadIdx.x; c < bd.ncols; c += blockDim.x) s_rr[c] = st->rr[c];
  __syncthreads();
  unsigned int gen = (unsigned int)s_gen;
  int iter = st->iter, since = st->iter_since_ru;
  double* part1 = a.part;
  double* part2 = a.part + (size_t)kMaxCols * a.stride;
  for (int it = 0; it < a.max_iters; ++it) {
    // pass 1: t = M p, |t|^2 per column -> alpha
    clear_columns(bd.ncols, sh_wcol);
    PEpiCG1<S> e1{a.tlo, bd.total};
    batch_stencil_pass<float, G, S, false, RB, PEpiCG1<S>, 2>(bd, a.plo, e1, 0, sh_wcol, sh_col);
    for (int c = threadIdx.x; c < bd.ncols; c += blockDim.x) part1[(size_t)c * a.stride + blockIdx.x] = sh_col[c];
    if (!grid_barrier(a, gen, &s_ok)) return;
    column_totals(part1, a.stride, bd.ncols, s_tot);
    __syncthreads();
    int bad = 0;
    if (threadIdx.x < bd.ncols) {
      const int c = threadIdx.x;
      const double tt = s_tot[c];
      if (st->done[c]) s_alpha[c] = 0.0;
      else if (!(tt > 0.0) || !isfinite(tt) || !isfinite(s_rr[c])) { s_alpha[c] = 0.0; bad = 1; }
      else s_alpha[c] = s_rr[c] / tt;
      if (blockIdx.x == 0) st->alpha[c] = s_alpha[c];
    }
    if (__syncthreads_or(bad)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) { st->breakdown = 1; st->halt = 1; st->iter = iter; }
      return;
    }
    // pass 2: r -= alpha M^dag t, x += alpha p, |r|^2 per column -> beta, halt decision
    clear_columns(bd.ncols, sh_wcol);
    PEpiCG2<S> e2{a.rlo, a.xlo, a.plo, bd.total, s_alpha};
    batch_stencil_pass<float, G, S, true, RB, PEpiCG2<S>, 2>(bd, a.tlo, e2, 0, sh_wcol, sh_col);
    for (int c = threadIdx.x; c < bd.ncols; c += blockDim.x) part2[(size_t)c * a.stride + blockIdx.x] = sh_col[c];
    if (!grid_barrier(a, gen, &s_ok)) return;
    column_totals(part2, a.stride, bd.ncols, s_tot);
    __syncthreads();
    int above = 0, trigger = 0, nonfinite = 0;
    if (threadIdx.x < bd.ncols) {
      const int c = threadIdx.x;
      const double rr_new = s_tot[c];
      if (blockIdx.x == 0 && st->hist && iter < st->hist_len)
        st->hist[(size_t)c * st->hist_len + iter] = sqrt(rr_new / st->phi2[c]);
      if (st->done[c]) {
        s_beta[c] = 0.0;
      } else {
        if (!isfinite(rr_new)) nonfinite = 1;
        s_beta[c] = rr_new / s_rr[c];
        if (blockIdx.x == 0) { st->rr_prev[c] = s_rr[c]; st->rr[c] = rr_new; st->beta[c] = s_beta[c]; }
        if (rr_new > st->stop2 * st->phi2[c]) above = 1;
        if (rr_new < st->delta2 * st->rr_ref[c]) trigger = 1;
      }
    }
    // every thread reads the column's old value before any writes the new one
    __syncthreads();
    if (threadIdx.x < bd.ncols && !st->done[threadIdx.x]) s_rr[threadIdx.x] = s_tot[threadIdx.x];
    const int any_above = __syncthreads_or(above);
    const int any_trigger = __syncthreads_or(trigger);
    const int any_nonfinite = __syncthreads_or(nonfinite);
    iter += 1;
    since += 1;
    const bool halt = !any_above || any_trigger || any_nonfinite || (st->ru_every > 0 && since >= st->ru_every) ||
                      iter >= st->maxiter;
    if (halt || it == a.max_iters - 1) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->iter = iter;
        st->iter_since_ru = since;
        if (any_nonfinite) st->breakdown = 1;
        if (halt) st->halt = 1;
      }
      if (halt) return;
    }
    // pass 3: p = r + beta p
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < bd.total; e += gridDim.x * blockDim.x) {
      const SysDesc& sd = bd.sys[system_of_element(bd, e)];
      const float beta = (float)s_beta[sd.col + (e - sd.off) / sd.geo.V];
      cplx<float> rv[12], pv[12];
      load_spinor<S, float, 2>(a.rlo, bd.total, e, rv);
      load_spinor<S, float, 2>(a.plo, bd.total, e, pv);
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        pv[q].re = fmaf(beta, pv[q].re, rv[q].re);
        pv[q].im = fmaf(beta, pv[q].im, rv[q].im);
      }
      store_spinor<S, float>(a.plo, bd.total, e, pv);
    }
    if (!grid_barrier(a, gen, &s_ok)) return;
  }
}

// Cooperative launch of the persistent iteration (grid: resident blocks, at most max_grid).
template <GStore G, SStore S>
cudaError_t launch_batch_persistent_t(const BatchDesc& bd, PersistArgs a, int sms, int max_grid, cudaStream_t st) {
  auto pick = [&](auto kern) -> cudaError_t {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, bd.tile, 0);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(std::min(bd.ntiles, max_grid), std::max(1, per_sm) * sms));
    if (grid > a.stride) return cudaErrorInvalidValue;
    void* args[] = {(void*)&bd, (void*)&a};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3(grid), dim3(bd.tile), args, 0, st);
  };
  switch (bd.rb) {
    case 2: return pick(&batch_persistent_kernel<G, S, 2>);
    case 3: return pick(&batch_persistent_kernel<G, S, 3>);
    case 4: return pick(&batch_persistent_kernel<G, S, 4>);
    default: return pick(&batch_persistent_kernel<G, S, 1>);
  }
}

// What one iteration of the batched solver needs (the fields live in the host-side workspace).
struct BatchIterArgs {
  SpinorRef plo, tlo, rlo, xlo;
  BatchState* st;
  BatchReduce br;
  int sms;        // SMs of the device
  int per_sm;     // resident blocks per SM used by the stencil passes (0: all that fit)
  cudaGraphConditionalHandle cond = 0;   // the device-side loop's condition (use_cond != 0)
  int use_cond = 0;
};

template <typename T, GStore G, SStore SI, bool DAG, int RB, class Epi, bool ONE>
void launch_batch_rb(const BatchDesc& bd, SpinorRef in, const Epi& epi, const BatchReduce& br, int use64, int sms,
                     int per_sm, cudaStream_t st) {
  auto kern = &batch_dslash_kernel<T, G, SI, DAG, RB, Epi, ONE>;
  static const int wave_all = resident_grid(reinterpret_cast<const void*>(kern), 256);
  // one wave of resident blocks (a second wave would sweep the lattice again and lose
  // the L2 reuse of neighbour spinors); per_sm > 0 caps the blocks per SM
  const int fit = std::max(1, wave_all / std::max(1, sms)) * (256 / bd.tile);
  const int wave = sms * (per_sm > 0 ? std::min(per_sm, fit) : fit);
  const int grid = std::max(1, std::min(std::min(bd.ntiles, br.max_blocks), wave));
  kern<<<grid, bd.tile, 0, st>>>(bd, in, epi, br, use64);
}

template <typename T, GStore G, SStore SI, bool DAG, class Epi>
void launch_batch(const BatchDesc& bd, SpinorRef in, const Epi& epi, const BatchReduce& br, int use64, int sms,
                  int per_sm, cudaStream_t st) {
  if constexpr (std::is_same<T, double>::value) {
    launch_batch_rb<T, G, SI, DAG, 1, Epi, false>(bd, in, epi, br, use64, sms, per_sm, st);   // FP64: one per thread
  } else if (bd.nsys == 1) {
    switch (bd.rb) {
      case 2: launch_batch_rb<T, G, SI, DAG, 2, Epi, true>(bd, in, epi, br, use64, sms, per_sm, st); break;
      case 3: launch_batch_rb<T, G, SI, DAG, 3, Epi, true>(bd, in, epi, br, use64, sms, per_sm, st); break;
      case 4: launch_batch_rb<T, G, SI, DAG, 4, Epi, true>(bd, in, epi, br, use64, sms, per_sm, st); break;
      default: launch_batch_rb<T, G, SI, DAG, 1, Epi, true>(bd, in, epi, br, use64, sms, per_sm, st); break;
    }
  } else {
    switch (bd.rb) {
      case 2: launch_batch_rb<T, G, SI, DAG, 2, Epi, false>(bd, in, epi, br, use64, sms, per_sm, st); break;
      case 3: launch_batch_rb<T, G, SI, DAG, 3, Epi, false>(bd, in, epi, br, use64, sms, per_sm, st); break;
      case 4: launch_batch_rb<T, G, SI, DAG, 4, Epi, false>(bd, in, epi, br, use64, sms, per_sm, st); break;
      default: launch_batch_rb<T, G, SI, DAG, 1, Epi, false>(bd, in, epi, br, use64, sms, per_sm, st); break;
    }
  }
}

// p = r + beta_col p (inner format), skipped when halted unless forced; use_cond: also sets
// the device-side iteration loop's condition cond
void launch_batch_xpay(const BatchDesc& bd, SStore s, SpinorRef r, SpinorRef p, BatchState* st, int forced,
                       int grid, cudaStream_t stream, cudaGraphConditionalHandle cond = 0, int use_cond = 0);

// One CG iteration (t = M p; r -= alpha M^dag t, x += alpha p; p = r + beta p) of the batch
// in the given storage, one translation unit per format (k_batch_f32.cu FP32-18,
// k_batch_f32_12.cu, k_batch_h16.cu FP16-12, k_batch_bf16.cu, k_batch_i16.cu).
void batch_iteration_f32(const BatchIterArgs& a, const BatchDesc& bd, int prec, cudaStream_t st);
void batch_iteration_f32_12(const BatchIterArgs& a, const BatchDesc& bd, int prec, cudaStream_t st);
void batch_iteration_h16(const BatchIterArgs& a, const BatchDesc& bd, int prec, cudaStream_t st);
void batch_iteration_bf16(const BatchIterArgs& a, const BatchDesc& bd, int prec, cudaStream_t st);
void batch_iteration_i16(const BatchIterArgs& a, const BatchDesc& bd, int prec, cudaStream_t st);
// The persistent form of the same iterations (one cooperative launch), per format.
cudaError_t batch_persistent_f32(const BatchDesc& bd, const PersistArgs& a, int prec, int sms, int max_grid,
                                 cudaStream_t st);
cudaError_t batch_persistent_f32_12(const BatchDesc& bd, const PersistArgs& a, int prec, int sms, int max_grid,
                                    cudaStream_t st);
cudaError_t batch_persistent_h16(const BatchDesc& bd, const PersistArgs& a, int prec, int sms, int max_grid,
                                 cudaStream_t st);
cudaError_t batch_persistent_bf16(const BatchDesc& bd, const PersistArgs& a, int prec, int sms, int max_grid,
                                  cudaStream_t st);
cudaError_t batch_persistent_i16(const BatchDesc& bd, const PersistArgs& a, int prec, int sms, int max_grid,
                                 cudaStream_t st);

// Double-float reliable update of the batch (k_batch_df.cu): x_df += x_lo, x_lo = 0
// (`accumulate`) and per column r = phi - M^dag M x_df with r to r_lo and the column's
// |r|^2 through reliable_update_column (`residual`).
struct BatchDfArgs {
  SpinorRef xlo, xdf, tmpdf, phidf, rlo;
  BatchState* st;
  BatchReduce br;
  const void* gauge_df[kMaxSys];   // per system: links as double-float pairs
  int flat_grid;
  bool accumulate, residual;       // which of the two steps to launch
  bool prefetch;                   // the double-float operator's prefetching variant
};
void batch_df_tail(const BatchDfArgs& a, const BatchDesc& bd, SStore s, cudaStream_t st);

template <GStore G, SStore S>
void batch_iteration_t(const BatchIterArgs& a, const BatchDesc& bd, cudaStream_t st) {
  BEpiCG1<S> e1{a.tlo, bd.total, a.st};
  launch_batch<float, G, S, false>(bd, a.plo, e1, a.br, 0, a.sms, a.per_sm, st);
  BEpiCG2<S> e2{a.rlo, a.xlo, a.plo, bd.total, a.st};
  launch_batch<float, G, S, true>(bd, a.tlo, e2, a.br, 0, a.sms, a.per_sm, st);
  launch_batch_xpay(bd, S, a.rlo, a.plo, a.st, 0, a.sms * 8, st, a.cond, a.use_cond);
}

}  // namespace lq
