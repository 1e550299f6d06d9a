// Batched CG on M^dag M: many right-hand sides sharing one gauge field, and
// independent lattices of different volumes and kappa, solved together in
// one launch per CG pass (the paper's CG routine, Sec. 3, over a batch of
// systems).
//
// Layout.  All systems share one set of fields of `total` elements; system
// k owns elements off_k .. off_k + V_k R_k - 1, its right-hand sides
// interleaved fastest (element off_k + site * R_k + r), so the threads of one
// site read the same link and the load is broadcast across the R_k lanes.
// Every field is [chunk][element] as in lq_device.cuh.
//
// Launch.  Blocks walk a list of tiles (tile t of system k covers elements
// (t - tile0_k) * tile .. + tile - 1 of that system); the tile size is a
// multiple of every R_k, so a thread's right-hand side is fixed by its lane.
// Each block accumulates per-column sums (column = system x right-hand side)
// in shared memory tile by tile, in a fixed order; the last block adds the
// per-block partials column by column: deterministic.
//
// Mixed precision.  The iterations run in FP32 (FP32 or 12-real FP32 links);
// every `reliable_every` iterations x is folded into FP64 and the FP64 true
// residual of every column is recomputed; a column whose true residual meets
// the tolerance is frozen (alpha = 0 from then on).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "lq_internal.h"

namespace lq {

constexpr int kMaxSys = 16;
constexpr int kMaxCols = 64;

struct SysDesc {
  Geom geo;
  const void* gauge_lo;   // inner-format links of the system (SoA, stride V)
  const void* gauge64;    // FP64 links
  double kappa;
  int R;                  // right-hand sides
  int off;                // first element in the batch fields
  int col;                // first reduction column
  int tile0;              // first tile
  const double* phi_in;   // canonical [R][V][4][3] complex (device)
  double* x_out;          // canonical [R][V][4][3] complex (device)
};

struct BatchDesc {
  int nsys, total, ncols, tile, ntiles;
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
  int iter, iter_since_ru, ru_every, maxiter, halt, breakdown, hist_len, pad_;
  double* hist;            // [ncols][hist_len] relative iterated residuals
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

// Column sums of one block (sh_col[ncols]) -> partials; the last block adds
// them up per column and calls fin(col_totals) in thread 0.
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
  for (int c = threadIdx.x; c < bd.ncols; c += blockDim.x) {
    double a = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) a += __ldcg(br.partials + (size_t)c * br.max_blocks + b);
    tot[c] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    fin(tot);
    *br.ticket = 0u;
  }
}

// Adds one tile's per-thread values v into sh_col, per column, in a fixed order.
__device__ __forceinline__ void tile_columns(const SysDesc& sd, double v, double* sh_tile, double* sh_col) {
  sh_tile[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < sd.R) {
    double a = 0.0;
    for (int j = threadIdx.x; j < (int)blockDim.x; j += sd.R) a += sh_tile[j];
    sh_col[sd.col + threadIdx.x] += a;
  }
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
  __device__ void finalize(const double*) const {}
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
  __device__ void finalize_cols(const double* tot, int ncols) const {
    for (int c = 0; c < ncols; ++c) {
      if (st->done[c]) { st->alpha[c] = 0.0; continue; }
      const double tt = tot[c];
      if (!(tt > 0.0) || !isfinite(tt)) { st->breakdown = 1; st->halt = 1; st->alpha[c] = 0.0; }
      else st->alpha[c] = st->rr[c] / tt;
    }
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
  __device__ void finalize_cols(const double* tot, int ncols) const {
    const int it = st->iter;
    bool all_below = true;
    for (int c = 0; c < ncols; ++c) {
      if (st->hist && it < st->hist_len) st->hist[(size_t)c * st->hist_len + it] = sqrt(tot[c] / st->phi2[c]);
      if (st->done[c]) { st->beta[c] = 0.0; continue; }
      const double rr_new = tot[c];
      if (!isfinite(rr_new)) { st->breakdown = 1; st->halt = 1; }
      st->beta[c] = rr_new / st->rr[c];
      st->rr_prev[c] = st->rr[c];
      st->rr[c] = rr_new;
      if (rr_new > st->stop2 * st->phi2[c]) all_below = false;
      if (rr_new < st->delta2 * st->rr_ref[c]) st->halt = 1;     // fell far: reliable update due
    }
    st->iter = it + 1;
    st->iter_since_ru += 1;
    if (all_below) st->halt = 1;
    if (st->ru_every > 0 && st->iter_since_ru >= st->ru_every) st->halt = 1;
    if (st->iter >= st->maxiter) st->halt = 1;
  }
};

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
  __device__ void finalize_cols(const double* tot, int ncols) const {
    for (int c = 0; c < ncols; ++c) {
      st->rr_true[c] = tot[c];
      if (st->done[c]) { st->beta[c] = 0.0; continue; }
      if (!isfinite(tot[c])) { st->breakdown = 1; continue; }
      if (tot[c] <= st->stop2 * st->phi2[c]) {       // converged: freeze the column
        st->done[c] = 1;
        st->conv_iter[c] = st->iter;
        st->beta[c] = 0.0;
        st->alpha[c] = 0.0;
      } else if (tot[c] > 100.0 * st->rr[c]) {
        // the low-precision recursion drifted far below the true residual: the
        // search direction no longer fits it, restart the column from r
        st->beta[c] = 0.0;
      } else {
        st->beta[c] = tot[c] / st->rr_prev[c];
      }
      st->rr[c] = tot[c];
      st->rr_ref[c] = tot[c];
    }
    st->iter_since_ru = 0;
    st->halt = 0;
  }
};

// ------------------------------------------------------------ kernels
template <typename T, GStore G, SStore SI, bool DAG, class Epi>
__global__ void __launch_bounds__(256) batch_dslash_kernel(BatchDesc bd, SpinorRef in, Epi epi, BatchReduce br,
                                                           int use64) {
  if (epi.halted()) return;
  extern __shared__ double smem[];
  double* sh_tile = smem;                 // [blockDim]
  double* sh_col = smem + blockDim.x;     // [ncols]
  for (int c = threadIdx.x; c < bd.ncols; c += blockDim.x) sh_col[c] = 0.0;
  __syncthreads();
  // A thread's column is fixed while the block stays inside one system (the
  // tile is a multiple of R), so it sums in a register and the block folds
  // the sums into sh_col only when the system changes (block-uniform).
  int cur = -1;
  double acc_v = 0.0;
  for (int t = blockIdx.x; t < bd.ntiles; t += gridDim.x) {
    const int k = system_of_tile(bd, t);
    if constexpr (Epi::REDUCE) {
      if (k != cur) {
        if (cur >= 0) tile_columns(bd.sys[cur], acc_v, sh_tile, sh_col);
        cur = k;
        acc_v = 0.0;
      }
    }
    const SysDesc& sd = bd.sys[k];
    const int e_loc = (t - sd.tile0) * bd.tile + threadIdx.x;
    double v = 0.0;
    if (e_loc < sd.geo.V * sd.R) {
      const int s = e_loc / sd.R, r = e_loc - s * sd.R;
      int c[4];
      site_coords(sd.geo, s, c);
      const BatchIndex ix{bd.total, sd.off, sd.R, r};
      const GaugeRef U{use64 ? sd.gauge64 : sd.gauge_lo};
      cplx<T> acc[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) acc[q] = {(T)0, (T)0};
      hop_dir<0, DAG, G, SI, T, BatchIndex>(sd.geo, U, in, s, c, acc, ix);
      hop_dir<1, DAG, G, SI, T, BatchIndex>(sd.geo, U, in, s, c, acc, ix);
      hop_dir<2, DAG, G, SI, T, BatchIndex>(sd.geo, U, in, s, c, acc, ix);
      hop_dir<3, DAG, G, SI, T, BatchIndex>(sd.geo, U, in, s, c, acc, ix);
      cplx<T> ctr[12];
      load_spinor<SI, T>(in, bd.total, ix(s), ctr);
      const T kappa = (T)sd.kappa;
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        acc[q].re = fma(-kappa, acc[q].re, ctr[q].re);
        acc[q].im = fma(-kappa, acc[q].im, ctr[q].im);
      }
      v = epi.apply(ix(s), sd.col + r, acc);
    }
    acc_v += v;
  }
  if constexpr (Epi::REDUCE) {
    if (cur >= 0) tile_columns(bd.sys[cur], acc_v, sh_tile, sh_col);
    auto fin = [&](const double* tot) { epi.finalize_cols(tot, bd.ncols); };
    batch_grid_sum(bd, sh_col, br, fin);
  }
}

// p = r + beta_col p (inner format), skipped when halted unless forced
template <SStore S>
__global__ void batch_xpay_kernel(BatchDesc bd, SpinorRef r, SpinorRef p, const BatchState* st, int forced) {
  if (!forced && *(volatile const int*)&st->halt) return;
  for (int t = blockIdx.x; t < bd.ntiles; t += gridDim.x) {
    const int k = system_of_tile(bd, t);
    const SysDesc& sd = bd.sys[k];
    const int e_loc = (t - sd.tile0) * bd.tile + threadIdx.x;
    if (e_loc >= sd.geo.V * sd.R) continue;
    const int e = sd.off + e_loc;
    const float beta = (float)st->beta[sd.col + e_loc % sd.R];
    cplx<float> rv[12], pv[12];
    load_spinor<S, float>(r, bd.total, e, rv);
    load_spinor<S, float, false>(p, bd.total, e, pv);
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      pv[q].re = fmaf(beta, pv[q].re, rv[q].re);
      pv[q].im = fmaf(beta, pv[q].im, rv[q].im);
    }
    store_spinor<S, float>(p, bd.total, e, pv);
  }
}

// Start: phi (canonical, per system) -> phi64; x64 = 0; x_lo = 0; r_lo = p_lo = phi; phi2 per column.
template <SStore S>
__global__ void batch_init_kernel(BatchDesc bd, SpinorRef phi64, SpinorRef x64, SpinorRef xlo, SpinorRef rlo,
                                  SpinorRef plo, BatchState* st, BatchReduce br) {
  extern __shared__ double smem[];
  double* sh_tile = smem;
  double* sh_col = smem + blockDim.x;
  for (int c = threadIdx.x; c < bd.ncols; c += blockDim.x) sh_col[c] = 0.0;
  __syncthreads();
  for (int t = blockIdx.x; t < bd.ntiles; t += gridDim.x) {
    const int k = system_of_tile(bd, t);
    const SysDesc& sd = bd.sys[k];
    const int e_loc = (t - sd.tile0) * bd.tile + threadIdx.x;
    double v = 0.0;
    if (e_loc < sd.geo.V * sd.R) {
      const int s = e_loc / sd.R, r = e_loc - s * sd.R;
      const int e = sd.off + e_loc;
      const double2* src = reinterpret_cast<const double2*>(sd.phi_in) + ((size_t)r * sd.geo.V + s) * 12;
      cplx<double> a[12], z[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        const double2 w = src[q];
        a[q] = {w.x, w.y};
        z[q] = {0.0, 0.0};
        v += w.x * w.x + w.y * w.y;
      }
      store_spinor<SStore::F64, double>(phi64, bd.total, e, a);
      store_spinor<SStore::F64, double>(x64, bd.total, e, z);
      store_spinor<xlo_store(S), double>(xlo, bd.total, e, z);
      store_spinor<S, double>(rlo, bd.total, e, a);
      store_spinor<S, double>(plo, bd.total, e, a);
    }
    tile_columns(sd, v, sh_tile, sh_col);
  }
  auto fin = [&](const double* tot) {
    for (int c = 0; c < bd.ncols; ++c) {
      st->phi2[c] = tot[c];
      st->rr[c] = st->rr_prev[c] = st->rr_true[c] = st->rr_ref[c] = tot[c];
      st->done[c] = tot[c] == 0.0 ? 1 : 0;
      st->conv_iter[c] = 0;
      st->alpha[c] = st->beta[c] = 0.0;
      if (!isfinite(tot[c])) st->breakdown = 1;
    }
  };
  batch_grid_sum(bd, sh_col, br, fin);
}

// x64 += x_lo; x_lo = 0
template <SStore S>
__global__ void batch_accumulate_kernel(int total, SpinorRef xlo, SpinorRef x64) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    cplx<double> a[12], b[12], z[12];
    load_spinor<xlo_store(S), double, false>(xlo, total, e, a);
    load_spinor<SStore::F64, double, false>(x64, total, e, b);
#pragma unroll
    for (int q = 0; q < 12; ++q) { b[q] = b[q] + a[q]; z[q] = {0.0, 0.0}; }
    store_spinor<SStore::F64, double>(x64, total, e, b);
    store_spinor<xlo_store(S), double>(xlo, total, e, z);
  }
}

// x64 -> canonical per system
__global__ void batch_unpack_kernel(BatchDesc bd, SpinorRef x64) {
  for (int t = blockIdx.x; t < bd.ntiles; t += gridDim.x) {
    const int k = system_of_tile(bd, t);
    const SysDesc& sd = bd.sys[k];
    const int e_loc = (t - sd.tile0) * bd.tile + threadIdx.x;
    if (e_loc >= sd.geo.V * sd.R) continue;
    const int s = e_loc / sd.R, r = e_loc - s * sd.R;
    cplx<double> a[12];
    load_spinor<SStore::F64, double>(x64, bd.total, sd.off + e_loc, a);
    double2* dst = reinterpret_cast<double2*>(sd.x_out) + ((size_t)r * sd.geo.V + s) * 12;
#pragma unroll
    for (int q = 0; q < 12; ++q) dst[q] = make_double2(a[q].re, a[q].im);
  }
}

// ------------------------------------------------------------ host side
namespace {

struct BatchWork {
  std::vector<int> key;           // signature: per system dims, R, antiperiodic, precision
  int total = 0, ncols = 0, grid_cap = 0;
  Field phi64, x64, r64, tmp64, plo, tlo, rlo, xlo;
  BatchState* st = nullptr;
  BatchState* st_host = nullptr;
  BatchReduce br{};
  double* hist = nullptr;
  int hist_cap = 0;
  int tile = 0;                   // tuned tile size
  // recorded iteration graphs with the descriptor they were recorded for
  std::vector<std::pair<BatchDesc, cudaGraphExec_t>> graphs;
};

// the fields of a descriptor the iteration kernels read (not the I/O pointers)
bool same_iteration_desc(const BatchDesc& a, const BatchDesc& b) {
  BatchDesc x = a, y = b;
  for (int k = 0; k < kMaxSys; ++k) {
    x.sys[k].phi_in = y.sys[k].phi_in = nullptr;
    x.sys[k].x_out = y.sys[k].x_out = nullptr;
  }
  return std::memcmp(&x, &y, sizeof(BatchDesc)) == 0;
}

void free_batch(BatchWork* w) {
  if (!w) return;
  for (auto& g : w->graphs) cudaGraphExecDestroy(g.second);
  for (Field* f : {&w->phi64, &w->x64, &w->r64, &w->tmp64, &w->plo, &w->tlo, &w->rlo, &w->xlo}) {
    if (f->data) cudaFree(f->data);
    if (f->norm) cudaFree(f->norm);
  }
  if (w->st) cudaFree(w->st);
  if (w->st_host) cudaFreeHost(w->st_host);
  if (w->br.partials) cudaFree(w->br.partials);
  if (w->br.ticket) cudaFree(w->br.ticket);
  if (w->hist) cudaFree(w->hist);
  delete w;
}

BatchDesc make_desc(lq_ctx** ctxs, int n, int R, const double* const* phi, double* const* x, const double* kappa,
                    int prec, int tile) {
  BatchDesc bd{};
  bd.nsys = n;
  bd.tile = tile;
  int off = 0, col = 0, t0 = 0;
  for (int k = 0; k < n; ++k) {
    SysDesc& sd = bd.sys[k];
    sd.geo = ctxs[k]->geo;
    sd.gauge_lo = ctxs[k]->gauge_lo[prec];
    sd.gauge64 = ctxs[k]->gauge64;
    sd.kappa = kappa[k];
    sd.R = R;
    sd.off = off;
    sd.col = col;
    sd.tile0 = t0;
    sd.phi_in = phi ? phi[k] : nullptr;
    sd.x_out = x ? x[k] : nullptr;
    off += sd.geo.V * R;
    col += R;
    t0 += (sd.geo.V * R + tile - 1) / tile;
  }
  bd.total = off;
  bd.ncols = col;
  bd.ntiles = t0;
  return bd;
}

// One wave of resident blocks: a second wave would sweep the lattice again
// after the first, losing the L2 reuse of neighbour spinors.
template <typename T, GStore G, SStore SI, bool DAG, class Epi>
void launch_batch(const BatchDesc& bd, SpinorRef in, const Epi& epi, const BatchReduce& br, int use64,
                  int grid_cap, cudaStream_t st) {
  const int wave = resident_grid(reinterpret_cast<const void*>(&batch_dslash_kernel<T, G, SI, DAG, Epi>), bd.tile);
  const int grid = std::min(std::min(bd.ntiles, grid_cap), wave);
  const size_t sh = sizeof(double) * (bd.tile + bd.ncols);
  batch_dslash_kernel<T, G, SI, DAG, Epi><<<grid, bd.tile, sh, st>>>(bd, in, epi, br, use64);
}

template <GStore G, SStore S>
void batch_iteration(BatchWork* w, const BatchDesc& bd, cudaStream_t st) {
  BEpiCG1<S> e1{w->tlo.ref(), bd.total, w->st};
  launch_batch<float, G, S, false>(bd, w->plo.ref(), e1, w->br, 0, w->grid_cap, st);
  BEpiCG2<S> e2{w->rlo.ref(), w->xlo.ref(), w->plo.ref(), bd.total, w->st};
  launch_batch<float, G, S, true>(bd, w->tlo.ref(), e2, w->br, 0, w->grid_cap, st);
  batch_xpay_kernel<S><<<std::min(bd.ntiles, w->grid_cap), bd.tile, 0, st>>>(bd, w->rlo.ref(), w->plo.ref(),
                                                                             w->st, 0);
}

void batch_iteration_prec(BatchWork* w, const BatchDesc& bd, int prec, cudaStream_t st) {
  switch (prec) {
    case LQ_F32_12: batch_iteration<GStore::F32_12, SStore::F32>(w, bd, st); break;
    case LQ_F16_12: batch_iteration<GStore::F16_12, SStore::F16>(w, bd, st); break;
    case LQ_I16_12: batch_iteration<GStore::I16_12, SStore::I16>(w, bd, st); break;
    default: batch_iteration<GStore::F32_18, SStore::F32>(w, bd, st); break;
  }
}

template <SStore S>
void batch_true_residual_s(BatchWork* w, const BatchDesc& bd, cudaStream_t st) {
  BEpiStore64 e0{w->tmp64.ref(), bd.total};
  launch_batch<double, GStore::F64_18, SStore::F64, false>(bd, w->x64.ref(), e0, w->br, 1, w->grid_cap, st);
  BEpiResidual<S> e1{w->phi64.ref(), w->r64.ref(), w->rlo.ref(), bd.total, w->st};
  launch_batch<double, GStore::F64_18, SStore::F64, true>(bd, w->tmp64.ref(), e1, w->br, 1, w->grid_cap, st);
}

void batch_true_residual(BatchWork* w, const BatchDesc& bd, int prec, cudaStream_t st) {
  switch (spinor_store_of(prec)) {
    case SStore::F16: batch_true_residual_s<SStore::F16>(w, bd, st); break;
    case SStore::I16: batch_true_residual_s<SStore::I16>(w, bd, st); break;
    default: batch_true_residual_s<SStore::F32>(w, bd, st); break;
  }
}

// the format-dependent element kernels of the host loop
void batch_init(BatchWork* w, const BatchDesc& bd, int prec, int grid, cudaStream_t st) {
  const size_t sh = sizeof(double) * (bd.tile + bd.ncols);
  switch (spinor_store_of(prec)) {
    case SStore::F16:
      batch_init_kernel<SStore::F16><<<grid, bd.tile, sh, st>>>(bd, w->phi64.ref(), w->x64.ref(), w->xlo.ref(),
                                                                w->rlo.ref(), w->plo.ref(), w->st, w->br);
      break;
    case SStore::I16:
      batch_init_kernel<SStore::I16><<<grid, bd.tile, sh, st>>>(bd, w->phi64.ref(), w->x64.ref(), w->xlo.ref(),
                                                                w->rlo.ref(), w->plo.ref(), w->st, w->br);
      break;
    default:
      batch_init_kernel<SStore::F32><<<grid, bd.tile, sh, st>>>(bd, w->phi64.ref(), w->x64.ref(), w->xlo.ref(),
                                                                w->rlo.ref(), w->plo.ref(), w->st, w->br);
      break;
  }
}
void batch_reliable_tail(BatchWork* w, const BatchDesc& bd, const BatchDesc& bd64, int prec, int grid,
                         cudaStream_t st) {
  switch (spinor_store_of(prec)) {
    case SStore::F16:
      batch_accumulate_kernel<SStore::F16><<<grid, bd.tile, 0, st>>>(bd.total, w->xlo.ref(), w->x64.ref());
      batch_true_residual(w, bd64, prec, st);
      batch_xpay_kernel<SStore::F16><<<grid, bd.tile, 0, st>>>(bd, w->rlo.ref(), w->plo.ref(), w->st, 1);
      break;
    case SStore::I16:
      batch_accumulate_kernel<SStore::I16><<<grid, bd.tile, 0, st>>>(bd.total, w->xlo.ref(), w->x64.ref());
      batch_true_residual(w, bd64, prec, st);
      batch_xpay_kernel<SStore::I16><<<grid, bd.tile, 0, st>>>(bd, w->rlo.ref(), w->plo.ref(), w->st, 1);
      break;
    default:
      batch_accumulate_kernel<SStore::F32><<<grid, bd.tile, 0, st>>>(bd.total, w->xlo.ref(), w->x64.ref());
      batch_true_residual(w, bd64, prec, st);
      batch_xpay_kernel<SStore::F32><<<grid, bd.tile, 0, st>>>(bd, w->rlo.ref(), w->plo.ref(), w->st, 1);
      break;
  }
}

}  // namespace

void destroy_batch_work(void* w) { free_batch(static_cast<BatchWork*>(w)); }

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_solve_batch(lq_ctx** ctxs, int n, double** x, const double** phi, const double* kappa,
                                    int nrhs, double tol, int maxiter, int inner_prec, int reliable_every,
                                    double* hist, int hist_len, int* iters, double* resid, lq_solve_stats* stats) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!ctxs || n <= 0 || n > kMaxSys || !ctxs[0]) return LQ_ERR_ARG;
  lq_ctx* c = ctxs[0];
  auto fail = [&](lq_status s, const std::string& m) { c->last_error = "lq_solve_batch: " + m; return s; };
  if (!x || !phi || !kappa) return fail(LQ_ERR_ARG, "null argument");
  if (nrhs <= 0 || nrhs > 16 || n * nrhs > kMaxCols) return fail(LQ_ERR_ARG, "need 1 <= nrhs <= 16, n * nrhs <= 64");
  if (!(tol > 0.0) || maxiter <= 0 || reliable_every <= 0) return fail(LQ_ERR_ARG, "bad tol, maxiter or reliable_every");
  if (inner_prec != LQ_F32 && inner_prec != LQ_F32_12 && inner_prec != LQ_F16_12 && inner_prec != LQ_I16_12)
    return fail(LQ_ERR_ARG, "inner precision must be LQ_F32, LQ_F32_12, LQ_F16_12 or LQ_I16_12");
  for (int k = 0; k < n; ++k) {
    if (!ctxs[k] || !ctxs[k]->gauge_set) return fail(LQ_ERR_STATE, "every context needs a gauge field");
    if (ctxs[k]->device != c->device) return fail(LQ_ERR_ARG, "all contexts must be on one device");
    cudaPointerAttributes a{};
    for (const void* p : {(const void*)x[k], (const void*)phi[k]}) {
      if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess ||
          (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(LQ_ERR_ARG, "x and phi must be device buffers");
      }
    }
  }
  cudaStream_t st = c->stream;
  // every system's links in the inner format, converted on the caller's stream
  for (int k = 0; k < n; ++k) {
    lq_ctx* ck = ctxs[k];
    if (!ck->gauge_lo[inner_prec]) {
      if (cudaMalloc(&ck->gauge_lo[inner_prec], gauge_bytes(gauge_store_of(inner_prec), ck->geo.V)) != cudaSuccess)
        return fail(LQ_ERR_CUDA, "cudaMalloc");
    }
    if (!ck->gauge_lo_valid[inner_prec]) {
      launch_convert_gauge(ck->geo, ck->gauge64, gauge_store_of(inner_prec), ck->gauge_lo[inner_prec], st);
      ck->gauge_lo_valid[inner_prec] = true;
    }
  }
  // workspace owned by the first context, rebuilt when the batch changes shape
  std::vector<int> key{n, nrhs, inner_prec};
  for (int k = 0; k < n; ++k)
    for (int m = 0; m < 4; ++m) key.push_back(ctxs[k]->geo.L[m]);
  for (int k = 0; k < n; ++k) key.push_back(ctxs[k]->geo.antiperiodic);
  BatchWork* w = static_cast<BatchWork*>(c->batch);
  if (!w || w->key != key) {
    free_batch(w);
    w = new BatchWork();
    c->batch = w;
    w->key = key;
    BatchDesc probe = make_desc(ctxs, n, nrhs, nullptr, nullptr, kappa, inner_prec, nrhs);
    w->total = probe.total;
    w->ncols = probe.ncols;
    bool ok = true;
    auto alloc = [&](Field& f, SStore s) {
      f.store = s;
      ok = ok && cudaMalloc(&f.data, spinor_bytes(s, w->total)) == cudaSuccess;
      if (s == SStore::F16 || s == SStore::I16) ok = ok && cudaMalloc(&f.norm, sizeof(float) * w->total) == cudaSuccess;
    };
    const SStore slo = spinor_store_of(inner_prec);
    alloc(w->phi64, SStore::F64); alloc(w->x64, SStore::F64); alloc(w->r64, SStore::F64); alloc(w->tmp64, SStore::F64);
    alloc(w->plo, slo); alloc(w->tlo, slo); alloc(w->rlo, slo); alloc(w->xlo, xlo_store(slo));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    w->grid_cap = std::max(1, sms) * 4;
    w->br.max_blocks = w->grid_cap;
    ok = ok && cudaMalloc(&w->br.partials, sizeof(double) * kMaxCols * w->br.max_blocks) == cudaSuccess;
    ok = ok && cudaMalloc(&w->br.ticket, sizeof(unsigned int)) == cudaSuccess;
    ok = ok && cudaMemset(w->br.ticket, 0, sizeof(unsigned int)) == cudaSuccess;
    ok = ok && cudaMalloc(&w->st, sizeof(BatchState)) == cudaSuccess;
    ok = ok && cudaMallocHost(&w->st_host, sizeof(BatchState)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      free_batch(w);
      c->batch = nullptr;
      return fail(LQ_ERR_CUDA, "workspace allocation failed");
    }
  }
  if (hist && hist_len > 0 && w->hist_cap < hist_len * w->ncols) {
    if (w->hist) cudaFree(w->hist);
    w->hist = nullptr;
    w->hist_cap = 0;
    if (cudaMalloc(&w->hist, sizeof(double) * hist_len * w->ncols) != cudaSuccess) return fail(LQ_ERR_CUDA, "cudaMalloc");
    w->hist_cap = hist_len * w->ncols;
  }
  // state
  BatchState h{};
  h.stop2 = tol * tol;
  h.delta2 = inner_prec == LQ_F32 || inner_prec == LQ_F32_12 ? 1e-6 : 1e-4;
  h.ru_every = reliable_every;
  h.maxiter = maxiter;
  h.hist = (hist && hist_len > 0) ? w->hist : nullptr;
  h.hist_len = (hist && hist_len > 0) ? hist_len : 0;
  *w->st_host = h;
  cudaMemcpyAsync(w->st, w->st_host, sizeof(BatchState), cudaMemcpyHostToDevice, st);
  lq_solve_stats s{};

  // autotune the tile (threads per block) once per workspace: multiples of
  // nrhs near 128 and 256 threads, timed over three iterations each
  const int base = nrhs;
  if (w->tile == 0) {
    std::vector<int> cand;
    for (int target : {128, 256}) {
      const int t = std::max(base, target / base * base);
      if (t <= 256 && std::find(cand.begin(), cand.end(), t) == cand.end()) cand.push_back(t);
    }
    BatchDesc bd0 = make_desc(ctxs, n, nrhs, phi, x, kappa, inner_prec, cand[0]);
    batch_init(w, bd0, inner_prec, std::min(bd0.ntiles, w->grid_cap), st);
    float best = 1e30f;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int t : cand) {
      BatchDesc bd = make_desc(ctxs, n, nrhs, phi, x, kappa, inner_prec, t);
      batch_iteration_prec(w, bd, inner_prec, st);   // warm-up
      cudaEventRecord(a, st);
      for (int i = 0; i < 3; ++i) batch_iteration_prec(w, bd, inner_prec, st);
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      s.kernel_launches += 12;
      if (ms < best) { best = ms; w->tile = t; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *w->st_host = h;
    cudaMemcpyAsync(w->st, w->st_host, sizeof(BatchState), cudaMemcpyHostToDevice, st);
  }
  const BatchDesc bd = make_desc(ctxs, n, nrhs, phi, x, kappa, inner_prec, w->tile);
  // FP64 passes (~250 registers per thread) use tiles of about 128 threads
  const BatchDesc bd64 = make_desc(ctxs, n, nrhs, phi, x, kappa, inner_prec, std::max(nrhs, 128 / nrhs * nrhs));
  const int grid = std::min(bd.ntiles, w->grid_cap);
  batch_init(w, bd, inner_prec, grid, st);
  s.kernel_launches += 1;

  // iterations as CUDA graphs of reliable_every iterations
  const int chunk = reliable_every;
  lq_status result = LQ_OK;
  cudaError_t err = cudaSuccess;
  for (long guard = 0; guard < (long)maxiter + 64; ++guard) {
    cudaGraphExec_t exec = nullptr;
    for (auto& gr : w->graphs)
      if (same_iteration_desc(gr.first, bd)) exec = gr.second;
    if (!exec) {
      cudaGraph_t g = nullptr;
      err = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
      if (err != cudaSuccess) break;
      for (int i = 0; i < chunk; ++i) batch_iteration_prec(w, bd, inner_prec, c->capture_stream);
      err = cudaStreamEndCapture(c->capture_stream, &g);
      if (err != cudaSuccess) break;
      err = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (err != cudaSuccess) break;
      // graphs bake in the kernel arguments (kappa, links, geometry): keep a
      // few, keyed by the descriptor they were recorded for
      if (w->graphs.size() >= 8) {
        cudaGraphExecDestroy(w->graphs.front().second);
        w->graphs.erase(w->graphs.begin());
      }
      w->graphs.emplace_back(bd, exec);
    }
    err = cudaGraphLaunch(exec, st);
    if (err != cudaSuccess) break;
    s.kernel_launches += 3 * chunk;
    // reliable update: fold x, FP64 true residual per column, freeze converged columns
    batch_reliable_tail(w, bd, bd64, inner_prec, grid, st);
    s.kernel_launches += 4;
    s.reliable_updates++;
    err = cudaMemcpyAsync(w->st_host, w->st, sizeof(BatchState), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) break;
    const BatchState& hs = *w->st_host;
    if (hs.breakdown) { result = fail(LQ_ERR_NAN, "non-finite value or CG breakdown"); break; }
    bool all = true;
    for (int col = 0; col < bd.ncols; ++col) all = all && hs.done[col];
    if (all) { s.converged = 1; break; }
    if (hs.iter >= maxiter) { result = fail(LQ_ERR_NOT_CONVERGED, "iteration limit reached"); break; }
  }
  if (err != cudaSuccess) {
    cudaGetLastError();
    return fail(LQ_ERR_CUDA, cudaGetErrorString(err));
  }
  batch_unpack_kernel<<<grid, bd.tile, 0, st>>>(bd, w->x64.ref());
  s.kernel_launches += 1;
  const BatchState& hs = *w->st_host;
  s.iterations = hs.iter;
  double worst = 0.0;
  for (int col = 0; col < bd.ncols; ++col) {
    const double rel = hs.phi2[col] > 0 ? std::sqrt(hs.rr_true[col] / hs.phi2[col]) : 0.0;
    worst = std::max(worst, rel);
    if (resid) resid[col] = rel;
    if (iters) iters[col] = hs.done[col] ? hs.conv_iter[col] : hs.iter;
  }
  s.true_rel_resid = worst;
  if (hist && hist_len > 0) {
    const int nh = std::min(hs.iter, hist_len);
    for (int col = 0; col < bd.ncols; ++col)
      cudaMemcpyAsync(hist + (size_t)col * hist_len, w->hist + (size_t)col * hist_len, sizeof(double) * nh,
                      cudaMemcpyDeviceToHost, st);
  }
  err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) return fail(LQ_ERR_CUDA, cudaGetErrorString(err));
  s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = s;
  return result;
}
