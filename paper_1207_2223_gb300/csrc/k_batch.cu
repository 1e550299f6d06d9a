// Batched CG on M^dag M: many right-hand sides sharing one gauge field, and
// independent lattices of different volumes and kappa, solved together with
// one launch per CG pass (the paper's CG routine, Sec. 3, over a batch of
// systems).
//
// Layout.  All systems share one set of fields of `total` elements; column r
// (right-hand side r) of system k owns elements off_k + r V_k .. off_k +
// (r + 1) V_k - 1, so consecutive threads read consecutive sites of one
// column and every load is coalesced.  Every field is [chunk][element] as in
// lq_device.cuh.  The caller's [nrhs][V][4][3] buffers map onto it directly.
//
// Work items.  A thread applies the stencil at one site to RB right-hand
// sides of its system at once (register blocking): each link is loaded and
// decoded (and, for 12-real storage, rebuilt) once and multiplied into RB
// half spinors.  Blocks walk a list of tiles of TILE sites of one rhs group
// of one system; inside a system the tiles run either site-major (the
// groups of one site tile are consecutive tiles, so one wave of blocks
// covers every right-hand side of a slab of sites and the links of the slab
// are re-read from L2 while they are still there) or group-major (every site
// tile of one group, then the next group).  A tile never spans two groups or
// systems, so the columns a thread reduces into are the same for the whole
// tile.  Per-column sums stay in registers while a block remains in one
// group, are reduced in the block when it changes (fixed order) and per block
// are added by the last block in block order: deterministic.
//
// Tuning.  The first call on a workspace times a few iterations for every
// candidate (tile order x threads per block x right-hand sides per thread x
// resident blocks per SM, i.e. how many sites each thread walks) and keeps
// the fastest.
//
// Mixed precision.  The iterations run in FP32 arithmetic on the storage of
// the inner precision; every `reliable_every` iterations (sooner for a column
// whose iterated residual fell far) x is folded into the high-precision
// solution and the true residual of every column is recomputed; a column
// whose true residual meets the tolerance is frozen (alpha = 0 from then on).
// The intermediate updates run in double-float arithmetic (k_batch_df.cu)
// unless the context asks for FP64 throughout; once every column is frozen,
// or every open column's iterated residual has met the tolerance, x is
// certified with the FP64 operator, which reopens any column that fails.
#include <algorithm>
#include <climits>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "lq_batch.cuh"

namespace lq {

// p = r + beta_col p (inner format), skipped when halted unless forced.  use_cond: the
// last kernel of an iteration inside the device-side loop; before anything else one thread
// sets the loop's condition (another iteration unless this one raised halt, counted against
// the iteration limit so that the loop ends even if the state never halts).
template <SStore S>
__global__ void batch_xpay_kernel(BatchDesc bd, SpinorRef r, SpinorRef p, BatchState* st, int forced,
                                  cudaGraphConditionalHandle cond, int use_cond) {
  const int halted = *(volatile const int*)&st->halt;
  if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) {
    const int g = ++st->guard_inner;
    st->loops[0]++;
    cudaGraphSetConditional(cond, (!halted && g <= st->maxiter) ? 1u : 0u);
  }
  if (!forced && halted) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < bd.total; e += gridDim.x * blockDim.x) {
    const SysDesc& sd = bd.sys[system_of_element(bd, e)];
    const float beta = (float)st->beta[sd.col + (e - sd.off) / sd.geo.V];
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

void launch_batch_xpay(const BatchDesc& bd, SStore s, SpinorRef r, SpinorRef p, BatchState* st, int forced,
                       int grid, cudaStream_t stream, cudaGraphConditionalHandle cond, int use_cond) {
  switch (s) {
    case SStore::F16:
      batch_xpay_kernel<SStore::F16><<<grid, 256, 0, stream>>>(bd, r, p, st, forced, cond, use_cond);
      break;
    case SStore::BF16:
      batch_xpay_kernel<SStore::BF16><<<grid, 256, 0, stream>>>(bd, r, p, st, forced, cond, use_cond);
      break;
    case SStore::I16:
      batch_xpay_kernel<SStore::I16><<<grid, 256, 0, stream>>>(bd, r, p, st, forced, cond, use_cond);
      break;
    default: batch_xpay_kernel<SStore::F32><<<grid, 256, 0, stream>>>(bd, r, p, st, forced, cond, use_cond); break;
  }
}

// Start: phi (canonical, per system) -> phi64; x64 = 0; x_lo = 0; r_lo = p_lo = phi; phi2 per column.
template <SStore S, int RB>
__global__ void batch_init_kernel(BatchDesc bd, SpinorRef phi64, SpinorRef x64, SpinorRef xlo, SpinorRef rlo,
                                  SpinorRef plo, BatchState* st, BatchReduce br) {
  __shared__ double sh_col[kMaxCols];
  __shared__ double sh_red[RB * 32];
  for (int c = threadIdx.x; c < bd.ncols; c += blockDim.x) sh_col[c] = 0.0;
  __syncthreads();
  int cur = -1;
  double red[RB];
#pragma unroll
  for (int j = 0; j < RB; ++j) red[j] = 0.0;
  for (int t = blockIdx.x; t < bd.ntiles; t += gridDim.x) {
    const TileWork w = tile_work(bd, t);
    const SysDesc& sd = bd.sys[w.k];
    const int col0 = sd.col + w.r0;
    if (col0 != cur) {
      if (cur >= 0) flush_columns<RB>(red, cur, sh_red, sh_col);
      cur = col0;
#pragma unroll
      for (int j = 0; j < RB; ++j) red[j] = 0.0;
    }
    if (w.s >= sd.geo.V) continue;
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      const int el = (w.r0 + j) * sd.geo.V + w.s;            // element within the system
      const double2* src = reinterpret_cast<const double2*>(sd.phi_in) + (size_t)el * 12;
      cplx<double> a[12], z[12];
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        const double2 x = src[q];
        a[q] = {x.x, x.y};
        z[q] = {0.0, 0.0};
        v += x.x * x.x + x.y * x.y;
      }
      const int e = sd.off + el;
      store_spinor<SStore::F64, double>(phi64, bd.total, e, a);
      store_spinor<SStore::F64, double>(x64, bd.total, e, z);
      store_spinor<xlo_store(S), double>(xlo, bd.total, e, z);
      store_spinor<S, double>(rlo, bd.total, e, a);
      store_spinor<S, double>(plo, bd.total, e, a);
      red[j] += v;
    }
  }
  if (cur >= 0) flush_columns<RB>(red, cur, sh_red, sh_col);
  auto fin = [&](const double* tot) {       // every thread of the last block: one column each
    for (int c = threadIdx.x; c < bd.ncols; c += blockDim.x) {
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

// x64 -> canonical per system (element off + r V + s is canonical entry r V + s of x_out)
__global__ void batch_unpack_kernel(BatchDesc bd, SpinorRef x64) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < bd.total; e += gridDim.x * blockDim.x) {
    const SysDesc& sd = bd.sys[system_of_element(bd, e)];
    cplx<double> a[12];
    load_spinor<SStore::F64, double>(x64, bd.total, e, a);
    double2* dst = reinterpret_cast<double2*>(sd.x_out) + (size_t)(e - sd.off) * 12;
#pragma unroll
    for (int q = 0; q < 12; ++q) dst[q] = make_double2(a[q].re, a[q].im);
  }
}

// ------------------------------------------------------------ host side
namespace {

enum { kFormChunk = 0, kFormLoop64 = 1, kFormLoopDF = 2 };

// Launch shape of the inner-format passes, picked by timing.
struct Tuning {
  int tile = 0;                   // threads per block (= sites per tile)
  int rb = 1;                     // right-hand sides per thread
  int per_sm = 0;                 // resident blocks per SM used (0: all that fit)
  int site_major = 1;             // tile order
};

struct BatchWork {
  std::vector<int> key;           // signature: per system dims, R, antiperiodic, precision
  int total = 0, ncols = 0, sms = 0, max_blocks = 0;
  Field phi64, x64, r64, tmp64, plo, tlo, rlo, xlo;
  Field phidf, xdf, tmpdf;        // double-float updates: phi, the solution, M x
  BatchState* st = nullptr;
  BatchState* st_host = nullptr;
  BatchReduce br{};
  double* hist = nullptr;
  int hist_cap = 0;
  Tuning tune;
  std::vector<double> tune_ms;    // timing of every candidate (for the caller's report)
  double* part = nullptr;         // persistent iteration: [2][kMaxCols][max_blocks] column sums
  unsigned int* bar = nullptr;    // persistent iteration: barrier arrivals, generation
  // recorded graphs with the descriptor and form they were recorded for
  struct Recorded {
    BatchDesc bd;
    int form;                     // kFormChunk, kFormLoop64, kFormLoopDF
    int chunk;                    // iterations of a chunk graph; operator variant of a loop graph
    cudaGraphExec_t exec;
  };
  std::vector<Recorded> graphs;
  cudaStream_t body_stream[2] = {nullptr, nullptr};   // record the bodies of conditional nodes
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

cudaGraphExec_t find_graph(const BatchWork* w, const BatchDesc& bd, int form, int chunk) {
  for (const auto& g : w->graphs)
    if (g.form == form && g.chunk == chunk && same_iteration_desc(g.bd, bd)) return g.exec;
  return nullptr;
}

// graphs bake in the kernel arguments (kappa, links, geometry): keep a few, keyed by
// the descriptor and form they were recorded for
void keep_graph(BatchWork* w, const BatchDesc& bd, int form, int chunk, cudaGraphExec_t exec) {
  if (w->graphs.size() >= 8) {
    cudaGraphExecDestroy(w->graphs.front().exec);
    w->graphs.erase(w->graphs.begin());
  }
  w->graphs.push_back({bd, form, chunk, exec});
}

void free_batch(BatchWork* w) {
  if (!w) return;
  for (auto& g : w->graphs) cudaGraphExecDestroy(g.exec);
  for (cudaStream_t s : w->body_stream)
    if (s) cudaStreamDestroy(s);
  for (Field* f : {&w->phi64, &w->x64, &w->r64, &w->tmp64, &w->plo, &w->tlo, &w->rlo, &w->xlo, &w->phidf, &w->xdf,
                   &w->tmpdf}) {
    if (f->data) cudaFree(f->data);
    if (f->norm) cudaFree(f->norm);
  }
  if (w->st) cudaFree(w->st);
  if (w->st_host) cudaFreeHost(w->st_host);
  if (w->br.partials) cudaFree(w->br.partials);
  if (w->br.ticket) cudaFree(w->br.ticket);
  if (w->hist) cudaFree(w->hist);
  if (w->part) cudaFree(w->part);
  if (w->bar) cudaFree(w->bar);
  delete w;
}

BatchDesc make_desc(lq_ctx** ctxs, int n, int R, const double* const* phi, double* const* x, const double* kappa,
                    int prec, int tile, int rb, int site_major) {
  BatchDesc bd{};
  bd.nsys = n;
  bd.tile = tile;
  bd.rb = rb;
  bd.site_major = site_major;
  int off = 0, col = 0, t0 = 0;
  for (int k = 0; k < n; ++k) {
    SysDesc& sd = bd.sys[k];
    sd.geo = ctxs[k]->geo;
    sd.gauge_lo = ctxs[k]->gauge_lo[prec];
    sd.gauge64 = ctxs[k]->gauge64;
    sd.gauge_df = ctxs[k]->gauge_lo[LQ_DF64];
    sd.kappa = kappa[k];
    sd.R = R;
    sd.off = off;
    sd.col = col;
    sd.tile0 = t0;
    sd.tpg = (sd.geo.V + tile - 1) / tile;
    sd.phi_in = phi ? phi[k] : nullptr;
    sd.x_out = x ? x[k] : nullptr;
    off += sd.geo.V * R;
    col += R;
    t0 += sd.tpg * (R / rb);
  }
  bd.total = off;
  bd.ncols = col;
  bd.ntiles = t0;
  return bd;
}

int flat_grid(const BatchWork* w) { return std::max(1, w->sms) * 8; }

BatchIterArgs iter_args(const BatchWork* w, const Tuning& tu) {
  return BatchIterArgs{w->plo.ref(), w->tlo.ref(), w->rlo.ref(), w->xlo.ref(), w->st, w->br, w->sms, tu.per_sm};
}

// use_cond: inside the device-side loop, whose condition the iteration's last kernel sets
void batch_iteration_prec(BatchWork* w, const BatchDesc& bd, int prec, const Tuning& tu, cudaStream_t st,
                          cudaGraphConditionalHandle cond = 0, int use_cond = 0) {
  BatchIterArgs a = iter_args(w, tu);
  a.cond = cond;
  a.use_cond = use_cond;
  switch (prec) {
    case LQ_F16_12: batch_iteration_h16(a, bd, prec, st); break;
    case LQ_BF16_12: batch_iteration_bf16(a, bd, prec, st); break;
    case LQ_I16_12: batch_iteration_i16(a, bd, prec, st); break;
    case LQ_F32_12: batch_iteration_f32_12(a, bd, prec, st); break;
    default: batch_iteration_f32(a, bd, prec, st); break;
  }
}

template <SStore S>
void batch_true_residual_s(BatchWork* w, const BatchDesc& bd64, cudaStream_t st) {
  BEpiStore64 e0{w->tmp64.ref(), bd64.total};
  launch_batch<double, GStore::F64_18, SStore::F64, false>(bd64, w->x64.ref(), e0, w->br, 1, w->sms, 0, st);
  BEpiResidual<S> e1{w->phi64.ref(), w->r64.ref(), w->rlo.ref(), bd64.total, w->st};
  launch_batch<double, GStore::F64_18, SStore::F64, true>(bd64, w->tmp64.ref(), e1, w->br, 1, w->sms, 0, st);
}

// the format-dependent element kernels of the host loop
template <SStore S>
void batch_init_s(BatchWork* w, const BatchDesc& bd, cudaStream_t st) {
  const int grid = std::max(1, std::min(bd.ntiles, w->br.max_blocks));
  auto args = [&](auto kern) {
    kern<<<grid, bd.tile, 0, st>>>(bd, w->phi64.ref(), w->x64.ref(), w->xlo.ref(), w->rlo.ref(), w->plo.ref(), w->st,
                                   w->br);
  };
  switch (bd.rb) {
    case 2: args(&batch_init_kernel<S, 2>); break;
    case 3: args(&batch_init_kernel<S, 3>); break;
    case 4: args(&batch_init_kernel<S, 4>); break;
    default: args(&batch_init_kernel<S, 1>); break;
  }
}
void batch_init(BatchWork* w, const BatchDesc& bd, int prec, cudaStream_t st) {
  switch (spinor_store_of(prec)) {
    case SStore::F16: batch_init_s<SStore::F16>(w, bd, st); break;
    case SStore::BF16: batch_init_s<SStore::BF16>(w, bd, st); break;
    case SStore::I16: batch_init_s<SStore::I16>(w, bd, st); break;
    default: batch_init_s<SStore::F32>(w, bd, st); break;
  }
}

// FP64 reliable update.  fold: x64 += x_lo first (otherwise x64 was just converted from
// the double-float solution).
template <SStore S>
void batch_reliable_tail_s(BatchWork* w, const BatchDesc& bd, const BatchDesc& bd64, bool fold, cudaStream_t st) {
  if (fold) batch_accumulate_kernel<S><<<flat_grid(w), 256, 0, st>>>(bd.total, w->xlo.ref(), w->x64.ref());
  batch_true_residual_s<S>(w, bd64, st);
  batch_xpay_kernel<S><<<flat_grid(w), 256, 0, st>>>(bd, w->rlo.ref(), w->plo.ref(), w->st, 1, 0, 0);
}
void batch_reliable_tail(BatchWork* w, const BatchDesc& bd, const BatchDesc& bd64, int prec, bool fold,
                         cudaStream_t st) {
  switch (spinor_store_of(prec)) {
    case SStore::F16: batch_reliable_tail_s<SStore::F16>(w, bd, bd64, fold, st); break;
    case SStore::BF16: batch_reliable_tail_s<SStore::BF16>(w, bd, bd64, fold, st); break;
    case SStore::I16: batch_reliable_tail_s<SStore::I16>(w, bd, bd64, fold, st); break;
    default: batch_reliable_tail_s<SStore::F32>(w, bd, bd64, fold, st); break;
  }
}
void batch_xpay_forced(BatchWork* w, const BatchDesc& bd, int prec, cudaStream_t st) {
  launch_batch_xpay(bd, spinor_store_of(prec), w->rlo.ref(), w->plo.ref(), w->st, 1, flat_grid(w), st);
}
Geom flat_geom(int total) {
  Geom g{};
  g.V = total;
  return g;
}

// ------------------------------------------------------------ device-side solve loop
// The whole solve as one CUDA graph: a while node over update cycles whose body holds a
// while node over CG iterations (until a reliable update is due), then the update, with if
// nodes around the double-float residual and the FP64 certification.  One-thread kernels
// read the state, take each decision and set the node's condition (the iteration loop's
// condition is set by the first thread of each iteration's last kernel, batch_xpay_kernel);
// every loop counts its bodies against a cap taken from the iteration limit, so the graph
// ends even if the state never halts.

// entering the iteration loop: run it unless a reliable update is already due
__global__ void cond_enter_kernel(BatchState* st, cudaGraphConditionalHandle inner) {
  st->guard_inner = 0;
  cudaGraphSetConditional(inner, st->halt ? 0u : 1u);
}
// the double-float residual unless every open column's iterated residual met the
// tolerance (that update goes straight to the FP64 certification)
__global__ void cond_df_kernel(BatchState* st, int ncols, cudaGraphConditionalHandle df) {
  int last = 1;
  for (int c = 0; c < ncols; ++c)
    if (!st->done[c] && !(st->rr[c] <= st->stop2 * st->phi2[c])) last = 0;
  st->df_last = last;
  if (!last) st->loops[2]++;
  cudaGraphSetConditional(df, last ? 0u : 1u);
}
// the FP64 certification once every column is frozen (or the double-float step was skipped)
__global__ void cond_cert_kernel(BatchState* st, int ncols, cudaGraphConditionalHandle cert) {
  int all = 1;
  for (int c = 0; c < ncols; ++c) all &= st->done[c] ? 1 : 0;
  const int go = st->df_last || (all && !st->breakdown);
  if (go) st->loops[3]++;
  cudaGraphSetConditional(cert, go ? 1u : 0u);
}
// another update cycle unless every column is frozen (certified), the iteration limit is
// reached or a breakdown was seen
__global__ void cond_continue_kernel(BatchState* st, int ncols, cudaGraphConditionalHandle outer) {
  int all = 1;
  for (int c = 0; c < ncols; ++c) all &= st->done[c] ? 1 : 0;
  const int g = ++st->guard_outer;
  st->loops[1]++;
  cudaGraphSetConditional(outer, (!all && !st->breakdown && st->iter < st->maxiter && g <= st->maxiter + 64) ? 1u
                                                                                                          : 0u);
}

// A condition handle on the graph being captured on `s`.
cudaError_t new_handle(cudaStream_t s, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  cudaError_t err = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr);
  if (err != cudaSuccess) return err;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  return cudaGraphConditionalHandleCreate(h, g, 0, 0);
}

// A conditional node on handle h at the current point of the capture on `s` (work captured
// on `s` afterwards follows it); returns its body graph.
cudaError_t add_conditional(cudaStream_t s, cudaGraphConditionalNodeType type, cudaGraphConditionalHandle h,
                            cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t err = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (err != cudaSuccess) return err;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  std::vector<cudaGraphNode_t> dv(deps, deps + nd);
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  err = cudaGraphAddNode(&node, g, dv.empty() ? nullptr : dv.data(), nullptr, dv.size(), &p);
  if (err != cudaSuccess) return err;
  *body = p.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Records `launches(stream)` into `body` on the stream.
template <class F>
cudaError_t record_body(cudaStream_t s, cudaGraph_t body, F&& launches) {
  cudaError_t err = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (err != cudaSuccess) return err;
  const cudaError_t e0 = launches(s);
  const cudaError_t e1 = cudaGetLastError();
  cudaGraph_t out = nullptr;
  err = cudaStreamEndCapture(s, &out);
  return err != cudaSuccess ? err : (e0 != cudaSuccess ? e0 : e1);
}

// dfa null: every reliable update in FP64
cudaError_t build_solve_graph(BatchWork* w, const BatchDesc& bd, const BatchDesc& bd64, int prec, const Tuning& tu,
                              const BatchDfArgs* dfa, cudaGraphExec_t* exec) {
  for (cudaStream_t& s : w->body_stream)
    if (!s) {
      const cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
    }
  cudaStream_t s1 = w->body_stream[0], s2 = w->body_stream[1];
  cudaGraph_t g = nullptr;
  cudaError_t err = cudaGraphCreate(&g, 0);
  if (err != cudaSuccess) return err;
  // top level: while (another update cycle), condition 1 at every launch
  cudaGraphConditionalHandle h_outer;
  err = cudaGraphConditionalHandleCreate(&h_outer, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h_outer;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t outer = nullptr;
  if (err == cudaSuccess) err = cudaGraphAddNode(&outer, g, nullptr, nullptr, 0, &p);
  const int ncols = bd.ncols;
  const SStore slo = spinor_store_of(prec);
  BatchState* st = w->st;
  if (err == cudaSuccess) {
    err = record_body(s1, p.conditional.phGraph_out[0], [&](cudaStream_t s) -> cudaError_t {
      // CG iterations until a reliable update is due
      cudaGraphConditionalHandle h_inner;
      cudaGraph_t body = nullptr;
      cudaError_t e = new_handle(s, &h_inner);
      if (e != cudaSuccess) return e;
      cond_enter_kernel<<<1, 1, 0, s>>>(st, h_inner);
      e = add_conditional(s, cudaGraphCondTypeWhile, h_inner, &body);
      if (e != cudaSuccess) return e;
      e = record_body(s2, body, [&](cudaStream_t q) -> cudaError_t {
        batch_iteration_prec(w, bd, prec, tu, q, h_inner, 1);   // its last kernel sets h_inner
        return cudaSuccess;
      });
      if (e != cudaSuccess) return e;
      if (!dfa) {
        batch_reliable_tail(w, bd, bd64, prec, true, s);
      } else {
        cudaGraphConditionalHandle h_df, h_cert;
        e = new_handle(s, &h_df);
        if (e == cudaSuccess) e = new_handle(s, &h_cert);
        if (e != cudaSuccess) return e;
        cond_df_kernel<<<1, 1, 0, s>>>(st, ncols, h_df);
        BatchDfArgs acc = *dfa;
        acc.accumulate = true;
        acc.residual = false;
        batch_df_tail(acc, bd, slo, s);
        // the double-float residual of every column
        e = add_conditional(s, cudaGraphCondTypeIf, h_df, &body);
        if (e != cudaSuccess) return e;
        e = record_body(s2, body, [&](cudaStream_t q) -> cudaError_t {
          BatchDfArgs res = *dfa;
          res.accumulate = false;
          res.residual = true;
          batch_df_tail(res, bd, slo, q);
          batch_xpay_forced(w, bd, prec, q);
          return cudaSuccess;
        });
        if (e != cudaSuccess) return e;
        // the FP64 certification
        cond_cert_kernel<<<1, 1, 0, s>>>(st, ncols, h_cert);
        e = add_conditional(s, cudaGraphCondTypeIf, h_cert, &body);
        if (e != cudaSuccess) return e;
        e = record_body(s2, body, [&](cudaStream_t q) -> cudaError_t {
          launch_convert_spinor(flat_geom(bd.total), SStore::DF64, w->xdf.ref(), SStore::F64, w->x64.ref(), q);
          batch_reliable_tail(w, bd, bd64, prec, false, q);
          return cudaSuccess;
        });
        if (e != cudaSuccess) return e;
      }
      cond_continue_kernel<<<1, 1, 0, s>>>(st, ncols, h_outer);
      return cudaSuccess;
    });
  }
  if (err == cudaSuccess) err = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  return err;
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
  if (inner_prec != LQ_F32 && inner_prec != LQ_F32_12 && inner_prec != LQ_F16_12 && inner_prec != LQ_BF16_12 &&
      inner_prec != LQ_I16_12)
    return fail(LQ_ERR_ARG, "inner precision must be LQ_F32, LQ_F32_12, LQ_F16_12, LQ_BF16_12 or LQ_I16_12");
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
  {
    // element indices of the batch fields are 32-bit (with room for a grid stride)
    long long elements = 0;
    for (int k = 0; k < n; ++k) elements += (long long)ctxs[k]->geo.V * nrhs;
    if (elements > (long long)(INT_MAX / 2)) return fail(LQ_ERR_SHAPE, "batch too large for 32-bit element indices");
  }
  cudaStream_t st = c->stream;
  const bool dfru = c->df_updates != 0;      // double-float intermediate reliable updates
  // every system's links in the inner format (and as double-float pairs), converted on
  // the caller's stream
  for (int k = 0; k < n; ++k) {
    lq_ctx* ck = ctxs[k];
    for (int prec : {inner_prec, dfru ? (int)LQ_DF64 : inner_prec}) {
      if (!ck->gauge_lo[prec]) {
        if (cudaMalloc(&ck->gauge_lo[prec], gauge_bytes(gauge_store_of(prec), ck->geo.V)) != cudaSuccess)
          return fail(LQ_ERR_CUDA, "cudaMalloc");
      }
      if (!ck->gauge_lo_valid[prec]) {
        launch_convert_gauge(ck->geo, ck->gauge64, gauge_store_of(prec), ck->gauge_lo[prec], st);
        ck->gauge_lo_valid[prec] = true;
      }
    }
  }
  // workspace owned by the first context, rebuilt when the batch changes shape
  std::vector<int> key{n, nrhs, inner_prec};
  for (int k = 0; k < n; ++k)
    for (int m = 0; m < 4; ++m) key.push_back(ctxs[k]->geo.L[m]);
  for (int k = 0; k < n; ++k) key.push_back(ctxs[k]->geo.antiperiodic);
  key.push_back(dfru);
  BatchWork* w = static_cast<BatchWork*>(c->batch);
  if (!w || w->key != key) {
    free_batch(w);
    w = new BatchWork();
    c->batch = w;
    w->key = key;
    BatchDesc probe = make_desc(ctxs, n, nrhs, nullptr, nullptr, kappa, inner_prec, 256, 1, 1);
    w->total = probe.total;
    w->ncols = probe.ncols;
    bool ok = true;
    auto alloc = [&](Field& f, SStore s) {
      f.store = s;
      ok = ok && cudaMalloc(&f.data, spinor_bytes(s, w->total)) == cudaSuccess;
      if (s == SStore::F16 || s == SStore::BF16 || s == SStore::I16)
        ok = ok && cudaMalloc(&f.norm, sizeof(float) * w->total) == cudaSuccess;
    };
    const SStore slo = spinor_store_of(inner_prec);
    alloc(w->phi64, SStore::F64); alloc(w->x64, SStore::F64); alloc(w->r64, SStore::F64); alloc(w->tmp64, SStore::F64);
    alloc(w->plo, slo); alloc(w->tlo, slo); alloc(w->rlo, slo); alloc(w->xlo, xlo_store(slo));
    if (dfru) { alloc(w->phidf, SStore::DF64); alloc(w->xdf, SStore::DF64); alloc(w->tmpdf, SStore::DF64); }
    cudaDeviceGetAttribute(&w->sms, cudaDevAttrMultiProcessorCount, c->device);
    w->sms = std::max(1, w->sms);
    w->max_blocks = w->sms * 8;
    w->br.max_blocks = w->max_blocks;
    ok = ok && cudaMalloc(&w->br.partials, sizeof(double) * kMaxCols * w->br.max_blocks) == cudaSuccess;
    ok = ok && cudaMalloc(&w->br.ticket, sizeof(unsigned int)) == cudaSuccess;
    ok = ok && cudaMemset(w->br.ticket, 0, sizeof(unsigned int)) == cudaSuccess;
    ok = ok && cudaMalloc(&w->st, sizeof(BatchState)) == cudaSuccess;
    ok = ok && cudaMallocHost(&w->st_host, sizeof(BatchState)) == cudaSuccess;
    ok = ok && cudaMalloc(&w->part, sizeof(double) * 2 * kMaxCols * w->max_blocks) == cudaSuccess;
    ok = ok && cudaMalloc(&w->bar, sizeof(unsigned int) * 2) == cudaSuccess;
    ok = ok && cudaMemset(w->bar, 0, sizeof(unsigned int) * 2) == cudaSuccess;
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
  h.delta2 = inner_prec == LQ_F32 || inner_prec == LQ_F32_12 ? 1e-6 : (inner_prec == LQ_BF16_12 ? 1e-2 : 1e-4);
  h.ru_every = reliable_every;
  h.maxiter = maxiter;
  h.hist = (hist && hist_len > 0) ? w->hist : nullptr;
  h.hist_len = (hist && hist_len > 0) ? hist_len : 0;
  *w->st_host = h;
  cudaMemcpyAsync(w->st, w->st_host, sizeof(BatchState), cudaMemcpyHostToDevice, st);
  lq_solve_stats s{};

  // the initialisation (|phi|^2 per column) in one fixed launch shape, so that the sums do
  // not depend on the shape the tuner picks
  const BatchDesc bdi = make_desc(ctxs, n, nrhs, phi, x, kappa, inner_prec, 256, 1, 1);
  // autotune once per workspace: tile order {site-major, group-major} x threads per block
  // {128, 256} x right-hand sides per thread {1, 2, 3, 4} (divisors of nrhs) x resident
  // blocks per SM {all that fit, 1}, each timed over three iterations on the real fields
  if (c->batch_rb > 0 && w->tune.tile == 0) {       // fixed by the caller: no timing
    if (nrhs % c->batch_rb != 0) return fail(LQ_ERR_ARG, "right-hand sides per thread must divide nrhs");
    w->tune.tile = 256;
    w->tune.rb = c->batch_rb;
    w->tune.per_sm = 0;
    w->tune.site_major = c->batch_order == 2 ? 0 : 1;
    w->tune_ms.clear();
  }
  if (w->tune.tile == 0) {
    std::vector<Tuning> cand;
    for (int order : {1, 0}) {
      if (c->batch_order != 0 && (c->batch_order == 1) != (order == 1)) continue;   // order fixed
      for (int rb : {1, 2, 3, 4})
        if (nrhs % rb == 0)
          for (int tile : {256, 128})
            for (int per_sm : {0, 1}) {
              if (per_sm == 1 && tile == 128) continue;
              Tuning t;
              t.tile = tile;
              t.rb = rb;
              t.per_sm = per_sm;
              t.site_major = order;
              cand.push_back(t);
            }
    }
    batch_init(w, bdi, inner_prec, st);
    // a state that never halts (no tolerance, no reliable-update trigger, no limit), reset
    // before every candidate, so that every candidate times full iterations
    BatchState ht = h;
    ht.stop2 = 0.0;
    ht.delta2 = 0.0;
    ht.ru_every = 0;
    ht.maxiter = 0x7fffffff;
    ht.hist = nullptr;
    ht.hist_len = 0;
    float best = 1e30f;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    w->tune_ms.clear();
    for (const Tuning& t : cand) {
      BatchDesc bd = make_desc(ctxs, n, nrhs, phi, x, kappa, inner_prec, t.tile, t.rb, t.site_major);
      // keep the per-column scalars the initialisation computed, clear the halt controls
      cudaMemcpyAsync(w->st_host, w->st, sizeof(BatchState), cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      w->st_host->stop2 = ht.stop2;
      w->st_host->delta2 = ht.delta2;
      w->st_host->ru_every = ht.ru_every;
      w->st_host->maxiter = ht.maxiter;
      w->st_host->halt = 0;
      w->st_host->iter = 0;
      w->st_host->iter_since_ru = 0;
      w->st_host->hist = nullptr;
      w->st_host->hist_len = 0;
      cudaMemcpyAsync(w->st, w->st_host, sizeof(BatchState), cudaMemcpyHostToDevice, st);
      batch_iteration_prec(w, bd, inner_prec, t, st);   // warm-up
      cudaEventRecord(a, st);
      for (int i = 0; i < 3; ++i) batch_iteration_prec(w, bd, inner_prec, t, st);
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      s.kernel_launches += 12;
      w->tune_ms.push_back(ms / 3.0);
      if (ms < best) { best = ms; w->tune = t; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *w->st_host = h;
    cudaMemcpyAsync(w->st, w->st_host, sizeof(BatchState), cudaMemcpyHostToDevice, st);
  }
  const Tuning tu = w->tune;
  const BatchDesc bd = make_desc(ctxs, n, nrhs, phi, x, kappa, inner_prec, tu.tile, tu.rb, tu.site_major);
  // FP64 passes (~250 registers per thread): one right-hand side per thread, 128 threads
  const BatchDesc bd64 = make_desc(ctxs, n, nrhs, phi, x, kappa, inner_prec, 128, 1, 1);
  batch_init(w, bdi, inner_prec, st);
  s.kernel_launches += 1;
  BatchDfArgs dfa{};
  if (dfru) {
    launch_convert_spinor(flat_geom(bd.total), SStore::F64, w->phi64.ref(), SStore::DF64, w->phidf.ref(), st);
    launch_zero_spinor(flat_geom(bd.total), SStore::DF64, w->xdf.ref(), st);
    s.kernel_launches += 2;
    dfa.xlo = w->xlo.ref();
    dfa.xdf = w->xdf.ref();
    dfa.tmpdf = w->tmpdf.ref();
    dfa.phidf = w->phidf.ref();
    dfa.rlo = w->rlo.ref();
    dfa.st = w->st;
    dfa.br = w->br;
    for (int k = 0; k < n; ++k) dfa.gauge_df[k] = ctxs[k]->gauge_lo[LQ_DF64];
    dfa.flat_grid = flat_grid(w);
    dfa.prefetch = c->df_prefetch != 0;
  }

  const int chunk = reliable_every;
  lq_status result = LQ_OK;
  cudaError_t err = cudaSuccess;
  const bool host_loop = c->batch_persistent || !c->batch_device_loop;
  if (!host_loop) {
    // the whole solve as one graph with conditional nodes; a launch that its loop caps
    // ended early is repeated (at most a few times)
    // the graph bakes in the double-float operator variant: part of its key
    const int form = dfru ? kFormLoopDF : kFormLoop64;
    const int variant = dfru && dfa.prefetch ? 1 : 0;
    cudaGraphExec_t exec = find_graph(w, bd, form, variant);
    if (!exec) {
      err = build_solve_graph(w, bd, bd64, inner_prec, tu, dfru ? &dfa : nullptr, &exec);
      if (err == cudaSuccess) keep_graph(w, bd, form, variant, exec);
    }
    for (int launch = 0; launch < 4 && err == cudaSuccess; ++launch) {
      err = cudaGraphLaunch(exec, st);
      if (err == cudaSuccess) err = cudaMemcpyAsync(w->st_host, w->st, sizeof(BatchState), cudaMemcpyDeviceToHost, st);
      if (err == cudaSuccess) err = cudaStreamSynchronize(st);
      if (err != cudaSuccess) break;
      const BatchState& hs = *w->st_host;
      if (hs.breakdown) { result = fail(LQ_ERR_NAN, "non-finite value or CG breakdown"); break; }
      bool all = true;
      for (int col = 0; col < bd.ncols; ++col) all = all && hs.done[col];
      if (all) { s.converged = 1; break; }
      if (hs.iter >= maxiter || launch == 3) {
        result = fail(LQ_ERR_NOT_CONVERGED, "iteration limit reached");
        break;
      }
    }
    // launches from the loop counts: an iteration is three passes (the last one sets the
    // loop's condition); an update cycle enters and leaves the loop around its update
    const int* L = w->st_host->loops;
    s.kernel_launches += 3 * L[0];
    if (dfru) {
      s.kernel_launches += 5 * L[1] + (2 * bd.ncols + 1) * L[2] + 4 * L[3];
      s.reliable_updates += L[2] + L[3];
    } else {
      s.kernel_launches += 6 * L[1];
      s.reliable_updates += L[1];
    }
  }
  // host loop: iterations as CUDA graphs of reliable_every iterations
  for (long guard = 0; host_loop && guard < (long)maxiter + 64; ++guard) {
    if (c->batch_persistent) {
      // one cooperative launch for the chunk: the three passes of every iteration with
      // device-wide barriers in between, no per-pass launches
      err = cudaMemsetAsync(w->bar, 0, sizeof(unsigned int), st);     // arrivals (the generation runs on)
      if (err != cudaSuccess) break;
      PersistArgs pa{w->plo.ref(), w->tlo.ref(), w->rlo.ref(), w->xlo.ref(), w->st, w->part, w->max_blocks,
                     w->bar, w->bar + 1, c->batch_barrier_extra, chunk, 2000000000LL};
      switch (inner_prec) {
        case LQ_F16_12: err = batch_persistent_h16(bd, pa, inner_prec, w->sms, w->max_blocks, st); break;
        case LQ_BF16_12: err = batch_persistent_bf16(bd, pa, inner_prec, w->sms, w->max_blocks, st); break;
        case LQ_I16_12: err = batch_persistent_i16(bd, pa, inner_prec, w->sms, w->max_blocks, st); break;
        case LQ_F32_12: err = batch_persistent_f32_12(bd, pa, inner_prec, w->sms, w->max_blocks, st); break;
        default: err = batch_persistent_f32(bd, pa, inner_prec, w->sms, w->max_blocks, st); break;
      }
      if (err != cudaSuccess) break;
      s.kernel_launches += 1;
      // a wait that gave up: the state says so; stop before the reliable update
      err = cudaMemcpyAsync(w->st_host, w->st, sizeof(BatchState), cudaMemcpyDeviceToHost, st);
      if (err == cudaSuccess) err = cudaStreamSynchronize(st);
      if (err != cudaSuccess) break;
      if (w->st_host->timeout) {
        result = fail(LQ_ERR_TIMEOUT, "a device-wide barrier of the persistent iteration timed out");
        break;
      }
    } else {
    cudaGraphExec_t exec = find_graph(w, bd, kFormChunk, chunk);
    if (!exec) {
      cudaGraph_t g = nullptr;
      err = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
      if (err != cudaSuccess) break;
      for (int i = 0; i < chunk; ++i) batch_iteration_prec(w, bd, inner_prec, tu, c->capture_stream);
      err = cudaStreamEndCapture(c->capture_stream, &g);
      if (err != cudaSuccess) break;
      err = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (err != cudaSuccess) break;
      keep_graph(w, bd, kFormChunk, chunk, exec);
    }
    err = cudaGraphLaunch(exec, st);
    if (err != cudaSuccess) break;
    s.kernel_launches += 3 * chunk;
    }
    // reliable update: fold x, true residual per column, freeze converged columns
    bool certify = true;
    if (dfru) {
      // double-float update, skipped (x_lo only folded) when every open column's
      // iterated residual has already met the tolerance: that update goes straight
      // to the FP64 certification
      err = cudaMemcpyAsync(w->st_host, w->st, sizeof(BatchState), cudaMemcpyDeviceToHost, st);
      if (err == cudaSuccess) err = cudaStreamSynchronize(st);
      if (err != cudaSuccess) break;
      bool last = true;
      for (int col = 0; col < bd.ncols; ++col)
        if (!w->st_host->done[col] && !(w->st_host->rr[col] <= w->st_host->stop2 * w->st_host->phi2[col]))
          last = false;
      dfa.accumulate = true;
      dfa.residual = !last;
      batch_df_tail(dfa, bd, spinor_store_of(inner_prec), st);
      s.kernel_launches += last ? 1 : 1 + 2 * bd.ncols;
      if (!last) {
        batch_xpay_forced(w, bd, inner_prec, st);
        s.kernel_launches += 1;
        s.reliable_updates++;
        err = cudaMemcpyAsync(w->st_host, w->st, sizeof(BatchState), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) break;
        for (int col = 0; col < bd.ncols; ++col) certify = certify && w->st_host->done[col];
        certify = certify && !w->st_host->breakdown;
      }
      if (certify) {
        launch_convert_spinor(flat_geom(bd.total), SStore::DF64, w->xdf.ref(), SStore::F64, w->x64.ref(), st);
        s.kernel_launches += 1;
      }
    }
    if (certify) {
      batch_reliable_tail(w, bd, bd64, inner_prec, !dfru, st);
      s.kernel_launches += dfru ? 3 : 4;
      s.reliable_updates++;
      err = cudaMemcpyAsync(w->st_host, w->st, sizeof(BatchState), cudaMemcpyDeviceToHost, st);
      if (err == cudaSuccess) err = cudaStreamSynchronize(st);
      if (err != cudaSuccess) break;
    }
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
  if (dfru) {
    // the solution lives in the double-float accumulator (x_lo already folded)
    launch_convert_spinor(flat_geom(bd.total), SStore::DF64, w->xdf.ref(), SStore::F64, w->x64.ref(), st);
    s.kernel_launches += 1;
  }
  batch_unpack_kernel<<<flat_grid(w), 256, 0, st>>>(bd, w->x64.ref());
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

extern "C" lq_status lq_batch_tuning(lq_ctx* c, int* tile, int* rhs_per_thread, int* blocks_per_sm,
                                     int* site_major, double* ms, int ms_len) {
  if (!c) return LQ_ERR_ARG;
  const BatchWork* w = static_cast<const BatchWork*>(c->batch);
  if (!w || w->tune.tile == 0) {
    c->last_error = "lq_batch_tuning: no batched solve has run on this context";
    return LQ_ERR_STATE;
  }
  if (tile) *tile = w->tune.tile;
  if (rhs_per_thread) *rhs_per_thread = w->tune.rb;
  if (blocks_per_sm) *blocks_per_sm = w->tune.per_sm;
  if (site_major) *site_major = w->tune.site_major;
  if (ms)
    for (int i = 0; i < ms_len && i < (int)w->tune_ms.size(); ++i) ms[i] = w->tune_ms[i];
  return LQ_OK;
}
