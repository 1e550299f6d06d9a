// C interface (include/lq.h): context management, buffer staging between
// the canonical layout and the internal formats, and the host driver of
// the CG solver (paper Sec. 3: the host sets up fields and calls the
// kernels; all vectors stay resident on the GPU, only scalars come back).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "lq_internal.h"

using namespace lq;

namespace {

thread_local std::string g_create_error;

lq_status fail(lq_ctx* c, lq_status code, const std::string& msg) {
  if (c) c->last_error = msg;
  else g_create_error = msg;
  return code;
}

lq_status cuda_check(lq_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LQ_OK;
  cudaGetLastError();
  return fail(c, LQ_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LQ_TRY(expr)                         \
  do {                                       \
    lq_status _s = (expr);                   \
    if (_s != LQ_OK) return _s;              \
  } while (0)
#define LQ_CUDA(c, call) LQ_TRY(cuda_check((c), (call), #call))

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// With LQ_OPT_HOST_DIRECT: the device address of a page-locked host buffer mapped into the
// device's address space (kernels then read or write it directly, no staging copy); null
// for device buffers, pageable host memory, or with the option off.
void* host_direct(const lq_ctx* c, const void* p) {
  if (!c->host_direct) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

lq_status alloc_field(lq_ctx* c, Field& f, SStore s) {
  if (f.data) return LQ_OK;
  f.store = s;
  LQ_CUDA(c, cudaMalloc(&f.data, spinor_bytes(s, c->geo.V)));
  if (s == SStore::F16 || s == SStore::BF16 || s == SStore::I16)
    LQ_CUDA(c, cudaMalloc(&f.norm, sizeof(float) * c->geo.V));
  return LQ_OK;
}

void free_field(Field& f) {
  if (f.data) cudaFree(f.data);
  if (f.norm) cudaFree(f.norm);
  f.data = nullptr;
  f.norm = nullptr;
}

lq_status require_gauge(lq_ctx* c, int prec) {
  if (!c->gauge_set) return fail(c, LQ_ERR_STATE, "no gauge field set (call lq_gauge_set first)");
  if (prec == LQ_F64) return LQ_OK;
  if (!c->gauge_lo[prec]) LQ_CUDA(c, cudaMalloc(&c->gauge_lo[prec], gauge_bytes(gauge_store_of(prec), c->geo.V)));
  if (!c->gauge_lo_valid[prec]) {
    launch_convert_gauge(c->geo, c->gauge64, gauge_store_of(prec), c->gauge_lo[prec], c->stream);
    LQ_CUDA(c, cudaGetLastError());
    c->gauge_lo_valid[prec] = true;
  }
  return LQ_OK;
}

lq_status check_prec(lq_ctx* c, int prec) {
  if (prec < LQ_F64 || prec > LQ_I16_12) return fail(c, LQ_ERR_ARG, "unknown precision");
  return LQ_OK;
}
lq_status check_inner(lq_ctx* c, int prec) {
  if (prec < LQ_F64 || prec > LQ_I16_12 || prec == LQ_DF64)
    return fail(c, LQ_ERR_ARG, "unknown or unsupported solver precision");
  return LQ_OK;
}

// Canonical spinor (host or device) -> device pointer to canonical data.
lq_status stage_spinor_in(lq_ctx* c, const double* in, const double** dev) {
  if (!in) return fail(c, LQ_ERR_ARG, "null spinor buffer");
  if (!aligned16(in)) return fail(c, LQ_ERR_ARG, "spinor buffer not 16-byte aligned");
  if (is_device_ptr(in)) { *dev = in; return LQ_OK; }
  if (const void* d = host_direct(c, in)) { *dev = static_cast<const double*>(d); return LQ_OK; }
  LQ_CUDA(c, cudaMemcpyAsync(c->stage_in, in, sizeof(double) * 24 * c->geo.V, cudaMemcpyHostToDevice, c->stream));
  *dev = c->stage_in;
  return LQ_OK;
}

// Unpack a field to the caller's canonical buffer (host or device).
lq_status deliver_spinor(lq_ctx* c, const Field& f, double* out) {
  if (!out) return fail(c, LQ_ERR_ARG, "null output buffer");
  if (!aligned16(out)) return fail(c, LQ_ERR_ARG, "output buffer not 16-byte aligned");
  if (is_device_ptr(out)) {
    launch_unpack_spinor(c->geo, f.store, f.ref(), out, c->stream);
    LQ_CUDA(c, cudaGetLastError());
    return LQ_OK;
  }
  if (void* d = host_direct(c, out)) {
    launch_unpack_spinor(c->geo, f.store, f.ref(), static_cast<double*>(d), c->stream);
    LQ_CUDA(c, cudaGetLastError());
    LQ_CUDA(c, cudaStreamSynchronize(c->stream));
    return LQ_OK;
  }
  launch_unpack_spinor(c->geo, f.store, f.ref(), c->stage_out, c->stream);
  LQ_CUDA(c, cudaGetLastError());
  LQ_CUDA(c, cudaMemcpyAsync(out, c->stage_out, sizeof(double) * 24 * c->geo.V, cudaMemcpyDeviceToHost, c->stream));
  LQ_CUDA(c, cudaStreamSynchronize(c->stream));
  return LQ_OK;
}

lq_status ensure_solver_fields(lq_ctx* c, int inner) {
  LQ_TRY(alloc_field(c, c->phi64, SStore::F64));
  LQ_TRY(alloc_field(c, c->x64, SStore::F64));
  LQ_TRY(alloc_field(c, c->r64, SStore::F64));
  LQ_TRY(alloc_field(c, c->tmp64, SStore::F64));
  if (inner == LQ_F64) {
    LQ_TRY(alloc_field(c, c->p64, SStore::F64));
    LQ_TRY(alloc_field(c, c->t64, SStore::F64));
  } else {
    const SStore s = spinor_store_of(inner);
    const int k = (int)s;
    LQ_TRY(alloc_field(c, c->r_lo[k], s));
    LQ_TRY(alloc_field(c, c->p_lo[k], s));
    LQ_TRY(alloc_field(c, c->t_lo[k], s));
    LQ_TRY(alloc_field(c, c->x_lo[k], xlo_store(s)));
  }
  return LQ_OK;
}

// Run n CG iterations as one CUDA graph (recorded once per context,
// precision, length and kappa); the kernels return at once after the
// device-side halt flag is raised.
lq_status run_chunk(lq_ctx* c, int inner, int n, double kappa) {
  if (!c->use_graphs) {
    for (int i = 0; i < n; ++i) {
      if (inner == LQ_F64) cg64_iteration(c, kappa, c->stream);
      else cglo_iteration(c, inner, kappa, c->stream);
    }
    LQ_CUDA(c, cudaGetLastError());
    return LQ_OK;
  }
  auto key = std::make_tuple(c->pair_sites + 2 * c->staged, inner, n, kappa);
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    cudaGraph_t graph = nullptr;
    LQ_CUDA(c, cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < n; ++i) {
      if (inner == LQ_F64) cg64_iteration(c, kappa, c->capture_stream);
      else cglo_iteration(c, inner, kappa, c->capture_stream);
    }
    LQ_CUDA(c, cudaStreamEndCapture(c->capture_stream, &graph));
    GraphEntry e;
    cudaError_t err = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    LQ_CUDA(c, err);
    it = c->graphs.emplace(key, e).first;
  }
  LQ_CUDA(c, cudaGraphLaunch(it->second.exec, c->stream));
  return LQ_OK;
}

lq_status read_state(lq_ctx* c) {
  LQ_CUDA(c, cudaMemcpyAsync(c->state_host, c->state, sizeof(SolverState), cudaMemcpyDeviceToHost, c->stream));
  LQ_CUDA(c, cudaStreamSynchronize(c->stream));
  return LQ_OK;
}

// Reliable update when the iterated residual fell by this factor (squared)
// since the last one: 16-bit storage loses accuracy faster than FP32.
double reliable_delta2(int inner) {
  switch (inner) {
    case LQ_BF16_12: return 1e-2;
    case LQ_F16_12: case LQ_I16_12: return 1e-4;
    default: return 1e-4;
  }
}

// Solve M^dag M x = phi with phi already in c->phi64; the solution is left in
// c->x64.  Host scalars come back once per CUDA graph of iterations.
lq_status solve_internal(lq_ctx* c, double kappa, double tol, int maxiter, int inner, int reliable_every,
                         double* hist_dev, int hist_len, lq_solve_stats* sout) {
  LQ_TRY(require_gauge(c, inner));
  LQ_TRY(ensure_solver_fields(c, inner));
  const Geom& g = c->geo;
  const bool mixed = inner != LQ_F64;
  const bool dfru = mixed && c->df_updates;     // double-float intermediate reliable updates
  SStore slo = spinor_store_of(inner);
  int k = (int)slo;
  if (dfru) {
    LQ_TRY(require_gauge(c, LQ_DF64));
    for (Field* f : {&c->phi_df, &c->x_df, &c->tmp_df, &c->r_df}) LQ_TRY(alloc_field(c, *f, SStore::DF64));
  }
  SolverState h{};
  h.stop2 = tol * tol;
  h.ru_every = mixed ? reliable_every : 0;
  h.delta2 = mixed ? reliable_delta2(inner) : 0.0;
  h.maxiter = maxiter;
  h.hist = hist_dev;
  h.hist_len = hist_dev ? hist_len : 0;
  *c->state_host = h;
  LQ_CUDA(c, cudaMemcpyAsync(c->state, c->state_host, sizeof(SolverState), cudaMemcpyHostToDevice, c->stream));
  if (mixed) {
    launch_zero_spinor(g, SStore::F64, c->x64.ref(), c->stream);
    if (dfru) {
      launch_convert_spinor(g, SStore::F64, c->phi64.ref(), SStore::DF64, c->phi_df.ref(), c->stream);
      launch_zero_spinor(g, SStore::DF64, c->x_df.ref(), c->stream);
    }
    launch_solver_init(g, c->phi64.ref(), slo, c->x_lo[k].ref(), slo, c->r_lo[k].ref(), slo, c->p_lo[k].ref(),
                       c->state, c->rs, c->stream);
  } else {
    launch_solver_init(g, c->phi64.ref(), SStore::F64, c->x64.ref(), SStore::F64, c->r64.ref(), SStore::F64,
                       c->p64.ref(), c->state, c->rs, c->stream);
  }
  LQ_CUDA(c, cudaGetLastError());
  LQ_TRY(read_state(c));

  lq_solve_stats& s = *sout;
  s = lq_solve_stats{};
  s.kernel_launches = mixed ? 2 : 1;      // (zero x,) initialise
  lq_status result = LQ_OK;
  double rel = 1.0;
  if (c->state_host->breakdown) {
    result = fail(c, LQ_ERR_NAN, "non-finite right-hand side");
  } else if (c->state_host->phi2 == 0.0) {
    rel = 0.0;
    s.converged = 1;
  } else {
    const int chunk = mixed ? (reliable_every > 0 ? reliable_every : 32) : 16;
    double best_rr = c->state_host->phi2;
    int stagnant = 0;
    for (long guard = 0; guard < (long)maxiter + 64; ++guard) {
      LQ_TRY(run_chunk(c, inner, chunk, kappa));
      s.kernel_launches += 3 * chunk;
      LQ_TRY(read_state(c));
      const SolverState& st = *c->state_host;
      if (st.breakdown) { result = fail(c, LQ_ERR_NAN, "CG breakdown (non-positive or non-finite curvature)"); break; }
      if (!st.halt) continue;
      // true residual; for mixed solves this is the reliable update
      if (dfru) {
        // double-float on the FP32 pipe; a residual meeting tol is certified in FP64.  When
        // the iterated residual has met tol the update is almost surely the last: it goes
        // straight to the FP64 certification.
        const bool last = st.rr <= st.stop2;
        if (last) {
          df_accumulate(c, inner, c->stream);
          s.kernel_launches += 1;
          rel = 0.0;
        } else {
          df_reliable_update(c, kappa, inner, c->stream);
          s.kernel_launches += 3;
          LQ_CUDA(c, cudaGetLastError());
          LQ_TRY(read_state(c));
          rel = std::sqrt(c->state_host->rr_true / c->state_host->phi2);
        }
        s.reliable_updates++;
        if (std::isfinite(rel) && rel <= tol) {
          launch_convert_spinor(g, SStore::DF64, c->x_df.ref(), SStore::F64, c->x64.ref(), c->stream);
          cg64_true_residual(c, kappa, inner, c->stream);
          s.kernel_launches += 3;
          LQ_CUDA(c, cudaGetLastError());
          LQ_TRY(read_state(c));
          rel = std::sqrt(c->state_host->rr_true / c->state_host->phi2);
          if (std::isfinite(rel) && rel <= tol) { s.converged = 1; break; }
          // not certified: continue from the FP64 residual
          launch_convert_spinor(g, SStore::F64, c->r64.ref(), SStore::DF64, c->r_df.ref(), c->stream);
          s.kernel_launches += 1;
        }
      } else {
        if (mixed) launch_accumulate_x(g, slo, c->x_lo[k].ref(), c->x64.ref(), c->stream);
        cg64_true_residual(c, kappa, inner, c->stream);
        s.kernel_launches += mixed ? 3 : 2;
        LQ_CUDA(c, cudaGetLastError());
        LQ_TRY(read_state(c));
        rel = std::sqrt(c->state_host->rr_true / c->state_host->phi2);
        if (mixed) s.reliable_updates++;
      }
      const double rr_true = c->state_host->rr_true;
      if (!std::isfinite(rel)) { result = fail(c, LQ_ERR_NAN, "non-finite residual"); break; }
      if (rel <= tol) { s.converged = 1; break; }
      if (c->state_host->iter >= maxiter) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "not converged after %d iterations (relative residual %.3e)",
                      c->state_host->iter, rel);
        result = fail(c, LQ_ERR_NOT_CONVERGED, buf);
        break;
      }
      // FP64 CG: the recursion met tol but the true residual did not ->
      // restart from the true residual.  Mixed: keep the search direction
      // unless the true residual has stopped improving.
      int restart = mixed ? 0 : 1;
      if (mixed) {
        if (rr_true < 0.5 * best_rr) { best_rr = rr_true; stagnant = 0; }
        else if (++stagnant >= 3) { restart = 1; stagnant = 0; }
      }
      if (restart && mixed && inner != LQ_F32) {
        // Defect correction fallback: the inner precision cannot make progress
        // on this system (its rounding times the condition number is too
        // large), so continue in FP32 from the FP64 iterate and residual.
        inner = LQ_F32;
        slo = SStore::F32;
        k = (int)slo;
        LQ_TRY(require_gauge(c, inner));
        LQ_TRY(ensure_solver_fields(c, inner));
        if (dfru)
          launch_inner_restart_df(g, c->r_df.ref(), slo, c->x_lo[k].ref(), c->r_lo[k].ref(), c->p_lo[k].ref(),
                                  c->stream);
        else
          launch_inner_restart(g, c->r64.ref(), slo, c->x_lo[k].ref(), c->r_lo[k].ref(), c->p_lo[k].ref(),
                               c->stream);
        SolverState& hs = *c->state_host;
        hs.rr = hs.rr_prev = hs.rr_ref = rr_true;
        hs.beta = 0.0;
        hs.iter_since_ru = 0;
        hs.halt = 0;
        hs.delta2 = reliable_delta2(inner);
        LQ_CUDA(c, cudaMemcpyAsync(c->state, c->state_host, sizeof(SolverState), cudaMemcpyHostToDevice, c->stream));
        s.restarts++;
        s.escalations++;
        s.kernel_launches += 1;
        LQ_CUDA(c, cudaGetLastError());
        continue;
      }
      if (restart) s.restarts++;
      launch_state_after_residual(c->state, restart, c->stream);
      if (mixed) launch_xpay_p(g, slo, c->r_lo[k].ref(), c->p_lo[k].ref(), c->state, true, c->stream);
      else launch_xpay_p(g, SStore::F64, c->r64.ref(), c->p64.ref(), c->state, true, c->stream);
      s.kernel_launches += 2;
      LQ_CUDA(c, cudaGetLastError());
    }
  }
  if (dfru && !s.converged) {
    // the current solution lives in the double-float accumulator
    launch_convert_spinor(g, SStore::DF64, c->x_df.ref(), SStore::F64, c->x64.ref(), c->stream);
    s.kernel_launches += 1;
  }
  s.iterations = c->state_host->iter;
  s.true_rel_resid = rel;
  return result;
}

lq_status ensure_md_fields(lq_ctx* c) {
  const size_t mb = sizeof(double) * 32 * (size_t)c->geo.V;
  if (!c->mom) LQ_CUDA(c, cudaMalloc(&c->mom, mb));
  if (!c->mom0) LQ_CUDA(c, cudaMalloc(&c->mom0, mb));
  if (!c->force) LQ_CUDA(c, cudaMalloc(&c->force, mb));
  if (!c->gauge_old) LQ_CUDA(c, cudaMalloc(&c->gauge_old, gauge_bytes(GStore::F64_18, c->geo.V)));
  LQ_TRY(alloc_field(c, c->y64, SStore::F64));
  LQ_TRY(alloc_field(c, c->chi64, SStore::F64));
  LQ_TRY(alloc_field(c, c->x64, SStore::F64));
  LQ_TRY(alloc_field(c, c->phi64, SStore::F64));
  return LQ_OK;
}

// canonical momenta / forces [V][32] (host or device) -> SoA [32][V]
lq_status stage_mom_in(lq_ctx* c, const double* p, double* soa) {
  if (!p) return fail(c, LQ_ERR_ARG, "null momentum buffer");
  if (!aligned16(p)) return fail(c, LQ_ERR_ARG, "momentum buffer not 16-byte aligned");
  const double* src = p;
  if (!is_device_ptr(p)) {
    if (!c->stage_mom) LQ_CUDA(c, cudaMalloc(&c->stage_mom, sizeof(double) * 32 * (size_t)c->geo.V));
    LQ_CUDA(c, cudaMemcpyAsync(c->stage_mom, p, sizeof(double) * 32 * (size_t)c->geo.V, cudaMemcpyHostToDevice,
                               c->stream));
    src = c->stage_mom;
  }
  launch_pack_mom(c->geo, src, soa, c->stream);
  LQ_CUDA(c, cudaGetLastError());
  return LQ_OK;
}

lq_status deliver_mom(lq_ctx* c, const double* soa, double* out) {
  if (!out) return fail(c, LQ_ERR_ARG, "null output buffer");
  if (!aligned16(out)) return fail(c, LQ_ERR_ARG, "output buffer not 16-byte aligned");
  if (is_device_ptr(out)) {
    launch_unpack_mom(c->geo, soa, out, c->stream);
    LQ_CUDA(c, cudaGetLastError());
    return LQ_OK;
  }
  if (!c->stage_mom) LQ_CUDA(c, cudaMalloc(&c->stage_mom, sizeof(double) * 32 * (size_t)c->geo.V));
  launch_unpack_mom(c->geo, soa, c->stage_mom, c->stream);
  LQ_CUDA(c, cudaMemcpyAsync(out, c->stage_mom, sizeof(double) * 32 * (size_t)c->geo.V, cudaMemcpyDeviceToHost,
                             c->stream));
  LQ_CUDA(c, cudaStreamSynchronize(c->stream));
  return LQ_OK;
}

void gauge_changed(lq_ctx* c) {
  for (int p = 0; p < kNumPrec; ++p) c->gauge_lo_valid[p] = false;
}

// Device time of the phases of a trajectory: CUDA event pairs on the work
// stream, summed once the trajectory has synchronised.
struct PhaseTimer {
  enum { kSolve, kGauge, kFermion, kLink, kN };
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[kN];
  cudaStream_t st;
  explicit PhaseTimer(cudaStream_t s) : st(s) {}
  void begin(int k) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
    ev[k].emplace_back(a, b);
  }
  void end(int k) { cudaEventRecord(ev[k].back().second, st); }
  double seconds(int k) {
    double t = 0.0;
    for (auto& p : ev[k]) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) t += ms * 1e-3;
    }
    return t;
  }
  ~PhaseTimer() {
    for (auto& v : ev)
      for (auto& p : v) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
      }
  }
};

// p -= eps (F_gauge + F_fermion) at the current links; one solve for X = (M^dag M)^{-1} phi
lq_status md_force_step(lq_ctx* c, const lq_hmc_params* hp, double eps, lq_traj_result* res, PhaseTimer& tm) {
  tm.begin(PhaseTimer::kGauge);
  launch_gauge_force(c->geo, c->gauge64, c->mom, hp->beta, eps, true, c->stream);
  tm.end(PhaseTimer::kGauge);
  lq_solve_stats s{};
  tm.begin(PhaseTimer::kSolve);
  lq_status st = solve_internal(c, hp->kappa, hp->tol, hp->maxiter, hp->inner_prec, hp->reliable_every, nullptr,
                                0, &s);
  tm.end(PhaseTimer::kSolve);
  res->solves += 1;
  res->cg_iterations += s.iterations;
  res->kernel_launches += s.kernel_launches + 3;
  if (st != LQ_OK) return st;
  tm.begin(PhaseTimer::kFermion);
  apply_M_prec(c->geo, LQ_F64, c->gauge64, c->x64.ref(), c->y64.ref(), hp->kappa, false, c->stream);
  launch_fermion_force(c->geo, c->gauge64, c->x64.ref(), c->y64.ref(), c->mom, hp->kappa, eps, true, c->stream);
  tm.end(PhaseTimer::kFermion);
  LQ_CUDA(c, cudaGetLastError());
  return LQ_OK;
}

lq_status read_scalars(lq_ctx* c) {
  LQ_CUDA(c, cudaMemcpyAsync(c->dscalar_host, c->dscalar, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream));
  LQ_CUDA(c, cudaStreamSynchronize(c->stream));
  return LQ_OK;
}

lq_status check_trajectory_args(lq_ctx* c, const lq_hmc_params* hp, lq_traj_result* out) {
  if (!hp || !out) return fail(c, LQ_ERR_ARG, "null parameters or result");
  if (hp->n_steps <= 0 || !(hp->tau > 0.0) || !(hp->tol > 0.0) || hp->maxiter <= 0 || hp->reliable_every < 0)
    return fail(c, LQ_ERR_ARG, "bad trajectory parameters");
  LQ_TRY(check_inner(c, hp->inner_prec));
  LQ_TRY(require_gauge(c, LQ_F64));
  LQ_TRY(ensure_md_fields(c));
  LQ_TRY(ensure_solver_fields(c, hp->inner_prec));
  return LQ_OK;
}

// The trajectory after its heat bath (Eq. 5; Sec. 2; Sec. 3 steps 1-3): c->mom holds the
// start momenta, c->chi64 the noise, u the Metropolis uniform.  p, when not null, receives
// the final momenta.
lq_status trajectory_after_heatbath(lq_ctx* c, const lq_hmc_params* hp, double u, double* p, lq_traj_result* out,
                                    std::chrono::steady_clock::time_point t0, int heatbath_launches) {
  lq_traj_result r{};
  const Geom& g = c->geo;
  // phi = M^dag chi; keep the start momenta and links
  LQ_CUDA(c, cudaMemcpyAsync(c->mom0, c->mom, sizeof(double) * 32 * (size_t)g.V, cudaMemcpyDeviceToDevice,
                             c->stream));
  apply_M_prec(g, LQ_F64, c->gauge64, c->chi64.ref(), c->phi64.ref(), hp->kappa, true, c->stream);
  LQ_CUDA(c, cudaMemcpyAsync(c->gauge_old, c->gauge64, gauge_bytes(GStore::F64_18, g.V), cudaMemcpyDeviceToDevice,
                             c->stream));
  r.kernel_launches += heatbath_launches + 1;
  // leapfrog: half step in p, then n x (full step in U, full step in p), last p step halved
  PhaseTimer tm(c->stream);
  const double eps = hp->tau / hp->n_steps;
  lq_status st = md_force_step(c, hp, 0.5 * eps, &r, tm);
  for (int i = 0; i < hp->n_steps && st == LQ_OK; ++i) {
    tm.begin(PhaseTimer::kLink);
    launch_link_update(g, c->gauge64, c->mom, eps, c->stream);
    tm.end(PhaseTimer::kLink);
    gauge_changed(c);
    r.kernel_launches += 1;
    st = md_force_step(c, hp, i < hp->n_steps - 1 ? eps : 0.5 * eps, &r, tm);
  }
  if (st == LQ_OK) {
    // S_f at the end: X = (M^dag M)^{-1} phi on the new links
    lq_solve_stats s{};
    tm.begin(PhaseTimer::kSolve);
    st = solve_internal(c, hp->kappa, hp->tol, hp->maxiter, hp->inner_prec, hp->reliable_every, nullptr, 0, &s);
    tm.end(PhaseTimer::kSolve);
    r.solves += 1;
    r.cg_iterations += s.iterations;
    r.kernel_launches += s.kernel_launches;
  }
  if (st != LQ_OK) {
    // leave the links as they were before the trajectory
    cudaMemcpyAsync(c->gauge64, c->gauge_old, gauge_bytes(GStore::F64_18, g.V), cudaMemcpyDeviceToDevice, c->stream);
    gauge_changed(c);
    cudaStreamSynchronize(c->stream);
    return st;
  }
  // Delta H from per-site differences
  launch_fermion_action_diff(g, c->phi64.ref(), c->x64.ref(), c->chi64.ref(), c->rs, c->dscalar + 0, c->stream);
  launch_kinetic_diff(g, c->mom, c->mom0, c->rs, c->dscalar + 1, c->stream);
  launch_plaquette(g, c->gauge_old, c->gauge64, c->rs, c->dscalar + 2, c->stream);
  r.kernel_launches += 3;
  LQ_CUDA(c, cudaGetLastError());
  LQ_TRY(read_scalars(c));
  r.dSf = c->dscalar_host[0];
  r.dK = c->dscalar_host[1];
  r.dSg = hp->beta / 3.0 * c->dscalar_host[3];       // sum (ReTr P_old - ReTr P_new)
  r.dH = r.dK + r.dSg + r.dSf;
  if (!std::isfinite(r.dH)) {
    cudaMemcpyAsync(c->gauge64, c->gauge_old, gauge_bytes(GStore::F64_18, g.V), cudaMemcpyDeviceToDevice, c->stream);
    gauge_changed(c);
    cudaStreamSynchronize(c->stream);
    *out = r;
    return fail(c, LQ_ERR_NAN, "non-finite Delta H; trajectory rejected");
  }
  r.accepted = (r.dH <= 0.0 || u < std::exp(-r.dH)) ? 1 : 0;
  if (!r.accepted) {
    LQ_CUDA(c, cudaMemcpyAsync(c->gauge64, c->gauge_old, gauge_bytes(GStore::F64_18, g.V),
                               cudaMemcpyDeviceToDevice, c->stream));
    gauge_changed(c);
  }
  launch_plaquette(g, c->gauge64, nullptr, c->rs, c->dscalar + 4, c->stream);
  r.kernel_launches += 1;
  LQ_TRY(read_scalars(c));
  r.plaquette = c->dscalar_host[4] / (18.0 * g.V);
  if (p) LQ_TRY(deliver_mom(c, c->mom, p));
  LQ_CUDA(c, cudaStreamSynchronize(c->stream));
  r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  r.seconds_solve = tm.seconds(PhaseTimer::kSolve);
  r.seconds_gauge_force = tm.seconds(PhaseTimer::kGauge);
  r.seconds_fermion_force = tm.seconds(PhaseTimer::kFermion);
  r.seconds_link_update = tm.seconds(PhaseTimer::kLink);
  *out = r;
  return LQ_OK;
}

}  // namespace

// Error text of calls that run without a context (read with lq_last_error(NULL)).
void lq_set_global_error(const std::string& msg) { g_create_error = msg; }

extern "C" {

const char* lq_version(void) { return "lq 0.1 (sm_103a)"; }

lq_status lq_create(lq_ctx** out, const int dims[4], int t_antiperiodic, void* cuda_stream) {
  if (!out || !dims) return fail(nullptr, LQ_ERR_ARG, "null argument");
  *out = nullptr;
  // the product is checked against the limit factor by factor, so it cannot overflow
  constexpr long long kMaxSites = (1LL << 31) / 64;
  long long V = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 2) return fail(nullptr, LQ_ERR_SHAPE, "every lattice extent must be >= 2");
    if (dims[m] >= kMaxSites || V * dims[m] >= kMaxSites) return fail(nullptr, LQ_ERR_SHAPE, "lattice volume too large");
    V *= dims[m];
  }
  lq_ctx* c = new lq_ctx();
  c->geo.V = (int)V;
  for (int m = 0; m < 4; ++m) c->geo.L[m] = dims[m];
  c->geo.stride[0] = 1;
  for (int m = 1; m < 4; ++m) c->geo.stride[m] = c->geo.stride[m - 1] * dims[m - 1];
  c->geo.antiperiodic = t_antiperiodic ? 1 : 0;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  lq_status st = LQ_OK;
  auto chk = [&](cudaError_t e, const char* what) {
    if (st == LQ_OK && e != cudaSuccess) {
      cudaGetLastError();
      g_create_error = std::string(what) + ": " + cudaGetErrorString(e);
      st = LQ_ERR_CUDA;
    }
  };
  chk(cudaGetDevice(&c->device), "cudaGetDevice");
  chk(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  for (cudaEvent_t& e : c->phase_ev) chk(cudaEventCreate(&e), "cudaEventCreate");
  const size_t spin = sizeof(double) * 24 * (size_t)V;
  chk(cudaMalloc(&c->gauge64, gauge_bytes(GStore::F64_18, (int)V)), "cudaMalloc gauge");
  chk(cudaMalloc(&c->stage_in, spin), "cudaMalloc stage");
  chk(cudaMalloc(&c->stage_out, spin), "cudaMalloc stage");
  c->rs.max_blocks = (int)((V + 63) / 64) + 1;
  chk(cudaMalloc(&c->rs.partials, sizeof(double) * 4 * c->rs.max_blocks), "cudaMalloc partials");
  chk(cudaMalloc(&c->rs.ticket, sizeof(unsigned int) * 4), "cudaMalloc ticket");
  if (st == LQ_OK) chk(cudaMemset(c->rs.ticket, 0, sizeof(unsigned int) * 4), "cudaMemset");
  chk(cudaMalloc(&c->state, sizeof(SolverState)), "cudaMalloc state");
  chk(cudaMallocHost(&c->state_host, sizeof(SolverState)), "cudaMallocHost");
  chk(cudaMalloc(&c->dscalar, sizeof(double) * 8), "cudaMalloc scalars");
  chk(cudaMallocHost(&c->dscalar_host, sizeof(double) * 8), "cudaMallocHost");
  if (st != LQ_OK) {
    lq_destroy(c);
    return st;
  }
  *out = c;
  return LQ_OK;
}

lq_status lq_destroy(lq_ctx* c) {
  if (!c) return LQ_OK;
  cudaStreamSynchronize(c->stream);
  destroy_batch_work(c->batch);
  for (auto& kv : c->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  for (cudaEvent_t e : c->phase_ev)
    if (e) cudaEventDestroy(e);
  if (c->gauge64) cudaFree(c->gauge64);
  for (int p = 0; p < kNumPrec; ++p)
    if (c->gauge_lo[p]) cudaFree(c->gauge_lo[p]);
  if (c->stage_in) cudaFree(c->stage_in);
  if (c->stage_out) cudaFree(c->stage_out);
  if (c->stage_gauge) cudaFree(c->stage_gauge);
  for (Field* f : {&c->phi64, &c->x64, &c->r64, &c->p64, &c->t64, &c->tmp64, &c->y64, &c->chi64, &c->phi_df,
                   &c->x_df, &c->tmp_df, &c->r_df})
    free_field(*f);
  for (double* d : {c->mom, c->mom0, c->force, c->stage_mom})
    if (d) cudaFree(d);
  if (c->gauge_old) cudaFree(c->gauge_old);
  for (int k = 0; k < kNumSStore; ++k) {
    free_field(c->r_lo[k]);
    free_field(c->p_lo[k]);
    free_field(c->t_lo[k]);
    free_field(c->x_lo[k]);
  }
  if (c->rs.partials) cudaFree(c->rs.partials);
  if (c->rs.ticket) cudaFree(c->rs.ticket);
  if (c->state) cudaFree(c->state);
  if (c->state_host) cudaFreeHost(c->state_host);
  if (c->dscalar) cudaFree(c->dscalar);
  if (c->dscalar_host) cudaFreeHost(c->dscalar_host);
  delete c;
  return LQ_OK;
}

const char* lq_last_error(const lq_ctx* c) { return c ? c->last_error.c_str() : g_create_error.c_str(); }

lq_status lq_set_stream(lq_ctx* c, void* cuda_stream) {
  if (!c) return LQ_ERR_ARG;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  return LQ_OK;
}

int64_t lq_volume(const lq_ctx* c) { return c ? (int64_t)c->geo.V : 0; }

lq_status lq_set_option(lq_ctx* c, int option, int value) {
  if (!c) return LQ_ERR_ARG;
  switch (option) {
    case LQ_OPT_CUDA_GRAPHS: c->use_graphs = value ? 1 : 0; return LQ_OK;
    case LQ_OPT_DF64_UPDATES: c->df_updates = value ? 1 : 0; return LQ_OK;
    case LQ_OPT_PAIR_SITES: c->pair_sites = value ? 1 : 0; return LQ_OK;
    case LQ_OPT_STAGED: c->staged = value ? 1 : 0; return LQ_OK;
    case LQ_OPT_BATCH_RHS_PER_THREAD:
      if (value < 0 || value > 4) return fail(c, LQ_ERR_ARG, "right-hand sides per thread must be 0 (tuned) or 1..4");
      c->batch_rb = value;
      if (c->batch) { destroy_batch_work(c->batch); c->batch = nullptr; }
      return LQ_OK;
    case LQ_OPT_BATCH_PERSISTENT: c->batch_persistent = value ? 1 : 0; return LQ_OK;
    case LQ_OPT_BATCH_DEVICE_LOOP: c->batch_device_loop = value ? 1 : 0; return LQ_OK;
    case LQ_OPT_HOST_DIRECT: c->host_direct = value ? 1 : 0; return LQ_OK;
    case LQ_OPT_DF64_PREFETCH: c->df_prefetch = value ? 1 : 0; return LQ_OK;
    case LQ_OPT_BATCH_TILE_ORDER:
      if (value < 0 || value > 2) return fail(c, LQ_ERR_ARG, "tile order is 0 (tuned), 1 or 2");
      c->batch_order = value;
      if (c->batch) { destroy_batch_work(c->batch); c->batch = nullptr; }
      return LQ_OK;
    case LQ_OPT_BATCH_BARRIER_TEST:
      if (value < 0 || value > 1) return fail(c, LQ_ERR_ARG, "barrier test option is 0 or 1");
      c->batch_barrier_extra = value;
      return LQ_OK;
    default: return fail(c, LQ_ERR_ARG, "unknown option");
  }
}

lq_status lq_gauge_set(lq_ctx* c, const double* U) {
  if (!c) return LQ_ERR_ARG;
  if (!U) return fail(c, LQ_ERR_ARG, "null gauge buffer");
  if (!aligned16(U)) return fail(c, LQ_ERR_ARG, "gauge buffer not 16-byte aligned");
  const double* src = U;
  if (const void* d = is_device_ptr(U) ? nullptr : host_direct(c, U)) {
    src = static_cast<const double*>(d);                    // read in place by the packing kernel
  } else if (!is_device_ptr(U)) {
    if (!c->stage_gauge) LQ_CUDA(c, cudaMalloc(&c->stage_gauge, sizeof(double) * 72 * (size_t)c->geo.V));
    LQ_CUDA(c, cudaMemcpyAsync(c->stage_gauge, U, sizeof(double) * 72 * (size_t)c->geo.V, cudaMemcpyHostToDevice,
                               c->stream));
    src = c->stage_gauge;
  }
  launch_pack_gauge64(c->geo, src, c->gauge64, c->stream);
  LQ_CUDA(c, cudaGetLastError());
  for (int p = 0; p < kNumPrec; ++p) c->gauge_lo_valid[p] = false;
  c->gauge_set = true;
  if (!is_device_ptr(U)) LQ_CUDA(c, cudaStreamSynchronize(c->stream));   // the host buffer may be reused at once
  return LQ_OK;
}

lq_status lq_gauge_get(lq_ctx* c, double* U) {
  if (!c) return LQ_ERR_ARG;
  if (!c->gauge_set) return fail(c, LQ_ERR_STATE, "no gauge field set");
  if (!U) return fail(c, LQ_ERR_ARG, "null gauge buffer");
  if (!aligned16(U)) return fail(c, LQ_ERR_ARG, "gauge buffer not 16-byte aligned");
  if (is_device_ptr(U)) {
    launch_unpack_gauge64(c->geo, c->gauge64, U, c->stream);
    LQ_CUDA(c, cudaGetLastError());
    return LQ_OK;
  }
  if (void* d = host_direct(c, U)) {
    launch_unpack_gauge64(c->geo, c->gauge64, static_cast<double*>(d), c->stream);
    LQ_CUDA(c, cudaGetLastError());
    LQ_CUDA(c, cudaStreamSynchronize(c->stream));
    return LQ_OK;
  }
  if (!c->stage_gauge) LQ_CUDA(c, cudaMalloc(&c->stage_gauge, sizeof(double) * 72 * (size_t)c->geo.V));
  launch_unpack_gauge64(c->geo, c->gauge64, c->stage_gauge, c->stream);
  LQ_CUDA(c, cudaGetLastError());
  LQ_CUDA(c, cudaMemcpyAsync(U, c->stage_gauge, sizeof(double) * 72 * (size_t)c->geo.V, cudaMemcpyDeviceToHost,
                             c->stream));
  LQ_CUDA(c, cudaStreamSynchronize(c->stream));
  return LQ_OK;
}

lq_status lq_apply_M(lq_ctx* c, double* out, const double* in, double kappa, int dagger, int prec) {
  if (!c) return LQ_ERR_ARG;
  LQ_TRY(check_prec(c, prec));
  LQ_TRY(require_gauge(c, prec));
  if (in == out) return fail(c, LQ_ERR_ARG, "in and out must not overlap");
  const SStore s = spinor_store_of(prec);
  Field& fin = (prec == LQ_F64) ? c->phi64 : c->p_lo[(int)s];
  Field& fout = (prec == LQ_F64) ? c->tmp64 : c->t_lo[(int)s];
  LQ_TRY(alloc_field(c, fin, s));
  LQ_TRY(alloc_field(c, fout, s));
  const double* din = nullptr;
  LQ_TRY(stage_spinor_in(c, in, &din));
  launch_pack_spinor(c->geo, din, s, fin.ref(), c->stream);
  const void* gauge = prec == LQ_F64 ? c->gauge64 : c->gauge_lo[prec];
  apply_M_prec(c->geo, prec, gauge, fin.ref(), fout.ref(), kappa, dagger != 0, c->stream, c->pair_sites, c->staged,
               c->df_prefetch);
  LQ_CUDA(c, cudaGetLastError());
  return deliver_spinor(c, fout, out);
}

lq_status lq_apply_MdagM(lq_ctx* c, double* out, const double* in, double kappa, int prec) {
  if (!c) return LQ_ERR_ARG;
  LQ_TRY(check_prec(c, prec));
  LQ_TRY(require_gauge(c, prec));
  if (in == out) return fail(c, LQ_ERR_ARG, "in and out must not overlap");
  const SStore s = spinor_store_of(prec);
  Field& fin = (prec == LQ_F64) ? c->phi64 : c->p_lo[(int)s];
  Field& fmid = (prec == LQ_F64) ? c->tmp64 : c->t_lo[(int)s];
  Field& fout = (prec == LQ_F64) ? c->r64 : c->r_lo[(int)s];
  LQ_TRY(alloc_field(c, fin, s));
  LQ_TRY(alloc_field(c, fmid, s));
  LQ_TRY(alloc_field(c, fout, s));
  const double* din = nullptr;
  LQ_TRY(stage_spinor_in(c, in, &din));
  launch_pack_spinor(c->geo, din, s, fin.ref(), c->stream);
  const void* gauge = prec == LQ_F64 ? c->gauge64 : c->gauge_lo[prec];
  apply_M_prec(c->geo, prec, gauge, fin.ref(), fmid.ref(), kappa, false, c->stream, c->pair_sites, c->staged,
               c->df_prefetch);
  apply_M_prec(c->geo, prec, gauge, fmid.ref(), fout.ref(), kappa, true, c->stream, c->pair_sites, c->staged,
               c->df_prefetch);
  LQ_CUDA(c, cudaGetLastError());
  return deliver_spinor(c, fout, out);
}

lq_status lq_solve_MdagM(lq_ctx* c, double* x, const double* phi, double kappa, double tol, int maxiter,
                         int inner, int reliable_every, double* hist, int hist_len, lq_solve_stats* stats) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!c) return LQ_ERR_ARG;
  LQ_TRY(check_inner(c, inner));
  if (!(tol > 0.0) || maxiter <= 0 || reliable_every < 0 || (hist && hist_len < 0))
    return fail(c, LQ_ERR_ARG, "bad tolerance, iteration limit or history length");
  LQ_TRY(require_gauge(c, LQ_F64));
  LQ_TRY(ensure_solver_fields(c, inner));
  double* hist_dev = nullptr;
  if (hist && hist_len > 0) LQ_CUDA(c, cudaMallocAsync((void**)&hist_dev, sizeof(double) * hist_len, c->stream));
  const double* dphi = nullptr;
  cudaEventRecord(c->phase_ev[0], c->stream);
  LQ_TRY(stage_spinor_in(c, phi, &dphi));
  launch_pack_spinor(c->geo, dphi, SStore::F64, c->phi64.ref(), c->stream);
  cudaEventRecord(c->phase_ev[1], c->stream);
  lq_solve_stats s{};
  lq_status result = solve_internal(c, kappa, tol, maxiter, inner, reliable_every, hist_dev, hist_len, &s);
  cudaEventRecord(c->phase_ev[2], c->stream);
  s.kernel_launches += 1;
  bool delivered = false;
  if (result == LQ_OK || result == LQ_ERR_NOT_CONVERGED) {
    lq_status d = deliver_spinor(c, c->x64, x);
    s.kernel_launches += 1;
    if (d != LQ_OK) result = d;
    else delivered = true;
  }
  cudaEventRecord(c->phase_ev[3], c->stream);
  if (hist_dev) {
    const int n = s.iterations < hist_len ? s.iterations : hist_len;
    if (n > 0) cudaMemcpyAsync(hist, hist_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(hist_dev, c->stream);
  }
  lq_status fin = cuda_check(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (result == LQ_OK) result = fin;
  s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  float ms[3] = {0.f, 0.f, 0.f};
  for (int k = 0; k < 3; ++k)
    if (cudaEventElapsedTime(&ms[k], c->phase_ev[k], c->phase_ev[k + 1]) != cudaSuccess) {
      cudaGetLastError();
      ms[k] = 0.f;
    }
  s.stage_ms = ms[0];
  s.solve_ms = ms[1];
  s.deliver_ms = delivered ? ms[2] : 0.0;
  if (stats) *stats = s;
  return result;
}

lq_status lq_time_dslash(lq_ctx* c, const double* in, double kappa, int dagger, int prec, int n, int flush_l2,
                         double* ms) {
  if (!c) return LQ_ERR_ARG;
  if (!ms || n <= 0) return fail(c, LQ_ERR_ARG, "need n > 0 and an output pointer");
  LQ_TRY(check_prec(c, prec));
  LQ_TRY(require_gauge(c, prec));
  const SStore s = spinor_store_of(prec);
  Field& fin = (prec == LQ_F64) ? c->phi64 : c->p_lo[(int)s];
  Field& fout = (prec == LQ_F64) ? c->tmp64 : c->t_lo[(int)s];
  LQ_TRY(alloc_field(c, fin, s));
  LQ_TRY(alloc_field(c, fout, s));
  const double* din = nullptr;
  LQ_TRY(stage_spinor_in(c, in, &din));
  launch_pack_spinor(c->geo, din, s, fin.ref(), c->stream);
  const void* gauge = prec == LQ_F64 ? c->gauge64 : c->gauge_lo[prec];
  const size_t flush_bytes = (size_t)256 << 20;
  void* flush = nullptr;
  if (flush_l2) LQ_CUDA(c, cudaMallocAsync(&flush, flush_bytes, c->stream));
  cudaEvent_t e0, e1;
  LQ_CUDA(c, cudaEventCreate(&e0));
  LQ_CUDA(c, cudaEventCreate(&e1));
  apply_M_prec(c->geo, prec, gauge, fin.ref(), fout.ref(), kappa, dagger != 0, c->stream, c->pair_sites, c->staged,
               c->df_prefetch);   // warm-up
  double total = 0.0;
  lq_status st = LQ_OK;
  if (flush_l2) {
    for (int i = 0; i < n && st == LQ_OK; ++i) {
      cudaMemsetAsync(flush, i & 0xff, flush_bytes, c->stream);
      cudaEventRecord(e0, c->stream);
      apply_M_prec(c->geo, prec, gauge, fin.ref(), fout.ref(), kappa, dagger != 0, c->stream, c->pair_sites, c->staged,
               c->df_prefetch);
      cudaEventRecord(e1, c->stream);
      st = cuda_check(c, cudaEventSynchronize(e1), "cudaEventSynchronize");
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      total += t;
    }
  } else {
    cudaEventRecord(e0, c->stream);
    for (int i = 0; i < n; ++i)
      apply_M_prec(c->geo, prec, gauge, fin.ref(), fout.ref(), kappa, dagger != 0, c->stream, c->pair_sites, c->staged,
               c->df_prefetch);
    cudaEventRecord(e1, c->stream);
    st = cuda_check(c, cudaEventSynchronize(e1), "cudaEventSynchronize");
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    total = t;
  }
  if (st == LQ_OK) st = cuda_check(c, cudaGetLastError(), "dslash launch");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (flush) cudaFreeAsync(flush, c->stream);
  cudaStreamSynchronize(c->stream);
  *ms = total / n;
  return st;
}

lq_status lq_plaquette(lq_ctx* c, double* plaq) {
  if (!c) return LQ_ERR_ARG;
  if (!plaq) return fail(c, LQ_ERR_ARG, "null output");
  LQ_TRY(require_gauge(c, LQ_F64));
  launch_plaquette(c->geo, c->gauge64, nullptr, c->rs, c->dscalar, c->stream);
  LQ_CUDA(c, cudaGetLastError());
  LQ_TRY(read_scalars(c));
  *plaq = c->dscalar_host[0] / (18.0 * c->geo.V);
  return LQ_OK;
}

lq_status lq_gauge_action(lq_ctx* c, double beta, double* S) {
  if (!c) return LQ_ERR_ARG;
  if (!S) return fail(c, LQ_ERR_ARG, "null output");
  LQ_TRY(require_gauge(c, LQ_F64));
  launch_plaquette(c->geo, c->gauge64, nullptr, c->rs, c->dscalar, c->stream);
  LQ_CUDA(c, cudaGetLastError());
  LQ_TRY(read_scalars(c));
  *S = beta * (6.0 * c->geo.V - c->dscalar_host[0] / 3.0);
  return LQ_OK;
}

lq_status lq_gauge_force(lq_ctx* c, double* F, double beta) {
  if (!c) return LQ_ERR_ARG;
  LQ_TRY(require_gauge(c, LQ_F64));
  LQ_TRY(ensure_md_fields(c));
  launch_gauge_force(c->geo, c->gauge64, c->force, beta, 0.0, false, c->stream);
  LQ_CUDA(c, cudaGetLastError());
  return deliver_mom(c, c->force, F);
}

lq_status lq_fermion_force(lq_ctx* c, double* F, const double* X, double kappa) {
  if (!c) return LQ_ERR_ARG;
  LQ_TRY(require_gauge(c, LQ_F64));
  LQ_TRY(ensure_md_fields(c));
  const double* dX = nullptr;
  LQ_TRY(stage_spinor_in(c, X, &dX));
  launch_pack_spinor(c->geo, dX, SStore::F64, c->x64.ref(), c->stream);
  apply_M_prec(c->geo, LQ_F64, c->gauge64, c->x64.ref(), c->y64.ref(), kappa, false, c->stream);
  launch_fermion_force(c->geo, c->gauge64, c->x64.ref(), c->y64.ref(), c->force, kappa, 0.0, false, c->stream);
  LQ_CUDA(c, cudaGetLastError());
  return deliver_mom(c, c->force, F);
}

lq_status lq_fermion_grad(lq_ctx* c, double* G, const double* X, double kappa) {
  if (!c) return LQ_ERR_ARG;
  if (!G) return fail(c, LQ_ERR_ARG, "null gradient buffer");
  if (!aligned16(G)) return fail(c, LQ_ERR_ARG, "gradient buffer not 16-byte aligned");
  LQ_TRY(require_gauge(c, LQ_F64));
  LQ_TRY(ensure_md_fields(c));
  const double* dX = nullptr;
  LQ_TRY(stage_spinor_in(c, X, &dX));
  launch_pack_spinor(c->geo, dX, SStore::F64, c->x64.ref(), c->stream);
  apply_M_prec(c->geo, LQ_F64, c->gauge64, c->x64.ref(), c->y64.ref(), kappa, false, c->stream);
  const size_t bytes = sizeof(double) * 72 * (size_t)c->geo.V;
  if (is_device_ptr(G)) {
    launch_fermion_grad(c->geo, c->x64.ref(), c->y64.ref(), G, kappa, c->stream);
    LQ_CUDA(c, cudaGetLastError());
    return LQ_OK;
  }
  if (!c->stage_gauge) LQ_CUDA(c, cudaMalloc(&c->stage_gauge, bytes));
  launch_fermion_grad(c->geo, c->x64.ref(), c->y64.ref(), c->stage_gauge, kappa, c->stream);
  LQ_CUDA(c, cudaGetLastError());
  LQ_CUDA(c, cudaMemcpyAsync(G, c->stage_gauge, bytes, cudaMemcpyDeviceToHost, c->stream));
  LQ_CUDA(c, cudaStreamSynchronize(c->stream));
  return LQ_OK;
}

lq_status lq_pseudofermion_action(lq_ctx* c, const double* phi, double kappa, double tol, int maxiter, int inner,
                                  int reliable_every, double* S, double* X) {
  if (!c) return LQ_ERR_ARG;
  if (!S) return fail(c, LQ_ERR_ARG, "null output");
  LQ_TRY(check_inner(c, inner));
  if (!(tol > 0.0) || maxiter <= 0 || reliable_every < 0)
    return fail(c, LQ_ERR_ARG, "bad tolerance or iteration limit");
  LQ_TRY(require_gauge(c, LQ_F64));
  LQ_TRY(ensure_solver_fields(c, inner));
  const double* dphi = nullptr;
  LQ_TRY(stage_spinor_in(c, phi, &dphi));
  launch_pack_spinor(c->geo, dphi, SStore::F64, c->phi64.ref(), c->stream);
  lq_solve_stats s{};
  LQ_TRY(solve_internal(c, kappa, tol, maxiter, inner, reliable_every, nullptr, 0, &s));
  launch_dot_re(c->geo, c->phi64.ref(), c->x64.ref(), c->rs, c->dscalar, c->stream);
  LQ_CUDA(c, cudaGetLastError());
  if (X) LQ_TRY(deliver_spinor(c, c->x64, X));
  LQ_TRY(read_scalars(c));
  *S = c->dscalar_host[0];
  return LQ_OK;
}

lq_status lq_link_update(lq_ctx* c, const double* p, double eps) {
  if (!c) return LQ_ERR_ARG;
  LQ_TRY(require_gauge(c, LQ_F64));
  LQ_TRY(ensure_md_fields(c));
  LQ_TRY(stage_mom_in(c, p, c->mom));
  launch_link_update(c->geo, c->gauge64, c->mom, eps, c->stream);
  LQ_CUDA(c, cudaGetLastError());
  gauge_changed(c);
  if (!is_device_ptr(p)) LQ_CUDA(c, cudaStreamSynchronize(c->stream));
  return LQ_OK;
}

lq_status lq_hmc_trajectory(lq_ctx* c, const lq_hmc_params* hp, double* p, const double* chi, double u,
                            lq_traj_result* out) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!c) return LQ_ERR_ARG;
  LQ_TRY(check_trajectory_args(c, hp, out));
  // heat bath inputs from the caller: p (momenta) and chi
  LQ_TRY(stage_mom_in(c, p, c->mom));
  const double* dchi = nullptr;
  LQ_TRY(stage_spinor_in(c, chi, &dchi));
  launch_pack_spinor(c->geo, dchi, SStore::F64, c->chi64.ref(), c->stream);
  return trajectory_after_heatbath(c, hp, u, p, out, t0, 2);
}

lq_status lq_hmc_trajectory_seeded(lq_ctx* c, const lq_hmc_params* hp, uint64_t seed, uint64_t traj_index,
                                   double* p_out, lq_traj_result* out) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!c) return LQ_ERR_ARG;
  if (!heatbath_counters_ok(seed, traj_index))
    return fail(c, LQ_ERR_ARG, "seed must fit in 32 bits and traj_index be below 2^30");
  LQ_TRY(check_trajectory_args(c, hp, out));
  // heat bath on the device: momenta and chi from their generator streams, u on the host
  launch_heatbath_momenta(c->geo, seed, traj_index, c->mom, nullptr, c->stream);
  launch_heatbath_chi(c->geo, seed, traj_index, c->chi64.ref(), nullptr, c->stream);
  LQ_CUDA(c, cudaGetLastError());
  return trajectory_after_heatbath(c, hp, metropolis_uniform(seed, traj_index), p_out, out, t0, 2);
}

lq_status lq_heatbath_draw(lq_ctx* c, uint64_t seed, uint64_t traj_index, double* p, double* chi, double* u) {
  if (!c) return LQ_ERR_ARG;
  if (!heatbath_counters_ok(seed, traj_index))
    return fail(c, LQ_ERR_ARG, "seed must fit in 32 bits and traj_index be below 2^30");
  for (const void* b : {(const void*)p, (const void*)chi})
    if (b && !aligned16(b)) return fail(c, LQ_ERR_ARG, "buffer not 16-byte aligned");
  if (p) {
    if (is_device_ptr(p)) {
      launch_heatbath_momenta(c->geo, seed, traj_index, nullptr, p, c->stream);
    } else {
      LQ_TRY(ensure_md_fields(c));
      launch_heatbath_momenta(c->geo, seed, traj_index, c->mom, nullptr, c->stream);
      LQ_CUDA(c, cudaGetLastError());
      LQ_TRY(deliver_mom(c, c->mom, p));
    }
    LQ_CUDA(c, cudaGetLastError());
  }
  if (chi) {
    if (is_device_ptr(chi)) {
      launch_heatbath_chi(c->geo, seed, traj_index, SpinorRef{nullptr, nullptr}, chi, c->stream);
    } else {
      launch_heatbath_chi(c->geo, seed, traj_index, SpinorRef{nullptr, nullptr}, c->stage_out, c->stream);
      LQ_CUDA(c, cudaGetLastError());
      LQ_CUDA(c, cudaMemcpyAsync(chi, c->stage_out, sizeof(double) * 24 * c->geo.V, cudaMemcpyDeviceToHost,
                                 c->stream));
      LQ_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    LQ_CUDA(c, cudaGetLastError());
  }
  if (u) *u = metropolis_uniform(seed, traj_index);
  return LQ_OK;
}

lq_status lq_apply_M_naive(lq_ctx* c, double* out, const double* in, double kappa, int dagger, int n, double* ms) {
  if (!c) return LQ_ERR_ARG;
  if (!out || !in || in == out || n < 0) return fail(c, LQ_ERR_ARG, "bad buffers or count");
  if (!is_device_ptr(out) || !is_device_ptr(in) || !aligned16(out) || !aligned16(in))
    return fail(c, LQ_ERR_ARG, "naive operator: device buffers, 16-byte aligned");
  LQ_TRY(require_gauge(c, LQ_F64));
  const size_t V = c->geo.V;
  int* nbr = nullptr;
  double* sgn = nullptr;
  double* Ucanon = nullptr;
  LQ_CUDA(c, cudaMallocAsync((void**)&nbr, sizeof(int) * 8 * V, c->stream));
  LQ_CUDA(c, cudaMallocAsync((void**)&sgn, sizeof(double) * 8 * V, c->stream));
  LQ_CUDA(c, cudaMallocAsync((void**)&Ucanon, sizeof(double) * 72 * V, c->stream));
  naive_setup(c, &nbr, &sgn);
  launch_unpack_gauge64(c->geo, c->gauge64, Ucanon, c->stream);
  launch_naive_dslash(c, nbr, sgn, Ucanon, in, out, kappa, dagger);
  lq_status st = cuda_check(c, cudaGetLastError(), "naive operator");
  if (st == LQ_OK && n > 0 && ms) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    for (int i = 0; i < n; ++i) launch_naive_dslash(c, nbr, sgn, Ucanon, in, out, kappa, dagger);
    cudaEventRecord(e1, c->stream);
    st = cuda_check(c, cudaEventSynchronize(e1), "cudaEventSynchronize");
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t / n;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  cudaFreeAsync(nbr, c->stream);
  cudaFreeAsync(sgn, c->stream);
  cudaFreeAsync(Ucanon, c->stream);
  lq_status fin = cuda_check(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  return st == LQ_OK ? fin : st;
}

lq_status lq_fermion_force_naive(lq_ctx* c, double* F, const double* X, double kappa, int n, double* ms) {
  if (!c) return LQ_ERR_ARG;
  if (!F || !X || n < 0) return fail(c, LQ_ERR_ARG, "bad buffers or count");
  if (!is_device_ptr(F) || !is_device_ptr(X) || !aligned16(F) || !aligned16(X))
    return fail(c, LQ_ERR_ARG, "naive force: device buffers, 16-byte aligned");
  LQ_TRY(require_gauge(c, LQ_F64));
  const size_t V = c->geo.V;
  int* nbr = nullptr;
  double *sgn = nullptr, *Ucanon = nullptr, *Y = nullptr, *Q = nullptr;
  LQ_CUDA(c, cudaMallocAsync((void**)&nbr, sizeof(int) * 8 * V, c->stream));
  LQ_CUDA(c, cudaMallocAsync((void**)&sgn, sizeof(double) * 8 * V, c->stream));
  LQ_CUDA(c, cudaMallocAsync((void**)&Ucanon, sizeof(double) * 72 * V, c->stream));
  LQ_CUDA(c, cudaMallocAsync((void**)&Y, sizeof(double) * 24 * V, c->stream));
  LQ_CUDA(c, cudaMallocAsync((void**)&Q, sizeof(double) * 72 * V, c->stream));
  naive_setup(c, &nbr, &sgn);
  launch_unpack_gauge64(c->geo, c->gauge64, Ucanon, c->stream);
  launch_naive_dslash(c, nbr, sgn, Ucanon, X, Y, kappa, 0);
  launch_naive_force(c, nbr, sgn, Ucanon, X, Y, Q, F, kappa);
  lq_status st = cuda_check(c, cudaGetLastError(), "naive force");
  if (st == LQ_OK && n > 0 && ms) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    for (int i = 0; i < n; ++i) launch_naive_force(c, nbr, sgn, Ucanon, X, Y, Q, F, kappa);
    cudaEventRecord(e1, c->stream);
    st = cuda_check(c, cudaEventSynchronize(e1), "cudaEventSynchronize");
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t / n;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  for (void* p : {(void*)nbr, (void*)sgn, (void*)Ucanon, (void*)Y, (void*)Q}) cudaFreeAsync(p, c->stream);
  lq_status fin = cuda_check(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  return st == LQ_OK ? fin : st;
}

lq_status lq_time_fermion_force(lq_ctx* c, const double* X, double kappa, int n, double* ms) {
  if (!c) return LQ_ERR_ARG;
  if (!ms || n <= 0) return fail(c, LQ_ERR_ARG, "need n > 0 and ms");
  LQ_TRY(require_gauge(c, LQ_F64));
  LQ_TRY(ensure_md_fields(c));
  const double* dX = nullptr;
  LQ_TRY(stage_spinor_in(c, X, &dX));
  launch_pack_spinor(c->geo, dX, SStore::F64, c->x64.ref(), c->stream);
  apply_M_prec(c->geo, LQ_F64, c->gauge64, c->x64.ref(), c->y64.ref(), kappa, false, c->stream);
  launch_fermion_force(c->geo, c->gauge64, c->x64.ref(), c->y64.ref(), c->force, kappa, 0.0, false, c->stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c->stream);
  for (int i = 0; i < n; ++i)
    launch_fermion_force(c->geo, c->gauge64, c->x64.ref(), c->y64.ref(), c->force, kappa, 0.0, false, c->stream);
  cudaEventRecord(e1, c->stream);
  lq_status st = cuda_check(c, cudaGetLastError(), "fermion force");
  lq_status sy = cuda_check(c, cudaEventSynchronize(e1), "cudaEventSynchronize");
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  *ms = t / n;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st == LQ_OK ? sy : st;
}

lq_status lq_time_cg_kernel(lq_ctx* c, const double* in, double kappa, int which, int prec, int n, double* ms) {
  if (!c) return LQ_ERR_ARG;
  if (!ms || n <= 0 || which < 0 || which > 3) return fail(c, LQ_ERR_ARG, "need 0 <= which <= 3, n > 0, ms");
  LQ_TRY(check_inner(c, prec));
  LQ_TRY(require_gauge(c, LQ_F64));
  LQ_TRY(require_gauge(c, prec));
  LQ_TRY(ensure_solver_fields(c, prec));
  const Geom& g = c->geo;
  const bool lo = prec != LQ_F64;
  const SStore s = spinor_store_of(prec);
  const int k = (int)s;
  Field& r = lo ? c->r_lo[k] : c->r64;
  Field& p = lo ? c->p_lo[k] : c->p64;
  Field& x = lo ? c->x_lo[k] : c->x64;
  const double* din = nullptr;
  LQ_TRY(stage_spinor_in(c, in, &din));
  launch_pack_spinor(g, din, SStore::F64, c->phi64.ref(), c->stream);
  // a state that never halts: stop2 = 0, no reliable updates, no iteration limit
  SolverState h{};
  h.maxiter = 0x7fffffff;
  *c->state_host = h;
  LQ_CUDA(c, cudaMemcpyAsync(c->state, c->state_host, sizeof(SolverState), cudaMemcpyHostToDevice, c->stream));
  launch_solver_init(g, c->phi64.ref(), s, x.ref(), s, r.ref(), s, p.ref(), c->state, c->rs, c->stream);
  if (lo) cglo_iteration(c, prec, kappa, c->stream);
  else cg64_iteration(c, kappa, c->stream);
  LQ_CUDA(c, cudaGetLastError());
  cudaEvent_t e0, e1;
  LQ_CUDA(c, cudaEventCreate(&e0));
  LQ_CUDA(c, cudaEventCreate(&e1));
  cudaEventRecord(e0, c->stream);
  for (int i = 0; i < n; ++i) {
    if (which == 0) {
      if (lo) cglo_iteration(c, prec, kappa, c->stream);
      else cg64_iteration(c, kappa, c->stream);
    } else if (which == 3) {
      launch_xpay_p(g, s, r.ref(), p.ref(), c->state, true, c->stream);
    } else {
      cg_step(c, prec, which, kappa, c->stream);
    }
  }
  cudaEventRecord(e1, c->stream);
  lq_status st = cuda_check(c, cudaEventSynchronize(e1), "cudaEventSynchronize");
  float tms = 0.f;
  cudaEventElapsedTime(&tms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == LQ_OK) st = cuda_check(c, cudaGetLastError(), "cg kernel launch");
  *ms = tms / n;
  return st;
}

}  // extern "C"
