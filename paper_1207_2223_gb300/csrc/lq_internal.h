// Host-side internals shared by the translation units of the library:
// the context object and the kernel launchers each unit provides.
#pragma once
#include <cuda_runtime.h>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "lq_device.cuh"
#include "lq_dslash.cuh"
#include "../../include/lq.h"

namespace lq {

constexpr int kNumPrec = 7;   // LQ_F64 .. LQ_I16_12
constexpr int kNumSStore = 6;

inline GStore gauge_store_of(int prec) {
  switch (prec) {
    case LQ_F64: return GStore::F64_18;
    case LQ_F32: return GStore::F32_18;
    case LQ_F32_12: return GStore::F32_12;
    case LQ_F16_12: return GStore::F16_12;
    case LQ_DF64: return GStore::DF64_18;
    case LQ_I16_12: return GStore::I16_12;
    default: return GStore::BF16_12;
  }
}
inline SStore spinor_store_of(int prec) {
  switch (prec) {
    case LQ_F64: return SStore::F64;
    case LQ_F32: case LQ_F32_12: return SStore::F32;
    case LQ_F16_12: return SStore::F16;
    case LQ_DF64: return SStore::DF64;
    case LQ_I16_12: return SStore::I16;
    default: return SStore::BF16;
  }
}
size_t spinor_bytes(SStore s, int V);        // chunk array only

// Storage of the low-precision solution x of a mixed solve: FP32 when the
// iteration vectors are 16-bit.  x is read and written once per iteration
// (not by the stencil), so FP32 costs 44 B per site each way.  It saves the
// per-site encode and decode of x in CG pass 2, and it keeps the accumulated
// correction free of 16-bit rounding.
constexpr SStore xlo_store(SStore s) {
  return (s == SStore::F16 || s == SStore::BF16 || s == SStore::I16) ? SStore::F32 : s;
}
size_t gauge_bytes(GStore g, int V);

// A spinor field in one storage format, owned by the context.
struct Field {
  SStore store = SStore::F64;
  void* data = nullptr;
  float* norm = nullptr;
  SpinorRef ref() const { return SpinorRef{data, norm}; }
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
};

}  // namespace lq

struct lq_ctx {
  lq::Geom geo{};
  int device = 0;
  cudaStream_t stream = nullptr;         // work stream (the caller's)
  cudaStream_t capture_stream = nullptr; // private stream used only to record graphs
  cudaEvent_t phase_ev[4] = {};          // phases of lq_solve_MdagM on the work stream
  std::string last_error;

  // gauge field: FP64 master copy and lazily built low-precision copies
  void* gauge64 = nullptr;
  void* gauge_lo[lq::kNumPrec] = {};
  bool gauge_lo_valid[lq::kNumPrec] = {};
  bool gauge_set = false;

  // canonical-layout staging buffers (device)
  double* stage_in = nullptr;            // V * 24 doubles
  double* stage_out = nullptr;           // V * 24 doubles
  double* stage_gauge = nullptr;         // V * 72 doubles

  // FP64 solver fields
  lq::Field phi64, x64, r64, p64, t64, tmp64;
  // low-precision solver fields, one set per storage format (indexed by SStore)
  lq::Field r_lo[lq::kNumSStore], p_lo[lq::kNumSStore], t_lo[lq::kNumSStore], x_lo[lq::kNumSStore];
  // double-float reliable updates: phi, the accumulated solution, M x, the residual
  lq::Field phi_df, x_df, tmp_df, r_df;

  // molecular dynamics: momenta / forces double [32][V], the start momenta,
  // the force buffer, the gauge field at the start of a trajectory, Y = M X
  // and the pseudofermion noise chi
  double* mom = nullptr;
  double* mom0 = nullptr;
  double* force = nullptr;
  double* stage_mom = nullptr;           // V * 32 doubles (canonical staging)
  void* gauge_old = nullptr;
  lq::Field y64, chi64;

  // reductions and solver scalars
  lq::ReduceScratch rs{};
  lq::SolverState* state = nullptr;      // device
  lq::SolverState* state_host = nullptr; // pinned mirror
  double* dscalar = nullptr;             // device scratch scalars [8]
  double* dscalar_host = nullptr;        // pinned mirror [8]

  std::map<std::tuple<int, int, int, double>, lq::GraphEntry> graphs;
  void* batch = nullptr;                 // workspace of lq_solve_batch (k_batch.cu)
  int use_graphs = 1;                    // CG iterations as CUDA graphs (lq_set_option)
  int df_updates = 1;                    // double-float intermediate reliable updates (lq_set_option)
  int pair_sites = 0;                    // two-site packed stencil for 16-bit storage (lq_set_option)
  int staged = 0;                        // links shared in-block through shared memory (lq_set_option)
  int batch_rb = 0;                      // batched solves: right-hand sides per thread (0: autotuned)
  int batch_persistent = 0;              // batched solves: one cooperative launch per chunk of iterations
  int batch_barrier_extra = 0;           // batched solves: phantom blocks the barrier waits for (timeout tests)
  int batch_device_loop = 1;             // batched solves: the whole solve as one graph with conditional nodes
  int batch_order = 0;                   // batched solves: tile order (0 tuned, 1 site-major, 2 group-major)
  int host_direct = 1;                   // kernels read / write mapped page-locked host buffers in place
  int df_prefetch = 0;                   // double-float operator: next hop's operands prefetched to shared memory
};

namespace lq {

// ---- naive operator for the register ablation (k_naive.cu)
void naive_setup(lq_ctx* c, int** nbr, double** sgn);
void launch_naive_dslash(lq_ctx* c, const int* nbr, const double* sgn, const double* Ucanon, const double* in,
                         double* out, double kappa, int dagger);
// naive fermion force: X, Y canonical, Q scratch [4V][18], F canonical [V][4][8]
void launch_naive_force(lq_ctx* c, const int* nbr, const double* sgn, const double* Ucanon, const double* X,
                        const double* Y, double* Q, double* F, double kappa);

// ---- batched solves (k_batch.cu)
void destroy_batch_work(void* w);

// ---- layout (k_layout.cu)
void launch_pack_gauge64(const Geom& g, const double* canon, void* soa, cudaStream_t st);
void launch_unpack_gauge64(const Geom& g, const void* soa, double* canon, cudaStream_t st);
void launch_convert_gauge(const Geom& g, const void* soa64, GStore dst, void* out, cudaStream_t st);
void launch_pack_spinor(const Geom& g, const double* canon, SStore s, SpinorRef out, cudaStream_t st);
void launch_unpack_spinor(const Geom& g, SStore s, SpinorRef in, double* canon, cudaStream_t st);
// FP64 <-> double-float field conversion
void launch_convert_spinor(const Geom& g, SStore a, SpinorRef in, SStore b, SpinorRef out, cudaStream_t st);

// ---- BLAS-1 (k_blas.cu)
// phi2 = |phi|^2 -> state; x = 0; r = phi; p = phi (each in its own format)
void launch_solver_init(const Geom& g, SpinorRef phi64, SStore sx, SpinorRef x, SStore sr, SpinorRef r,
                        SStore sp, SpinorRef p, SolverState* st, const ReduceScratch& rs, cudaStream_t stream);
// p = r + beta p (skipped when halted unless forced)
void launch_xpay_p(const Geom& g, SStore s, SpinorRef r, SpinorRef p, SolverState* st, bool forced,
                   cudaStream_t stream);
// x_hi += x_lo ; x_lo = 0
void launch_accumulate_x(const Geom& g, SStore slo, SpinorRef xlo, SpinorRef xhi, cudaStream_t stream);
// after a true-residual pass: beta = rr_true / rr_prev (0 when restart), rr = rr_ref = rr_true, resume
void launch_state_after_residual(SolverState* st, int restart, cudaStream_t stream);
void launch_zero_spinor(const Geom& g, SStore s, SpinorRef f, cudaStream_t stream);
// x = 0, r = p = src64 in format s (restart of the inner iteration)
void launch_inner_restart(const Geom& g, SpinorRef src64, SStore s, SpinorRef x, SpinorRef r, SpinorRef p,
                          cudaStream_t stream);

// ---- Wilson operator applications (k_apply.cu): out = M in or M^dag in
// (pair: the two-site packed stencil where it applies, 16-bit fixed point)
// (staged: the stencil that shares x and y links inside a block through shared memory,
// FP32-arithmetic formats)
void apply_M_prec(const Geom& g, int prec, const void* gauge, SpinorRef in, SpinorRef out, double kappa,
                  bool dagger, cudaStream_t stream, bool pair = false, bool staged = false,
                  bool df_prefetch = false);

// ---- two-site packed stencil for 16-bit fixed-point storage (k_pair.cu);
// it pairs x with x + L_t/2 in time, so it needs an even L_t
inline bool pair_geometry(const Geom& g) { return g.L[3] % 2 == 0; }
void pair_apply(const Geom& g, const void* gauge, SpinorRef in, SpinorRef out, double kappa, bool dagger,
                cudaStream_t stream);
void pair_cg1(lq_ctx* c, const void* gauge, double kappa, cudaStream_t stream);   // t = M p, |t|^2
void pair_cg2(lq_ctx* c, const void* gauge, double kappa, cudaStream_t stream);   // r -= alpha M^dag t, x += alpha p

// ---- FP64 CG pieces (k_cg64.cu)
void cg64_iteration(lq_ctx* c, double kappa, cudaStream_t stream);
void cg64_true_residual(lq_ctx* c, double kappa, int store_lo_prec, cudaStream_t stream);

// ---- double-float reliable update (k_cgdf.cu): x_df += x_lo; r = phi_df - M^dag M x_df
// stored as r_df and in the inner format r_lo[prec]; |r|^2 -> state->rr_true
void df_reliable_update(lq_ctx* c, double kappa, int inner_prec, cudaStream_t stream);
// x_df += x_lo; x_lo = 0 (no residual)
void df_accumulate(lq_ctx* c, int inner_prec, cudaStream_t stream);
// x = 0, r = p = src in format s, from a double-float residual
void launch_inner_restart_df(const Geom& g, SpinorRef src, SStore s, SpinorRef x, SpinorRef r, SpinorRef p,
                             cudaStream_t stream);

// ---- low-precision CG iteration (k_cglo.cu)
void cglo_iteration(lq_ctx* c, int prec, double kappa, cudaStream_t stream);
// single steps (which = 1: t = M p with |t|^2; 2: r -= alpha M^dag t, x += alpha p, |r|^2)
void cg64_step(lq_ctx* c, int which, double kappa, cudaStream_t stream);
void cglo_step(lq_ctx* c, int prec, int which, double kappa, cudaStream_t stream);
inline void cg_step(lq_ctx* c, int prec, int which, double kappa, cudaStream_t stream) {
  if (prec == LQ_F64) cg64_step(c, which, kappa, stream);
  else cglo_step(c, prec, which, kappa, stream);
}

}  // namespace lq

namespace lq {
// ---- heat bath on the device (k_heatbath.cu): momenta into the SoA [32][V] and/or the
// canonical [V][4][8]; chi into an FP64 field and/or a canonical spinor; the Metropolis
// uniform (host); counters are 32-bit words (seed < 2^32, traj < 2^30)
bool heatbath_counters_ok(uint64_t seed, uint64_t traj);
void launch_heatbath_momenta(const Geom& g, uint64_t seed, uint64_t traj, double* soa, double* canon,
                             cudaStream_t st);
void launch_heatbath_chi(const Geom& g, uint64_t seed, uint64_t traj, SpinorRef soa, double* canon, cudaStream_t st);
double metropolis_uniform(uint64_t seed, uint64_t traj);

// ---- gauge side (k_gauge.cu); momenta / forces are double [32][V]
void launch_plaquette(const Geom& g, const void* ga, const void* gb, const ReduceScratch& rs, double* out,
                      cudaStream_t st);
void launch_gauge_force(const Geom& g, const void* gauge, double* f, double beta, double eps, bool update,
                        cudaStream_t st);
void launch_link_update(const Geom& g, void* gauge, const double* p, double eps, cudaStream_t st);
void launch_pack_mom(const Geom& g, const double* canon, double* soa, cudaStream_t st);
void launch_unpack_mom(const Geom& g, const double* soa, double* canon, cudaStream_t st);
void launch_kinetic_diff(const Geom& g, const double* p, const double* p0, const ReduceScratch& rs, double* out,
                         cudaStream_t st);
// ---- fermion side (k_force.cu)
void launch_fermion_force(const Geom& g, const void* gauge, SpinorRef X, SpinorRef Y, double* f, double kappa,
                          double eps, bool update, cudaStream_t st);
void launch_fermion_grad(const Geom& g, SpinorRef X, SpinorRef Y, double* G, double kappa, cudaStream_t st);
void launch_dot_re(const Geom& g, SpinorRef a, SpinorRef b, const ReduceScratch& rs, double* out, cudaStream_t st);
void launch_fermion_action_diff(const Geom& g, SpinorRef phi, SpinorRef X, SpinorRef chi, const ReduceScratch& rs,
                                double* out, cudaStream_t st);
}  // namespace lq
