/*
 * lq.h - C interface of a GB300 (sm_103a) library for two-flavour
 * Wilson-fermion Hybrid Monte Carlo, following Chakrabarty & Majumdar,
 * "Hybrid Monte Carlo with Wilson Dirac operator on the Fermi GPU".
 *
 * The paper's program applies the Wilson-Dirac matrix M = D + m and its
 * adjoint to the pseudofermion field inside a conjugate-gradient inversion
 * of M^dag M (Eq. 4, Sec. 1 and Sec. 3 kernel 1), computes the gauge and
 * fermion driving forces (Sec. 3 kernels 2 and 3), evolves momenta and
 * links by leapfrog (Sec. 3 kernel 4; Sec. 2) and accepts or rejects the
 * trajectory on H_new - H_old (Eq. 5; Sec. 3, trajectory step 3).  Each
 * entry point below is one of those operations.
 *
 * Conventions (the paper fixes none of them; these are the readings the
 * library takes and its tests pin):
 *   lattice     Lx x Ly x Lz x Lt, direction mu = 0..3 = x, y, z, t,
 *               site s = x + Lx*(y + Ly*(z + Lz*t))
 *   operator    M psi(x) = psi(x) - kappa sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu)
 *                                              + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
 *               (Wilson r = 1, hopping-parameter normalisation, M^dag = g5 M g5),
 *               gamma matrices in the DeGrand-Rossi basis
 *   boundary    periodic in x, y, z; antiperiodic in t when t_antiperiodic != 0
 *   su(3)       t_a = lambda_a / sqrt(2), p = sum_a p_a t_a, kinetic term (1/2) sum p_a^2
 *
 * Canonical buffer layouts (all FP64, complex numbers interleaved re, im):
 *   gauge field   double [V][4][3][3][2]   U_mu(s) row-major
 *   spinor        double [V][4][3][2]      spin-major, colour fastest
 *   momentum /
 *   force         double [V][4][8]         su(3) coefficients
 * Every buffer argument may live in device memory or in host memory (the
 * library asks the CUDA runtime which).  Buffers must be 16-byte aligned.
 * The caller owns every buffer it passes; the context owns its internal
 * copies (site-major structure-of-arrays, several precisions) and
 * workspaces, and frees them in lq_destroy.
 *
 * Ordering: work is issued on the context's CUDA stream.  A call whose
 * arguments are all device buffers and that returns no host scalar is
 * asynchronous; a call that writes a host buffer or a host scalar
 * synchronises the stream before it returns.
 *
 * Errors: every call returns an lq_status; nothing throws across this
 * interface.  lq_last_error() returns a description of the last failure
 * on that context.  A context must not be used from two host threads at
 * the same time.
 */
#ifndef LQ_H
#define LQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lq_ctx lq_ctx;

typedef enum {
  LQ_OK = 0,
  LQ_ERR_ARG = 1,            /* bad argument: null pointer, misaligned buffer, bad precision, ... */
  LQ_ERR_SHAPE = 2,          /* lattice extents not allowed */
  LQ_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  LQ_ERR_NOT_CONVERGED = 4,  /* iteration limit reached; the best iterate was still written */
  LQ_ERR_NAN = 5,            /* a non-finite value appeared (input or breakdown) */
  LQ_ERR_STATE = 6,          /* call out of order, e.g. no gauge field set yet */
  LQ_ERR_TIMEOUT = 7         /* a bounded device-side wait gave up (persistent batched iteration) */
} lq_status;

/* Storage / arithmetic precision of the operator and of the inner solver.
 *   LQ_F64      FP64 links (18 reals) and spinors, FP64 arithmetic
 *   LQ_F32      FP32 links (18 reals) and spinors, FP32 arithmetic
 *   LQ_F32_12   FP32 links stored as 12 reals (row 3 rebuilt), FP32 spinors
 *   LQ_F16_12   FP16 links (12 reals), FP16 spinors scaled by a per-site FP32 norm,
 *               FP32 arithmetic
 *   LQ_BF16_12  as LQ_F16_12 with BF16 storage
 *   LQ_DF64     links and spinors as double-float pairs (hi + lo FP32, ~48 bits),
 *               double-float arithmetic on the FP32 pipe: operator applications only
 *               (lq_apply_M, lq_apply_MdagM, lq_time_dslash); the solver can use it for
 *               its intermediate reliable updates (LQ_OPT_DF64_UPDATES)
 *   LQ_I16_12   16-bit fixed point: links (12 reals) as q/32767, spinors as q/32767
 *               times a per-site FP32 norm (15 bits relative to the site maximum),
 *               FP32 arithmetic */
typedef enum { LQ_F64 = 0, LQ_F32 = 1, LQ_F32_12 = 2, LQ_F16_12 = 3, LQ_BF16_12 = 4, LQ_DF64 = 5,
               LQ_I16_12 = 6 } lq_prec;

typedef struct {
  int iterations;           /* CG iterations (inner iterations for a mixed solve) */
  int reliable_updates;     /* FP64 true-residual recomputations that fed back into the solve */
  int restarts;             /* restarts of the search direction from the true residual */
  int converged;            /* 1 when true_rel_resid <= tol */
  double true_rel_resid;    /* ||phi - M^dag M x|| / ||phi||, recomputed in FP64 */
  double seconds;           /* host wall-clock of the call, from entry to the final synchronisation */
  int64_t kernel_launches;  /* kernels this call launched (every node of a CUDA graph counts once) */
  int escalations;          /* times the inner precision was raised to FP32 because it stagnated */
  /* lq_solve_MdagM only (0 elsewhere): time on the context's stream (CUDA events) of staging
   * the right-hand side (host-to-device copy and packing), of the solve, and of delivering
   * the solution (unpacking and the device-to-host copy) */
  double stage_ms, solve_ms, deliver_ms;
} lq_solve_stats;

/* Library version string. */
const char* lq_version(void);

/* Create a context for an Lx x Ly x Lz x Lt lattice (dims[0..3] = Lx, Ly,
 * Lz, Lt, each >= 2, V = product < 2^31 / 64), on the current CUDA device,
 * issuing work on `cuda_stream` (a cudaStream_t; NULL = the legacy default
 * stream).  Lattice of Sec. 1 ("Lambda", N_site points, d x N_site links).
 * Errors: LQ_ERR_ARG (null out), LQ_ERR_SHAPE, LQ_ERR_CUDA. */
lq_status lq_create(lq_ctx** out, const int dims[4], int t_antiperiodic, void* cuda_stream);

/* Free the context and everything it owns.  Synchronises its stream. */
lq_status lq_destroy(lq_ctx* ctx);

/* Description of the last error on ctx (never NULL; "" when none). */
const char* lq_last_error(const lq_ctx* ctx);

/* Issue subsequent work on another stream (a cudaStream_t). */
lq_status lq_set_stream(lq_ctx* ctx, void* cuda_stream);

/* Options of a context.
 *   LQ_OPT_CUDA_GRAPHS  1 (default): CG iterations are recorded once as CUDA graphs and
 *                       replayed; 0: every kernel is launched from the host (to measure
 *                       the launch overhead the graphs remove; paper Sec. 4, Fig. 1 reads
 *                       a per-call overhead off CG time against iteration count).
 *   LQ_OPT_DF64_UPDATES 1 (default): the intermediate reliable updates of a mixed-precision
 *                       solve in double-float arithmetic (LQ_DF64, ~48 bits) on the FP32 pipe,
 *                       the final residual always recomputed and certified in FP64 (an update
 *                       triggered by the iterated residual meeting tol goes straight to the
 *                       FP64 certification); 0: every reliable update in FP64.  Same
 *                       iterations; on GB300 the double-float operator takes 1.5 ms against
 *                       3.3 ms for FP64 at 32^3 x 64.  Batched solves (lq_solve_batch) read
 *                       the option of their first context: double-float updates per column,
 *                       FP64 certification once every column is frozen, which reopens a
 *                       column whose FP64 residual misses tol.
 *   LQ_OPT_PAIR_SITES   0 (default): one site per thread; 1: with LQ_I16_12 and an even
 *                       L_t, the operator and the CG passes apply the stencil at two sites
 *                       per thread (x and x + L_t/2 in time) with packed FP32x2 arithmetic.
 *                       Same operator, results differ only by FP32 rounding.  (On this part
 *                       option 1 issues 35% fewer instructions but is slower: a packed FMA
 *                       holds the FMA pipe for two cycles and the occupancy halves.)
 *   LQ_OPT_STAGED       0 (default): every thread loads and decodes the links of its eight hops;
 *                       1: with an FP32-arithmetic precision, a block of 256 consecutive sites
 *                       decodes each x and y link once for the forward hop of x and the backward
 *                       hop of x+mu, handing the latter to the neighbour's thread through shared
 *                       memory (Sec. 3 kernel 1 with in-block sharing); the operator and the CG
 *                       passes.  Same operator, results differ only by FP32 rounding order.
 *   LQ_OPT_BATCH_RHS_PER_THREAD  0 (default): lq_solve_batch tunes its launch shape; 1..4:
 *                       every thread applies each link to this many right-hand sides (must
 *                       divide nrhs), 256 threads per block, no timing.  Changing it drops
 *                       the batch workspace of the context.
 *   LQ_OPT_BATCH_PERSISTENT  0 (default): lq_solve_batch runs its iterations as CUDA graphs of
 *                       one launch per CG pass (LQ_OPT_BATCH_DEVICE_LOOP says how the host
 *                       drives them); 1: one persistent cooperative launch per chunk
 *                       of reliable_every iterations runs every pass of every iteration, with
 *                       device-wide barriers between the passes.  The barrier waits are
 *                       bounded (about one second); a wait that runs out makes the call
 *                       return LQ_ERR_TIMEOUT and leaves the context usable.
 *   LQ_OPT_BATCH_DEVICE_LOOP  1 (default): without the persistent launch, lq_solve_batch runs
 *                       the whole solve as one CUDA graph whose conditional nodes (a while
 *                       loop over CG iterations inside a while loop over reliable updates,
 *                       if nodes around the double-float residual and the FP64
 *                       certification) take every convergence decision on the device; the
 *                       host waits once.  Each loop stops at a cap taken from maxiter.
 *                       0: the host launches a graph of reliable_every iterations, runs the
 *                       reliable update and reads the state back once per chunk.
 *   LQ_OPT_BATCH_TILE_ORDER  0 (default): the autotuner of lq_solve_batch tries both tile orders;
 *                       1: site-major only (the right-hand-side groups of one site tile are
 *                       consecutive tiles); 2: group-major only (every site tile of one group,
 *                       then the next).  With LQ_OPT_BATCH_RHS_PER_THREAD set, 0 and 1 mean
 *                       site-major.  Changing it drops the batch workspace of the context.
 *   LQ_OPT_DF64_PREFETCH  0 (default): the double-float operator (LQ_DF64 applications and the
 *                       double-float reliable updates) loads each hop's links and spinors as
 *                       it needs them; 1: a variant that copies the next hop's operands into
 *                       shared memory with asynchronous copies while the current hop computes.
 *                       Same arithmetic in the same order: identical results.  Measured slower
 *                       on GB300 (1.64 against 1.50 ms at 32^3 x 64), so off.
 *   LQ_OPT_HOST_DIRECT  1 (default): page-locked host buffers mapped into the device's address
 *                       space are read (gauge field, right-hand sides) and written (solutions,
 *                       lq_gauge_get) in place by the packing kernels, which access the
 *                       canonical records in contiguous runs; 0: they are copied through
 *                       device staging buffers (cudaMemcpyAsync).  Pageable host buffers are
 *                       always staged.  On the GB300 machine the in-place path moves 1.6 GB in
 *                       and 0.4 GB out per solve at the copy engines' rate without the
 *                       occasional 10x slower staged copy.
 *   LQ_OPT_BATCH_BARRIER_TEST  0 (default); 1: the persistent iteration's barrier also waits for
 *                       one block that does not exist, so every wait runs out: exercises the
 *                       LQ_ERR_TIMEOUT path (tests of the failure detection only). */
enum { LQ_OPT_CUDA_GRAPHS = 1, LQ_OPT_DF64_UPDATES = 2, LQ_OPT_PAIR_SITES = 3, LQ_OPT_STAGED = 4,
       LQ_OPT_BATCH_RHS_PER_THREAD = 5, LQ_OPT_BATCH_PERSISTENT = 6, LQ_OPT_BATCH_BARRIER_TEST = 7,
       LQ_OPT_BATCH_DEVICE_LOOP = 8, LQ_OPT_HOST_DIRECT = 9, LQ_OPT_BATCH_TILE_ORDER = 10,
       LQ_OPT_DF64_PREFETCH = 11 };
lq_status lq_set_option(lq_ctx* ctx, int option, int value);

/* Number of lattice sites V. */
int64_t lq_volume(const lq_ctx* ctx);

/* Load the gauge field U_{n,mu} in SU(3) (Sec. 1: "U_{n,mu} ... defined on
 * the link (n, mu)"), canonical layout, host or device.  Low-precision
 * copies are rebuilt from it on first use.  Links stored with 12 reals are
 * reconstructed assuming det U = 1.  Errors: LQ_ERR_ARG. */
lq_status lq_gauge_set(lq_ctx* ctx, const double* U);

/* Copy the context's current gauge field to U (canonical layout). */
lq_status lq_gauge_get(lq_ctx* ctx, double* U);

/* out = M in (dagger = 0) or M^dag in (dagger = 1) in precision `prec`
 * (Eq. 4; Sec. 3 kernel 1: the Dirac operator and its hermitian conjugate
 * acting on the pseudofermion field).  in and out are canonical spinors
 * and must not overlap.  Low precisions convert on the way in and out.
 * Errors: LQ_ERR_ARG, LQ_ERR_STATE (no gauge field). */
lq_status lq_apply_M(lq_ctx* ctx, double* out, const double* in, double kappa, int dagger, int prec);

/* out = M^dag M in, precision `prec` (the matrix of Eq. 4). */
lq_status lq_apply_MdagM(lq_ctx* ctx, double* out, const double* in, double kappa, int prec);

/* Solve M^dag M x = phi by conjugate gradient (Sec. 1 after Eq. 3; Sec. 3,
 * "conjugate gradient routine") from x0 = 0, until the FP64 true residual
 * ||phi - M^dag M x|| / ||phi|| <= tol.
 *   inner_prec      LQ_F64: plain FP64 CG.  Otherwise the iterations run
 *                   in that precision (the low-precision solution is kept
 *                   in FP32 when the precision is a 16-bit format) and the
 *                   solution and residual are corrected in FP64 ("reliable
 *                   updates"): the low-precision solution is added to the
 *                   FP64 one and the FP64 residual is recomputed after
 *                   `reliable_every` iterations (0: no fixed interval), or
 *                   sooner when the iterated residual has dropped by a
 *                   factor 100 since the last update (10 for LQ_BF16_12),
 *                   and when it has met tol.  If three reliable updates in
 *                   a row fail to halve the true residual, the iterations
 *                   continue in FP32 from there (counted in
 *                   stats->escalations).
 *   maxiter         iteration limit (> 0)
 *   hist, hist_len  optional host array receiving the relative iterated
 *                   residual of each iteration (NULL / 0 to skip)
 *   stats           optional, filled on return
 * x receives the FP64 solution, also when LQ_ERR_NOT_CONVERGED is returned.
 * phi = 0 gives x = 0.  Synchronises.  Errors: LQ_ERR_ARG, LQ_ERR_STATE,
 * LQ_ERR_NOT_CONVERGED, LQ_ERR_NAN (non-finite input or CG breakdown). */
lq_status lq_solve_MdagM(lq_ctx* ctx, double* x, const double* phi, double kappa, double tol, int maxiter,
                         int inner_prec, int reliable_every, double* hist, int hist_len,
                         lq_solve_stats* stats);

/* Batched CG: n independent systems solved together, one launch per CG pass
 * (the CG routine of Sec. 3 over a batch).  System k is the lattice and gauge
 * field of ctxs[k] (volumes and kappa[k] may differ; all contexts on one
 * device) with nrhs right-hand sides phi[k] (device, canonical spinors stored
 * one after another: [nrhs][V_k][4][3] complex), solution x[k] (device, same
 * layout).  Right-hand sides of one system share its links, which are read
 * once per site for all of them: a thread applies each decoded link to several right-hand
 * sides held in registers.  Iterations run in FP32 arithmetic on the storage
 * of inner_prec (LQ_F32, LQ_F32_12, LQ_F16_12, LQ_BF16_12 or LQ_I16_12) with reliable updates
 * every reliable_every iterations (sooner when a column's iterated residual fell by 1e-2,
 * 16-bit storage, or 1e-3, FP32; a column whose true residual turns out far above its
 * iterated one restarts its search direction): double-float updates per column
 * (LQ_OPT_DF64_UPDATES of ctxs[0]), and once every column meets tol an FP64
 * certification that reopens any column whose FP64 true residual misses it; the solve
 * ends when every column's FP64 true residual meets tol.  1 <= n <= 16, 1 <= nrhs <= 16,
 * n * nrhs <= 64.  The launch shape (tile order, threads per block, right-hand sides per
 * thread, resident blocks per SM) is picked by timing the candidates on the first call
 * for a batch shape (autotuning; lq_batch_tuning reports the choice).  Everything runs on
 * ctxs[0]'s stream, which owns the workspace: by default the whole solve as one CUDA
 * graph with conditional nodes (LQ_OPT_BATCH_DEVICE_LOOP), or per-chunk graphs, or
 * persistent launches (LQ_OPT_BATCH_PERSISTENT).
 *   hist     optional host array [n * nrhs][hist_len]: relative iterated residual
 *            of every column per iteration
 *   iters    optional host int[n * nrhs]: iterations until each column was frozen
 *   resid    optional host double[n * nrhs]: final FP64 true relative residuals
 * Synchronises.  Errors: LQ_ERR_ARG (host buffers, sizes), LQ_ERR_SHAPE (more than 2^30
 * sites x right-hand sides in all), LQ_ERR_STATE, LQ_ERR_NOT_CONVERGED, LQ_ERR_NAN,
 * LQ_ERR_TIMEOUT (persistent launch), LQ_ERR_CUDA (message on ctxs[0]). */
lq_status lq_solve_batch(lq_ctx** ctxs, int n, double** x, const double** phi, const double* kappa, int nrhs,
                         double tol, int maxiter, int inner_prec, int reliable_every, double* hist, int hist_len,
                         int* iters, double* resid, lq_solve_stats* stats);

/* The launch shape the autotuner of lq_solve_batch picked for the last batch shape solved
 * with ctx as ctxs[0]: threads per block (= sites per tile), right-hand sides per thread,
 * resident blocks per SM (0: all that fit), tile order (1: site-major, the right-hand-side
 * groups of one site tile are consecutive tiles; 0: group-major); ms[0 .. ms_len) receives
 * the measured time of one iteration for every candidate in the order tried (site-major
 * first, then group-major; in each, rhs per thread 1, 2, 3, 4 among the divisors of nrhs;
 * for each, 256 threads with all blocks, 256 threads with one block per SM, 128 threads).
 * Any output may be NULL.  Errors: LQ_ERR_STATE (no batched solve yet). */
lq_status lq_batch_tuning(lq_ctx* ctx, int* tile, int* rhs_per_thread, int* blocks_per_sm, int* site_major,
                          double* ms, int ms_len);

/* ---------------------------------------------------------------- MD */

/* Parameters of one HMC trajectory (Sec. 3, the three steps of the evolution). */
typedef struct {
  double beta;          /* gauge coupling of the Wilson plaquette action */
  double kappa;         /* hopping parameter */
  double tau;           /* trajectory length; step eps = tau / n_steps */
  int n_steps;          /* leapfrog steps (> 0) */
  double tol;           /* CG tolerance of every solve (FP64 true relative residual) */
  int maxiter;          /* CG iteration limit per solve */
  int inner_prec;       /* lq_prec of the CG iterations (LQ_F64 or mixed) */
  int reliable_every;   /* reliable-update interval of mixed solves */
} lq_hmc_params;

typedef struct {
  double dH, dK, dSg, dSf;   /* H_new - H_old and its kinetic, gauge and pseudofermion parts */
  int accepted;              /* Metropolis decision */
  double plaquette;          /* of the configuration kept (accepted or restored) */
  int solves;                /* CG solves in the trajectory (n_steps + 2) */
  int64_t cg_iterations;     /* their total iterations */
  int64_t kernel_launches;   /* kernels launched by the call */
  double seconds;            /* host wall-clock of the call */
  /* device time per routine (CUDA events), the paper's per-routine timing (Sec. 4) */
  double seconds_solve;          /* CG solves (the inversions) */
  double seconds_gauge_force;    /* gauge force fused with the momentum update */
  double seconds_fermion_force;  /* Y = M X and the fermion force fused with the momentum update */
  double seconds_link_update;    /* exp(i eps p) U and reunitarisation */
} lq_traj_result;

/* Average plaquette <Re tr U_P / 3> over the 6 V plaquettes (1 for U = 1);
 * the measurement made at the end of each trajectory (Sec. 3).  Synchronises. */
lq_status lq_plaquette(lq_ctx* ctx, double* plaq);

/* Wilson gauge action S_g = beta sum_P (1 - Re tr U_P / 3) (S_g of Eq. 1, 5).
 * Synchronises. */
lq_status lq_gauge_action(lq_ctx* ctx, double beta, double* S);

/* Gauge force F_a(x, mu) = dS_g / d omega_a under U_mu(x) -> exp(i omega_a t_a) U_mu(x),
 * i.e. (beta/3) Im tr(t_a U_mu(x) Sigma_mu(x)) with the six staples Sigma_mu
 * (Sec. 3 kernel 2).  F: canonical [V][4][8].  FP64. */
lq_status lq_gauge_force(lq_ctx* ctx, double* F, double beta);

/* Fermion force F_a(x, mu) = dS_f / d omega_a for S_f = phi^dag (M^dag M)^{-1} phi, given
 * the solution X = (M^dag M)^{-1} phi (canonical spinor); Y = M X is formed inside
 * (Sec. 3 kernel 3).  F: canonical [V][4][8].  FP64. */
lq_status lq_fermion_force(lq_ctx* ctx, double* F, const double* X, double kappa);

/* Complex gradient G = dS_f / dconj(U) of S_f = phi^dag (M^dag M)^{-1} phi with respect
 * to the entries of the gauge field, given X = (M^dag M)^{-1} phi: the convention of
 * torch.autograd for a real function of complex inputs (dS = Re sum conj(G) dU).  The
 * su(3) force of lq_fermion_force is F_a = -Im tr(t_a U G^dag).  Adjoint of the fermion
 * part of Eq. 5 (the derivative behind Sec. 3 kernel 3).  G: canonical [V][4][3][3]
 * complex.  FP64. */
lq_status lq_fermion_grad(lq_ctx* ctx, double* G, const double* X, double kappa);

/* S_f = phi^dag (M^dag M)^{-1} phi (the pseudofermion term of Eq. 4, 5): one solve
 * (arguments as in lq_solve_MdagM) and an FP64 reduction; *S on the host; X, when not
 * NULL, receives the solution.  Synchronises. */
lq_status lq_pseudofermion_action(lq_ctx* ctx, const double* phi, double kappa, double tol, int maxiter,
                                  int inner_prec, int reliable_every, double* S, double* X);

/* Link update U_mu(x) <- exp(i eps P_mu(x)) U_mu(x), P = sum_a p_a t_a, then
 * reunitarisation (Gram-Schmidt rows 1, 2; row 3 = conj(row1 x row2)) (Sec. 3
 * kernel 4; Sec. 2: U and exp(ip) conjugate).  p: canonical [V][4][8].  The
 * context's gauge field changes. */
lq_status lq_link_update(lq_ctx* ctx, const double* p, double eps);

/* One HMC trajectory on the context's gauge field (Eq. 5; Sec. 2; Sec. 3 steps 1-3):
 *   heat bath   p (canonical [V][4][8], su(3) coefficients N(0,1)) and chi
 *               (canonical spinor, density exp(-chi^dag chi)) are the caller's draws;
 *               phi = M^dag chi; S_f at the start is chi^dag chi
 *   leapfrog    p -= eps/2 F; n_steps x (U <- exp(i eps p) U; p -= eps F), the
 *               last momentum step eps/2; F = gauge + fermion force, every solve
 *               from x0 = 0 to the tolerance of params
 *   Metropolis  accept iff u < exp(-Delta H), u in [0, 1) the caller's draw;
 *               Delta H summed from per-site differences in FP64
 * On return p holds the momenta at the end of the leapfrog, the context holds
 * the new links if accepted and the old ones otherwise.  A failed solve leaves
 * the old links and returns its status.  Synchronises. */
lq_status lq_hmc_trajectory(lq_ctx* ctx, const lq_hmc_params* params, double* p, const double* chi, double u,
                            lq_traj_result* result);

/* One HMC trajectory with its heat bath drawn on the device (Sec. 2: Gaussian momenta
 * at the start of every trajectory; Sec. 3 step 1: chi Gaussian, phi = M^dag chi; Sec. 3
 * step 3: the Metropolis test), otherwise as lq_hmc_trajectory.  The random numbers come
 * from the counter-based generator Philox4x32-10 (Salmon et al., SC'11) with key
 * (seed, stream) and counters (all 32-bit words):
 *   momenta  stream 1, counter (site, mu + 4 traj_index, k, 0), k = 0..3: coefficients
 *            2k, 2k+1 of link (site, mu) are the Box-Muller pair of call k
 *   chi      stream 2, counter (site, traj_index, k, 0), k = 0..11: complex component
 *            k = 3 spin + colour is (z0 + i z1) sqrt(1/2)
 *   u        stream 3, counter (traj_index, 0, 0, 0): 53-bit uniform of words 0, 1
 * Uniforms: ((w0 >> 5) 2^26 + (w1 >> 6)) 2^-53; Box-Muller r = sqrt(-2 log(1 - u1)),
 * angle 2 pi u2, with the logarithm and sine / cosine evaluated by fixed series in
 * correctly rounded FP64 operations, so the draws are reproducible bit for bit by any
 * implementation that performs the same operations.  seed < 2^32, traj_index < 2^30
 * (else LQ_ERR_ARG).  p_out (canonical [V][4][8], host or device, may be NULL) receives
 * the final momenta.  Nothing is copied from the host.  Synchronises. */
lq_status lq_hmc_trajectory_seeded(lq_ctx* ctx, const lq_hmc_params* params, uint64_t seed, uint64_t traj_index,
                                   double* p_out, lq_traj_result* result);

/* The heat-bath draws of lq_hmc_trajectory_seeded for (seed, traj_index), written to the
 * caller's buffers: p momenta (canonical [V][4][8]), chi noise (canonical spinor), u the
 * Metropolis uniform (host); any may be NULL; p and chi host or device.  Synchronises when
 * a host buffer is written.  Errors: LQ_ERR_ARG. */
lq_status lq_heatbath_draw(lq_ctx* ctx, uint64_t seed, uint64_t traj_index, double* p, double* chi, double* u);

/* Philox4x32-10 on the device: for i < n, out[i][0..3] = the generator's four output
 * words for counter in[i][0..3] and key in[i][4..5] (the heat bath's generator, exposed
 * for its known-answer tests).  in, out: device buffers of uint32.  Asynchronous. */
lq_status lq_philox4x32_10(lq_ctx* ctx, const uint32_t* in, uint32_t* out, int n);

/* Measurement: apply M (dagger = 0) or M^dag (1) `n` times in precision
 * `prec` to `in` (packed once, outside the timed region) and return the
 * average device time of one application in *ms, measured with CUDA events
 * on the context's stream.  flush_l2 != 0 writes a 256 MB buffer before
 * each application (outside its timing) so no operand is L2-resident.
 * This is the hot kernel of the solve (Sec. 2: repeated multiplication of
 * M takes most of the molecular-dynamics time).  Synchronises. */
lq_status lq_time_dslash(lq_ctx* ctx, const double* in, double kappa, int dagger, int prec, int n, int flush_l2,
                         double* ms);

/* out = M^dag M in, FP64, without allocating any device memory.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot let a library allocate GPU memory: programs that give all device
 * memory to their own pool allocator and forbid cudaMalloc once they are
 * running, or plugins that live inside a host application under a fixed
 * device-memory budget.  It needs no context (lq_create allocates): U, in
 * and out are the caller's device buffers in the canonical layouts above
 * (U [V][4][3][3] complex, in / out [V][4][3] complex, 16-byte aligned),
 * dims and t_antiperiodic as in lq_create, and the work is issued on
 * `cuda_stream` (a cudaStream_t) without synchronising.  out may equal in.
 *
 * The intermediate field M in is kept in one array compiled into the
 * library (12 MiB, held on every GPU that loads the library until the
 * process exits), so the lattice may have at most 65,536 sites (e.g. 16^4);
 * larger lattices return LQ_ERR_SHAPE.  All calls share that array: two
 * calls whose work overlaps on the GPU (different streams, or different
 * host threads without ordering) race and give wrong results; calls on the
 * same stream are ordered and safe.  Every call overwrites the whole part
 * of the array it uses before reading it, so no state carries over.
 * The first call on each device looks up the array's device address (one
 * cudaGetSymbolAddress with that device current) and keeps it for the life
 * of the process; make that first call before capturing the stream into a
 * CUDA graph.  Calls after a device reset (cudaDeviceReset, or a reset of
 * the primary context) are not supported: the address kept belongs to the
 * module instance the reset unloaded.
 * Errors: LQ_ERR_ARG (null or misaligned buffer, or a buffer that is not
 * device memory: host buffers are refused, never read by a kernel),
 * LQ_ERR_SHAPE (an extent < 2, or more sites than the array holds),
 * LQ_ERR_CUDA; the message is returned by lq_last_error(NULL). */
lq_status lq_apply_MdagM_static(double* out, const double* U, const double* in, const int dims[4],
                                int t_antiperiodic, double kappa, void* cuda_stream);

/* Measurement: the fused multiply-add rate of this GPU in *tflops (TFLOP/s, 2 flop per
 * multiply-add) for prec = LQ_F64 or LQ_F32: eight independent multiply-add chains per
 * thread, four blocks of 256 threads per SM, best of five launches timed with CUDA events
 * on the context's stream.  The FP64 operator is bound by this rate rather than by HBM
 * bandwidth on this part, so it is the denominator of the FP64 operator's roofline
 * (the paper's FP64 kernels, Sec. 3, are here limited by the FP64 pipe).  Synchronises. */
lq_status lq_time_fma_peak(lq_ctx* ctx, int prec, double* tflops);

/* Measurement: the average device time in *ms of one CG iteration (which = 0)
 * or of one of its three passes (1: t = M p with |t|^2; 2: r -= alpha M^dag t,
 * x += alpha p with |r|^2; 3: p = r + beta p) in precision `prec`, run `n`
 * times on a CG state started from `in` (canonical spinor) that never halts.
 * CUDA events on the context's stream; the context's solver fields are
 * overwritten.  The iteration is the paper's CG routine (Sec. 3).  Synchronises. */
lq_status lq_time_cg_kernel(lq_ctx* ctx, const double* in, double kappa, int which, int prec, int n, double* ms);

/* Ablation of the paper's register observation (Sec. 3 and 4: the array variables of
 * the kernels moved from global memory into registers, a fivefold speed-up on Fermi).
 * out = M in (dagger 0) or M^dag in (1), FP64, computed by a naive kernel: canonical
 * array-of-structures layout, a neighbour table in global memory, dense 4x4 spin
 * matrices and accumulation through global memory.  in, out: device, canonical.
 * When n > 0 and ms != NULL, the kernel is then launched n more times and *ms receives
 * its average device time (CUDA events on the context's stream).  Synchronises. */
lq_status lq_apply_M_naive(lq_ctx* ctx, double* out, const double* in, double kappa, int dagger, int n, double* ms);

/* The force half of the same ablation (Sec. 3 kernel 3 written naively).  F = the fermion
 * force of lq_fermion_force for the given X, computed with Y = M X from the naive operator
 * and a naive force kernel: one thread per link, canonical layouts, the neighbour table in
 * global memory, dense 4x4 spin matrices on full four-spinors, the colour matrix
 * accumulated in global memory.  F: device, canonical [V][4][8]; X: device, canonical.
 * When n > 0 and ms != NULL, the force kernel is launched n more times and *ms receives
 * its average device time.  Synchronises. */
lq_status lq_fermion_force_naive(lq_ctx* ctx, double* F, const double* X, double kappa, int n, double* ms);

/* Average device time of the optimised fermion-force kernel (Sec. 3 kernel 3, the one
 * lq_fermion_force and the trajectory use) over n launches, for X (canonical spinor, host
 * or device) with Y = M X formed once beforehand and not timed.  The context's force
 * buffer is overwritten.  Synchronises. */
lq_status lq_time_fermion_force(lq_ctx* ctx, const double* X, double kappa, int n, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* LQ_H */
