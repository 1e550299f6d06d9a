// Level-1 vector kernels of the CG solver: start-up, the search-direction
// update p = r + beta p, folding the low-precision solution into the FP64
// one at a reliable update, and the scalar bookkeeping after a true
// residual.  All reductions are FP64 and deterministic (lq_device.cuh).
#include "lq_internal.h"

namespace lq {

static constexpr int kBS = 256;

template <SStore S>
__global__ void __launch_bounds__(kBS) solver_init_kernel(int V, SpinorRef phi64, SpinorRef x, SpinorRef r,
                                                          SpinorRef p, SolverState* st, ReduceScratch rs) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double red[1] = {0.0};
  if (s < V) {
    cplx<double> v[12], z[12];
    load_spinor<SStore::F64, double>(phi64, V, s, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) { red[0] += v[k].re * v[k].re + v[k].im * v[k].im; z[k] = {0.0, 0.0}; }
    store_spinor<xlo_store(S), double>(x, V, s, z);
    store_spinor<S, double>(r, V, s, v);
    store_spinor<S, double>(p, V, s, v);
  }
  double tot[1];
  if (grid_sum<1>(red, rs, tot)) {
    st->phi2 = tot[0];
    st->stop2 = st->stop2 * tot[0];     // host stored tol^2 there
    st->rr = tot[0];
    st->rr_prev = tot[0];
    st->rr_ref = tot[0];
    st->rr_true = tot[0];
    if (!isfinite(tot[0])) { st->breakdown = 1; st->halt = 1; }
  }
}

template <SStore S>
__global__ void __launch_bounds__(kBS) xpay_p_kernel(int V, SpinorRef r, SpinorRef p, const SolverState* st,
                                                     int forced) {
  if (!forced && *(volatile const int*)&st->halt) return;
  // one site per thread: a grid-stride loop over one resident wave would make
  // the empty launches after a halt cheaper, but measured slower (91% against
  // 97% of HBM) on the launches that do the work
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  using T = typename std::conditional<S == SStore::F64, double, float>::type;
  const T beta = (T)st->beta;
  cplx<T> rv[12], pv[12];
  load_spinor<S, T>(r, V, s, rv);
  load_spinor<S, T, false>(p, V, s, pv);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    pv[k].re = fma(beta, pv[k].re, rv[k].re);
    pv[k].im = fma(beta, pv[k].im, rv[k].im);
  }
  store_spinor<S, T>(p, V, s, pv);
}

template <SStore S>
__global__ void __launch_bounds__(kBS) accumulate_x_kernel(int V, SpinorRef xlo, SpinorRef xhi) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  cplx<double> a[12], b[12], z[12];
  load_spinor<xlo_store(S), double, false>(xlo, V, s, a);
  load_spinor<SStore::F64, double, false>(xhi, V, s, b);
#pragma unroll
  for (int k = 0; k < 12; ++k) { b[k] = b[k] + a[k]; z[k] = {0.0, 0.0}; }
  store_spinor<SStore::F64, double>(xhi, V, s, b);
  store_spinor<xlo_store(S), double>(xlo, V, s, z);
}

template <SStore S>
__global__ void __launch_bounds__(kBS) zero_spinor_kernel(int V, SpinorRef f) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  cplx<double> z[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) z[k] = {0.0, 0.0};
  store_spinor<S, double>(f, V, s, z);
}

// Restart the inner iteration from an FP64 residual: r = p = src, x = 0.
template <SStore S>
__global__ void __launch_bounds__(kBS) inner_restart_kernel(int V, SpinorRef src64, SpinorRef x, SpinorRef r,
                                                            SpinorRef p) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  cplx<double> v[12], z[12];
  load_spinor<SStore::F64, double>(src64, V, s, v);
#pragma unroll
  for (int k = 0; k < 12; ++k) z[k] = {0.0, 0.0};
  store_spinor<xlo_store(S), double>(x, V, s, z);
  store_spinor<S, double>(r, V, s, v);
  store_spinor<S, double>(p, V, s, v);
}

__global__ void state_after_residual_kernel(SolverState* st, int restart) {
  const double rr = st->rr_true;
  st->beta = restart ? 0.0 : rr / st->rr_prev;
  st->rr = rr;
  st->rr_ref = rr;
  st->iter_since_ru = 0;
  st->halt = 0;
  if (!isfinite(rr)) { st->breakdown = 1; st->halt = 1; }
}

#define LQ_DISPATCH_S(S, CALL)                               \
  switch (S) {                                               \
    case SStore::F64: { constexpr SStore SS = SStore::F64; CALL; } break;   \
    case SStore::F32: { constexpr SStore SS = SStore::F32; CALL; } break;   \
    case SStore::F16: { constexpr SStore SS = SStore::F16; CALL; } break;   \
    case SStore::BF16: { constexpr SStore SS = SStore::BF16; CALL; } break; \
    case SStore::DF64: { constexpr SStore SS = SStore::DF64; CALL; } break; \
    case SStore::I16: { constexpr SStore SS = SStore::I16; CALL; } break;   \
  }

void launch_solver_init(const Geom& g, SpinorRef phi64, SStore sx, SpinorRef x, SStore sr, SpinorRef r,
                        SStore sp, SpinorRef p, SolverState* st, const ReduceScratch& rs, cudaStream_t stream) {
  (void)sr; (void)sp;   // r and p share one format; x is stored as xlo_store() of it
  const int grid = grid_for(g.V, kBS);
  LQ_DISPATCH_S(sx, (solver_init_kernel<SS><<<grid, kBS, 0, stream>>>(g.V, phi64, x, r, p, st, rs)));
}

void launch_xpay_p(const Geom& g, SStore s, SpinorRef r, SpinorRef p, SolverState* st, bool forced,
                   cudaStream_t stream) {
  const int grid = grid_for(g.V, kBS);
  LQ_DISPATCH_S(s, (xpay_p_kernel<SS><<<grid, kBS, 0, stream>>>(g.V, r, p, st, forced ? 1 : 0)));
}

void launch_accumulate_x(const Geom& g, SStore slo, SpinorRef xlo, SpinorRef xhi, cudaStream_t stream) {
  const int grid = grid_for(g.V, kBS);
  LQ_DISPATCH_S(slo, (accumulate_x_kernel<SS><<<grid, kBS, 0, stream>>>(g.V, xlo, xhi)));
}

void launch_zero_spinor(const Geom& g, SStore s, SpinorRef f, cudaStream_t stream) {
  const int grid = grid_for(g.V, kBS);
  LQ_DISPATCH_S(s, (zero_spinor_kernel<SS><<<grid, kBS, 0, stream>>>(g.V, f)));
}

void launch_inner_restart(const Geom& g, SpinorRef src64, SStore s, SpinorRef x, SpinorRef r, SpinorRef p,
                          cudaStream_t stream) {
  const int grid = grid_for(g.V, kBS);
  LQ_DISPATCH_S(s, (inner_restart_kernel<SS><<<grid, kBS, 0, stream>>>(g.V, src64, x, r, p)));
}

void launch_state_after_residual(SolverState* st, int restart, cudaStream_t stream) {
  state_after_residual_kernel<<<1, 1, 0, stream>>>(st, restart);
}

}  // namespace lq
