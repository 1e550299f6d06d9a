// Double-float reliable update of the mixed-precision CG (the CG routine of
// Sec. 3 with the mixed precision the paper names as future work in Sec. 4):
//   x_df += x_lo, x_lo = 0;   tmp = M x_df;   r = phi - M^dag tmp
// with links and spinors stored as hi/lo float pairs, the arithmetic of
// lq_df64.cuh on the FP32 pipe and two threads per site (lq_dfsplit.cuh).  The residual goes to a double-float field
// (r_df) and to the inner format (r_lo), |r|^2 to state->rr_true.
#include "lq_internal.h"
#include "lq_dfsplit.cuh"

namespace lq {

static constexpr int kBS = 256;

// x_df += x_lo; x_lo = 0
template <SStore SLO>
__global__ void __launch_bounds__(kBS) accumulate_df_kernel(int V, SpinorRef xlo, SpinorRef xdf) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  cplx<float> a[12], z[12];
  cplx<df64> b[12];
  load_spinor<xlo_store(SLO), float, false>(xlo, V, s, a);
  load_spinor<SStore::DF64, df64, false>(xdf, V, s, b);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    b[k] = {b[k].re + df64(a[k].re), b[k].im + df64(a[k].im)};
    z[k] = {0.f, 0.f};
  }
  store_spinor<SStore::DF64, df64>(xdf, V, s, b);
  store_spinor<xlo_store(SLO), float>(xlo, V, s, z);
}

// x = 0, r = p = src (double-float) in format S
template <SStore S>
__global__ void __launch_bounds__(kBS) inner_restart_df_kernel(int V, SpinorRef src, SpinorRef x, SpinorRef r,
                                                               SpinorRef p) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  cplx<df64> v[12], z[12];
  load_spinor<SStore::DF64, df64>(src, V, s, v);
#pragma unroll
  for (int k = 0; k < 12; ++k) z[k] = {df64(0.f), df64(0.f)};
  store_spinor<xlo_store(S), df64>(x, V, s, z);
  store_spinor<S, df64>(r, V, s, v);
  store_spinor<S, df64>(p, V, s, v);
}

template <SStore SLO>
static void ru(lq_ctx* c, double kappa, cudaStream_t stream) {
  const Geom& g = c->geo;
  const int k = (int)SLO;
  accumulate_df_kernel<SLO><<<grid_for(g.V, kBS), kBS, 0, stream>>>(g.V, c->x_lo[k].ref(), c->x_df.ref());
  DFEpiStore e0{c->tmp_df.ref()};
  launch_dslash_dfsplit<false>(g, c->gauge_lo[LQ_DF64], c->x_df.ref(), kappa, e0, c->rs, stream, -1, 0,
                               c->df_prefetch);
  DFEpiResidual<SLO> e1{c->phi_df.ref(), c->r_df.ref(), c->r_lo[k].ref(), DFFinSolver{c->state}};
  launch_dslash_dfsplit<true>(g, c->gauge_lo[LQ_DF64], c->tmp_df.ref(), kappa, e1, c->rs, stream, -1, 0,
                              c->df_prefetch);
}

template <SStore SLO>
static void acc_only(lq_ctx* c, cudaStream_t stream) {
  const Geom& g = c->geo;
  accumulate_df_kernel<SLO><<<grid_for(g.V, kBS), kBS, 0, stream>>>(g.V, c->x_lo[(int)SLO].ref(), c->x_df.ref());
}

void df_accumulate(lq_ctx* c, int inner_prec, cudaStream_t stream) {
  switch (spinor_store_of(inner_prec)) {
    case SStore::F32: acc_only<SStore::F32>(c, stream); break;
    case SStore::F16: acc_only<SStore::F16>(c, stream); break;
    case SStore::BF16: acc_only<SStore::BF16>(c, stream); break;
    case SStore::I16: acc_only<SStore::I16>(c, stream); break;
    default: break;
  }
}

void df_reliable_update(lq_ctx* c, double kappa, int inner_prec, cudaStream_t stream) {
  switch (spinor_store_of(inner_prec)) {
    case SStore::F32: ru<SStore::F32>(c, kappa, stream); break;
    case SStore::F16: ru<SStore::F16>(c, kappa, stream); break;
    case SStore::BF16: ru<SStore::BF16>(c, kappa, stream); break;
    case SStore::I16: ru<SStore::I16>(c, kappa, stream); break;
    default: break;
  }
}

void launch_inner_restart_df(const Geom& g, SpinorRef src, SStore s, SpinorRef x, SpinorRef r, SpinorRef p,
                             cudaStream_t stream) {
  const int grid = grid_for(g.V, kBS);
  switch (s) {
    case SStore::F32: inner_restart_df_kernel<SStore::F32><<<grid, kBS, 0, stream>>>(g.V, src, x, r, p); break;
    case SStore::F16: inner_restart_df_kernel<SStore::F16><<<grid, kBS, 0, stream>>>(g.V, src, x, r, p); break;
    case SStore::BF16: inner_restart_df_kernel<SStore::BF16><<<grid, kBS, 0, stream>>>(g.V, src, x, r, p); break;
    case SStore::I16: inner_restart_df_kernel<SStore::I16><<<grid, kBS, 0, stream>>>(g.V, src, x, r, p); break;
    default: break;
  }
}

}  // namespace lq
