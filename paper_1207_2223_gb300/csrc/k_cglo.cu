// Low-precision CG iteration for mixed-precision solves: the same three
// fused passes as the FP64 iteration, on FP32 or 16-bit storage with FP32
// arithmetic and FP64 reductions; the low-precision solution x is FP32 for
// the 16-bit formats (xlo_store).  The FP64 solution and residual are
// corrected by reliable updates driven from the host (api.cu).
#include "lq_internal.h"
#include "lq_staged.cuh"

namespace lq {

// One stencil pass: the plain kernel, or the one sharing x and y links in-block (option LQ_OPT_STAGED).
template <GStore G, SStore S, bool DAG, class Epi>
static void pass(const lq_ctx* c, GaugeRef U, SpinorRef in, double kappa, const Epi& e, cudaStream_t stream) {
  if (c->staged) launch_dslash_staged<float, G, S, DAG>(c->geo, U, in, kappa, e, c->rs, stream);
  else launch_dslash<float, G, S, DAG>(c->geo, U, in, kappa, e, c->rs, stream);
}

template <GStore G, SStore S>
static void step(lq_ctx* c, const void* gauge, int which, double kappa, cudaStream_t stream) {
  GaugeRef U{gauge};
  const int k = (int)S;
  if (which == 1) {
    EpiCG1<S> e1{c->t_lo[k].ref(), c->state};
    pass<G, S, false>(c, U, c->p_lo[k].ref(), kappa, e1, stream);
  } else {
    EpiCG2<S, xlo_store(S), S> e2{c->r_lo[k].ref(), c->x_lo[k].ref(), c->p_lo[k].ref(), c->state};
    pass<G, S, true>(c, U, c->t_lo[k].ref(), kappa, e2, stream);
  }
}

template <GStore G, SStore S>
static void iteration(lq_ctx* c, const void* gauge, double kappa, cudaStream_t stream) {
  const int k = (int)S;
  step<G, S>(c, gauge, 1, kappa, stream);
  step<G, S>(c, gauge, 2, kappa, stream);
  launch_xpay_p(c->geo, S, c->r_lo[k].ref(), c->p_lo[k].ref(), c->state, false, stream);
}

// The two-site packed passes replace the one-site ones for 16-bit fixed point
// (the same fields, formats and solver state).
static bool use_pair(const lq_ctx* c, int prec) {
  return prec == LQ_I16_12 && c->pair_sites && pair_geometry(c->geo);
}

void cglo_step(lq_ctx* c, int prec, int which, double kappa, cudaStream_t stream) {
  const void* gauge = c->gauge_lo[prec];
  if (use_pair(c, prec)) {
    if (which == 1) pair_cg1(c, gauge, kappa, stream);
    else pair_cg2(c, gauge, kappa, stream);
    return;
  }
  switch (prec) {
    case LQ_F32: step<GStore::F32_18, SStore::F32>(c, gauge, which, kappa, stream); break;
    case LQ_F32_12: step<GStore::F32_12, SStore::F32>(c, gauge, which, kappa, stream); break;
    case LQ_F16_12: step<GStore::F16_12, SStore::F16>(c, gauge, which, kappa, stream); break;
    case LQ_BF16_12: step<GStore::BF16_12, SStore::BF16>(c, gauge, which, kappa, stream); break;
    case LQ_I16_12: step<GStore::I16_12, SStore::I16>(c, gauge, which, kappa, stream); break;
    default: break;
  }
}

void cglo_iteration(lq_ctx* c, int prec, double kappa, cudaStream_t stream) {
  const void* gauge = c->gauge_lo[prec];
  if (use_pair(c, prec)) {
    const int k = (int)SStore::I16;
    pair_cg1(c, gauge, kappa, stream);
    pair_cg2(c, gauge, kappa, stream);
    launch_xpay_p(c->geo, SStore::I16, c->r_lo[k].ref(), c->p_lo[k].ref(), c->state, false, stream);
    return;
  }
  switch (prec) {
    case LQ_F32: iteration<GStore::F32_18, SStore::F32>(c, gauge, kappa, stream); break;
    case LQ_F32_12: iteration<GStore::F32_12, SStore::F32>(c, gauge, kappa, stream); break;
    case LQ_F16_12: iteration<GStore::F16_12, SStore::F16>(c, gauge, kappa, stream); break;
    case LQ_BF16_12: iteration<GStore::BF16_12, SStore::BF16>(c, gauge, kappa, stream); break;
    case LQ_I16_12: iteration<GStore::I16_12, SStore::I16>(c, gauge, kappa, stream); break;
    default: break;
  }
}

}  // namespace lq
