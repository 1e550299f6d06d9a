// FP64 conjugate gradient on M^dag M (Sec. 1 after Eq. 3; Sec. 3): one
// iteration is three fused passes over the lattice,
//   k1  t = M p,                         tt = |t|^2, alpha = rr / tt
//   k2  r -= alpha M^dag t, x += alpha p, rr = |r|^2, beta
//   k3  p = r + beta p
// and the FP64 true residual r = phi - M^dag (M x) used to stop the solve
// and, for mixed-precision solves, as the reliable update.
#include "lq_internal.h"

namespace lq {

void cg64_step(lq_ctx* c, int which, double kappa, cudaStream_t stream) {
  const Geom& g = c->geo;
  GaugeRef U{c->gauge64};
  if (which == 1) {
    EpiCG1<SStore::F64> e1{c->t64.ref(), c->state};
    launch_dslash<double, GStore::F64_18, SStore::F64, false>(g, U, c->p64.ref(), kappa, e1, c->rs, stream);
  } else {
    EpiCG2<SStore::F64, SStore::F64, SStore::F64> e2{c->r64.ref(), c->x64.ref(), c->p64.ref(), c->state};
    launch_dslash<double, GStore::F64_18, SStore::F64, true>(g, U, c->t64.ref(), kappa, e2, c->rs, stream);
  }
}

void cg64_iteration(lq_ctx* c, double kappa, cudaStream_t stream) {
  const Geom& g = c->geo;
  GaugeRef U{c->gauge64};
  EpiCG1<SStore::F64> e1{c->t64.ref(), c->state};
  launch_dslash<double, GStore::F64_18, SStore::F64, false>(g, U, c->p64.ref(), kappa, e1, c->rs, stream);
  EpiCG2<SStore::F64, SStore::F64, SStore::F64> e2{c->r64.ref(), c->x64.ref(), c->p64.ref(), c->state};
  launch_dslash<double, GStore::F64_18, SStore::F64, true>(g, U, c->t64.ref(), kappa, e2, c->rs, stream);
  launch_xpay_p(g, SStore::F64, c->r64.ref(), c->p64.ref(), c->state, false, stream);
}

template <SStore SLO>
static void residual_lo(lq_ctx* c, double kappa, SpinorRef rlo, cudaStream_t stream) {
  EpiResidual<SLO, true> e{c->phi64.ref(), c->r64.ref(), rlo, c->state};
  launch_dslash<double, GStore::F64_18, SStore::F64, true>(c->geo, GaugeRef{c->gauge64}, c->tmp64.ref(), kappa, e,
                                                           c->rs, stream);
}

void cg64_true_residual(lq_ctx* c, double kappa, int store_lo_prec, cudaStream_t stream) {
  const Geom& g = c->geo;
  GaugeRef U{c->gauge64};
  EpiStore<SStore::F64> e0{c->tmp64.ref()};
  launch_dslash<double, GStore::F64_18, SStore::F64, false>(g, U, c->x64.ref(), kappa, e0, c->rs, stream);
  if (store_lo_prec == LQ_F64) {
    EpiResidual<SStore::F64, false> e{c->phi64.ref(), c->r64.ref(), SpinorRef{nullptr, nullptr}, c->state};
    launch_dslash<double, GStore::F64_18, SStore::F64, true>(g, U, c->tmp64.ref(), kappa, e, c->rs, stream);
    return;
  }
  const SStore slo = spinor_store_of(store_lo_prec);
  SpinorRef rlo = c->r_lo[(int)slo].ref();
  switch (slo) {
    case SStore::F32: residual_lo<SStore::F32>(c, kappa, rlo, stream); break;
    case SStore::F16: residual_lo<SStore::F16>(c, kappa, rlo, stream); break;
    case SStore::BF16: residual_lo<SStore::BF16>(c, kappa, rlo, stream); break;
    case SStore::I16: residual_lo<SStore::I16>(c, kappa, rlo, stream); break;
    default: break;
  }
}

}  // namespace lq
