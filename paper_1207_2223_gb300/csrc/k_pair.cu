// Launchers of the two-site packed stencil (lq_pair.cuh) for 16-bit
// fixed-point storage: the plain operator and the two fused CG passes.
#include "lq_internal.h"
#include "lq_pair.cuh"

namespace lq {

template <bool DAG, class Epi>
static void launch_pair(const Geom& geo, const void* gauge, SpinorRef in, double kappa, const Epi& epi,
                        const ReduceScratch& rs, cudaStream_t stream) {
  constexpr int bs = LQ_PAIR_BLOCK;
  static const int wave = resident_grid(reinterpret_cast<const void*>(&dslash_pair_kernel<DAG, Epi>), bs);
  const int grid = std::min(grid_for(geo.V / 2, bs), wave);
  dslash_pair_kernel<DAG, Epi><<<grid, bs, 0, stream>>>(geo, GaugeRef{gauge}, in, (float)kappa, epi, rs);
}

void pair_apply(const Geom& g, const void* gauge, SpinorRef in, SpinorRef out, double kappa, bool dagger,
                cudaStream_t stream) {
  PairStore epi{{out}};
  ReduceScratch none{nullptr, nullptr, 0};
  if (dagger) launch_pair<true>(g, gauge, in, kappa, epi, none, stream);
  else launch_pair<false>(g, gauge, in, kappa, epi, none, stream);
}

void pair_cg1(lq_ctx* c, const void* gauge, double kappa, cudaStream_t stream) {
  const int k = (int)SStore::I16;
  PairCG1 e1{{c->t_lo[k].ref(), c->state}};
  launch_pair<false>(c->geo, gauge, c->p_lo[k].ref(), kappa, e1, c->rs, stream);
}

void pair_cg2(lq_ctx* c, const void* gauge, double kappa, cudaStream_t stream) {
  const int k = (int)SStore::I16;
  PairCG2 e2{{c->r_lo[k].ref(), c->x_lo[k].ref(), c->p_lo[k].ref(), c->state}};
  launch_pair<true>(c->geo, gauge, c->t_lo[k].ref(), kappa, e2, c->rs, stream);
}

}  // namespace lq
