// Plain applications of M and M^dag (Eq. 4; Sec. 3 kernel 1) in each
// precision: out = M in, no reduction.
#include "lq_internal.h"
#include "lq_staged.cuh"
#include "lq_dfsplit.cuh"

namespace lq {

template <typename T, GStore G, SStore S>
static void apply_one(const Geom& g, const void* gauge, SpinorRef in, SpinorRef out, double kappa, bool dagger,
                      cudaStream_t stream, bool staged = false) {
  EpiStore<S> epi{out};
  ReduceScratch none{nullptr, nullptr, 0};
  if constexpr (std::is_same<T, float>::value) {
    if (staged) {
      if (dagger) launch_dslash_staged<T, G, S, true>(g, GaugeRef{gauge}, in, kappa, epi, none, stream);
      else launch_dslash_staged<T, G, S, false>(g, GaugeRef{gauge}, in, kappa, epi, none, stream);
      return;
    }
  }
  if (dagger) launch_dslash<T, G, S, true>(g, GaugeRef{gauge}, in, kappa, epi, none, stream);
  else launch_dslash<T, G, S, false>(g, GaugeRef{gauge}, in, kappa, epi, none, stream);
}

void apply_M_prec(const Geom& g, int prec, const void* gauge, SpinorRef in, SpinorRef out, double kappa,
                  bool dagger, cudaStream_t stream, bool pair, bool staged, bool df_prefetch) {
  if (pair && prec == LQ_I16_12 && pair_geometry(g)) {
    pair_apply(g, gauge, in, out, kappa, dagger, stream);
    return;
  }
  switch (prec) {
    case LQ_F64: apply_one<double, GStore::F64_18, SStore::F64>(g, gauge, in, out, kappa, dagger, stream); break;
    case LQ_F32: apply_one<float, GStore::F32_18, SStore::F32>(g, gauge, in, out, kappa, dagger, stream, staged); break;
    case LQ_F32_12: apply_one<float, GStore::F32_12, SStore::F32>(g, gauge, in, out, kappa, dagger, stream, staged); break;
    case LQ_F16_12: apply_one<float, GStore::F16_12, SStore::F16>(g, gauge, in, out, kappa, dagger, stream, staged); break;
    case LQ_BF16_12: apply_one<float, GStore::BF16_12, SStore::BF16>(g, gauge, in, out, kappa, dagger, stream, staged); break;
    case LQ_DF64: {
      // the two-threads-per-site double-float operator (lq_dfsplit.cuh)
      DFEpiStore epi{out};
      ReduceScratch none{nullptr, nullptr, 0};
      if (dagger) launch_dslash_dfsplit<true>(g, gauge, in, kappa, epi, none, stream, -1, 0, df_prefetch);
      else launch_dslash_dfsplit<false>(g, gauge, in, kappa, epi, none, stream, -1, 0, df_prefetch);
      break;
    }
    case LQ_I16_12: apply_one<float, GStore::I16_12, SStore::I16>(g, gauge, in, out, kappa, dagger, stream, staged); break;
  }
}

}  // namespace lq
