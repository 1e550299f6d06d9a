// The batched solver's iteration for FP16 and BF16 storage (12-real links, per-site norms).
#include "lq_batch.cuh"

namespace lq {

void batch_iteration_h16(const BatchIterArgs& a, const BatchDesc& bd, int prec, cudaStream_t st) {
  if (prec == LQ_BF16_12) batch_iteration_t<GStore::BF16_12, SStore::BF16>(a, bd, st);
  else batch_iteration_t<GStore::F16_12, SStore::F16>(a, bd, st);
}

cudaError_t batch_persistent_h16(const BatchDesc& bd, const PersistArgs& a, int prec, int sms, int max_grid,
                                 cudaStream_t st) {
  if (prec == LQ_BF16_12) return launch_batch_persistent_t<GStore::BF16_12, SStore::BF16>(bd, a, sms, max_grid, st);
  return launch_batch_persistent_t<GStore::F16_12, SStore::F16>(bd, a, sms, max_grid, st);
}

}  // namespace lq
