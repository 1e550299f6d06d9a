// The batched solver's iteration for BF16 storage (12-real links, per-site norms).
#include "lq_batch.cuh"

namespace lq {

void batch_iteration_bf16(const BatchIterArgs& a, const BatchDesc& bd, int, cudaStream_t st) {
  batch_iteration_t<GStore::BF16_12, SStore::BF16>(a, bd, st);
}

cudaError_t batch_persistent_bf16(const BatchDesc& bd, const PersistArgs& a, int, int sms, int max_grid,
                                  cudaStream_t st) {
  return launch_batch_persistent_t<GStore::BF16_12, SStore::BF16>(bd, a, sms, max_grid, st);
}

}  // namespace lq
