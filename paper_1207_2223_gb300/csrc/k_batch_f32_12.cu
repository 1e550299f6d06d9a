// The batched solver's iteration for FP32 storage with 12 reals per link.
#include "lq_batch.cuh"

namespace lq {

void batch_iteration_f32_12(const BatchIterArgs& a, const BatchDesc& bd, int, cudaStream_t st) {
  batch_iteration_t<GStore::F32_12, SStore::F32>(a, bd, st);
}

cudaError_t batch_persistent_f32_12(const BatchDesc& bd, const PersistArgs& a, int, int sms, int max_grid,
                                    cudaStream_t st) {
  return launch_batch_persistent_t<GStore::F32_12, SStore::F32>(bd, a, sms, max_grid, st);
}

}  // namespace lq
