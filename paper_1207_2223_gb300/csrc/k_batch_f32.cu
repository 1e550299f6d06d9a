// The batched solver's iteration for FP32 storage (18 and 12 reals per link).
#include "lq_batch.cuh"

namespace lq {

void batch_iteration_f32(const BatchIterArgs& a, const BatchDesc& bd, int prec, cudaStream_t st) {
  if (prec == LQ_F32_12) batch_iteration_t<GStore::F32_12, SStore::F32>(a, bd, st);
  else batch_iteration_t<GStore::F32_18, SStore::F32>(a, bd, st);
}

cudaError_t batch_persistent_f32(const BatchDesc& bd, const PersistArgs& a, int prec, int sms, int max_grid,
                                 cudaStream_t st) {
  if (prec == LQ_F32_12) return launch_batch_persistent_t<GStore::F32_12, SStore::F32>(bd, a, sms, max_grid, st);
  return launch_batch_persistent_t<GStore::F32_18, SStore::F32>(bd, a, sms, max_grid, st);
}

}  // namespace lq
