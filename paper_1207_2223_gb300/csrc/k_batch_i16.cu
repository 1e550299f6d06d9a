// The batched solver's iteration for 16-bit fixed-point storage.
#include "lq_batch.cuh"

namespace lq {

void batch_iteration_i16(const BatchIterArgs& a, const BatchDesc& bd, int, cudaStream_t st) {
  batch_iteration_t<GStore::I16_12, SStore::I16>(a, bd, st);
}

cudaError_t batch_persistent_i16(const BatchDesc& bd, const PersistArgs& a, int, int sms, int max_grid,
                                 cudaStream_t st) {
  return launch_batch_persistent_t<GStore::I16_12, SStore::I16>(bd, a, sms, max_grid, st);
}

}  // namespace lq
