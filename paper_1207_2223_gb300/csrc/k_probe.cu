// Arithmetic peak of the GPU this library runs on, measured: the FP64 operator
// is bound by the FP64 pipe, not by HBM, so its roofline needs the FP64 fused
// multiply-add rate of the part (and the FP32 rate for comparison).
//
// Every thread runs eight independent multiply-add chains (enough independent
// work to hide the pipe latency at four blocks of 256 threads per SM), the
// grid covers every SM, and the device time of the launch (CUDA events on the
// context's stream) gives 2 flop per multiply-add.
#include "lq_internal.h"

namespace lq {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains_kernel(T a, T b, int iters, T* out) {
  T x0 = (T)threadIdx.x * a, x1 = x0 + b, x2 = x1 + b, x3 = x2 + b, x4 = x3 + b, x5 = x4 + b, x6 = x5 + b,
    x7 = x6 + b;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

template <typename T>
lq_status time_chains(lq_ctx* c, int iters, double* tflops) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    c->last_error = "lq_time_fma_peak: cannot read the SM count";
    return LQ_ERR_CUDA;
  }
  const int bs = 256, grid = sms * 4;
  T* out = nullptr;
  if (cudaMallocAsync((void**)&out, sizeof(T) * grid * bs, c->stream) != cudaSuccess) {
    cudaGetLastError();
    c->last_error = "lq_time_fma_peak: cudaMallocAsync";
    return LQ_ERR_CUDA;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains_kernel<T><<<grid, bs, 0, c->stream>>>((T)0.999999, (T)1e-7, iters / 8, out);   // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0, c->stream);
    fma_chains_kernel<T><<<grid, bs, 0, c->stream>>>((T)0.999999, (T)1e-7, iters, out);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 0.f && ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, c->stream);
  cudaStreamSynchronize(c->stream);
  if (err != cudaSuccess) {
    c->last_error = std::string("lq_time_fma_peak: ") + cudaGetErrorString(err);
    return LQ_ERR_CUDA;
  }
  const double flop = 2.0 * 8.0 * (double)iters * grid * bs;
  *tflops = flop / (best * 1e-3) / 1e12;
  return LQ_OK;
}

}  // namespace
}  // namespace lq

extern "C" lq_status lq_time_fma_peak(lq_ctx* c, int prec, double* tflops) {
  using namespace lq;
  if (!c) return LQ_ERR_ARG;
  if (!tflops || (prec != LQ_F64 && prec != LQ_F32)) {
    c->last_error = "lq_time_fma_peak: prec must be LQ_F64 or LQ_F32, tflops non-null";
    return LQ_ERR_ARG;
  }
  return prec == LQ_F64 ? time_chains<double>(c, 4096, tflops) : time_chains<float>(c, 65536, tflops);
}
