// FP32 and FP64 FMA throughput of the device (the CUDA-core roofline denominators): every SM runs
// eight 256-thread CTAs whose threads each advance eight independent FMA chains in registers, so
// the FMA pipes, not latency or memory, set the time.
#include "common.cuh"
#include "internal.h"

namespace pt {

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(T* __restrict__ out, int iters, T a, T b) {
  T x0 = T(threadIdx.x), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
  T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = fma(x0, a, b);
      x1 = fma(x1, a, b);
      x2 = fma(x2, a, b);
      x3 = fma(x3, a, b);
      x4 = fma(x4, a, b);
      x5 = fma(x5, a, b);
      x6 = fma(x6, a, b);
      x7 = fma(x7, a, b);
    }
  }
  // the sum keeps every chain live
  out[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <class T>
double fma_tflops(pt_ctx* ctx, int iters, cudaStream_t st) {
  const int blocks = ctx->num_sms * 8, threads = 256;
  T* out = static_cast<T*>(ctx->get("peaks_out", size_t(blocks) * threads * sizeof(T)));
  PT_LAUNCH(k_fma_chains<T>, blocks, threads, 0, st, out, 10, T(0.999), T(0.001));  // warm-up
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PT_CUDA_CHECK(cudaEventCreate(&e0));
  PT_CUDA_CHECK(cudaEventCreate(&e1));
  float ms = 0.f;
  try {
    PT_CUDA_CHECK(cudaEventRecord(e0, st));
    PT_LAUNCH(k_fma_chains<T>, blocks, threads, 0, st, out, iters, T(0.999), T(0.001));
    PT_CUDA_CHECK(cudaEventRecord(e1, st));
    PT_CUDA_CHECK(cudaEventSynchronize(e1));
    PT_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * 8 * 16 * double(iters) * blocks * threads;
  return flops / (double(ms) * 1e-3) / 1e12;
}

}  // namespace

void alu_peaks(pt_ctx* ctx, double* fp32_tflops, double* fp64_tflops, cudaStream_t st) {
  *fp32_tflops = fma_tflops<float>(ctx, 20000, st);  // ~1.6 PFLOP of work: tens of ms
  *fp64_tflops = fma_tflops<double>(ctx, 400, st);
}

}  // namespace pt
