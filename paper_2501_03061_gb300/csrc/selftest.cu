// Self-test of the bounded device waits: one CTA waits on a shared-memory mbarrier through the
// deadline-bounded wait of the TMA and tensor-core pipelines.  When nothing arrives the wait gives
// up at its deadline, the kernel records the expiry in device memory and returns normally, and
// the host turns the record into PT_TIMEOUT; the context stays usable.
#include "common.cuh"
#include "internal.h"
#include "tma.cuh"

namespace pt {

namespace {

__global__ void k_wait_selftest(int arrive, unsigned long long timeout_ns, int* __restrict__ err) {
  __shared__ __align__(8) unsigned long long bar_storage;
  const uint32_t bar = smem_u32(&bar_storage);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
    if (!mbar_wait(bar, 0, timeout_ns)) *err = 1;
  }
}

}  // namespace

void wait_selftest(pt_ctx* ctx, int arrive, double timeout_s, cudaStream_t st) {
  int* err = static_cast<int*>(ctx->get("selftest_err", sizeof(int)));
  PT_CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st));
  PT_LAUNCH(k_wait_selftest, 1, 32, 0, st, arrive, static_cast<unsigned long long>(timeout_s * 1e9), err);
  int h = 0;
  PT_CUDA_CHECK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PT_CUDA_CHECK(cudaStreamSynchronize(st));
  if (h) fail(PT_TIMEOUT, "self-test: the device wait gave up at its deadline");
}

}  // namespace pt
