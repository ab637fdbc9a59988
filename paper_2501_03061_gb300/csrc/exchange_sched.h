// Pair schedule of the exchange: batches of pairs (i, j) whose pair fields share one scratch
// slot, and per batch the list of targets with the contributions (pair, partner orbital,
// occupation, conjugation) each target accumulates.
#pragma once

#include <memory>
#include <vector>

#include "common.cuh"
#include "exchange_plan.h"
#include "fft.cuh"

namespace pt {

__device__ __forceinline__ bool pair_skipped(const PairDesc& pd, const double* occ) {
  return occ[pd.o1] == 0.0 && (pd.o2 < 0 || occ[pd.o2] == 0.0);
}

struct ScheduleImpl {
  int N = 0, M = 0, B = 0;
  bool sym = false;
  std::vector<int> pair_off, tgt_off;  // per batch offsets (size nbatch+1)
  PairDesc* d_pairs = nullptr;
  TargetDesc* d_tgts = nullptr;
  Contrib* d_contribs = nullptr;
  std::vector<PairDesc> h_pairs;
  std::vector<TargetDesc> h_tgts;
  std::vector<Contrib> h_contribs;
  int max_pairs = 0, max_tgts = 0;
  long long total_pairs = 0;
  ~ScheduleImpl() {
    cudaFree(d_pairs);
    cudaFree(d_tgts);
    cudaFree(d_contribs);
  }
};

// plan_pairs (tiles of B x B orbitals) with its tables copied to the device
std::shared_ptr<ScheduleImpl> build_schedule(int N, int M, bool sym, int B);

// the three generic tile passes for one pair batch on caller-provided device buffers
template <class T>
void exchange_batch_generic(const GridPlan& gp, const cx<T>* src, const cx<T>* tgt, const double* occ,
                            const PairDesc* pairs, int np, const TargetDesc* tgts, int nt, const Contrib* contribs,
                            const T* ktab, const cx<T>* tw, cx<T>* scratch, cx<T>* out, cudaStream_t st);
// the same passes with compile-time FFT kernels for a cubic grid of side n (fixed_cubic)
// (ft: threads per CTA of the tile kernels, 256, or in FP32 also 128 or 512)
template <class T>
void exchange_batch_fixed(int n, const cx<T>* src, const cx<T>* tgt, const double* occ, const PairDesc* pairs, int np,
                          const TargetDesc* tgts, int nt, const Contrib* contribs, const T* ktab, const cx<T>* tw,
                          cx<T>* scratch, cx<T>* out, cudaStream_t st, int ft = 256);
double kernel_value(const pt_kernel& k, double G2);

bool exchange64_applies(const pt_grid& g);
// FP32 64^3 path with TMA staging; sets a device error word on a wait timeout (see exchange_check)
// fused: the three-role form (A, B, and CD: C's inverse plane transforms inside the accumulate)
void exchange64_tma(pt_ctx* ctx, const ScheduleImpl& sch, const c64* src, const double* occ, const c64* tgt, int M,
                    c64* out, const float* ktab, const c64* tw, cudaStream_t st, bool fused = false);
// FP32 64^3 path as one persistent cooperative launch (exchange64_persist.cu); returns the pair FFTs
long long exchange64_persist(pt_ctx* ctx, const c64* src, const double* occ, int N, const c64* tgt, int M, bool sym,
                             c64* out, const float* ktab, const c64* tw, cudaStream_t st);
// synchronise st and fail with PT_TIMEOUT if a bounded device wait expired
void exchange_check(pt_ctx* ctx, cudaStream_t st);

}  // namespace pt
