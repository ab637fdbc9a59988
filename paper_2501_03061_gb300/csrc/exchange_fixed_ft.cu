// FP32 compile-time pair-FFT exchange batches with 128 or 512 threads per CTA in the tile kernels:
// the CTA sizes besides the default 256 that the batched form's autotuner times per grid (a
// separate translation unit so that the instantiations compile in parallel).
#include "exchange_fixed_kernels.cuh"

namespace pt {

void exchange_batch_fixed_ft(int ft, int n, const c64* src, const c64* tgt, const double* occ, const PairDesc* pairs,
                             int np, const TargetDesc* tgts, int nt, const Contrib* contribs, const float* ktab,
                             const c64* tw, c64* scratch, c64* out, cudaStream_t st) {
  switch (n) {
#define PT_CASE(s)                                                                                          \
  case s:                                                                                                   \
    if (ft == 128)                                                                                          \
      batch_n<s, float, 128>(src, tgt, occ, pairs, np, tgts, nt, contribs, ktab, tw, scratch, out, st);     \
    else                                                                                                    \
      batch_n<s, float, 512>(src, tgt, occ, pairs, np, tgts, nt, contribs, ktab, tw, scratch, out, st);     \
    return;
    PT_FIXED_SIZES(PT_CASE)
#undef PT_CASE
    default:
      fail(PT_INVALID_ARG, "no compile-time FFT kernels for this grid side");
  }
}

}  // namespace pt
