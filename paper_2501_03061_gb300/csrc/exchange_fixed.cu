// Pair-FFT exchange on cubic grids with a compile-time side N (Sec. IV-A1, Eq. vxdiag): dispatch of
// one pair batch to the kernels of exchange_fixed_kernels.cuh, with 256 threads per CTA here and,
// in FP32, 128 or 512 from exchange_fixed_ft.cu when the context's "fft_threads" asks for them.
#include "exchange_fixed_kernels.cuh"

namespace pt {

// FP32 batches with 128 or 512 threads per CTA (exchange_fixed_ft.cu)
void exchange_batch_fixed_ft(int ft, int n, const c64* src, const c64* tgt, const double* occ, const PairDesc* pairs,
                             int np, const TargetDesc* tgts, int nt, const Contrib* contribs, const float* ktab,
                             const c64* tw, c64* scratch, c64* out, cudaStream_t st);

template <class T>
void exchange_batch_fixed(int n, const cx<T>* src, const cx<T>* tgt, const double* occ, const PairDesc* pairs, int np,
                          const TargetDesc* tgts, int nt, const Contrib* contribs, const T* ktab, const cx<T>* tw,
                          cx<T>* scratch, cx<T>* out, cudaStream_t st, int ft) {
  if constexpr (sizeof(T) == 4) {
    if (ft == 128 || ft == 512) {
      exchange_batch_fixed_ft(ft, n, src, tgt, occ, pairs, np, tgts, nt, contribs, ktab, tw, scratch, out, st);
      return;
    }
  }
  switch (n) {
#define PT_CASE(s)                                                                                      \
  case s:                                                                                               \
    batch_n<s, T, 256>(src, tgt, occ, pairs, np, tgts, nt, contribs, ktab, tw, scratch, out, st);            \
    return;
    PT_FIXED_SIZES(PT_CASE)
#undef PT_CASE
    default:
      fail(PT_INVALID_ARG, "no compile-time FFT kernels for this grid side");
  }
}

template void exchange_batch_fixed<float>(int, const c64*, const c64*, const double*, const PairDesc*, int,
                                          const TargetDesc*, int, const Contrib*, const float*, const c64*, c64*, c64*,
                                          cudaStream_t, int);
template void exchange_batch_fixed<double>(int, const c128*, const c128*, const double*, const PairDesc*, int,
                                           const TargetDesc*, int, const Contrib*, const double*, const c128*, c128*,
                                           c128*, cudaStream_t, int);

}  // namespace pt
