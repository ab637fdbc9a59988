// Compile-time pair-FFT exchange kernels (Sec. IV-A1, Eq. vxdiag) on cubic grids with side N, with
// FT threads per CTA in the three tile kernels; included by the translation units that instantiate
// them (exchange_fixed.cu: FT = 256; exchange_fixed_ft.cu: the other CTA sizes the batched form's
// autotuner chooses from).
//
// Four passes per pair batch, all on L2-resident pair fields (one scratch field per pair):
//   plane:      rho = conj(src_i) tgt_j on one z-plane, FFT along x and y;
//   column:     on the (z, x) slab of one y-row: FFT along z, multiply by K(G)/Ng, inverse along z;
//   inv plane:  inverse FFT along y and x of one z-plane, in place (once per pair: with tgt == src
//               the mirrored contribution uses v_ji = conj(v_ij));
//   accumulate: W_t -= sum_c d_c partner_c v_c for every target of the batch (streaming).
// The FFT stages come from fft_fixed.cuh, so all tile index arithmetic is compile-time.
#pragma once

#include <algorithm>

#include "exchange_sched.h"
#include "fft_fixed.cuh"
#include "internal.h"

namespace pt {

namespace {

constexpr int AT = 256;  // threads per CTA of the accumulate kernel
constexpr int AE = 4;    // elements per thread of the accumulate kernel

template <int N, class T>
constexpr size_t tile_smem() {
  return size_t(N) * kPitch<N> * sizeof(cx<T>) + size_t(N) * sizeof(cx<T>);
}

template <int N, class T, int FT>
__global__ void __launch_bounds__(FT) k_fx_fwd_plane(const cx<T>* __restrict__ src, const cx<T>* __restrict__ tgt,
                                                     const double* __restrict__ occ,
                                                     const PairDesc* __restrict__ pairs, cx<T>* __restrict__ scratch,
                                                     const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = buf + N * kPitch<N>;
  constexpr int PL = N * N;
  constexpr size_t NG = size_t(N) * N * N;
  const int z = blockIdx.x, p = blockIdx.y;
  const PairDesc pd = pairs[p];
  if (pair_skipped(pd, occ)) return;
  for (int t = threadIdx.x; t < N; t += FT) tw[t] = twg[t];
  const cx<T>* a = src + size_t(pd.i) * NG + size_t(z) * PL;
  const cx<T>* b = tgt + size_t(pd.j) * NG + size_t(z) * PL;
#pragma unroll 4
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int y = e / N, x = e - y * N;
    buf[y * kPitch<N> + x] = cmulc(a[e], b[e]);
  }
  __syncthreads();
  cfft_fast<N, false, FT>(buf, tw);  // x
  cfft_slow<N, false, FT>(buf, tw);  // y
  cx<T>* o = scratch + size_t(p) * NG + size_t(z) * PL;
#pragma unroll 4
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int y = e / N, x = e - y * N;
    o[e] = buf[y * kPitch<N> + x];
  }
}

template <int N, class T, int FT>
__global__ void __launch_bounds__(FT) k_fx_column(cx<T>* __restrict__ scratch, const T* __restrict__ ktab,
                                                  const double* __restrict__ occ, const PairDesc* __restrict__ pairs,
                                                  const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = buf + N * kPitch<N>;
  constexpr size_t NG = size_t(N) * N * N;
  const int y = blockIdx.x, p = blockIdx.y;
  const PairDesc pd = pairs[p];
  if (pair_skipped(pd, occ)) return;
  for (int t = threadIdx.x; t < N; t += FT) tw[t] = twg[t];
  cx<T>* f = scratch + size_t(p) * NG;
  // slab tile: row z, column x (z slow, x fast)
#pragma unroll 4
  for (int e = threadIdx.x; e < N * N; e += FT) {
    const int z = e / N, x = e - z * N;
    buf[z * kPitch<N> + x] = f[(size_t(z) * N + y) * N + x];
  }
  __syncthreads();
  cfft_slow<N, false, FT>(buf, tw);  // z
#pragma unroll 4
  for (int e = threadIdx.x; e < N * N; e += FT) {
    const int z = e / N, x = e - z * N;
    buf[z * kPitch<N> + x] = buf[z * kPitch<N> + x] * ktab[(size_t(z) * N + y) * N + x];
  }
  __syncthreads();
  cfft_slow<N, true, FT>(buf, tw);  // inverse z
#pragma unroll 4
  for (int e = threadIdx.x; e < N * N; e += FT) {
    const int z = e / N, x = e - z * N;
    f[(size_t(z) * N + y) * N + x] = buf[z * kPitch<N> + x];
  }
}

template <int N, class T, int FT>
__global__ void __launch_bounds__(FT) k_fx_inv_plane(cx<T>* __restrict__ scratch, const double* __restrict__ occ,
                                                     const PairDesc* __restrict__ pairs,
                                                     const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = buf + N * kPitch<N>;
  constexpr int PL = N * N;
  constexpr size_t NG = size_t(N) * N * N;
  const int z = blockIdx.x, p = blockIdx.y;
  const PairDesc pd = pairs[p];
  if (pair_skipped(pd, occ)) return;
  for (int t = threadIdx.x; t < N; t += FT) tw[t] = twg[t];
  cx<T>* f = scratch + size_t(p) * NG + size_t(z) * PL;
#pragma unroll 4
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int y = e / N, x = e - y * N;
    buf[y * kPitch<N> + x] = f[e];
  }
  __syncthreads();
  cfft_slow<N, true, FT>(buf, tw);  // inverse y
  cfft_fast<N, true, FT>(buf, tw);  // inverse x
#pragma unroll 4
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int y = e / N, x = e - y * N;
    f[e] = buf[y * kPitch<N> + x];
  }
}

// W_t(r) -= sum_c d_c partner_c(r) v_c(r)  (v conjugated for the mirrored half of a symmetric pair)
template <class T>
__global__ void __launch_bounds__(AT) k_fx_accumulate(const cx<T>* __restrict__ scratch, const cx<T>* __restrict__ src,
                                                      const double* __restrict__ occ,
                                                      const TargetDesc* __restrict__ tgts,
                                                      const Contrib* __restrict__ contribs, cx<T>* __restrict__ out,
                                                      size_t ng) {
  const TargetDesc td = tgts[blockIdx.y];
  const size_t e0 = size_t(blockIdx.x) * (AT * AE) + threadIdx.x;
  cx<T> acc[AE];
#pragma unroll
  for (int u = 0; u < AE; ++u) acc[u] = czero<T>();
  for (int c = td.cbeg; c < td.cend; ++c) {
    const Contrib cb = contribs[c];
    const T coef = T(occ[cb.occ]);
    if (coef == T(0)) continue;  // a skipped pair left its scratch field unwritten
    const cx<T>* v = scratch + size_t(cb.slot) * ng;
    const cx<T>* pp = src + size_t(cb.partner) * ng;
#pragma unroll
    for (int u = 0; u < AE; ++u) {
      const size_t e = e0 + size_t(u) * AT;
      if (e < ng) {
        cx<T> w = v[e];
        if (cb.conj) w.im = -w.im;
        acc[u] = acc[u] + cmul(pp[e], w) * coef;
      }
    }
  }
  cx<T>* o = out + size_t(td.t) * ng;
#pragma unroll
  for (int u = 0; u < AE; ++u) {
    const size_t e = e0 + size_t(u) * AT;
    if (e < ng) o[e] = td.first ? czero<T>() - acc[u] : o[e] - acc[u];
  }
}

template <int N, class T, int FT>
void set_fx_attrs() {
  static DeviceOnce once;
  once([] {
    const int bytes = int(tile_smem<N, T>());
    PT_CUDA_CHECK(
        cudaFuncSetAttribute(k_fx_fwd_plane<N, T, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_fx_column<N, T, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PT_CUDA_CHECK(
        cudaFuncSetAttribute(k_fx_inv_plane<N, T, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  });
}

// the four passes of one pair batch with FT threads per CTA in the three tile kernels
template <int N, class T, int FT>
void batch_n(const cx<T>* src, const cx<T>* tgt, const double* occ, const PairDesc* pairs, int np,
             const TargetDesc* tgts, int nt, const Contrib* contribs, const T* ktab, const cx<T>* tw, cx<T>* scratch,
             cx<T>* out, cudaStream_t st) {
  set_fx_attrs<N, T, FT>();
  const size_t smem = tile_smem<N, T>();
  constexpr size_t NG = size_t(N) * N * N;
  PT_LAUNCH((k_fx_fwd_plane<N, T, FT>), dim3(N, np), FT, smem, st, src, tgt, occ, pairs, scratch, tw);
  PT_LAUNCH((k_fx_column<N, T, FT>), dim3(N, np), FT, smem, st, scratch, ktab, occ, pairs, tw);
  PT_LAUNCH((k_fx_inv_plane<N, T, FT>), dim3(N, np), FT, smem, st, scratch, occ, pairs, tw);
  const unsigned chunks = unsigned((NG + AT * AE - 1) / (AT * AE));
  PT_LAUNCH(k_fx_accumulate<T>, dim3(chunks, nt), AT, 0, st, scratch, src, occ, tgts, contribs, out, NG);
}

}  // namespace

}  // namespace pt
