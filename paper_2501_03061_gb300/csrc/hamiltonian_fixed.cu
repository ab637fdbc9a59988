// H psi = P_sph[ 1/2 (-i grad + A)^2 psi + V_loc psi + alpha X ] (Eq. 1) on cubic grids with a
// compile-time side N: the three passes of hamiltonian.cu (x/y plane transforms of psi and of
// y = V_loc psi + alpha X; one column kernel that transforms both along z, combines
// |G + A|^2/2 FFT(psi) + FFT(y) inside the sphere |G|^2/2 <= Ecut and transforms back along z; an
// inverse plane pass), with the FFT stages of fft_fixed.cuh.
#include <algorithm>

#include "fft_fixed.cuh"
#include "internal.h"

namespace pt {

namespace {

constexpr int FT = 256;

template <int N, class T>
constexpr size_t tile_bytes_n() {
  return size_t(N) * kPitch<N> * sizeof(cx<T>);
}

// item k of the batch: psi_{j0+k/2} (k even) or y_{j0+k/2} = V_loc psi + alpha X (k odd)
template <int N, class T>
__global__ void __launch_bounds__(FT) k_hx_fwd_plane(const cx<T>* __restrict__ psi, const T* __restrict__ vloc,
                                                     const cx<T>* __restrict__ X, T alpha, int j0,
                                                     cx<T>* __restrict__ scratch, const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = buf + N * kPitch<N>;
  constexpr int PL = N * N;
  constexpr size_t NG = size_t(N) * N * N;
  const int z = blockIdx.x, k = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += FT) tw[t] = twg[t];
  const size_t off = size_t(j0 + (k >> 1)) * NG + size_t(z) * PL;
  const cx<T>* f = psi + off;
  if (k & 1) {
    const T* v = vloc + size_t(z) * PL;
    const cx<T>* xx = X ? X + off : nullptr;
#pragma unroll 8
    for (int e = threadIdx.x; e < PL; e += FT) {
      const int yy = e / N, x = e - yy * N;
      cx<T> val = f[e] * v[e];
      if (xx) val = val + xx[e] * alpha;
      buf[yy * kPitch<N> + x] = val;
    }
  } else {
#pragma unroll 8
    for (int e = threadIdx.x; e < PL; e += FT) {
      const int yy = e / N, x = e - yy * N;
      buf[yy * kPitch<N> + x] = f[e];
    }
  }
  __syncthreads();
  cfft_fast<N, false, FT>(buf, tw);
  cfft_slow<N, false, FT>(buf, tw);
  cx<T>* o = scratch + size_t(k) * NG + size_t(z) * PL;
#pragma unroll 8
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int yy = e / N, x = e - yy * N;
    o[e] = buf[yy * kPitch<N> + x];
  }
}

template <int N, class T>
__global__ void __launch_bounds__(FT) k_hx_column(cx<T>* __restrict__ scratch, const double* __restrict__ g2,
                                                  double ecut, KinField kf, T inv_ng,
                                                  const cx<T>* __restrict__ twg,
                                                  const unsigned long long* __restrict__ masks) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* ba = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* bb = ba + N * kPitch<N>;
  cx<T>* tw = bb + N * kPitch<N>;
  constexpr size_t NG = size_t(N) * N * N;
  const int yrow = blockIdx.x, j = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += FT) tw[t] = twg[t];
  // FP32 form: the sphere test from the exact FP64 masks, the kinetic factor in FP32 from per-axis
  // terms (an FP64 operation per grid point would take this pass's time on this part's FP64 pipe)
  __shared__ unsigned long long mrow[N];
  __shared__ float kx[N], kz[N];
  __shared__ float ky;
  if constexpr (sizeof(T) == 4) {
    for (int t = threadIdx.x; t < N; t += FT) {
      mrow[t] = masks[size_t(yrow) * N + t];
      const double w = double(wrapped_freq(t, N));
      kx[t] = float(0.5 * g2[t] + (kf.on ? w * kf.c[0] : 0.0));
      kz[t] = float(0.5 * g2[2 * N + t] + (kf.on ? w * kf.c[2] : 0.0));
    }
    if (threadIdx.x == 0)
      ky = float(0.5 * g2[N + yrow] + (kf.on ? double(wrapped_freq(yrow, N)) * kf.c[1] + kf.a2h : 0.0));
  }
  cx<T>* fa = scratch + size_t(2 * j) * NG;
  cx<T>* fb = fa + NG;
#pragma unroll 8
  for (int e = threadIdx.x; e < N * N; e += FT) {
    const int z = e / N, x = e - z * N;
    const size_t gi = (size_t(z) * N + yrow) * N + x;
    ba[z * kPitch<N> + x] = fa[gi];
    bb[z * kPitch<N> + x] = fb[gi];
  }
  __syncthreads();
  cfft_slow<N, false, FT>(ba, tw);
  cfft_slow<N, false, FT>(bb, tw);
  if constexpr (sizeof(T) == 4) {
#pragma unroll 8
    for (int e = threadIdx.x; e < N * N; e += FT) {
      const int z = e / N, x = e - z * N;
      cx<T> v = czero<T>();
      if ((mrow[x] >> z) & 1ull) {
        const float kin = kx[x] + (ky + kz[z]);  // 1/2 |G + A|^2
        v = (ba[z * kPitch<N> + x] * kin + bb[z * kPitch<N> + x]) * inv_ng;
      }
      ba[z * kPitch<N> + x] = v;
    }
  } else {
    // |G|^2 and the sphere test in FP64 so that the cutoff boundary does not depend on the precision
    const double* g2x = g2;
    const double* g2y = g2 + N;
    const double* g2z = g2 + 2 * N;
#pragma unroll 8
    for (int e = threadIdx.x; e < N * N; e += FT) {
      const int z = e / N, x = e - z * N;
      const double half = 0.5 * (g2x[x] + g2y[yrow] + g2z[z]);
      cx<T> v = czero<T>();
      if (half <= ecut) {
        const double kin = half + kin_shift(kf, x, yrow, z, N, N, N);  // 1/2 |G + A|^2
        v = (ba[z * kPitch<N> + x] * T(kin) + bb[z * kPitch<N> + x]) * inv_ng;
      }
      ba[z * kPitch<N> + x] = v;
    }
  }
  __syncthreads();
  cfft_slow<N, true, FT>(ba, tw);
#pragma unroll 8
  for (int e = threadIdx.x; e < N * N; e += FT) {
    const int z = e / N, x = e - z * N;
    fa[(size_t(z) * N + yrow) * N + x] = ba[z * kPitch<N> + x];
  }
}

template <int N, class T>
__global__ void __launch_bounds__(FT) k_hx_inv_plane(const cx<T>* __restrict__ scratch, int j0, cx<T>* __restrict__ out,
                                                     const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = buf + N * kPitch<N>;
  constexpr int PL = N * N;
  constexpr size_t NG = size_t(N) * N * N;
  const int z = blockIdx.x, j = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += FT) tw[t] = twg[t];
  const cx<T>* f = scratch + size_t(2 * j) * NG + size_t(z) * PL;
#pragma unroll 8
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int yy = e / N, x = e - yy * N;
    buf[yy * kPitch<N> + x] = f[e];
  }
  __syncthreads();
  cfft_slow<N, true, FT>(buf, tw);
  cfft_fast<N, true, FT>(buf, tw);
  cx<T>* o = out + size_t(j0 + j) * NG + size_t(z) * PL;
#pragma unroll 8
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int yy = e / N, x = e - yy * N;
    o[e] = buf[yy * kPitch<N> + x];
  }
}

template <int N, class T>
void h_batch_n(const cx<T>* psi, const T* vloc, const cx<T>* X, T alpha, int j0, int nb, cx<T>* scratch,
               const double* g2d, double ecut, KinField kf, const cx<T>* tw, cx<T>* out, cudaStream_t st,
               const unsigned long long* masks) {
  static DeviceOnce once;
  const size_t one = tile_bytes_n<N, T>() + N * sizeof(cx<T>);
  const size_t two = 2 * tile_bytes_n<N, T>() + N * sizeof(cx<T>);
  once([&] {
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_hx_fwd_plane<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(one)));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_hx_inv_plane<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(one)));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_hx_column<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(two)));
  });
  constexpr double ng = double(N) * N * N;
  PT_LAUNCH((k_hx_fwd_plane<N, T>), dim3(N, 2 * nb), FT, one, st, psi, vloc, X, alpha, j0, scratch, tw);
  PT_LAUNCH((k_hx_column<N, T>), dim3(N, nb), FT, two, st, scratch, g2d, ecut, kf, T(1.0 / ng), tw, masks);
  PT_LAUNCH((k_hx_inv_plane<N, T>), dim3(N, nb), FT, one, st, scratch, j0, out, tw);
}

}  // namespace

template <class T>
void apply_h_batch_fixed(int n, const cx<T>* psi, const T* vloc, const cx<T>* X, double alpha, int j0, int nb,
                         cx<T>* scratch, const double* g2d, double ecut, KinField kf, const cx<T>* tw, cx<T>* out,
                         cudaStream_t st, const unsigned long long* masks) {
  if (sizeof(T) == 4 && !masks) fail(PT_INVALID_ARG, "FP32 column pass without its sphere masks");
  switch (n) {
#define PT_CASE(s)                                                                                     \
  case s:                                                                                              \
    h_batch_n<s, T>(psi, vloc, X, T(alpha), j0, nb, scratch, g2d, ecut, kf, tw, out, st, masks);       \
    return;
    PT_FIXED_SIZES(PT_CASE)
#undef PT_CASE
    default:
      fail(PT_INVALID_ARG, "no compile-time FFT kernels for this grid side");
  }
}

template void apply_h_batch_fixed<float>(int, const c64*, const float*, const c64*, double, int, int, c64*,
                                         const double*, double, KinField, const c64*, c64*, cudaStream_t,
                                         const unsigned long long*);
template void apply_h_batch_fixed<double>(int, const c128*, const double*, const c128*, double, int, int, c128*,
                                          const double*, double, KinField, const c128*, c128*, cudaStream_t,
                                          const unsigned long long*);

}  // namespace pt
