// Orbitals as their plane-wave coefficients in the Ecut sphere (the orbital basis of Sec. VI:
// plane waves with |G|^2/2 <= Ecut), on cubic grids with a compile-time side N <= 64.
//
// c_j(G) = FFT(phi_j)(G) / sqrt(Ng) for the plane waves G of the sphere.  The transform is
// unitary, so every inner product over the grid (with its volume element dV) is the same sum over
// the coefficients, and a field inside the sphere is represented exactly by them.  The PT-IM step
// holds its orbital blocks (iterates, Anderson history, ACE operator, residuals) as coefficient
// vectors: at 64^3 with Ecut = 10 Ha, 13,037 plane waves against 262,144 grid points.  Real space
// is entered only where the method needs it: the local potential of H, the exchange and the
// density.
//
// Layout of a coefficient vector: the (y, x) columns of the grid in row-major order and, in each,
// the z of the sphere ascending; col_off[y N + x] is the index of the column's first plane wave.
// Vectors are padded with zeros to npad (a multiple of 64); every kernel here that writes a vector
// writes its padding as zeros.
//
// Transforms, with the FFT stages of fft_fixed.cuh on N x N shared-memory tiles and one
// N^3 scratch field per orbital of a batch:
//   to coefficients  plane pass (x, y transforms of each z plane) -> column pass (z transforms of
//                    each y slab, gather of the sphere, 1/sqrt(Ng))
// Only the y slabs that hold sphere points (29 of 64 at 64^3, Ecut = 10 Ha) are transformed along z
// and moved between the passes; the plane pass takes the others as zeros (the input conversion,
// which measures the weight outside the sphere, transforms every slab).
//   to real space    column pass (scatter into zeroed columns, inverse z) -> plane pass (inverse
//                    y, x, 1/sqrt(Ng))
//   H                column pass (scatter, inverse z) -> plane pass (inverse y, x; times V_loc;
//                    forward x, y) -> column pass (forward z; |G + A|^2/2 c + FFT(V psi)/Ng +
//                    alpha X at the sphere points): Eq. 1 with the sphere projection
#include <algorithm>
#include <cmath>
#include <vector>

#include "fft_fixed.cuh"
#include "internal.h"

namespace pt {

namespace {

constexpr int FT = 256;

struct PwTables {
  int* col_off = nullptr;
  int* xyz = nullptr;
  int* yact = nullptr;
  ~PwTables() {
    cudaFree(col_off);
    cudaFree(xyz);
    cudaFree(yact);
  }
};

template <int N, class T>
constexpr size_t pw_tile_bytes() {
  return size_t(N) * kPitch<N> * sizeof(cx<T>);
}

// x, y transforms of plane z of orbital j0 + j (real space) into scratch field j
template <int N, class T>
__global__ void __launch_bounds__(FT) k_pw_fwd_plane(const cx<T>* __restrict__ src, int j0, cx<T>* __restrict__ scratch,
                                                     unsigned long long ykeep, const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = buf + N * kPitch<N>;
  constexpr int PL = N * N;
  constexpr size_t NG = size_t(N) * N * N;
  const int z = blockIdx.x, j = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += FT) tw[t] = twg[t];
  const cx<T>* f = src + size_t(j0 + j) * NG + size_t(z) * PL;
#pragma unroll 8
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int yy = e / N, x = e - yy * N;
    buf[yy * kPitch<N> + x] = f[e];
  }
  __syncthreads();
  cfft_fast<N, false, FT>(buf, tw);
  cfft_slow<N, false, FT>(buf, tw);
  cx<T>* o = scratch + size_t(j) * NG + size_t(z) * PL;
#pragma unroll 8
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int yy = e / N, x = e - yy * N;
    if ((ykeep >> yy) & 1ull) o[e] = buf[yy * kPitch<N> + x];  // rows the column pass reads
  }
}

// z transforms of slab y of scratch field j, then at the sphere points:
//   COMB = false: out = v * scale, with the per-(j, y) sums of |v|^2 inside and outside the sphere
//                 in part[2 (j N + y) + {0, 1}] (the test that the field lay in the sphere);
//   COMB = true:  out = |G + A|^2/2 cin + v * scale + alpha X  (H of the column pass).
template <int N, class T, bool COMB>
__global__ void __launch_bounds__(FT) k_pw_fwd_col(const cx<T>* __restrict__ scratch, int j0, cx<T>* __restrict__ out,
                                                   size_t npw, size_t npad, const int* __restrict__ col_off,
                                                   const unsigned long long* __restrict__ masks, T scale,
                                                   double* __restrict__ part, const cx<T>* __restrict__ cin,
                                                   const cx<T>* __restrict__ X, T alpha,
                                                   const double* __restrict__ g2, KinField kf,
                                                   const int* __restrict__ ylist, const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* ba = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = ba + N * kPitch<N>;
  constexpr size_t NG = size_t(N) * N * N;
  const int yrow = ylist ? ylist[blockIdx.x] : int(blockIdx.x), j = blockIdx.y;
  __shared__ unsigned long long mrow[N];
  __shared__ int coff[N];
  __shared__ float kxf[N], kzf[N];
  __shared__ float kyf;
  for (int t = threadIdx.x; t < N; t += FT) {
    tw[t] = twg[t];
    mrow[t] = masks[size_t(yrow) * N + t];
    coff[t] = col_off[size_t(yrow) * N + t];
    if constexpr (COMB && sizeof(T) == 4) {
      const double w = double(wrapped_freq(t, N));
      kxf[t] = float(0.5 * g2[t] + (kf.on ? w * kf.c[0] : 0.0));
      kzf[t] = float(0.5 * g2[2 * N + t] + (kf.on ? w * kf.c[2] : 0.0));
    }
  }
  if constexpr (COMB && sizeof(T) == 4) {
    if (threadIdx.x == 0)
      kyf = float(0.5 * g2[N + yrow] + (kf.on ? double(wrapped_freq(yrow, N)) * kf.c[1] + kf.a2h : 0.0));
  }
  const cx<T>* fa = scratch + size_t(j) * NG;
#pragma unroll 8
  for (int e = threadIdx.x; e < N * N; e += FT) {
    const int z = e / N, x = e - z * N;
    ba[z * kPitch<N> + x] = fa[(size_t(z) * N + yrow) * N + x];
  }
  __syncthreads();
  cfft_slow<N, false, FT>(ba, tw);
  cx<T>* o = out + size_t(j0 + j) * npad;
  float s_in = 0.f, s_out = 0.f;  // the sphere test needs no more (and FP64 per point is slow here)
  for (int e = threadIdx.x; e < N * N; e += FT) {
    const int z = e / N, x = e - z * N;
    const unsigned long long m = mrow[x];
    const cx<T> v = ba[z * kPitch<N> + x];
    if ((m >> z) & 1ull) {
      const size_t p = size_t(coff[x]) + size_t(__popcll(m & ((1ull << z) - 1ull)));
      if constexpr (COMB) {
        const cx<T>* ci = cin + size_t(j0 + j) * npad;
        T kin;
        if constexpr (sizeof(T) == 4) {
          kin = kxf[x] + (kyf + kzf[z]);  // 1/2 |G + A|^2, as in the grid form's column pass
        } else {
          kin = 0.5 * (g2[x] + g2[N + yrow] + g2[2 * N + z]) + kin_shift(kf, x, yrow, z, N, N, N);
        }
        cx<T> r = ci[p] * kin + v * scale;
        if (X) r = r + X[size_t(j0 + j) * npad + p] * alpha;
        o[p] = r;
      } else {
        o[p] = v * scale;
        s_in += float(v.re) * float(v.re) + float(v.im) * float(v.im);
      }
    } else if constexpr (!COMB) {
      s_out += float(v.re) * float(v.re) + float(v.im) * float(v.im);
    }
  }
  if (blockIdx.x == 0)
    for (size_t p = npw + threadIdx.x; p < npad; p += FT) o[p] = czero<T>();
  if constexpr (!COMB) {
    for (int off = 16; off; off >>= 1) {
      s_in += __shfl_down_sync(0xffffffffu, s_in, off);
      s_out += __shfl_down_sync(0xffffffffu, s_out, off);
    }
    __shared__ float red[2][FT / 32];
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = s_in;
      red[1][threadIdx.x >> 5] = s_out;
    }
    __syncthreads();
    if (threadIdx.x == 0 && part) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < FT / 32; ++w) {
        a += red[0][w];
        b += red[1][w];
      }
      part[2 * (size_t(j0 + j) * N + yrow)] = a;
      part[2 * (size_t(j0 + j) * N + yrow) + 1] = b;
    }
  }
}

// slab y of scratch field j: the sphere coefficients of orbital j0 + j scattered into zeroed z
// columns, inverse z transforms
template <int N, class T>
__global__ void __launch_bounds__(FT) k_pw_inv_col(const cx<T>* __restrict__ c, int j0, size_t npad,
                                                   cx<T>* __restrict__ scratch, const int* __restrict__ col_off,
                                                   const unsigned long long* __restrict__ masks,
                                                   const int* __restrict__ ylist, const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* ba = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = ba + N * kPitch<N>;
  constexpr size_t NG = size_t(N) * N * N;
  const int yrow = ylist[blockIdx.x], j = blockIdx.y;
  __shared__ unsigned long long mrow[N];
  __shared__ int coff[N];
  for (int t = threadIdx.x; t < N; t += FT) {
    tw[t] = twg[t];
    mrow[t] = masks[size_t(yrow) * N + t];
    coff[t] = col_off[size_t(yrow) * N + t];
  }
  __syncthreads();
  const cx<T>* ci = c + size_t(j0 + j) * npad;
  for (int e = threadIdx.x; e < N * N; e += FT) {
    const int z = e / N, x = e - z * N;
    const unsigned long long m = mrow[x];
    cx<T> v = czero<T>();
    if ((m >> z) & 1ull) v = ci[size_t(coff[x]) + size_t(__popcll(m & ((1ull << z) - 1ull)))];
    ba[z * kPitch<N> + x] = v;
  }
  __syncthreads();
  cfft_slow<N, true, FT>(ba, tw);
  cx<T>* fa = scratch + size_t(j) * NG;
#pragma unroll 8
  for (int e = threadIdx.x; e < N * N; e += FT) {
    const int z = e / N, x = e - z * N;
    fa[(size_t(z) * N + yrow) * N + x] = ba[z * kPitch<N> + x];
  }
}

// plane z of scratch field j: inverse y, x transforms;
//   VMUL = false: out (real space, orbital j0 + j) = result * scale;
//   VMUL = true:  result * V_loc, forward x, y transforms, back into the scratch plane.
template <int N, class T, bool VMUL>
__global__ void __launch_bounds__(FT) k_pw_inv_plane(cx<T>* __restrict__ scratch, int j0, cx<T>* __restrict__ out,
                                                     const T* __restrict__ vloc, T scale, unsigned long long ykeep,
                                                     const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = buf + N * kPitch<N>;
  constexpr int PL = N * N;
  constexpr size_t NG = size_t(N) * N * N;
  const int z = blockIdx.x, j = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += FT) tw[t] = twg[t];
  cx<T>* f = scratch + size_t(j) * NG + size_t(z) * PL;
#pragma unroll 8
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int yy = e / N, x = e - yy * N;
    // rows ky outside the sphere's extent are zero: not written by the column pass, not read here
    buf[yy * kPitch<N> + x] = ((ykeep >> yy) & 1ull) ? f[e] : czero<T>();
  }
  __syncthreads();
  cfft_slow<N, true, FT>(buf, tw);
  cfft_fast<N, true, FT>(buf, tw);
  if constexpr (VMUL) {
    const T* v = vloc + size_t(z) * PL;
#pragma unroll 8
    for (int e = threadIdx.x; e < PL; e += FT) {
      const int yy = e / N, x = e - yy * N;
      buf[yy * kPitch<N> + x] = buf[yy * kPitch<N> + x] * v[e];
    }
    __syncthreads();
    cfft_fast<N, false, FT>(buf, tw);
    cfft_slow<N, false, FT>(buf, tw);
#pragma unroll 8
    for (int e = threadIdx.x; e < PL; e += FT) {
      const int yy = e / N, x = e - yy * N;
      if ((ykeep >> yy) & 1ull) f[e] = buf[yy * kPitch<N> + x];
    }
  } else {
    cx<T>* o = out + size_t(j0 + j) * NG + size_t(z) * PL;
#pragma unroll 8
    for (int e = threadIdx.x; e < PL; e += FT) {
      const int yy = e / N, x = e - yy * N;
      o[e] = buf[yy * kPitch<N> + x] * scale;
    }
  }
}

// the two sums of part over (j, y) in a fixed order
__global__ void k_pw_part_sum(const double* __restrict__ part, size_t n, double* __restrict__ out) {
  double a = 0.0, b = 0.0;
  for (size_t e = threadIdx.x; e < n; e += blockDim.x) {
    a += part[2 * e];
    b += part[2 * e + 1];
  }
  __shared__ double red[2][32];
  for (int off = 16; off; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      s += red[0][w];
      t += red[1][w];
    }
    out[0] = s;
    out[1] = t;
  }
}

// 1/2 |G + A|^2 of every plane wave (FP64), zero on the padding
__global__ void k_pw_kinetic(const int* __restrict__ xyz, size_t npad, int n, const double* __restrict__ g2, KinField kf,
                             double* __restrict__ kin) {
  const size_t p = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= npad) return;
  const int c = xyz[p];
  if (c < 0) {
    kin[p] = 0.0;
    return;
  }
  const int x = c & 255, y = (c >> 8) & 255, z = c >> 16;
  kin[p] = 0.5 * (g2[x] + g2[n + y] + g2[2 * n + z]) + kin_shift(kf, x, y, z, n, n, n);
}

// r_j(G) <- r_j(G) / (1 + i dt/2 (|G + A|^2/2 - Re A_jj)) at every plane wave of every orbital
template <class T>
__global__ void k_pw_precond(cx<T>* __restrict__ r, int M, size_t npw, size_t npad, const double* __restrict__ kin,
                             const c128* __restrict__ A, int lda, T hdt) {
  const size_t total = size_t(M) * npad;
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += size_t(gridDim.x) * blockDim.x) {
    const size_t j = e / npad, p = e - j * npad;
    if (p >= npw) continue;
    const T th = hdt * T(kin[p] - A[j * size_t(lda) + j].re);
    const T s = T(1) / (T(1) + th * th);
    r[e] = cmul(r[e], cx<T>{s, -th * s});  // (1 - i th) / (1 + th^2)
  }
}

__global__ void k_pw_to_float(const double* __restrict__ a, size_t n, float* __restrict__ b) {
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x)
    b[e] = float(a[e]);
}

template <int N, class T>
void set_pw_attrs() {
  static DeviceOnce once;
  once([] {
    const int bytes = int(pw_tile_bytes<N, T>() + N * sizeof(cx<T>));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pw_fwd_plane<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pw_fwd_col<N, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pw_fwd_col<N, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pw_inv_col<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PT_CUDA_CHECK(
        cudaFuncSetAttribute(k_pw_inv_plane<N, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pw_inv_plane<N, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  });
}

// orbitals per batch: one N^3 scratch field each, within the context's scratch budget (the same
// buffer as the Hamiltonian's grid form, which holds two fields per orbital of its batches)
template <class T>
int pw_batch(pt_ctx* ctx, const pt_grid& g, int M, cx<T>** scratch) {
  const size_t field = ng_of(g) * sizeof(cx<T>);
  const int mb = int(std::max<size_t>(1, exchange_scratch_budget(ctx) / (2 * field)));
  const int pb = std::min(M, 2 * mb);
  *scratch = static_cast<cx<T>*>(ctx->get("h_scratch", size_t(pb) * field));  // no more than M fields
  return pb;
}

enum class PwOp { ToPw, ToGrid, H };

template <int N, class T>
void pw_run_n(pt_ctx* ctx, const PwBasis& b, PwOp op, const cx<T>* in, int M, cx<T>* out, double* part, const T* vloc,
              const cx<T>* X, T alpha, KinField kf, const pt_grid& g, cudaStream_t st) {
  set_pw_attrs<N, T>();
  const FftTables& ft = fft_tables(ctx, g, sizeof(T) == 4 ? PT_FP32 : PT_FP64);
  const cx<T>* tw = static_cast<const cx<T>*>(ft.tw);
  const double* g2d = static_cast<const double*>(ft.g2d);
  const size_t bytes = pw_tile_bytes<N, T>() + N * sizeof(cx<T>);
  constexpr double ng = double(N) * N * N;
  const T unit = T(1.0 / std::sqrt(ng));
  cx<T>* scratch = nullptr;
  const int pb = pw_batch<T>(ctx, g, M, &scratch);
  for (int j0 = 0; j0 < M; j0 += pb) {
    const int nb = std::min(pb, M - j0);
    switch (op) {
      case PwOp::ToPw:
        if (part) {  // the sphere test sums |FFT|^2 over every slab
          PT_LAUNCH((k_pw_fwd_plane<N, T>), dim3(N, nb), FT, bytes, st, in, j0, scratch, ~0ull, tw);
          PT_LAUNCH((k_pw_fwd_col<N, T, false>), dim3(N, nb), FT, bytes, st, scratch, j0, out, b.npw, b.npad,
                    b.col_off, b.masks, unit, part, nullptr, nullptr, T(0), g2d, kf, nullptr, tw);
        } else {  // the slabs that hold sphere points only
          PT_LAUNCH((k_pw_fwd_plane<N, T>), dim3(N, nb), FT, bytes, st, in, j0, scratch, b.ymask, tw);
          PT_LAUNCH((k_pw_fwd_col<N, T, false>), dim3(b.ny_act, nb), FT, bytes, st, scratch, j0, out, b.npw, b.npad,
                    b.col_off, b.masks, unit, nullptr, nullptr, nullptr, T(0), g2d, kf, b.yact, tw);
        }
        break;
      case PwOp::ToGrid:
        PT_LAUNCH((k_pw_inv_col<N, T>), dim3(b.ny_act, nb), FT, bytes, st, in, j0, b.npad, scratch, b.col_off, b.masks,
                  b.yact, tw);
        PT_LAUNCH((k_pw_inv_plane<N, T, false>), dim3(N, nb), FT, bytes, st, scratch, j0, out, nullptr, unit, b.ymask,
                  tw);
        break;
      case PwOp::H:
        PT_LAUNCH((k_pw_inv_col<N, T>), dim3(b.ny_act, nb), FT, bytes, st, in, j0, b.npad, scratch, b.col_off, b.masks,
                  b.yact, tw);
        PT_LAUNCH((k_pw_inv_plane<N, T, true>), dim3(N, nb), FT, bytes, st, scratch, j0, nullptr, vloc, T(1), b.ymask,
                  tw);
        PT_LAUNCH((k_pw_fwd_col<N, T, true>), dim3(b.ny_act, nb), FT, bytes, st, scratch, j0, out, b.npw, b.npad,
                  b.col_off, b.masks, T(1.0 / ng), nullptr, in, X, alpha, g2d, kf, b.yact, tw);
        break;
    }
  }
}

template <class T>
void pw_run(pt_ctx* ctx, const PwBasis& b, PwOp op, const cx<T>* in, int M, cx<T>* out, double* part, const T* vloc,
            const cx<T>* X, T alpha, KinField kf, cudaStream_t st) {
  switch (b.grid.nx) {
#define PT_CASE(s)                                                                                 \
  case s:                                                                                          \
    pw_run_n<s, T>(ctx, b, op, in, M, out, part, vloc, X, alpha, kf, b.grid, st);                  \
    return;
    PT_FIXED_SIZES(PT_CASE)
#undef PT_CASE
    default:
      fail(PT_INVALID_ARG, "plane-wave basis: no compile-time FFT kernels for this grid side");
  }
}

}  // namespace

bool pw_applies(const pt_grid& g) { return fixed_cubic(g) && g.nx <= 64; }

const PwBasis& pw_basis(pt_ctx* ctx, const pt_grid& g, double ecut, cudaStream_t st) {
  if (!pw_applies(g)) fail(PT_INVALID_ARG, "plane-wave basis: cubic grids of side <= 64 with compile-time FFTs");
  char key[192];
  snprintf(key, sizeof(key), "pw_basis:%d:%.17g:%.17g:%.17g:%.17g", g.nx, g.L[0], g.L[1], g.L[2], ecut);
  auto it = ctx->caches.find(key);
  if (it != ctx->caches.end()) return *std::static_pointer_cast<PwBasis>(it->second);
  const int n = g.nx;
  const FftTables& ft = fft_tables(ctx, g, PT_FP64);
  const unsigned long long* masks = sphere_masks(ctx, g, static_cast<const double*>(ft.g2d), ecut, st);
  std::vector<unsigned long long> hm(size_t(n) * n);
  PT_CUDA_CHECK(cudaMemcpyAsync(hm.data(), masks, hm.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  PT_CUDA_CHECK(cudaStreamSynchronize(st));
  std::vector<int> off(size_t(n) * n);
  std::vector<int> xyz;
  for (int y = 0; y < n; ++y)
    for (int x = 0; x < n; ++x) {
      off[size_t(y) * n + x] = int(xyz.size());
      const unsigned long long m = hm[size_t(y) * n + x];
      for (int z = 0; z < n; ++z)
        if ((m >> z) & 1ull) xyz.push_back(x | (y << 8) | (z << 16));
    }
  std::vector<int> yact;
  unsigned long long ymask = 0;
  for (int y = 0; y < n; ++y)
    for (int x = 0; x < n; ++x)
      if (hm[size_t(y) * n + x]) {
        yact.push_back(y);
        ymask |= 1ull << y;
        break;
      }
  auto b = std::make_shared<PwBasis>();
  auto tables = std::make_shared<PwTables>();
  b->grid = g;
  b->ecut = ecut;
  b->npw = xyz.size();
  b->npad = std::max<size_t>(64, (b->npw + 63) / 64 * 64);
  xyz.resize(b->npad, -1);
  PT_CUDA_CHECK(cudaMalloc(&tables->col_off, off.size() * sizeof(int)));
  PT_CUDA_CHECK(cudaMalloc(&tables->xyz, xyz.size() * sizeof(int)));
  PT_CUDA_CHECK(cudaMalloc(&tables->yact, std::max<size_t>(1, yact.size()) * sizeof(int)));
  PT_CUDA_CHECK(cudaMemcpyAsync(tables->col_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  PT_CUDA_CHECK(cudaMemcpyAsync(tables->xyz, xyz.data(), xyz.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  if (!yact.empty())
    PT_CUDA_CHECK(cudaMemcpyAsync(tables->yact, yact.data(), yact.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  PT_CUDA_CHECK(cudaStreamSynchronize(st));  // the host vectors go out of scope
  b->masks = masks;
  b->col_off = tables->col_off;
  b->xyz = tables->xyz;
  b->yact = tables->yact;
  b->ny_act = int(yact.size());
  b->ymask = ymask;
  b->tables = tables;
  ctx->caches[key] = b;
  return *b;
}

template <class T>
double pw_from_grid(pt_ctx* ctx, const PwBasis& b, const cx<T>* phi, int M, cx<T>* c, cudaStream_t st, bool check) {
  const int n = b.grid.nx;
  double* part = static_cast<double*>(ctx->get("pw_part", 2 * size_t(M) * n * sizeof(double) + 2 * sizeof(double)));
  pw_run<T>(ctx, b, PwOp::ToPw, phi, M, c, part, nullptr, nullptr, T(0), KinField{{0, 0, 0}, 0, 0}, st);
  if (!check) return 0.0;
  double* sums = part + 2 * size_t(M) * n;
  PT_LAUNCH(k_pw_part_sum, 1, 1024, 0, st, part, size_t(M) * n, sums);
  double h[2] = {0.0, 0.0};
  PT_CUDA_CHECK(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st));
  PT_CUDA_CHECK(cudaStreamSynchronize(st));
  const double all = h[0] + h[1];
  return all > 0.0 ? h[1] / all : 0.0;
}

template <class T>
void pw_to_grid(pt_ctx* ctx, const PwBasis& b, const cx<T>* c, int M, cx<T>* phi, cudaStream_t st) {
  pw_run<T>(ctx, b, PwOp::ToGrid, c, M, phi, nullptr, nullptr, nullptr, T(0), KinField{{0, 0, 0}, 0, 0}, st);
}

template <class T>
void pw_apply_h(pt_ctx* ctx, const PwBasis& b, const cx<T>* c, int M, cx<T>* out, const double* vloc, const cx<T>* X,
                double alpha, const double* Avec, cudaStream_t st) {
  const size_t ng = ng_of(b.grid);
  const T* vl = nullptr;
  if constexpr (sizeof(T) == 4) {
    float* v32 = static_cast<float*>(ctx->get("pw_vloc32", ng * sizeof(float)));
    PT_LAUNCH(k_pw_to_float, int(std::min<size_t>((ng + 255) / 256, size_t(ctx->num_sms) * 8)), 256, 0, st, vloc, ng,
              v32);
    vl = v32;
  } else {
    vl = vloc;
  }
  pw_run<T>(ctx, b, PwOp::H, c, M, out, nullptr, vl, X, T(alpha), make_kin_field(b.grid, Avec), st);
}

template <class T>
void pw_precondition(pt_ctx* ctx, const PwBasis& b, cx<T>* r, int M, const c128* A, double dt, const double* Avec,
                     cudaStream_t st) {
  const FftTables& ft = fft_tables(ctx, b.grid, PT_FP64);
  double* kin = static_cast<double*>(ctx->get("pw_kinetic", b.npad * sizeof(double)));
  PT_LAUNCH(k_pw_kinetic, int((b.npad + 255) / 256), 256, 0, st, b.xyz, b.npad, b.grid.nx,
            static_cast<const double*>(ft.g2d), make_kin_field(b.grid, Avec), kin);
  const size_t total = size_t(M) * b.npad;
  const int blocks = int(std::max<size_t>(1, std::min<size_t>((total + 255) / 256, size_t(ctx->num_sms) * 8)));
  PT_LAUNCH(k_pw_precond<T>, blocks, 256, 0, st, r, M, b.npw, b.npad, kin, A, M, T(0.5 * dt));
}

template double pw_from_grid<float>(pt_ctx*, const PwBasis&, const c64*, int, c64*, cudaStream_t, bool);
template double pw_from_grid<double>(pt_ctx*, const PwBasis&, const c128*, int, c128*, cudaStream_t, bool);
template void pw_to_grid<float>(pt_ctx*, const PwBasis&, const c64*, int, c64*, cudaStream_t);
template void pw_to_grid<double>(pt_ctx*, const PwBasis&, const c128*, int, c128*, cudaStream_t);
template void pw_apply_h<float>(pt_ctx*, const PwBasis&, const c64*, int, c64*, const double*, const c64*, double,
                                const double*, cudaStream_t);
template void pw_apply_h<double>(pt_ctx*, const PwBasis&, const c128*, int, c128*, const double*, const c128*, double,
                                 const double*, cudaStream_t);
template void pw_precondition<float>(pt_ctx*, const PwBasis&, c64*, int, const c128*, double, const double*,
                                     cudaStream_t);
template void pw_precondition<double>(pt_ctx*, const PwBasis&, c128*, int, const c128*, double, const double*,
                                      cudaStream_t);

}  // namespace pt
