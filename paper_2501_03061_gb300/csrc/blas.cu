// Complex contractions over the grid (CUDA-core form) and streaming vector kernels.
//
//   gram:    C[i][j] = scale * sum_r conj(A_i(r)) B_j(r)      (A: Ng x N1, B: Ng x N2, orbital-major;
//            C: N1 x N2 complex128 row-major).  Split over r, FP64 reduction of the splits.
//   rotate:  Out_j(r) = alpha * sum_k A_k(r) Bm[k][j] + sum_e c_e E_e,j(r)
//            (Bm: N1 x N2 complex128 row-major, converted to the orbital precision).
//   lincomb, sqnorms: streaming kernels over orbital blocks.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace pt {

namespace {

// Summation in the orbital precision: FP64 adds directly; FP32 carries a Kahan
// compensation so long sums keep ~FP32-ulp accuracy without FP64 arithmetic in the
// inner loop (FP64 throughput is a small fraction of FP32 on this part).
template <class T>
struct Acc {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T x) {
    if constexpr (sizeof(T) == 8) {
      s += x;
    } else {
      const T y = x - c;
      const T t = s + y;
      c = (t - s) - y;
      s = t;
    }
  }
  __device__ __forceinline__ double value() const { return double(s) - double(c); }
};

// ---------------------------------------------------------------- gram (A^H B) ----
constexpr int GT = 32;      // output tile (i and j)
constexpr int GK = 32;      // grid points per smem stage
constexpr int GTHREADS = 256;

template <class T>
__global__ void __launch_bounds__(GTHREADS) k_gram(const cx<T>* __restrict__ A, const cx<T>* __restrict__ B,
                                                    int N1, int N2, size_t ng, size_t chunk,
                                                    c128* __restrict__ part) {
  __shared__ cx<T> As[GK][GT + 1];
  __shared__ cx<T> Bs[GK][GT + 1];
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  const size_t r_begin = size_t(blockIdx.z) * chunk;
  const size_t r_end = std::min(ng, r_begin + chunk);
  const int tid = threadIdx.x;
  const int ti = tid % 16, tj = tid / 16;
  Acc<T> acc_re[2][2], acc_im[2][2];
  for (size_t r0 = r_begin; r0 < r_end; r0 += GK) {
    cx<T> acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) acc[a][b] = czero<T>();
    // load 32 orbitals x 32 points of A and B (points fastest: coalesced)
#pragma unroll
    for (int pass = 0; pass < (GT * GK) / GTHREADS; ++pass) {
      const int e = tid + pass * GTHREADS;
      const int k = e % GK, o = e / GK;
      const size_t r = r0 + k;
      cx<T> va = czero<T>(), vb = czero<T>();
      if (r < r_end) {
        if (i0 + o < N1) va = A[size_t(i0 + o) * ng + r];
        if (j0 + o < N2) vb = B[size_t(j0 + o) * ng + r];
      }
      As[k][o] = va;
      Bs[k][o] = vb;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < GK; ++k) {
      const cx<T> a0 = As[k][ti], a1 = As[k][ti + 16];
      const cx<T> b0 = Bs[k][tj], b1 = Bs[k][tj + 16];
      cfma(acc[0][0], conjc(a0), b0);
      cfma(acc[0][1], conjc(a0), b1);
      cfma(acc[1][0], conjc(a1), b0);
      cfma(acc[1][1], conjc(a1), b1);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        acc_re[a][b].add(acc[a][b].re);
        acc_im[a][b].add(acc[a][b].im);
      }
    __syncthreads();
  }
  c128* P = part + size_t(blockIdx.z) * N1 * N2;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + ti + 16 * a, j = j0 + tj + 16 * b;
      if (i < N1 && j < N2) P[size_t(i) * N2 + j] = c128{acc_re[a][b].value(), acc_im[a][b].value()};
    }
}

// FP32 Gram tile of 64 x 64 outputs, 4 x 4 complex per thread, 16 grid points per stage; the
// per-stage sums are folded into Kahan-compensated totals.  With herm, only tiles on or above
// the diagonal run (the reduction mirrors the rest).
constexpr int G4T = 64, G4K = 16, G4THREADS = 256;

__global__ void __launch_bounds__(G4THREADS, 2) k_gram64(const c64* __restrict__ A, const c64* __restrict__ B,
                                                         int N1, int N2, size_t ng, size_t chunk, int herm,
                                                         c128* __restrict__ part) {
  if (herm && blockIdx.y < blockIdx.x) return;
  __shared__ c64 As[G4K][G4T + 1];
  __shared__ c64 Bs[G4K][G4T + 1];
  const int i0 = blockIdx.x * G4T, j0 = blockIdx.y * G4T;
  const size_t r_begin = size_t(blockIdx.z) * chunk;
  const size_t r_end = std::min(ng, r_begin + chunk);
  const int tid = threadIdx.x;
  const int ti = tid % 16, tj = tid / 16;
  Acc<float> sre[4][4], sim[4][4];
  for (size_t r0 = r_begin; r0 < r_end; r0 += G4K) {
#pragma unroll
    for (int pass = 0; pass < (G4T * G4K) / G4THREADS; ++pass) {
      const int e = tid + pass * G4THREADS;
      const int k = e % G4K, o = e / G4K;
      const size_t r = r0 + k;
      c64 va = czero<float>(), vb = czero<float>();
      if (r < r_end) {
        if (i0 + o < N1) va = A[size_t(i0 + o) * ng + r];
        if (j0 + o < N2) vb = B[size_t(j0 + o) * ng + r];
      }
      As[k][o] = va;
      Bs[k][o] = vb;
    }
    __syncthreads();
    c64 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = czero<float>();
#pragma unroll 4
    for (int k = 0; k < G4K; ++k) {
      c64 av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = conjc(As[k][ti + 16 * a]);
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tj + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cfma(acc[a][b], av[a], bv[b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        sre[a][b].add(acc[a][b].re);
        sim[a][b].add(acc[a][b].im);
      }
    __syncthreads();
  }
  c128* P = part + size_t(blockIdx.z) * N1 * N2;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ti + 16 * a, j = j0 + tj + 16 * b;
      if (i < N1 && j < N2) P[size_t(i) * N2 + j] = c128{sre[a][b].value(), sim[a][b].value()};
    }
}

// C = scale * sum of split partials; herm_tile > 0: elements whose tile row is below the tile
// column were not computed and are taken as the conjugate of the mirrored element
__global__ void k_reduce_parts(const c128* __restrict__ part, int nsplit, int N1, int N2, double scale,
                               int herm_tile, c128* __restrict__ C) {
  const size_t n = size_t(N1) * N2;
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int i = int(e / N2), j = int(e % N2);
  const bool mirror = herm_tile > 0 && (i / herm_tile) > (j / herm_tile);
  const size_t src = mirror ? size_t(j) * N2 + i : e;
  double re = 0, im = 0;
  for (int s = 0; s < nsplit; ++s) {
    re += part[size_t(s) * n + src].re;
    im += part[size_t(s) * n + src].im;
  }
  C[e] = mirror ? c128{re * scale, -im * scale} : c128{re * scale, im * scale};
}

// ---------------------------------------------------------------- rotate (A Bm + E) ----
constexpr int RT = 128;   // grid points per CTA
constexpr int JT = 32;    // output orbitals per CTA
constexpr int KC = 16;    // k per smem stage
constexpr int RTHREADS = 256;

template <class T>
struct Epi {
  const cx<T>* e[3];
  cx<T> c[3];
};

template <class T>
__global__ void __launch_bounds__(RTHREADS) k_rotate(const cx<T>* __restrict__ A, const c128* __restrict__ Bm,
                                                      int ldb, int N1, int N2, size_t ng, cx<T> alpha, Epi<T> epi,
                                                      cx<T>* __restrict__ out) {
  __shared__ cx<T> As[KC][RT];
  __shared__ cx<T> Bs[KC][JT];
  const size_t r0 = size_t(blockIdx.x) * RT;
  const int j0 = blockIdx.y * JT;
  const int tid = threadIdx.x;
  const int tr = tid % 32, tj = tid / 32;  // 32 x 8
  cx<T> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = czero<T>();
  for (int k0 = 0; k0 < N1; k0 += KC) {
#pragma unroll
    for (int pass = 0; pass < (KC * RT) / RTHREADS; ++pass) {
      const int e = tid + pass * RTHREADS;
      const int r = e % RT, kk = e / RT;
      const size_t rr = r0 + r;
      cx<T> v = czero<T>();
      if (k0 + kk < N1 && rr < ng) v = A[size_t(k0 + kk) * ng + rr];
      As[kk][r] = v;
    }
    for (int e = tid; e < KC * JT; e += RTHREADS) {
      const int j = e % JT, kk = e / JT;
      cx<T> v = czero<T>();
      if (k0 + kk < N1 && j0 + j < N2) v = to_cx<T>(Bm[size_t(k0 + kk) * ldb + j0 + j]);
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      cx<T> av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][tr + 32 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tj + 8 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cfma(acc[a][b], av[a], bv[b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int j = j0 + tj + 8 * b;
    if (j >= N2) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const size_t r = r0 + tr + 32 * a;
      if (r >= ng) continue;
      const size_t idx = size_t(j) * ng + r;
      cx<T> v = cmul(alpha, acc[a][b]);
#pragma unroll
      for (int t = 0; t < 3; ++t)
        if (epi.e[t]) v = v + cmul(epi.c[t], epi.e[t][idx]);
      out[idx] = v;
    }
  }
}

// ---------------------------------------------------------------- streaming kernels ----
template <class T>
__global__ void k_lincomb(cx<T>* __restrict__ out, size_t n, Epi<T> t, const cx<T>* __restrict__ x3, cx<T> c3) {
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x) {
    cx<T> v = czero<T>();
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (t.e[k]) v = v + cmul(t.c[k], t.e[k][e]);
    if (x3) v = v + cmul(c3, x3[e]);
    out[e] = v;
  }
}

// out_j(r) = v(r) psi_j(r) + a * X_j(r)   (v real, FP64 on input)
template <class T>
__global__ void k_potential_apply(cx<T>* __restrict__ out, const cx<T>* __restrict__ psi,
                                  const double* __restrict__ v, size_t ng, size_t n, const cx<T>* __restrict__ X,
                                  T a) {
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x) {
    const T vv = T(v[e % ng]);
    cx<T> o = psi[e] * vv;
    if (X) o = o + X[e] * a;
    out[e] = o;
  }
}

// one value per vector from the per-block partials part[a * nblk + b]
__global__ void k_reduce_dots(const double* __restrict__ part, int nblk, int m, double* __restrict__ out) {
  const int a = blockIdx.x;
  double x = 0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) x += part[size_t(a) * nblk + b];
  __shared__ double red[32];
  for (int off = 16; off; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
    out[a] = t;
  }
}

int stream_blocks(pt_ctx* ctx, size_t n, int threads) {
  const size_t want = (n + threads - 1) / threads;
  return int(std::max<size_t>(1, std::min<size_t>(want, size_t(ctx->num_sms) * 8)));
}

}  // namespace

// ------------------------------------------------------------------------------------------
template <class T>
void gram(pt_ctx* ctx, const cx<T>* A, const cx<T>* B, int N1, int N2, size_t ng, double scale, c128* C,
          cudaStream_t st, bool herm) {
  if constexpr (sizeof(T) == 4) {
    if (ctx->bf16_requested) {
      gram_bf16(ctx, A, B, N1, N2, ng, scale, C, st, herm);
      return;
    }
    if (ctx->active_tc && gram_tc_applies(A, B, ng)) {
      if (ctx->tc_gram_wide && N2 > 64)
        gram_tc_wide(ctx, A, B, C, nullptr, nullptr, N1, N2, ng, scale, st, herm, ctx->active_tc == 1);
      else
        gram_tc(ctx, A, B, N1, N2, ng, scale, C, st, herm, ctx->active_tc == 1);
      return;
    }
  }
  const bool f32 = sizeof(T) == 4;
  const int tile = f32 ? G4T : GT;
  const int kstep = f32 ? G4K : GK;
  herm = herm && (N1 == N2);
  const int ti = (N1 + tile - 1) / tile, tj = (N2 + tile - 1) / tile;
  const int tiles = herm ? ti * (ti + 1) / 2 : ti * tj;
  // enough splits along r to fill the GPU about four times (two CTAs per SM for the FP32 tile)
  int splits = std::max(1, (ctx->num_sms * 4 + tiles - 1) / tiles);
  size_t chunk = (ng + splits - 1) / splits;
  chunk = (chunk + kstep - 1) / kstep * kstep;
  splits = int((ng + chunk - 1) / chunk);
  c128* part = static_cast<c128*>(ctx->get("gram_parts", size_t(splits) * N1 * N2 * sizeof(c128)));
  if constexpr (sizeof(T) == 4) {
    PT_LAUNCH(k_gram64, dim3(ti, tj, splits), G4THREADS, 0, st, A, B, N1, N2, ng, chunk, int(herm), part);
  } else {
    herm = false;
    PT_LAUNCH(k_gram<T>, dim3(ti, tj, splits), GTHREADS, 0, st, A, B, N1, N2, ng, chunk, part);
  }
  const size_t n = size_t(N1) * N2;
  PT_LAUNCH(k_reduce_parts, dim3(unsigned((n + 255) / 256)), 256, 0, st, part, splits, N1, N2, scale,
            herm ? tile : 0, C);
}

template <class T>
void gram2(pt_ctx* ctx, const cx<T>* A, const cx<T>* B0, c128* C0, const cx<T>* B1, c128* C1, int N1, int N2,
           size_t ng, double scale, cudaStream_t st, bool herm) {
  if constexpr (sizeof(T) == 4) {
    if (!ctx->bf16_requested && ctx->active_tc && ctx->tc_gram_wide && gram_tc_applies(A, B0, ng) &&
        gram_tc_applies(A, B1, ng)) {
      gram_tc_wide(ctx, A, B0, C0, B1, C1, N1, N2, ng, scale, st, herm, ctx->active_tc == 1);
      return;
    }
  }
  gram<T>(ctx, A, B0, N1, N2, ng, scale, C0, st, herm);
  gram<T>(ctx, A, B1, N1, N2, ng, scale, C1, st, herm);
}

template <class T>
void rotate(pt_ctx* ctx, const cx<T>* A, const c128* Bm, int ldb, int N1, int N2, size_t ng, c128 alpha,
            const Term* terms, int nterms, cx<T>* out, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (ctx->bf16_requested && nterms <= 3) {
      rotate_bf16(ctx, A, Bm, ldb, N1, N2, ng, alpha, terms, nterms, out, st);
      return;
    }
    if (ctx->active_tc && nterms <= 3 && rotate_tc_applies(A, ng)) {
      rotate_tc(ctx, A, Bm, ldb, N1, N2, ng, alpha, terms, nterms, out, st, ctx->active_tc == 1);
      return;
    }
  }
  Epi<T> epi{};
  for (int t = 0; t < 3; ++t) {
    epi.e[t] = (t < nterms) ? static_cast<const cx<T>*>(terms[t].x) : nullptr;
    epi.c[t] = (t < nterms) ? to_cx<T>(terms[t].c) : czero<T>();
  }
  dim3 grid(unsigned((ng + RT - 1) / RT), unsigned((N2 + JT - 1) / JT));
  PT_LAUNCH(k_rotate<T>, grid, RTHREADS, 0, st, A, Bm, ldb, N1, N2, ng, to_cx<T>(alpha), epi, out);
}

template <class T>
void lincomb(pt_ctx* ctx, cx<T>* out, size_t n, const Term* terms, int nterms, cudaStream_t st) {
  Epi<T> t{};
  for (int k = 0; k < 3; ++k) {
    t.e[k] = (k < nterms) ? static_cast<const cx<T>*>(terms[k].x) : nullptr;
    t.c[k] = (k < nterms) ? to_cx<T>(terms[k].c) : czero<T>();
  }
  const cx<T>* x3 = nterms > 3 ? static_cast<const cx<T>*>(terms[3].x) : nullptr;
  const cx<T> c3 = nterms > 3 ? to_cx<T>(terms[3].c) : czero<T>();
  PT_LAUNCH(k_lincomb<T>, stream_blocks(ctx, n, 256), 256, 0, st, out, n, t, x3, c3);
}

template <class T>
void potential_apply(pt_ctx* ctx, cx<T>* out, const cx<T>* psi, const double* v, size_t ng, int M,
                     const cx<T>* X, double a, cudaStream_t st) {
  const size_t n = ng * size_t(M);
  PT_LAUNCH(k_potential_apply<T>, stream_blocks(ctx, n, 256), 256, 0, st, out, psi, v, ng, n, X, T(a));
}


template void gram<float>(pt_ctx*, const c64*, const c64*, int, int, size_t, double, c128*, cudaStream_t, bool);
template void gram<double>(pt_ctx*, const c128*, const c128*, int, int, size_t, double, c128*, cudaStream_t, bool);
template void gram2<float>(pt_ctx*, const c64*, const c64*, c128*, const c64*, c128*, int, int, size_t, double,
                           cudaStream_t, bool);
template void gram2<double>(pt_ctx*, const c128*, const c128*, c128*, const c128*, c128*, int, int, size_t, double,
                            cudaStream_t, bool);
template void rotate<float>(pt_ctx*, const c64*, const c128*, int, int, int, size_t, c128, const Term*, int, c64*,
                            cudaStream_t);
template void rotate<double>(pt_ctx*, const c128*, const c128*, int, int, int, size_t, c128, const Term*, int,
                             c128*, cudaStream_t);
template void lincomb<float>(pt_ctx*, c64*, size_t, const Term*, int, cudaStream_t);
template void lincomb<double>(pt_ctx*, c128*, size_t, const Term*, int, cudaStream_t);
template void potential_apply<float>(pt_ctx*, c64*, const c64*, const double*, size_t, int, const c64*, double,
                                     cudaStream_t);
template void potential_apply<double>(pt_ctx*, c128*, const c128*, const double*, size_t, int, const c128*, double,
                                      cudaStream_t);
// ---------------------------------------------------------------- squared norms ----
// out[q] = w1 ||a_q||^2 + w2 ||s_q||^2 for two two-segment vectors (q = 0, 1): one streaming pass
// with 16-byte loads, compensated per-thread sums in the orbital precision, FP64 across threads.
constexpr int NRT = 256;

template <class T>
__global__ void __launch_bounds__(NRT) k_sqnorms(const cx<T>* __restrict__ a0, const cx<T>* __restrict__ a1, size_t n1,
                                                 const c128* __restrict__ s0, const c128* __restrict__ s1, size_t n2,
                                                 double w1, double w2, int vec, double* __restrict__ part) {
  Acc<T> acc[2];
  const size_t tid = size_t(blockIdx.x) * blockDim.x + threadIdx.x, stride = size_t(gridDim.x) * blockDim.x;
  if (sizeof(T) == 4 && vec) {
    // two complex64 per float4
    const size_t n4 = n1 / 2;
    const float4* p0 = reinterpret_cast<const float4*>(a0);
    const float4* p1 = reinterpret_cast<const float4*>(a1);
    for (size_t e = tid; e < n4; e += stride) {
      const float4 u = p0[e], v = p1[e];
      acc[0].add(T(fmaf(u.x, u.x, fmaf(u.y, u.y, fmaf(u.z, u.z, u.w * u.w)))));
      acc[1].add(T(fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, v.w * v.w)))));
    }
    if ((n1 & 1) && tid == 0) {
      const cx<T> u = a0[n1 - 1], v = a1[n1 - 1];
      acc[0].add(u.re * u.re + u.im * u.im);
      acc[1].add(v.re * v.re + v.im * v.im);
    }
  } else {
    for (size_t e = tid; e < n1; e += stride) {
      const cx<T> u = a0[e], v = a1[e];
      acc[0].add(u.re * u.re + u.im * u.im);
      acc[1].add(v.re * v.re + v.im * v.im);
    }
  }
  double s[2] = {w1 * acc[0].value(), w1 * acc[1].value()};
  for (size_t e = tid; e < n2; e += stride) {
    const c128 u = s0[e], v = s1[e];
    s[0] += w2 * (u.re * u.re + u.im * u.im);
    s[1] += w2 * (v.re * v.re + v.im * v.im);
  }
  __shared__ double red[2][NRT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    double x = s[q];
    for (int off = 16; off; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0) red[q][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double x = 0;
    for (int w = 0; w < NRT / 32; ++w) x += red[threadIdx.x][w];
    part[size_t(threadIdx.x) * gridDim.x + blockIdx.x] = x;
  }
}

template <class T>
void sqnorms(pt_ctx* ctx, const cx<T>* a0, const c128* s0, const cx<T>* a1, const c128* s1, size_t n1, size_t n2,
             double w1, double w2, double* out, cudaStream_t st) {
  const int nblk = ctx->num_sms * 4;
  double* part = static_cast<double*>(ctx->get("sqnorm_part", size_t(2) * nblk * sizeof(double)));
  const int vec = ((reinterpret_cast<uintptr_t>(a0) | reinterpret_cast<uintptr_t>(a1)) % 16) == 0;
  PT_LAUNCH(k_sqnorms<T>, nblk, NRT, 0, st, a0, a1, n1, s0, s1, n2, w1, w2, vec, part);
  PT_LAUNCH(k_reduce_dots, 2, 256, 0, st, part, nblk, 2, out);
}

template void sqnorms<float>(pt_ctx*, const c64*, const c128*, const c64*, const c128*, size_t, size_t, double, double,
                             double*, cudaStream_t);
template void sqnorms<double>(pt_ctx*, const c128*, const c128*, const c128*, const c128*, size_t, size_t, double,
                              double, double*, cudaStream_t);



}  // namespace pt
