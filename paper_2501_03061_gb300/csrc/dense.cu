// FP64 dense linear algebra on N x N complex matrices (N up to a few hundred), on the GPU.
//
//   zgemm        C = alpha op(A) op(B) + beta C, op in {N, C (conjugate transpose), T}
//   zgemm_add    C = alpha op(A) op(B) + beta D (D read-only, may differ from C)
//   heev         Hermitian eigen-decomposition by parallel two-sided cyclic Jacobi
//                (round-robin pairing; one launch per round; every 2x2 block of the
//                matrix is updated by J_k^H X J_l in the same launch; entries below the
//                stopping level are not rotated, so late sweeps are mostly copies)
//   cholesky     blocked lower Cholesky (32-wide panels), error flag on a non-positive or
//                non-finite pivot
//   tri_inv      L^{-1} of a lower-triangular matrix, one CTA per column
//   small_solve  m x m (m <= 24) Gaussian elimination with partial pivoting, one thread
// All matrices are row-major complex128: a[i*ld + j].
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace pt {

namespace {

template <class T>
__device__ __forceinline__ cx<T> opval(const cx<T>* A, int lda, char op, int i, int k) {
  // element (i, k) of op(A)
  if (op == 'N') return A[size_t(i) * lda + k];
  cx<T> v = A[size_t(k) * lda + i];
  if (op == 'C') v.im = -v.im;
  return v;
}

constexpr int ZT = 16;

// C = alpha op(A) op(B) + beta D  (D may be C itself, or another matrix with leading dimension ldd)
template <class T>
__global__ void __launch_bounds__(ZT* ZT) k_gemm(char opA, char opB, int m, int n, int k, cx<T> alpha,
                                                 const cx<T>* __restrict__ A, int lda, const cx<T>* __restrict__ B,
                                                 int ldb, cx<T> beta, const cx<T>* D, int ldd, cx<T>* C, int ldc) {
  __shared__ cx<T> As[ZT][ZT + 1];
  __shared__ cx<T> Bs[ZT][ZT + 1];
  const int tx = threadIdx.x % ZT, ty = threadIdx.x / ZT;
  const int i = blockIdx.y * ZT + ty, j = blockIdx.x * ZT + tx;
  cx<T> acc = czero<T>();
  for (int k0 = 0; k0 < k; k0 += ZT) {
    const int ka = k0 + tx, kb = k0 + ty;
    As[ty][tx] = (i < m && ka < k) ? opval(A, lda, opA, i, ka) : czero<T>();
    Bs[ty][tx] = (kb < k && j < n) ? opval(B, ldb, opB, kb, j) : czero<T>();
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < ZT; ++kk) cfma(acc, As[ty][kk], Bs[kk][tx]);
    __syncthreads();
  }
  if (i < m && j < n) {
    cx<T> v = cmul(alpha, acc);
    if (beta.re != T(0) || beta.im != T(0)) v = v + cmul(beta, D[size_t(i) * ldd + j]);
    C[size_t(i) * ldc + j] = v;
  }
}

// ---------------------------------------------------------------- Jacobi ----
// pair partner of position k in round r of the circle method on Np (even) players
__device__ __forceinline__ void jacobi_pair(int k, int r, int Np, int* p, int* q) {
  auto idx = [&](int i) { return i == 0 ? 0 : ((i - 1 + r) % (Np - 1)) + 1; };
  const int a = idx(k), b = idx(Np - 1 - k);
  *p = min(a, b);
  *q = max(a, b);
}

struct Rot {
  double c, s;
  c128 u;  // J = [[c, s u], [-s conj(u), c]]
};

// the rotation that annihilates a_pq, or the identity (s = 0) when |a_pq|^2 <= thr2 (threshold
// Jacobi: an entry already below the stopping level is left in place)
__device__ __forceinline__ Rot jacobi_rot(const c128* A, int N, int p, int q, double thr2) {
  Rot r{1.0, 0.0, c128{1.0, 0.0}};
  if (q >= N) return r;  // padding player
  const c128 apq = A[size_t(p) * N + q];
  const double b2 = apq.re * apq.re + apq.im * apq.im;
  if (!(b2 > thr2)) return r;
  const double app = A[size_t(p) * N + p].re, aqq = A[size_t(q) * N + q].re;
  // reciprocal square roots in place of square roots and divisions (each a long FP64 sequence on
  // the round's critical path)
  const double rb = rsqrt(b2);  // 1 / |a_pq|
  const double zeta = (aqq - app) * (0.5 * rb);
  const double az = fabs(zeta);
  double t;
  if (az > 1e100) {
    t = 0.5 / az;  // 1 / (|zeta| + sqrt(1 + zeta^2)) to double precision
  } else {
    const double q2 = 1.0 + zeta * zeta;
    t = 1.0 / (az + q2 * rsqrt(q2));
  }
  if (zeta < 0.0) t = -t;
  r.c = rsqrt(1.0 + t * t);
  r.s = t * r.c;
  r.u = c128{apq.re * rb, apq.im * rb};
  return r;
}

constexpr int JB = 8;  // pairs per CTA side (16 x 16 elements): (N/16)^2 CTAs spread over every SM

__global__ void __launch_bounds__(JB* JB) k_jacobi_round(const c128* __restrict__ Ain, c128* __restrict__ Aout,
                                                         c128* __restrict__ V, int N, int Np, int r, double thr2) {
  __shared__ Rot rk[JB], rl[JB];
  __shared__ int pk[JB], qk[JB], pl[JB], ql[JB];
  const int kb = blockIdx.y * JB, lb = blockIdx.x * JB;
  const int half = Np / 2;
  const int t = threadIdx.x;
  pdl_wait();  // the previous round's A and V
  pdl_launch_dependents();
  if (t < JB) {
    const int k = kb + t;
    if (k < half) {
      jacobi_pair(k, r, Np, &pk[t], &qk[t]);
      rk[t] = jacobi_rot(Ain, N, pk[t], qk[t], thr2);
    }
  } else if (t < 2 * JB) {
    const int l = lb + t - JB;
    if (l < half) {
      jacobi_pair(l, r, Np, &pl[t - JB], &ql[t - JB]);
      rl[t - JB] = jacobi_rot(Ain, N, pl[t - JB], ql[t - JB], thr2);
    }
  }
  __syncthreads();
  const int tk = t / JB, tl = t % JB;
  const int k = kb + tk, l = lb + tl;
  if (k < half && l < half) {
    const int p1 = pk[tk], q1 = qk[tk], p2 = pl[tl], q2 = ql[tl];
    const Rot a = rk[tk], b = rl[tl];
    auto get = [&](int i, int j) -> c128 {
      return (i < N && j < N) ? Ain[size_t(i) * N + j] : czero<double>();
    };
    const c128 x00 = get(p1, p2), x01 = get(p1, q2), x10 = get(q1, p2), x11 = get(q1, q2);
    auto put = [&](int i, int j, c128 v) {
      if (i < N && j < N) Aout[size_t(i) * N + j] = v;
    };
    if (a.s == 0.0 && b.s == 0.0) {  // both rotations the identity: the block is carried over
      put(p1, p2, x00);
      put(p1, q2, x01);
      put(q1, p2, x10);
      put(q1, q2, x11);
    } else {
      // Y = J_a^H X:  J^H = [[c, -s u], [s conj(u), c]]
      const c128 su = a.u * a.s, suc = conjc(a.u) * a.s;
      const c128 y00 = x00 * a.c - cmul(su, x10), y01 = x01 * a.c - cmul(su, x11);
      const c128 y10 = cmul(suc, x00) + x10 * a.c, y11 = cmul(suc, x01) + x11 * a.c;
      // Z = Y J_b:  J = [[c, s u], [-s conj(u), c]]
      const c128 tu = b.u * b.s, tuc = conjc(b.u) * b.s;
      c128 z00 = y00 * b.c - cmul(y01, tuc), z01 = cmul(y00, tu) + y01 * b.c;
      c128 z10 = y10 * b.c - cmul(y11, tuc), z11 = cmul(y10, tu) + y11 * b.c;
      if (k == l) {  // the 2x2 block this rotation diagonalises
        z01 = czero<double>();
        z10 = czero<double>();
        z00.im = 0.0;
        z11.im = 0.0;
      }
      put(p1, p2, z00);
      put(p1, q2, z01);
      put(q1, p2, z10);
      put(q1, q2, z11);
    }
  }
  // V <- V J for the column pairs of this CTA's l-range; the rows are split over the CTAs of the
  // same l-range so every CTA of the grid shares the update
  {
    const int rows_per = (N + gridDim.y - 1) / gridDim.y;
    const int r0 = blockIdx.y * rows_per, r1 = min(N, r0 + rows_per);
    for (int e = t; e < (r1 - r0) * JB; e += JB * JB) {
      const int row = r0 + e / JB, tl2 = e % JB;
      const int l2 = lb + tl2;
      if (l2 >= half) continue;
      const int p2 = pl[tl2], q2 = ql[tl2];
      if (q2 >= N) continue;
      const Rot b = rl[tl2];
      if (b.s == 0.0) continue;  // identity
      const c128 vp = V[size_t(row) * N + p2], vq = V[size_t(row) * N + q2];
      const c128 tu = b.u * b.s, tuc = conjc(b.u) * b.s;
      V[size_t(row) * N + p2] = vp * b.c - cmul(vq, tuc);
      V[size_t(row) * N + q2] = cmul(vp, tu) + vq * b.c;
    }
  }
}

// A = (S + S^*)/2 and V = V0 (identity when V0 is NULL)
__global__ void k_herm_part_and_basis(const c128* __restrict__ S, c128* __restrict__ A, const c128* __restrict__ V0,
                                      c128* __restrict__ V, int N) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const int i = e / N, j = e % N;
  const c128 a = S[size_t(i) * N + j], b = S[size_t(j) * N + i];
  A[e] = c128{0.5 * (a.re + b.re), 0.5 * (a.im - b.im)};
  V[e] = V0 ? V0[e] : c128{i == j ? 1.0 : 0.0, 0.0};
}

// sums of |offdiag|^2 and |all|^2: one partial pair per block (OFF_BLOCKS blocks), then one thread
// adds the partials in order
constexpr int OFF_BLOCKS = 64;
__global__ void __launch_bounds__(256) k_offnorm_part(const c128* __restrict__ A, int N, double* __restrict__ part) {
  pdl_wait();  // the last Jacobi round
  double off = 0, all = 0;
  for (int e = blockIdx.x * 256 + threadIdx.x; e < N * N; e += OFF_BLOCKS * 256) {
    const double v = A[e].re * A[e].re + A[e].im * A[e].im;
    all += v;
    if (e / N != e % N) off += v;
  }
  __shared__ double so[8], sa[8];
  for (int o = 16; o; o >>= 1) {
    off += __shfl_down_sync(0xffffffffu, off, o);
    all += __shfl_down_sync(0xffffffffu, all, o);
  }
  if ((threadIdx.x & 31) == 0) {
    so[threadIdx.x >> 5] = off;
    sa[threadIdx.x >> 5] = all;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < 8; ++w) {
      a += so[w];
      b += sa[w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}
__global__ void k_offnorm_sum(const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < OFF_BLOCKS; ++k) {
      a += part[2 * k];
      b += part[2 * k + 1];
    }
    out[0] = a;
    out[1] = b;
  }
}

// ascending sort of the diagonal with the matching columns of V: a rank sort on order-preserving
// integer keys of the doubles (an FP64 comparison issues at the FP64 rate here), then the column
// permutation over the whole grid
__device__ __forceinline__ unsigned long long order_key(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__global__ void k_eig_keys(const c128* __restrict__ A, int N, unsigned long long* __restrict__ key) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) key[i] = order_key(A[size_t(i) * N + i].re);
}
__global__ void k_eig_rank(const c128* __restrict__ A, const unsigned long long* __restrict__ key, int N,
                           int* __restrict__ rank, double* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned long long ki = key[i];
  int r = 0;
  for (int j = 0; j < N; ++j) {
    const unsigned long long kj = key[j];  // the same j across the warp: one broadcast load
    r += (kj < ki) || (kj == ki && j < i);
  }
  rank[i] = r;
  d[r] = A[size_t(i) * N + i].re;
}
__global__ void k_eig_permute(const c128* __restrict__ V, const int* __restrict__ rank, int N, c128* __restrict__ Q) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const int row = e / N, i = e - row * N;
  Q[size_t(row) * N + rank[i]] = V[e];
}

// ---------------------------------------------------------------- Cholesky ----
// Right-looking blocked Cholesky with CB-wide panels.  Per panel: the diagonal block is
// factored (and inverted) in one CTA's shared memory, the panel below is solved against the
// inverse of the diagonal block, and the trailing lower triangle gets a rank-CB update.
constexpr int CB = 32;

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

template <class T>
__global__ void __launch_bounds__(256) k_chol_diag(cx<T>* __restrict__ A, int N, int kb, int bs,
                                                   cx<T>* __restrict__ Winv, int* __restrict__ info) {
  __shared__ cx<T> a[CB][CB + 1];
  __shared__ cx<T> x[CB][CB + 1];
  // lower triangle (i >= j) listed column by column: entry (j, i) at j*bs - j(j-1)/2 + (i - j), so
  // the trailing triangle of step k (j > k) is one contiguous range and no thread idles on the
  // upper half
  __shared__ unsigned short tri[CB * (CB + 1) / 2];
  pdl_wait();  // the previous panel's trailing update
  pdl_launch_dependents();
  if (*info) return;
  const int tid = threadIdx.x;
  for (int e = tid; e < bs * bs; e += blockDim.x) {
    const int i = e / bs, j = e % bs;
    a[i][j] = A[size_t(kb + i) * N + kb + j];
    if (i >= j) tri[j * bs - j * (j - 1) / 2 + (i - j)] = static_cast<unsigned short>((j << 8) | i);
  }
  __syncthreads();
  const int tri_end = bs * (bs + 1) / 2;
  // FP64 square roots and divisions are long instruction sequences on the FP64 pipe: one thread
  // takes them and broadcasts the results
  __shared__ T rdiag[CB];
  __shared__ T s_rk;
  for (int k = 0; k < bs; ++k) {
    const T piv = a[k][k].re;
    if (!(piv > 0.0) || !isfinite(piv)) {
      if (tid == 0) *info = kb + k + 1;
      return;  // uniform: every thread read the same pivot
    }
    __syncthreads();
    if (tid == 0) {
      // one reciprocal square root instead of a square root and a division (each a long FP64
      // sequence on the pivot's critical path)
      const T rk0 = rsq(piv);
      a[k][k] = cx<T>{piv * rk0, T(0)};
      s_rk = rk0;
      rdiag[k] = rk0;
    }
    __syncthreads();
    const T rk = s_rk;
    for (int i = k + 1 + tid; i < bs; i += blockDim.x) a[i][k] = a[i][k] * rk;
    __syncthreads();
    for (int e = (k + 1) * bs - (k + 1) * k / 2 + tid; e < tri_end; e += blockDim.x) {
      const int i = tri[e] & 255, j = tri[e] >> 8;
      a[i][j] = a[i][j] - cmulc(a[j][k], a[i][k]);
    }
    __syncthreads();
  }
  // inverse X of the lower-triangular factor, one row at a time with all threads:
  //   X[i][i] = 1 / L[i][i],  X[i][j] = -(sum_{p=j}^{i-1} L[i][p] X[p][j]) / L[i][i]  (j < i);
  // thread (part, j) sums every 8th p, the 8 parts meet in shared memory
  __shared__ cx<T> red[8][CB];
  {
    const int j = tid & (CB - 1), part = tid >> 5;
    for (int i = 0; i < bs; ++i) {
      cx<T> acc = czero<T>();
      if (j < i)
        for (int p = j + part; p < i; p += 8) acc = acc + cmul(a[i][p], x[p][j]);
      red[part][j] = acc;
      __syncthreads();
      if (part == 0) {
        cx<T> t = czero<T>();
        for (int q = 0; q < 8; ++q) t = t + red[q][j];
        const T inv = rdiag[i];
        x[i][j] = j < i ? t * (-inv) : (j == i ? cx<T>{inv, T(0)} : czero<T>());
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < bs * bs; e += blockDim.x) {
    const int i = e / bs, j = e % bs;
    if (j <= i) A[size_t(kb + i) * N + kb + j] = a[i][j];
    Winv[i * CB + j] = x[i][j];
  }
}

// L_ik = A_ik L_kk^{-*} for the rows below the diagonal block (8 rows per CTA)
template <class T>
__global__ void __launch_bounds__(256) k_chol_panel(cx<T>* __restrict__ A, int N, int kb, int bs,
                                                    const cx<T>* __restrict__ Winv, const int* __restrict__ info) {
  __shared__ cx<T> w[CB][CB + 1];
  __shared__ cx<T> r[8][CB + 1];
  pdl_wait();  // the diagonal block and its inverse
  pdl_launch_dependents();
  if (*info) return;
  const int tid = threadIdx.x;
  const int i0 = kb + bs + blockIdx.x * 8;
  for (int e = tid; e < bs * bs; e += blockDim.x) w[e / bs][e % bs] = Winv[(e / bs) * CB + (e % bs)];
  for (int e = tid; e < 8 * bs; e += blockDim.x) {
    const int ii = e / bs, p = e % bs;
    r[ii][p] = (i0 + ii < N) ? A[size_t(i0 + ii) * N + kb + p] : czero<T>();
  }
  __syncthreads();
  const int ii = tid / CB, j = tid % CB;
  if (i0 + ii < N && j < bs) {
    cx<T> acc = czero<T>();
    // (L_kk^{-*})[p][j] = conj(Winv[j][p]), nonzero for p <= j
    for (int p = 0; p <= j; ++p) acc = acc + cmul(r[ii][p], conjc(w[j][p]));
    A[size_t(i0 + ii) * N + kb + j] = acc;
  }
}

// trailing update A[i][j] -= sum_p L[i][kb+p] conj(L[j][kb+p]) for kb+bs <= j <= i < N
template <class T>
__global__ void __launch_bounds__(256) k_chol_update(cx<T>* __restrict__ A, int N, int kb, int bs,
                                                     const int* __restrict__ info) {
  pdl_wait();  // the panel below the diagonal block
  pdl_launch_dependents();
  if (*info) return;
  const int t0 = kb + bs;
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  __shared__ cx<T> li[16][CB + 1], lj[16][CB + 1];
  const int tid = threadIdx.x;
  const int ib = t0 + bi * 16, jb = t0 + bj * 16;
  for (int e = tid; e < 16 * bs; e += blockDim.x) {
    const int q = e / bs, p = e % bs;
    li[q][p] = (ib + q < N) ? A[size_t(ib + q) * N + kb + p] : czero<T>();
    lj[q][p] = (jb + q < N) ? A[size_t(jb + q) * N + kb + p] : czero<T>();
  }
  __syncthreads();
  const int i = ib + tid / 16, j = jb + tid % 16;
  if (i < N && j < N && j <= i) {
    cx<T> acc = czero<T>();
    for (int p = 0; p < bs; ++p) acc = acc + cmulc(lj[tid % 16][p], li[tid / 16][p]);
    A[size_t(i) * N + j] = A[size_t(i) * N + j] - acc;
  }
}

template <class T>
__global__ void k_chol_finish(const cx<T>* __restrict__ A, int N, cx<T>* __restrict__ L, const int* __restrict__ info) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N || *info) return;
  const int i = e / N, j = e % N;
  L[e] = (j > i) ? czero<T>() : A[e];
}

// out = U diag(f(lam)) (scale columns), f = lam^power
__global__ void k_scale_cols_pow(const c128* __restrict__ U, const double* __restrict__ lam, int N, double power,
                                 c128* __restrict__ out, int* __restrict__ info) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const int j = e % N;
  const double l = lam[j];
  if (!(l > 0.0)) {
    *info = 1;
    out[e] = czero<double>();
    return;
  }
  out[e] = U[e] * pow(l, power);
}

__global__ void k_small_solve(const double* __restrict__ G, const double* __restrict__ rhs, int m, double reg,
                              double* __restrict__ x) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a[24][25];
  double tr = 0;
  for (int i = 0; i < m; ++i) tr += G[i * m + i];
  const double shift = reg * (tr > 0 ? tr / m : 1.0);
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) a[i][j] = G[i * m + j] + (i == j ? shift : 0.0);
    a[i][m] = rhs[i];
  }
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    if (piv != c)
      for (int j = c; j <= m; ++j) {
        const double t = a[c][j];
        a[c][j] = a[piv][j];
        a[piv][j] = t;
      }
    const double d = a[c][c];
    if (d == 0.0) continue;
    for (int r = c + 1; r < m; ++r) {
      const double f = a[r][c] / d;
      for (int j = c; j <= m; ++j) a[r][j] -= f * a[c][j];
    }
  }
  for (int c = m - 1; c >= 0; --c) {
    double s = a[c][m];
    for (int j = c + 1; j < m; ++j) s -= a[c][j] * x[j];
    x[c] = (a[c][c] != 0.0) ? s / a[c][c] : 0.0;
  }
}

}  // namespace

// ------------------------------------------------------------------------------------------
template <class T>
void gemm(char opA, char opB, int m, int n, int k, cx<T> alpha, const cx<T>* A, int lda, const cx<T>* B, int ldb,
          cx<T> beta, const cx<T>* D, int ldd, cx<T>* C, int ldc, cudaStream_t st) {
  dim3 grid((n + ZT - 1) / ZT, (m + ZT - 1) / ZT);
  PT_LAUNCH(k_gemm<T>, grid, ZT * ZT, 0, st, opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, D, ldd, C, ldc);
}
template void gemm<float>(char, char, int, int, int, c64, const c64*, int, const c64*, int, c64, const c64*, int, c64*,
                          int, cudaStream_t);
template void gemm<double>(char, char, int, int, int, c128, const c128*, int, const c128*, int, c128, const c128*, int,
                           c128*, int, cudaStream_t);

void zgemm(char opA, char opB, int m, int n, int k, c128 alpha, const c128* A, int lda, const c128* B, int ldb,
           c128 beta, c128* C, int ldc, cudaStream_t st) {
  gemm<double>(opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, C, ldc, st);
}

void zgemm_add(char opA, char opB, int m, int n, int k, c128 alpha, const c128* A, int lda, const c128* B, int ldb,
               c128 beta, const c128* D, int ldd, c128* C, int ldc, cudaStream_t st) {
  gemm<double>(opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, D, ldd, C, ldc, st);
}

int heev(pt_ctx* ctx, const c128* S, int N, c128* Q, double* d, cudaStream_t st, int max_sweeps, const c128* Q0,
         double rel_tol) {
  const int Np = N + (N & 1);
  c128* A0 = static_cast<c128*>(ctx->get("heev_A0", size_t(N) * N * sizeof(c128)));
  c128* A1 = static_cast<c128*>(ctx->get("heev_A1", size_t(N) * N * sizeof(c128)));
  c128* V = static_cast<c128*>(ctx->get("heev_V", size_t(N) * N * sizeof(c128)));
  double* nrm = static_cast<double*>(ctx->get("heev_norm", (2 * OFF_BLOCKS + 2) * sizeof(double)));
  if (Q0) {
    // warm start: rotate into the basis Q0 (Jacobi then starts from a nearly diagonal matrix when
    // Q0 diagonalises a nearby matrix) and accumulate the rotations onto Q0
    zgemm('N', 'N', N, N, N, c128{1, 0}, S, N, Q0, N, c128{0, 0}, A1, N, st);
    zgemm('C', 'N', N, N, N, c128{1, 0}, Q0, N, A1, N, c128{0, 0}, V, N, st);
    PT_LAUNCH(k_herm_part_and_basis, (N * N + 255) / 256, 256, 0, st, V, A0, Q0, A1, N);
    std::swap(V, A1);
  } else {
    PT_LAUNCH(k_herm_part_and_basis, (N * N + 255) / 256, 256, 0, st, S, A0, nullptr, V, N);
  }
  const int half = Np / 2;
  dim3 grid((half + JB - 1) / JB, (half + JB - 1) / JB);
  double h[2] = {0, 0};
  double prev_off = INFINITY;
  int sweeps = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    PT_LAUNCH_PDL(k_offnorm_part, OFF_BLOCKS, 256, 0, st, A0, N, nrm + 2);
    PT_LAUNCH(k_offnorm_sum, 1, 32, 0, st, nrm + 2, nrm);
    PT_CUDA_CHECK(cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, st));
    PT_CUDA_CHECK(cudaStreamSynchronize(st));
    if (!std::isfinite(h[1])) fail(PT_NONFINITE, "non-finite entry in the matrix to diagonalise");
    // Converged when the off-diagonal norm is at the FP64 rounding floor (eps * sqrt(N) * ||A||),
    // or when, already small, a sweep no longer reduces it (cyclic Jacobi converges
    // quadratically, so a stalled sweep means rounding noise).
    const double floor2 = 1e-32 * double(N) * h[1];
    if (h[0] <= floor2 || h[0] == 0.0) break;
    if (h[0] <= rel_tol * rel_tol * h[1]) break;
    if (h[0] <= 1e-24 * h[1] && h[0] > 0.25 * prev_off) break;
    prev_off = h[0];
    // entries with |a_pq|^2 at or below the stopping level spread over all N^2 entries are not
    // rotated: all of them together stay within the stopping test, and late sweeps, where most
    // entries are there, skip their FP64 arithmetic
    const double stop2 = rel_tol > 0.0 ? rel_tol * rel_tol * h[1] : floor2;
    const double thr2 = std::max(1e-280, stop2 / (double(N) * double(N)));
    for (int r = 0; r < Np - 1; ++r) {
      PT_LAUNCH_PDL(k_jacobi_round, grid, JB * JB, 0, st, A0, A1, V, N, Np, r, thr2);
      std::swap(A0, A1);
    }
    ++sweeps;
  }
  auto* key = static_cast<unsigned long long*>(ctx->get("heev_key", size_t(N) * sizeof(unsigned long long)));
  int* rank = static_cast<int*>(ctx->get("heev_rank", size_t(N) * sizeof(int)));
  PT_LAUNCH(k_eig_keys, (N + 255) / 256, 256, 0, st, A0, N, key);
  PT_LAUNCH(k_eig_rank, (N + 127) / 128, 128, 0, st, A0, key, N, rank, d);
  PT_LAUNCH(k_eig_permute, (N * N + 255) / 256, 256, 0, st, V, rank, N, Q);
  return sweeps;
}

template <class T>
void cholesky(pt_ctx* ctx, cx<T>* A, int N, cx<T>* L, int* info, cudaStream_t st) {
  // the inverses of all diagonal blocks are kept (rows kb..kb+bs of an N x CB array) for tri_inv_lower
  cx<T>* winv_all = static_cast<cx<T>*>(
      ctx->get(sizeof(T) == 8 ? "chol_winv_all" : "chol_winv_all32", size_t(N) * CB * sizeof(cx<T>)));
  PT_CUDA_CHECK(cudaMemsetAsync(info, 0, sizeof(int), st));
  for (int kb = 0; kb < N; kb += CB) {
    const int bs = std::min(CB, N - kb);
    cx<T>* winv = winv_all + size_t(kb) * CB;
    PT_LAUNCH_PDL(k_chol_diag<T>, 1, 256, 0, st, A, N, kb, bs, winv, info);
    const int rest = N - kb - bs;
    if (rest <= 0) break;
    PT_LAUNCH_PDL(k_chol_panel<T>, (rest + 7) / 8, 256, 0, st, A, N, kb, bs, winv, info);
    const int nt = (rest + 15) / 16;
    PT_LAUNCH_PDL(k_chol_update<T>, dim3(nt, nt), 256, 0, st, A, N, kb, bs, info);
  }
  PT_LAUNCH(k_chol_finish<T>, (N * N + 255) / 256, 256, 0, st, A, N, L, info);
}
template void cholesky<float>(pt_ctx*, c64*, int, c64*, int*, cudaStream_t);
template void cholesky<double>(pt_ctx*, c128*, int, c128*, int*, cudaStream_t);

// X = 0 except the diagonal CB-blocks, which take the inverses cholesky() kept
template <class T>
__global__ void k_tri_inv_leaves(const cx<T>* __restrict__ winv_all, int N, cx<T>* __restrict__ X) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const int i = e / N, j = e % N;
  const int bi = i / CB, bj = j / CB;
  X[e] = (bi == bj) ? winv_all[size_t(i) * CB + (j - bj * CB)] : czero<T>();
}

template <class T>
void tri_inv_lower(pt_ctx* ctx, const cx<T>* L, int N, cx<T>* X, cudaStream_t st) {
  // Bottom-up block inversion: for [L11 0; L21 L22] with X11 = L11^{-1}, X22 = L22^{-1} known,
  // X21 = -X22 (L21 X11).  Leaves are the CB x CB inverses from the preceding cholesky().
  const cx<T>* winv_all = static_cast<const cx<T>*>(
      ctx->get(sizeof(T) == 8 ? "chol_winv_all" : "chol_winv_all32", size_t(N) * CB * sizeof(cx<T>)));
  cx<T>* Tm = static_cast<cx<T>*>(ctx->get(sizeof(T) == 8 ? "tri_inv_T" : "tri_inv_T32", size_t(N) * N * sizeof(cx<T>)));
  PT_LAUNCH(k_tri_inv_leaves<T>, (N * N + 255) / 256, 256, 0, st, winv_all, N, X);
  const cx<T> one{T(1), T(0)}, mone{T(-1), T(0)}, zero{T(0), T(0)};
  for (int s = CB; s < N; s *= 2) {
    for (int i0 = 0; i0 + s < N; i0 += 2 * s) {
      const int n1 = s, n2 = std::min(s, N - i0 - s);
      const cx<T>* X11 = X + size_t(i0) * N + i0;
      const cx<T>* X22 = X + size_t(i0 + s) * N + (i0 + s);
      const cx<T>* L21 = L + size_t(i0 + s) * N + i0;
      cx<T>* X21 = X + size_t(i0 + s) * N + i0;
      gemm<T>('N', 'N', n2, n1, n1, one, L21, N, X11, N, zero, Tm, n1, Tm, n1, st);
      gemm<T>('N', 'N', n2, n1, n2, mone, X22, N, Tm, n1, zero, X21, N, X21, N, st);
    }
  }
}
template void tri_inv_lower<float>(pt_ctx*, const c64*, int, c64*, cudaStream_t);
template void tri_inv_lower<double>(pt_ctx*, const c128*, int, c128*, cudaStream_t);

void scale_cols_pow(const c128* U, const double* lam, int N, double power, c128* out, int* info, cudaStream_t st) {
  PT_LAUNCH(k_scale_cols_pow, (N * N + 255) / 256, 256, 0, st, U, lam, N, power, out, info);
}

__global__ void k_set_identity(c128* __restrict__ A, int N) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < N * N) A[e] = c128{(e / N == e % N) ? 1.0 : 0.0, 0.0};
}

__global__ void k_add_diagonal(c128* __restrict__ A, int N, double v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) A[size_t(i) * N + i].re += v;
}

void set_identity(c128* A, int N, cudaStream_t st) {
  PT_LAUNCH(k_set_identity, (N * N + 255) / 256, 256, 0, st, A, N);
}

void add_diagonal(c128* A, int N, double v, cudaStream_t st) {
  PT_LAUNCH(k_add_diagonal, (N + 255) / 256, 256, 0, st, A, N, v);
}

void small_solve(const double* G, const double* rhs, int m, double reg, double* x, cudaStream_t st) {
  if (m > 24) fail(PT_INVALID_ARG, "small_solve supports m <= 24");
  PT_LAUNCH(k_small_solve, 1, 32, 0, st, G, rhs, m, reg, x);
}

}  // namespace pt
