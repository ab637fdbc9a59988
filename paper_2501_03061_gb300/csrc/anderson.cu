// Anderson mixing (type II, real coefficients) on x = (Phi, sigma), streaming form.
//
// History entries a = 1..m hold dR_a = r_a - r_{a-1} and Z_a = dX_a + beta dR_a (dX_a = x_a - x_{a-1}).
// Per iteration k two passes touch the orbital block:
//   prepare: dR_s = r_k - r_{k-1};  Z_s = dXpend + beta dR_s  (dXpend = x_k - x_{k-1} from the last
//            update);  dots <dR_a, dR_s> and <dR_a, r_k> for every other entry a, plus
//            <dR_s, dR_s> and <dR_s, r_k>;
//   update:  x_{k+1} = x_k + beta r_k - sum_a gamma_a Z_a,  dXpend = x_{k+1} - x_k,
// with gamma solving the m x m normal equations (FP64, on the device).  History pointers
// travel in the kernel parameters.  The dots steer the mixing only (they do not enter the
// fixed point) and are accumulated in the orbital precision per thread, in FP64 across threads.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace pt {

namespace {

constexpr int HMAX = 20;
constexpr int AT = 256;

template <class T>
struct HistPtrs {
  const cx<T>* v[HMAX];
};

template <class T>
__device__ __forceinline__ T rdot(cx<T> a, cx<T> b) {
  return a.re * b.re + a.im * b.im;
}

// out partial layout: [2*MO + 2][nblk] per segment call, written at column offset blk_off.  The
// number of other entries MO is a template constant, so a call with a short history holds only
// the accumulators it needs (registers, and with them the resident warps that keep this streaming
// pass's loads in flight, fall with MO).
template <class T, int MO>
__global__ void __launch_bounds__(AT) k_and_prepare(const cx<T>* __restrict__ rk, const cx<T>* __restrict__ rprev,
                                                    const cx<T>* __restrict__ dxp, cx<T>* __restrict__ dRs,
                                                    cx<T>* __restrict__ Zs, HistPtrs<T> dR, T beta, size_t n,
                                                    double w, double* __restrict__ part, int ld, int blk_off) {
  constexpr int NV = 2 * MO + 2;
  T s[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) s[a] = T(0);
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x) {
    const cx<T> r = rk[e];
    const cx<T> d = r - rprev[e];
    dRs[e] = d;
    Zs[e] = dxp[e] + d * beta;
    s[2 * MO] += rdot(d, d);
    s[2 * MO + 1] += rdot(d, r);
#pragma unroll
    for (int a = 0; a < MO; ++a) {
      const cx<T> h = dR.v[a][e];
      s[2 * a] += rdot(h, d);
      s[2 * a + 1] += rdot(h, r);
    }
  }
  // block sums: warp shuffles, then one value per warp in shared memory
  __shared__ double red[NV][AT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double x = double(s[q]);
    for (int off = 16; off; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0) red[q][warp] = x;
  }
  __syncthreads();
  // output order: the pairs of the other entries, then the two values of the new entry
  if (threadIdx.x < NV) {
    double t = 0;
    for (int k = 0; k < AT / 32; ++k) t += red[threadIdx.x][k];
    part[size_t(threadIdx.x) * ld + blk_off + blockIdx.x] = w * t;
  }
}

template <class T, int MO = 0>
void launch_prepare(int mo, int blocks, cudaStream_t st, const cx<T>* rk, const cx<T>* rprev, const cx<T>* dxp,
                    cx<T>* dRs, cx<T>* Zs, const HistPtrs<T>& h, T beta, size_t n, double w, double* part, int ld,
                    int blk_off) {
  if constexpr (MO < HMAX) {
    if (mo != MO) {
      launch_prepare<T, MO + 1>(mo, blocks, st, rk, rprev, dxp, dRs, Zs, h, beta, n, w, part, ld, blk_off);
      return;
    }
    PT_LAUNCH((k_and_prepare<T, MO>), blocks, AT, 0, st, rk, rprev, dxp, dRs, Zs, h, beta, n, w, part, ld, blk_off);
  } else {
    fail(PT_INVALID_ARG, "Anderson history too deep");
  }
}

__global__ void k_and_reduce(const double* __restrict__ part, int ld, int nvals, double* __restrict__ out) {
  const int q = blockIdx.x;
  if (q >= nvals) return;
  double x = 0;
  for (int b = threadIdx.x; b < ld; b += blockDim.x) x += part[size_t(q) * ld + b];
  __shared__ double red[32];
  for (int off = 16; off; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < int(blockDim.x >> 5); ++k) t += red[k];
    out[q] = t;
  }
}

// Gram update and packed normal equations.  dots: [<dR_o,dR_s>, <dR_o,r>]_o..., <dR_s,dR_s>, <dR_s,r>
// where o runs over `others` (slot indices); G is kept by slot in a HMAX x HMAX array.
__global__ void k_and_gram(double* __restrict__ G, const double* __restrict__ dots, int s, const int* __restrict__ others,
                           int mo, const int* __restrict__ order, int m, double* __restrict__ Gp,
                           double* __restrict__ rhs) {
  if (threadIdx.x == 0) {
    for (int a = 0; a < mo; ++a) {
      G[s * HMAX + others[a]] = dots[2 * a];
      G[others[a] * HMAX + s] = dots[2 * a];
    }
    G[s * HMAX + s] = dots[2 * mo];
  }
  __syncthreads();
  // rhs in packed order: slot s -> <dR_s, r>; slot others[a] -> <dR_a, r>
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    const int sl = order[p];
    double v = dots[2 * mo + 1];
    for (int a = 0; a < mo; ++a)
      if (others[a] == sl) v = dots[2 * a + 1];
    rhs[p] = v;
    for (int q = 0; q < m; ++q) Gp[p * m + q] = G[sl * HMAX + order[q]];
  }
}

template <class T>
__global__ void __launch_bounds__(AT) k_and_update(cx<T>* __restrict__ x, const cx<T>* __restrict__ r,
                                                   HistPtrs<T> Z, const double* __restrict__ gamma, int m, T beta,
                                                   cx<T>* __restrict__ dxp, size_t n) {
  __shared__ T g[HMAX];
  if (threadIdx.x < HMAX) g[threadIdx.x] = threadIdx.x < m ? T(gamma[threadIdx.x]) : T(0);
  __syncthreads();
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x) {
    cx<T> dx = r[e] * beta;
#pragma unroll
    for (int a = 0; a < HMAX; ++a)
      if (a < m) dx = dx - Z.v[a][e] * g[a];
    x[e] = x[e] + dx;
    dxp[e] = dx;
  }
}

int blocks_for(pt_ctx* ctx, size_t n) {
  return int(std::max<size_t>(1, std::min<size_t>((n + AT - 1) / AT, size_t(ctx->num_sms) * 4)));
}

}  // namespace

template <class T>
void anderson_prepare(pt_ctx* ctx, const AndersonSeg<T>& phi, const AndersonSeg<double>& sig, int mo, double beta,
                      double w_phi, double* dots, cudaStream_t st) {
  if (mo > HMAX - 1) fail(PT_INVALID_ARG, "Anderson history too deep");
  const int b1 = blocks_for(ctx, phi.n), b2 = blocks_for(ctx, sig.n);
  const int ld = b1 + b2;
  const int nv = 2 * mo + 2;
  double* part = static_cast<double*>(ctx->get("and_part", size_t(2 * HMAX + 2) * ld * sizeof(double)));
  HistPtrs<T> h1{};
  HistPtrs<double> h2{};
  for (int a = 0; a < mo; ++a) {
    h1.v[a] = phi.dR[a];
    h2.v[a] = sig.dR[a];
  }
  launch_prepare<T>(mo, b1, st, phi.rk, phi.rprev, phi.dxp, phi.dRs, phi.Zs, h1, T(beta), phi.n, w_phi, part, ld, 0);
  launch_prepare<double>(mo, b2, st, sig.rk, sig.rprev, sig.dxp, sig.dRs, sig.Zs, h2, beta, sig.n, 1.0, part, ld, b1);
  PT_LAUNCH(k_and_reduce, nv, 256, 0, st, part, ld, nv, dots);
}

void anderson_gram(double* G, const double* dots, int s, const int* others_d, int mo, const int* order_d, int m,
                   double* Gp, double* rhs, cudaStream_t st) {
  PT_LAUNCH(k_and_gram, 1, 32, 0, st, G, dots, s, others_d, mo, order_d, m, Gp, rhs);
}

template <class T>
void anderson_update(pt_ctx* ctx, cx<T>* x, const cx<T>* r, const cx<T>* const* Z, int m, const double* gamma,
                     double beta, cx<T>* dxp, size_t n, cudaStream_t st) {
  if (m > HMAX) fail(PT_INVALID_ARG, "Anderson history too deep");
  HistPtrs<T> h{};
  for (int a = 0; a < m; ++a) h.v[a] = Z[a];
  PT_LAUNCH(k_and_update<T>, blocks_for(ctx, n), AT, 0, st, x, r, h, gamma, m, T(beta), dxp, n);
}

template void anderson_prepare<float>(pt_ctx*, const AndersonSeg<float>&, const AndersonSeg<double>&, int, double,
                                      double, double*, cudaStream_t);
template void anderson_prepare<double>(pt_ctx*, const AndersonSeg<double>&, const AndersonSeg<double>&, int, double,
                                       double, double*, cudaStream_t);
template void anderson_update<float>(pt_ctx*, c64*, const c64*, const c64* const*, int, const double*, double, c64*,
                                     size_t, cudaStream_t);
template void anderson_update<double>(pt_ctx*, c128*, const c128*, const c128* const*, int, const double*, double,
                                      c128*, size_t, cudaStream_t);

}  // namespace pt
