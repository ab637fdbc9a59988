// Adaptively compressed exchange (Sec. IV-A2, Eq. vx_ace; the construction of the cited ACE paper).
//
//   W = V_x phi,  M = <phi|W> (N x N, Hermitian negative definite),  -M = L L^* (FP64 Cholesky),
//   xi = W L^{-*},  V_ACE = -xi xi^*  so that  V_ACE phi = -W L^{-*} L^{-1} <W|phi> = W.
//   Applying it:  V_ACE psi = -xi <xi|psi>  (two contractions over the grid).
#include "common.cuh"
#include "internal.h"

namespace pt {

namespace {

// A = -(M + M^H)/2
__global__ void k_neg_herm(const c128* __restrict__ M, int N, c128* __restrict__ A) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const int i = e / N, j = e % N;
  const c128 a = M[size_t(i) * N + j], b = M[size_t(j) * N + i];
  A[e] = c128{-0.5 * (a.re + b.re), -0.5 * (a.im - b.im)};
}

__global__ void k_conj_transpose(const c128* __restrict__ A, int N, c128* __restrict__ B) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const int i = e / N, j = e % N;
  const c128 a = A[size_t(j) * N + i];
  B[e] = c128{a.re, -a.im};
}

}  // namespace

void conj_transpose(const c128* A, int N, c128* B, cudaStream_t st) {
  PT_LAUNCH(k_conj_transpose, (N * N + 255) / 256, 256, 0, st, A, N, B);
}

void ace_from_w(pt_ctx* ctx, const void* W, const void* phi, int N, const pt_grid& g, pt_precision prec, void* xi,
                cudaStream_t st, size_t nvec) {
  const size_t ng = nvec ? nvec : ng_of(g);
  const double dV = dv_of(g);
  const size_t nn = size_t(N) * N * sizeof(c128);
  c128* M = static_cast<c128*>(ctx->get("ace_M", nn));
  c128* A = static_cast<c128*>(ctx->get("ace_A", nn));
  c128* L = static_cast<c128*>(ctx->get("ace_L", nn));
  c128* Li = static_cast<c128*>(ctx->get("ace_Linv", nn));
  c128* LiH = static_cast<c128*>(ctx->get("ace_LinvH", nn));
  int* info = static_cast<int*>(ctx->get("ace_info", sizeof(int)));
  if (prec == PT_FP64)
    gram<double>(ctx, static_cast<const c128*>(phi), static_cast<const c128*>(W), N, N, ng, dV, M, st);
  else
    gram<float>(ctx, static_cast<const c64*>(phi), static_cast<const c64*>(W), N, N, ng, dV, M, st);
  PT_LAUNCH(k_neg_herm, (N * N + 255) / 256, 256, 0, st, M, N, A);
  cholesky(ctx, A, N, L, info, st);
  int h_info = 0;
  PT_CUDA_CHECK(cudaMemcpyAsync(&h_info, info, sizeof(int), cudaMemcpyDeviceToHost, st));
  PT_CUDA_CHECK(cudaStreamSynchronize(st));
  if (h_info) fail(PT_NOT_PD, "ACE: -<phi|V_x phi> is not positive definite (pivot " + std::to_string(h_info) + ")");
  tri_inv_lower(ctx, L, N, Li, st);
  conj_transpose(Li, N, LiH, st);
  // xi_k = sum_j conj(Linv[k][j]) W_j  ->  rotate with Bm = Linv^H
  if (prec == PT_FP64)
    rotate<double>(ctx, static_cast<const c128*>(W), LiH, N, N, N, ng, c128{1.0, 0.0}, nullptr, 0,
                   static_cast<c128*>(xi), st);
  else
    rotate<float>(ctx, static_cast<const c64*>(W), LiH, N, N, N, ng, c128{1.0, 0.0}, nullptr, 0,
                  static_cast<c64*>(xi), st);
}

void ace_apply(pt_ctx* ctx, const void* xi, int N, const void* psi, int M, void* out, const pt_grid& g,
               pt_precision prec, cudaStream_t st, size_t nvec) {
  const size_t ng = nvec ? nvec : ng_of(g);
  const double dV = dv_of(g);
  c128* C = static_cast<c128*>(ctx->get("ace_C", size_t(N) * M * sizeof(c128)));
  if (prec == PT_FP64) {
    gram<double>(ctx, static_cast<const c128*>(xi), static_cast<const c128*>(psi), N, M, ng, dV, C, st);
    rotate<double>(ctx, static_cast<const c128*>(xi), C, M, N, M, ng, c128{-1.0, 0.0}, nullptr, 0,
                   static_cast<c128*>(out), st);
  } else {
    gram<float>(ctx, static_cast<const c64*>(xi), static_cast<const c64*>(psi), N, M, ng, dV, C, st);
    rotate<float>(ctx, static_cast<const c64*>(xi), C, M, N, M, ng, c128{-1.0, 0.0}, nullptr, 0,
                  static_cast<c64*>(out), st);
  }
}

}  // namespace pt
