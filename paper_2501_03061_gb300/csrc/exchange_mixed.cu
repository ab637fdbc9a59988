// The undiagonalised mixed-state exchange on the GPU: Algorithm 2's triple loop (Sec. III-B;
// Sec. II-B Eq. mixed_vx), the baseline that the occupation-matrix diagonalisation of Sec. IV-A1
// (Eq. vxdiag, the library's pt_apply_exchange) replaces.
//
//   (V_x tgt_j)(r) = - sum_{k, i} sigma_ik phi_i(r) IFFT[ K(G) FFT[ conj(phi_k) tgt_j ] ](r) / Ng
//
// In Algorithm 2's order: for every k, for every i, the pair fields conj(phi_k) tgt_j of a batch of
// targets are transformed, multiplied by K/Ng and transformed back, and sigma_ik phi_i times the
// result is accumulated into W_j — N * N * M pair FFTs, the pair FFT of (k, j) recomputed for every
// i exactly as the listing's innermost loop does (the multi-batch form of Sec. III-B batches the j
// loop).  The equation's minus sign is followed (the listing accumulates with a plus).  No sigma_ik
// is skipped.  The passes are the library's batched pair-FFT kernels (compile-time kernels on
// cubic grids, runtime-plan kernels otherwise): for a fixed (k, i) the pair product's source is
// phi_k and the accumulate partner is the field sigma_ik phi_i, both held in a two-field buffer.
#include <algorithm>
#include <cstring>

#include "exchange_sched.h"
#include "fft_fixed.cuh"
#include "internal.h"

namespace pt {

namespace {

// dst = sigma[i][k] * phi_i (sigma complex128, row-major N x N)
template <class T>
__global__ void k_scale_by_sigma(cx<T>* __restrict__ dst, const cx<T>* __restrict__ phi_i,
                                 const c128* __restrict__ sigma, int N, int i, int k, size_t ng) {
  const c128 s = sigma[size_t(i) * N + k];
  const cx<T> c{T(s.re), T(s.im)};
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < ng; e += size_t(gridDim.x) * blockDim.x)
    dst[e] = cmul(phi_i[e], c);
}

// the per-batch schedule of one (k, i) pass: pairs (source slot 0, target j), one contribution per
// target (pair slot, partner slot 1, coefficient index 1, no conjugation); two target lists, the
// first (k, i) pass overwriting W, the others accumulating
struct MixedPlan {
  std::vector<int> off;  // batch offsets into the pair list (size nbatch + 1)
  PairDesc* pairs = nullptr;
  TargetDesc* tgt_first = nullptr;
  TargetDesc* tgt_acc = nullptr;
  Contrib* contribs = nullptr;
  double* coef = nullptr;  // {0, 1}
  ~MixedPlan() {
    cudaFree(pairs);
    cudaFree(tgt_first);
    cudaFree(tgt_acc);
    cudaFree(contribs);
    cudaFree(coef);
  }
};

std::shared_ptr<MixedPlan> make_mixed_plan(int M, int mb) {
  auto pl = std::make_shared<MixedPlan>();
  std::vector<PairDesc> pairs;
  std::vector<TargetDesc> first, acc;
  std::vector<Contrib> cons;
  pl->off.push_back(0);
  for (int j0 = 0; j0 < M; j0 += mb) {
    const int j1 = std::min(M, j0 + mb);
    for (int j = j0; j < j1; ++j) {
      const int slot = j - j0;
      pairs.push_back({0, j, 1, -1});
      const int c = int(cons.size());
      cons.push_back({slot, 1, 1, 0});
      first.push_back({j, c, c + 1, 1});
      acc.push_back({j, c, c + 1, 0});
    }
    pl->off.push_back(int(pairs.size()));
  }
  const double coef[2] = {0.0, 1.0};
  auto up = [](auto** d, const auto& h) {
    using E = typename std::remove_reference<decltype(h)>::type::value_type;
    PT_CUDA_CHECK(cudaMalloc(reinterpret_cast<void**>(d), h.size() * sizeof(E)));
    PT_CUDA_CHECK(cudaMemcpy(*d, h.data(), h.size() * sizeof(E), cudaMemcpyHostToDevice));
  };
  up(&pl->pairs, pairs);
  up(&pl->tgt_first, first);
  up(&pl->tgt_acc, acc);
  up(&pl->contribs, cons);
  PT_CUDA_CHECK(cudaMalloc(&pl->coef, sizeof(coef)));
  PT_CUDA_CHECK(cudaMemcpy(pl->coef, coef, sizeof(coef), cudaMemcpyHostToDevice));
  return pl;
}

template <class T>
long long exchange_mixed_t(pt_ctx* ctx, const cx<T>* phi, const c128* sigma, int N, const cx<T>* tgt, int M,
                           cx<T>* out, const pt_grid& g, const pt_kernel& kern, pt_precision prec, cudaStream_t st) {
  if (!tgt) {
    tgt = phi;
    M = N;
  }
  const FftTables& ft = fft_tables(ctx, g, prec);
  const T* ktab = static_cast<const T*>(kernel_table(ctx, g, kern, prec));
  const size_t ng = ng_of(g);
  const size_t field = ng * sizeof(cx<T>);
  const int mb = std::max(1, std::min<int>(M, int(exchange_scratch_budget(ctx) / field)));
  char key[96];
  snprintf(key, sizeof(key), "mixed:%d:%d", M, mb);
  std::shared_ptr<MixedPlan> pl;
  auto it = ctx->caches.find(key);
  if (it == ctx->caches.end()) {
    pl = make_mixed_plan(M, mb);
    ctx->caches[key] = pl;
  } else {
    pl = std::static_pointer_cast<MixedPlan>(it->second);
  }
  cx<T>* two = static_cast<cx<T>*>(ctx->get(ctx->tagged("mixed_src"), 2 * field));  // [phi_k | sigma_ik phi_i]
  cx<T>* scratch = static_cast<cx<T>*>(ctx->get(ctx->tagged("exchange_scratch"), size_t(mb) * field));
  const cx<T>* twg = static_cast<const cx<T>*>(ft.tw);
  const bool fixed = fixed_cubic(g);
  const GridPlan& gp = ft.plan;
  const int nbatch = int(pl->off.size()) - 1;
  const int sblocks = std::max(1, std::min<int>(ctx->num_sms * 8, int((ng + 255) / 256)));
  for (int k = 0; k < N; ++k) {
    PT_CUDA_CHECK(cudaMemcpyAsync(two, phi + size_t(k) * ng, field, cudaMemcpyDeviceToDevice, st));
    for (int i = 0; i < N; ++i) {
      PT_LAUNCH(k_scale_by_sigma<T>, sblocks, 256, 0, st, two + ng, phi + size_t(i) * ng, sigma, N, i, k, ng);
      const TargetDesc* tl = (k == 0 && i == 0) ? pl->tgt_first : pl->tgt_acc;
      for (int b = 0; b < nbatch; ++b) {
        const int p0 = pl->off[b], np = pl->off[b + 1] - p0;
        if (fixed)
          exchange_batch_fixed<T>(g.nx, two, tgt, pl->coef, pl->pairs + p0, np, tl + p0, np, pl->contribs, ktab, twg,
                                  scratch, out, st);
        else
          exchange_batch_generic<T>(gp, two, tgt, pl->coef, pl->pairs + p0, np, tl + p0, np, pl->contribs, ktab, twg,
                                    scratch, out, st);
      }
    }
  }
  return (long long)N * N * M;
}

}  // namespace

long long exchange_mixed(pt_ctx* ctx, const void* phi, const c128* sigma, int N, const void* tgt, int M, void* out,
                         const pt_grid& g, const pt_kernel& k, pt_precision prec, cudaStream_t st) {
  if (prec == PT_FP64)
    return exchange_mixed_t<double>(ctx, static_cast<const c128*>(phi), sigma, N, static_cast<const c128*>(tgt), M,
                                    static_cast<c128*>(out), g, k, prec, st);
  return exchange_mixed_t<float>(ctx, static_cast<const c64*>(phi), sigma, N, static_cast<const c64*>(tgt), M,
                                 static_cast<c64*>(out), g, k, prec, st);
}

}  // namespace pt
