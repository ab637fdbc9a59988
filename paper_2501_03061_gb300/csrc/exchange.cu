// Occupation-weighted screened Fock exchange  W_j = V_x tgt_j  (Sec. IV-A1, Eq. vxdiag).
//
// For every pair (i, j):  rho = conj(src_i) tgt_j -> FFT -> * K(G)/Ng -> IFFT -> v_ij,
// then W_j -= d_i src_i v_ij.  Pairs are processed in batches whose pair fields
// (one Ng-point scratch field per pair) stay resident in L2 between the three
// passes of the 3-D FFT:
//   pass 1 (plane):   pair product and the x, y transforms of one z-plane;
//   pass 2 (column):  forward z transform, kernel multiply, inverse z transform;
//   pass 3 (plane):   inverse y, x transforms and the d_i-weighted accumulate of
//                     every pair of the batch that contributes to one target plane.
// With tgt == src the kernel symmetry v_ji = conj(v_ij) (K real and even) lets
// one pair FFT serve both W_j (with d_i src_i) and W_i (with d_j src_j conj v).
// Pairs whose every contribution has d = 0 are skipped on the device.
#include <algorithm>
#include <cstring>

#include "exchange_sched.h"
#include "fft.cuh"
#include "fft_fixed.cuh"
#include "internal.h"

namespace pt {

namespace {

constexpr int NT = 512;          // threads per CTA of the tile kernels
constexpr int MAXE = kMaxDim * kMaxDim;  // tile elements (64 x 64)
constexpr int EPT = (MAXE + NT - 1) / NT;

template <class T>
__device__ __forceinline__ void load_twiddles(cx<T>* tw, const cx<T>* twg, int n) {
  for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
}

// pass 1: rho = conj(src_i) tgt_j on plane z, then FFT along x and y
template <class T>
__global__ void __launch_bounds__(NT) k_pair_fwd_plane(GridPlan gp, const cx<T>* __restrict__ src,
                                                       const cx<T>* __restrict__ tgt,
                                                       const double* __restrict__ occ,
                                                       const PairDesc* __restrict__ pairs,
                                                       cx<T>* __restrict__ scratch,
                                                       const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf = tw + 3 * kMaxDim;
  const int z = blockIdx.x, p = blockIdx.y;
  const PairDesc pd = pairs[p];
  if (pair_skipped(pd, occ)) return;
  const int nx = gp.nx, ny = gp.ny, pitch = gp.pitch_x;
  const int plane = nx * ny;
  const size_t ng = size_t(plane) * gp.nz;
  load_twiddles(tw, twg, nx + ny + gp.nz);
  const cx<T>* a = src + size_t(pd.i) * ng + size_t(z) * plane;
  const cx<T>* b = tgt + size_t(pd.j) * ng + size_t(z) * plane;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int y = e / nx, x = e - y * nx;
    buf[y * pitch + x] = cmulc(a[e], b[e]);
  }
  __syncthreads();
  fft_lines<false, NT, MAXE>(buf, gp.ax[0], ny, pitch, 1, tw);       // x
  fft_lines<false, NT, MAXE>(buf, gp.ax[1], nx, 1, pitch, tw + nx);  // y
  cx<T>* o = scratch + size_t(p) * ng + size_t(z) * plane;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int y = e / nx, x = e - y * nx;
    o[e] = buf[y * pitch + x];
  }
}

// pass 2: on the (z, x) slab of row y: FFT along z, multiply by K/Ng, inverse FFT along z
template <class T>
__global__ void __launch_bounds__(NT) k_pair_column(GridPlan gp, cx<T>* __restrict__ scratch,
                                                    const T* __restrict__ ktab,
                                                    const double* __restrict__ occ,
                                                    const PairDesc* __restrict__ pairs,
                                                    const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf = tw + 3 * kMaxDim;
  const int y = blockIdx.x, p = blockIdx.y;
  const PairDesc pd = pairs[p];
  if (pair_skipped(pd, occ)) return;
  const int nx = gp.nx, ny = gp.ny, nz = gp.nz, pitch = gp.pitch_x;
  const size_t ng = size_t(nx) * ny * nz;
  load_twiddles(tw, twg, nx + ny + nz);
  cx<T>* f = scratch + size_t(p) * ng;
  const int slab = nz * nx;
  for (int e = threadIdx.x; e < slab; e += NT) {
    const int z = e / nx, x = e - z * nx;
    buf[z * pitch + x] = f[(size_t(z) * ny + y) * nx + x];
  }
  __syncthreads();
  fft_lines<false, NT, MAXE>(buf, gp.ax[2], nx, 1, pitch, tw + nx + ny);
  for (int e = threadIdx.x; e < slab; e += NT) {
    const int z = e / nx, x = e - z * nx;
    buf[z * pitch + x] = buf[z * pitch + x] * ktab[(size_t(z) * ny + y) * nx + x];
  }
  __syncthreads();
  fft_lines<true, NT, MAXE>(buf, gp.ax[2], nx, 1, pitch, tw + nx + ny);
  for (int e = threadIdx.x; e < slab; e += NT) {
    const int z = e / nx, x = e - z * nx;
    f[(size_t(z) * ny + y) * nx + x] = buf[z * pitch + x];
  }
}

// pass 3: for target t and plane z, inverse y/x FFT of each contributing pair and
// acc += d * partner * v (v conjugated for the mirrored half of a symmetric pair)
template <class T>
__global__ void __launch_bounds__(NT) k_pair_inv_acc(GridPlan gp, const cx<T>* __restrict__ scratch,
                                                     const cx<T>* __restrict__ src,
                                                     const double* __restrict__ occ,
                                                     const TargetDesc* __restrict__ tgts,
                                                     const Contrib* __restrict__ contribs,
                                                     cx<T>* __restrict__ out,
                                                     const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf = tw + 3 * kMaxDim;
  const int z = blockIdx.x;
  const TargetDesc td = tgts[blockIdx.y];
  const int nx = gp.nx, ny = gp.ny, pitch = gp.pitch_x;
  const int plane = nx * ny;
  const size_t ng = size_t(plane) * gp.nz;
  load_twiddles(tw, twg, nx + ny + gp.nz);
  cx<T> acc[EPT];
#pragma unroll
  for (int u = 0; u < EPT; ++u) acc[u] = czero<T>();
  for (int c = td.cbeg; c < td.cend; ++c) {
    const Contrib cb = contribs[c];
    const T coef = T(occ[cb.occ]);
    if (coef == T(0)) continue;
    const cx<T>* f = scratch + size_t(cb.slot) * ng + size_t(z) * plane;
    for (int e = threadIdx.x; e < plane; e += NT) {
      const int y = e / nx, x = e - y * nx;
      buf[y * pitch + x] = f[e];
    }
    __syncthreads();
    fft_lines<true, NT, MAXE>(buf, gp.ax[1], nx, 1, pitch, tw + nx);  // y
    fft_lines<true, NT, MAXE>(buf, gp.ax[0], ny, pitch, 1, tw);       // x
    const cx<T>* pp = src + size_t(cb.partner) * ng + size_t(z) * plane;
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int e = threadIdx.x + u * NT;
      if (e < plane) {
        const int y = e / nx, x = e - y * nx;
        cx<T> v = buf[y * pitch + x];
        if (cb.conj) v.im = -v.im;
        acc[u] = acc[u] + cmul(pp[e], v) * coef;
      }
    }
    __syncthreads();
  }
  cx<T>* o = out + size_t(td.t) * ng + size_t(z) * plane;
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    const int e = threadIdx.x + u * NT;
    if (e < plane) o[e] = td.first ? czero<T>() - acc[u] : o[e] - acc[u];
  }
}

// ------------------------------------------------------------------------------------------
// host: pair schedule
// ------------------------------------------------------------------------------------------
}  // namespace

std::shared_ptr<ScheduleImpl> build_schedule(int N, int M, bool sym, int B) {
  auto s = std::make_shared<ScheduleImpl>();
  PairPlan plan = plan_pairs(N, M, sym, B);
  s->N = N;
  s->M = M;
  s->B = B;
  s->sym = sym;
  s->pair_off = std::move(plan.pair_off);
  s->tgt_off = std::move(plan.tgt_off);
  s->max_pairs = plan.max_pairs;
  s->max_tgts = plan.max_tgts;
  s->total_pairs = (long long)plan.pairs.size();
  s->h_pairs = std::move(plan.pairs);
  s->h_tgts = std::move(plan.tgts);
  s->h_contribs = std::move(plan.contribs);
  const auto& pairs = s->h_pairs;
  const auto& tgts = s->h_tgts;
  const auto& cons = s->h_contribs;
  PT_CUDA_CHECK(cudaMalloc(&s->d_pairs, pairs.size() * sizeof(PairDesc)));
  PT_CUDA_CHECK(cudaMalloc(&s->d_tgts, tgts.size() * sizeof(TargetDesc)));
  PT_CUDA_CHECK(cudaMalloc(&s->d_contribs, cons.size() * sizeof(Contrib)));
  PT_CUDA_CHECK(cudaMemcpy(s->d_pairs, pairs.data(), pairs.size() * sizeof(PairDesc), cudaMemcpyHostToDevice));
  PT_CUDA_CHECK(cudaMemcpy(s->d_tgts, tgts.data(), tgts.size() * sizeof(TargetDesc), cudaMemcpyHostToDevice));
  PT_CUDA_CHECK(cudaMemcpy(s->d_contribs, cons.data(), cons.size() * sizeof(Contrib), cudaMemcpyHostToDevice));
  return s;
}

namespace {

size_t tile_smem_bytes(size_t esize) { return (3 * kMaxDim + size_t(kMaxDim) * (kMaxDim + 1)) * esize; }

template <class T>
void set_smem_attrs() {
  static DeviceOnce once;
  once([] {
    const int bytes = int(tile_smem_bytes(sizeof(cx<T>)));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pair_fwd_plane<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pair_column<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pair_inv_acc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  });
}

template <class T>
long long exchange_t(pt_ctx* ctx, const cx<T>* src, const double* occ, int N, const cx<T>* tgt, int M,
                     cx<T>* out, const pt_grid& g, const pt_kernel& k, pt_precision prec, cudaStream_t st) {
  const bool sym = (tgt == nullptr);
  if (sym) {
    tgt = src;
    M = N;
  }
  const FftTables& ft = fft_tables(ctx, g, prec);
  const T* ktab = static_cast<const T*>(kernel_table(ctx, g, k, prec));
  if constexpr (sizeof(T) == 4) {
    if (exchange64_applies(g) && ctx->exchange64_engine == 2) {
      const long long np = exchange64_persist(ctx, src, occ, N, tgt, M, sym, out, ktab,
                                              static_cast<const cx<T>*>(ft.tw), st);
      if (!ctx->defer_checks) exchange_check(ctx, st);
      return np;
    }
  }
  const size_t ng = ng_of(g);
  const size_t field = ng * sizeof(cx<T>);
  // Pair batch: as many pair fields as fit a budget that keeps them L2-resident (the 64^3 TMA
  // pipeline takes its own, larger budget: see pt_ctx::tma64_budget).
  const bool tma64 =
      sizeof(T) == 4 && exchange64_applies(g) && (ctx->exchange64_engine == 0 || ctx->exchange64_engine == 3);
  const size_t budget = ctx->budget_override ? ctx->budget_override
                                             : (tma64 ? ctx->tma64_budget : exchange_scratch_budget(ctx));
  int B = int(std::floor(std::sqrt(double(std::max<size_t>(1, budget / field)))));
  B = std::max(1, std::min(B, std::max(N, M)));
  if (tma64) B = std::min(B, kExchange64MaxTile);
  char key[128];
  snprintf(key, sizeof(key), "sched:%d:%d:%d:%d", N, M, int(sym), B);
  auto it = ctx->caches.find(key);
  std::shared_ptr<ScheduleImpl> sch;
  if (it == ctx->caches.end()) {
    sch = build_schedule(N, M, sym, B);
    ctx->caches[key] = sch;
  } else {
    sch = std::static_pointer_cast<ScheduleImpl>(it->second);
  }
  if constexpr (sizeof(T) == 4) {
    if (exchange64_applies(g) && (ctx->exchange64_engine == 0 || ctx->exchange64_engine == 3)) {
      exchange64_tma(ctx, *sch, src, occ, tgt, M, out, ktab, static_cast<const cx<T>*>(ft.tw), st,
                     ctx->exchange64_engine == 3);
      if (!ctx->defer_checks) exchange_check(ctx, st);
      return sch->total_pairs;
    }
  }
  cx<T>* scratch = static_cast<cx<T>*>(ctx->get(ctx->tagged("exchange_scratch"), size_t(sch->max_pairs) * field));
  const cx<T>* twg = static_cast<const cx<T>*>(ft.tw);
  const int nbatch = int(sch->pair_off.size()) - 1;
  if (fixed_cubic(g)) {
    // compile-time FFT kernels for this side; inverse plane transforms once per pair
    for (int b = 0; b < nbatch; ++b) {
      const int p0 = sch->pair_off[b], np = sch->pair_off[b + 1] - p0;
      const int t0 = sch->tgt_off[b], nt = sch->tgt_off[b + 1] - t0;
      exchange_batch_fixed<T>(g.nx, src, tgt, occ, sch->d_pairs + p0, np, sch->d_tgts + t0, nt, sch->d_contribs,
                              ktab, twg, scratch, out, st, ctx->fft_threads);
    }
    return sch->total_pairs;
  }
  set_smem_attrs<T>();
  const size_t smem = tile_smem_bytes(sizeof(cx<T>));
  for (int b = 0; b < nbatch; ++b) {
    const int p0 = sch->pair_off[b], np = sch->pair_off[b + 1] - p0;
    const int t0 = sch->tgt_off[b], nt = sch->tgt_off[b + 1] - t0;
    PT_LAUNCH(k_pair_fwd_plane<T>, dim3(g.nz, np), NT, smem, st, ft.plan, src, tgt, occ, sch->d_pairs + p0,
              scratch, twg);
    PT_LAUNCH(k_pair_column<T>, dim3(g.ny, np), NT, smem, st, ft.plan, scratch, ktab, occ, sch->d_pairs + p0,
              twg);
    PT_LAUNCH(k_pair_inv_acc<T>, dim3(g.nz, nt), NT, smem, st, ft.plan, scratch, src, occ, sch->d_tgts + t0,
              sch->d_contribs, out, twg);
  }
  return sch->total_pairs;
}

}  // namespace

template <class T>
void exchange_batch_generic(const GridPlan& gp, const cx<T>* src, const cx<T>* tgt, const double* occ,
                            const PairDesc* pairs, int np, const TargetDesc* tgts, int nt, const Contrib* contribs,
                            const T* ktab, const cx<T>* tw, cx<T>* scratch, cx<T>* out, cudaStream_t st) {
  set_smem_attrs<T>();
  const size_t smem = tile_smem_bytes(sizeof(cx<T>));
  PT_LAUNCH(k_pair_fwd_plane<T>, dim3(gp.nz, np), NT, smem, st, gp, src, tgt, occ, pairs, scratch, tw);
  PT_LAUNCH(k_pair_column<T>, dim3(gp.ny, np), NT, smem, st, gp, scratch, ktab, occ, pairs, tw);
  PT_LAUNCH(k_pair_inv_acc<T>, dim3(gp.nz, nt), NT, smem, st, gp, scratch, src, occ, tgts, contribs, out, tw);
}

template void exchange_batch_generic<float>(const GridPlan&, const c64*, const c64*, const double*, const PairDesc*,
                                            int, const TargetDesc*, int, const Contrib*, const float*, const c64*,
                                            c64*, c64*, cudaStream_t);
template void exchange_batch_generic<double>(const GridPlan&, const c128*, const c128*, const double*,
                                             const PairDesc*, int, const TargetDesc*, int, const Contrib*,
                                             const double*, const c128*, c128*, c128*, cudaStream_t);

size_t exchange_scratch_budget(const pt_ctx* ctx) { return ctx->scratch_budget; }

bool exchange64_applies(const pt_grid& g) { return g.nx == 64 && g.ny == 64 && g.nz == 64; }

void exchange_check(pt_ctx* ctx, cudaStream_t st) {
  int* err = static_cast<int*>(ctx->get("exchange_err", sizeof(int)));
  int h = 0;
  PT_CUDA_CHECK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PT_CUDA_CHECK(cudaStreamSynchronize(st));
  if (h) fail(PT_TIMEOUT, "exchange: a TMA wait timed out on the device (code " + std::to_string(h) + ")");
}

long long exchange(pt_ctx* ctx, const void* src, const double* occ, int N, const void* tgt, int M, void* out,
                   const pt_grid& g, const pt_kernel& k, pt_precision prec, cudaStream_t st) {
  if (prec == PT_FP64)
    return exchange_t<double>(ctx, static_cast<const c128*>(src), occ, N, static_cast<const c128*>(tgt), M,
                              static_cast<c128*>(out), g, k, prec, st);
  return exchange_t<float>(ctx, static_cast<const c64*>(src), occ, N, static_cast<const c64*>(tgt), M,
                           static_cast<c64*>(out), g, k, prec, st);
}

}  // namespace pt
