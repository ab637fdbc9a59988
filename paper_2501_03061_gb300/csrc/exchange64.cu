// Pair-FFT exchange specialised for 64^3 grids (the 128-site cell and the largest batched grids).
//
// A 64-point line transform is held by a group of 8 lanes, lane t holding x[t + 8a] (a < 8):
// radix-8 DFT over a in registers, twiddle w64^{t k1} (derived in registers from w64^t), an
// 8 x 8 transpose through a swizzled per-group shared-memory tile (warp-synchronous, no CTA
// barrier), radix-8 DFT over t.  The result sits in the same layout (lane k1 holds
// X[k1 + 8 k2]), so forward and inverse transforms chain without data movement.
//
// Four roles of one kernel, software-pipelined over pair batches on four scratch slots
// (launch k runs A of batch k, B of k-1, C of k-2, D of k-3), so one launch per batch keeps
// every SM busy and each pair is transformed exactly once forward and once back:
//   A (plane z of a pair):   rho = conj(src_i) tgt_j, FFT along x, CTA transpose, FFT along y.
//   B (slab ky of pairs):    FFT along z, multiply by K/Ng, inverse FFT along z.
//   C (plane z of a pair):   inverse FFT along y, CTA transpose, inverse FFT along x -> v_ij.
//   D (plane z of a target): acc = sum over contributing pairs of d * partner * v (v conjugated
//                            for the mirrored half of a symmetric pair); W = -acc (or W -= acc).
#include <algorithm>

#include "exchange_sched.h"
#include "fft.cuh"
#include "internal.h"

namespace pt {

namespace {

constexpr int G = 64;
constexpr int PITCH = 68;   // plane row pitch (complex): rows and columns both conflict-free (68 = 4 mod 16)
constexpr int GSTR = 72;    // per-group transpose tile stride (complex): 4 groups of a warp in 2 wavefronts
constexpr int THREADS = 512;
constexpr int GROUPS = THREADS / 8;
constexpr int PPC = 4;      // pairs per pass-B CTA (K(G) reused from registers)

template <class T>
struct Smem {
  cx<T> tw[G];
  cx<T> plane[G * PITCH];
  cx<T> grp[GROUPS * GSTR];
};

// in-group 64-point transform: lane t holds x[t + 8a] in v[a]; on exit X[t + 8k] in v[k]
template <bool INV, class T>
__device__ __forceinline__ void fft64g(cx<T> (&v)[8], int t, cx<T>* gs, const cx<T>* tw) {
  dft8<INV>(v);
  // w^k for k = 1..7 from w = w64^t in at most three products (error a few ulp)
  cx<T> w1 = tw[t];
  if (INV) w1.im = -w1.im;
  const cx<T> w2 = cmul(w1, w1), w4 = cmul(w2, w2);
  v[1] = cmul(v[1], w1);
  v[2] = cmul(v[2], w2);
  v[3] = cmul(v[3], cmul(w1, w2));
  v[4] = cmul(v[4], w4);
  v[5] = cmul(v[5], cmul(w1, w4));
  v[6] = cmul(v[6], cmul(w2, w4));
  v[7] = cmul(v[7], cmul(cmul(w1, w2), w4));
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 8; ++k) gs[k * 8 + (t ^ k)] = v[k];
  __syncwarp();
#pragma unroll
  for (int s = 0; s < 8; ++s) v[s] = gs[t * 8 + (s ^ t)];
  dft8<INV>(v);
}

struct Launch {
  // roles A, B, C, D on four batches; a count of 0 leaves the role idle
  int nA, nB, nC, nD;        // CTAs of each role
  int a_pair0, b_pair0, b_np, c_pair0;
  int d_tgt0;                // target range of batch d (nD = 64 * nt)
  int slotA, slotB, slotC, slotD;
};

template <class T>
__global__ void __launch_bounds__(THREADS, sizeof(T) == 4 ? 2 : 1)
    k_exchange64(Launch L, const cx<T>* __restrict__ src, const cx<T>* __restrict__ tgt,
                 const double* __restrict__ occ, const PairDesc* __restrict__ pairs,
                 const TargetDesc* __restrict__ tgts, const Contrib* __restrict__ contribs,
                 const T* __restrict__ ktab, cx<T>* __restrict__ scratch, size_t slot_elems,
                 cx<T>* __restrict__ out, const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  Smem<T>& sm = *reinterpret_cast<Smem<T>*>(smem_raw);
  const int tid = threadIdx.x;
  const int grp = tid >> 3, t = tid & 7;
  cx<T>* gs = sm.grp + grp * GSTR;
  if (tid < G) sm.tw[tid] = twg[tid];
  __syncthreads();
  constexpr size_t ng = size_t(G) * G * G;
  int bid = blockIdx.x;

  if (bid < L.nA) {
    // ---------------- pass A: pair product, x and y transforms of plane z ----------------
    const int z = bid % G, p = bid / G;
    const PairDesc pd = pairs[L.a_pair0 + p];
    if (pair_skipped(pd, occ)) return;
    const int y = grp;
    const cx<T>* a = src + size_t(pd.i) * ng + size_t(z) * G * G + y * G;
    const cx<T>* b = tgt + size_t(pd.j) * ng + size_t(z) * G * G + y * G;
    cx<T> v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = cmulc(a[t + 8 * q], b[t + 8 * q]);
    fft64g<false>(v, t, gs, sm.tw);
#pragma unroll
    for (int k = 0; k < 8; ++k) sm.plane[y * PITCH + t + 8 * k] = v[k];
    __syncthreads();
    const int kx = grp;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = sm.plane[(t + 8 * q) * PITCH + kx];
    fft64g<false>(v, t, gs, sm.tw);
    cx<T>* o = scratch + size_t(L.slotA) * slot_elems + size_t(p) * ng + size_t(z) * G * G + kx;
#pragma unroll
    for (int k = 0; k < 8; ++k) o[(t + 8 * k) * G] = v[k];
    return;
  }
  bid -= L.nA;
  if (bid < L.nB) {
    // ---------------- pass B: z transform, kernel multiply, inverse z transform ----------------
    const int ky = bid % G, chunk = bid / G;
    const int kx = grp;
    T kv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) kv[k] = ktab[(size_t(t + 8 * k) * G + ky) * G + kx];
    const int p0 = chunk * PPC, p1 = min(L.b_np, p0 + PPC);
    for (int p = p0; p < p1; ++p) {
      const PairDesc pd = pairs[L.b_pair0 + p];
      if (pair_skipped(pd, occ)) continue;
      cx<T>* f = scratch + size_t(L.slotB) * slot_elems + size_t(p) * ng + size_t(ky) * G + kx;
      cx<T> v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = f[size_t(t + 8 * q) * G * G];
      fft64g<false>(v, t, gs, sm.tw);
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = v[k] * kv[k];
      fft64g<true>(v, t, gs, sm.tw);
#pragma unroll
      for (int k = 0; k < 8; ++k) f[size_t(t + 8 * k) * G * G] = v[k];
    }
    return;
  }
  bid -= L.nB;
  if (bid < L.nC) {
    // ---------------- pass C: inverse y and x transforms of plane z -> v_ij ----------------
    const int z = bid % G, p = bid / G;
    const PairDesc pd = pairs[L.c_pair0 + p];
    if (pair_skipped(pd, occ)) return;
    cx<T>* f = scratch + size_t(L.slotC) * slot_elems + size_t(p) * ng + size_t(z) * G * G;
    const int kx = grp, y = grp;
    cx<T> v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = f[(t + 8 * q) * G + kx];
    fft64g<true>(v, t, gs, sm.tw);
#pragma unroll
    for (int k = 0; k < 8; ++k) sm.plane[(t + 8 * k) * PITCH + kx] = v[k];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = sm.plane[y * PITCH + t + 8 * q];
    fft64g<true>(v, t, gs, sm.tw);
    __syncthreads();  // every column read of f is done before the rows are overwritten
#pragma unroll
    for (int k = 0; k < 8; ++k) f[y * G + t + 8 * k] = v[k];
    return;
  }
  bid -= L.nC;
  {
    // ---------------- pass D: weighted accumulate of v into the target plane ----------------
    const int z = bid % G;
    const TargetDesc td = tgts[L.d_tgt0 + bid / G];
    constexpr int EPT = G * G / THREADS;
    cx<T> acc[EPT];
#pragma unroll
    for (int u = 0; u < EPT; ++u) acc[u] = czero<T>();
    for (int c = td.cbeg; c < td.cend; ++c) {
      const Contrib cb = contribs[c];
      const T coef = T(occ[cb.occ]);
      if (coef == T(0)) continue;
      const cx<T>* f = scratch + size_t(L.slotD) * slot_elems + size_t(cb.slot) * ng + size_t(z) * G * G;
      const cx<T>* pp = src + size_t(cb.partner) * ng + size_t(z) * G * G;
#pragma unroll
      for (int u = 0; u < EPT; ++u) {
        const int e = tid + u * THREADS;
        cx<T> w = f[e];
        if (cb.conj) w.im = -w.im;
        acc[u] = acc[u] + cmul(pp[e], w) * coef;
      }
    }
    cx<T>* o = out + size_t(td.t) * ng + size_t(z) * G * G;
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int e = tid + u * THREADS;
      o[e] = td.first ? czero<T>() - acc[u] : o[e] - acc[u];
    }
  }
}

template <class T>
void set_attr() {
  static bool done = false;
  if (done) return;
  PT_CUDA_CHECK(cudaFuncSetAttribute(k_exchange64<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(sizeof(Smem<T>))));
  done = true;
}

}  // namespace

bool exchange64_applies(const pt_grid& g) { return g.nx == 64 && g.ny == 64 && g.nz == 64; }

template <class T>
void exchange64(pt_ctx* ctx, const ScheduleImpl& sch, const cx<T>* src, const double* occ, const cx<T>* tgt,
                cx<T>* out, const T* ktab, const cx<T>* tw, cudaStream_t st) {
  constexpr size_t ng = size_t(G) * G * G;
  const size_t slot_elems = size_t(sch.max_pairs) * ng;
  cx<T>* scratch = static_cast<cx<T>*>(ctx->get("exchange64_scratch", 4 * slot_elems * sizeof(cx<T>)));
  set_attr<T>();
  const int nb = int(sch.pair_off.size()) - 1;
  for (int k = 0; k < nb + 3; ++k) {
    Launch L{};
    if (k < nb) {
      L.a_pair0 = sch.pair_off[k];
      L.nA = G * (sch.pair_off[k + 1] - L.a_pair0);
      L.slotA = k % 4;
    }
    const int b = k - 1, c = k - 2, d = k - 3;
    if (b >= 0 && b < nb) {
      L.b_pair0 = sch.pair_off[b];
      L.b_np = sch.pair_off[b + 1] - L.b_pair0;
      L.nB = G * ((L.b_np + PPC - 1) / PPC);
      L.slotB = b % 4;
    }
    if (c >= 0 && c < nb) {
      L.c_pair0 = sch.pair_off[c];
      L.nC = G * (sch.pair_off[c + 1] - L.c_pair0);
      L.slotC = c % 4;
    }
    if (d >= 0) {
      L.d_tgt0 = sch.tgt_off[d];
      L.nD = G * (sch.tgt_off[d + 1] - L.d_tgt0);
      L.slotD = d % 4;
    }
    const int grid = L.nA + L.nB + L.nC + L.nD;
    if (grid == 0) continue;
    PT_LAUNCH(k_exchange64<T>, grid, THREADS, sizeof(Smem<T>), st, L, src, tgt, occ, sch.d_pairs, sch.d_tgts,
              sch.d_contribs, ktab, scratch, slot_elems, out, tw);
  }
}

template void exchange64<float>(pt_ctx*, const ScheduleImpl&, const c64*, const double*, const c64*, c64*,
                                const float*, const c64*, cudaStream_t);
template void exchange64<double>(pt_ctx*, const ScheduleImpl&, const c128*, const double*, const c128*, c128*,
                                 const double*, const c128*, cudaStream_t);

}  // namespace pt
