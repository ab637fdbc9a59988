// FP32 pair-FFT exchange for 64^3 grids as ONE persistent launch per application (Sec. IV-A1,
// Eq. vxdiag; the batched pair products of Sec. III-B).
//
// The four roles of the pipelined TMA kernel — A: pair product and x/y transforms of a plane;
// B: z transform, K(G)/Ng and inverse z transform of two slabs; C: inverse y/x transforms of two
// planes; D: the occupation-weighted accumulate of a tile's contributions into half a target
// plane — run as items of one cooperative launch (every CTA resident).  Each CTA takes the next
// item from a global counter.  The items follow a software pipeline over the pairs of the
// schedule ("waves"): wave w holds, oldest stage first, the D items of the tile whose last pair is
// w - LD, the C items of pair w - LC, the B items of pair w - LB and the A items of pair w.  An
// item waits (bounded) for the counters of the items it depends on, all of which come earlier in
// the order, so the lowest unfinished item can always run:
//   B(p) after the 64 A items of p;  C(p) after the 32 B items of p;
//   D(tile) after the C items of all its pairs;
//   A(p) after the D items of the tile of pair p - R, the last user of p's ring slot;
//   D(tile, target t, half-plane h) after D(previous tile touching t, h) (W is read-modify-written).
// Pair fields live in a ring of R slots (R * 2 MiB), small enough to stay in L2 between the
// passes, instead of whole tiles' worth of fields in HBM.  Counters are released with a
// gpu-scope fence after the CTA's barrier and acquired before the dependent loads (with an
// async-proxy fence before TMA reads of data that plain stores wrote).  Every wait is bounded by a
// %globaltimer deadline: on expiry the CTA records an error word and stops, and the other CTAs
// stop at their next item.
#include <algorithm>
#include <cstring>

#include "exchange64_common.cuh"
#include "exchange_sched.h"
#include "internal.h"

namespace pt {

void encode_tmap_4d_u64(CUtensorMap* map, const void* base, const uint64_t dims[4], const uint64_t strides_bytes[3],
                        const uint32_t box[4], CUtensorMapSwizzle swizzle);

namespace {

using namespace x64;

constexpr int ZH = 2 * G;  // D items per target: (plane, half)

struct PArgs {
  const PairDesc* pairs;     // [P] plan order
  const int* pair_batch;     // [P] tile of each pair
  const int* batch_pair0;    // [nbatch] first pair of each tile
  const int* batch_ndone;    // [nbatch] D items of each tile
  const int* batch_npairs;   // [nbatch]
  const int* batch_tgt0;     // [nbatch] first target descriptor of each tile
  const TargetDesc* tgts;    // [ntgt] with global contribution ranges
  const Contrib* contribs;   // slot = pair index within its tile
  const int* tgt_seq;        // [ntgt] earlier tiles that touched the same target
  const int2* waves;         // [nwaves + 1] {first item, D tile or -1}
  int nwaves, total, npairs, ring, lagB, lagC, lagD;
  int* next;                 // item counter
  int* cntA;                 // [P]
  int* cntB;                 // [P]
  int* cntC;                 // [nbatch]
  int* cntD;                 // [nbatch]
  int* wseq;                 // [M * ZH]
  int* err;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// thread 0 only: wait until *c >= target (or the error word is set / the deadline passes)
__device__ bool wait_count(const int* c, int target, int* err, int code) {
  if (ld_acquire(c) >= target) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    __nanosleep(100);
    if (ld_acquire(c) >= target) return true;
    if (*reinterpret_cast<volatile int*>(err)) return false;
    if (globaltimer_ns() - t0 > TIMEOUT_NS) {
      atomicOr(err, code);
      return false;
    }
  }
}

// all threads: the CTA's writes are done; thread 0 publishes them with one increment
__device__ __forceinline__ void signal_add(int* c, int tid) {
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    atomicAdd(c, 1);
  }
}

__global__ void __launch_bounds__(THREADS, 2)
    k_exchange64_persist(const __grid_constant__ CUtensorMap tm_src, const __grid_constant__ CUtensorMap tm_tgt,
                         const __grid_constant__ CUtensorMap tm_plane, const __grid_constant__ CUtensorMap tm_slab,
                         const __grid_constant__ PArgs A, const c64* __restrict__ src,
                         const double* __restrict__ occ, const float* __restrict__ ktab, const c64* __restrict__ twg,
                         c64* __restrict__ scratch, c64* __restrict__ out) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ int s_item, s_ok;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  c64* P = reinterpret_cast<c64*>(sm + OFF_P);
  c64* tw = reinterpret_cast<c64*>(sm + OFF_TW);
  const uint32_t bar = base + OFF_BAR;
  const int tid = threadIdx.x, grp = tid >> 3, t = tid & 7;
  const int gpar = (grp & 1) << 3;
  constexpr size_t ng = size_t(G) * G * G;
  constexpr int H = G / 2;
  if (tid < G) tw[tid] = twg[tid];
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 8, 1);
    mbar_init(bar + 16, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t ph[3] = {0u, 0u, 0u};  // completed phases of the three barriers (same in every thread)
  int wave = 0;                   // cursor into the wave table (items are taken in increasing order)
  for (;;) {
    if (tid == 0) s_item = *reinterpret_cast<volatile int*>(A.err) ? A.total : atomicAdd(A.next, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= A.total) break;
    while (A.waves[wave + 1].x <= item) ++wave;
    int u = item - A.waves[wave].x;
    const int dtile = A.waves[wave].y;
    const int nD = dtile >= 0 ? A.batch_ndone[dtile] : 0;
    const int pC = wave - A.lagC, pB = wave - A.lagB, pA = wave;
    const int nC = (pC >= 0 && pC < A.npairs) ? H : 0;
    const int nB = (pB >= 0 && pB < A.npairs) ? H : 0;
    // every thread takes the same branch: the item is uniform over the CTA
    if (u < nD) {
      // ---------------- D: half a target plane, the contributions of one tile ----------------
      const int k = A.batch_tgt0[dtile] + u / ZH;
      const int zh = u % ZH, z = zh >> 1, half = zh & 1;
      const TargetDesc td = A.tgts[k];
      const int seq = A.tgt_seq[k];
      int* wq = A.wseq + size_t(td.t) * ZH + zh;
      if (tid == 0) {
        bool ok = wait_count(A.cntC + dtile, H * A.batch_npairs[dtile], A.err, 64);
        ok = ok && wait_count(wq, seq, A.err, 128);
        if (ok) fence_proxy_async_global();
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) break;
      constexpr int EPT = G * G / (2 * THREADS);
      constexpr uint32_t HB = G * G / 2 * sizeof(c64);
      constexpr int DS = 3;
      const size_t zoff = size_t(z) * G * G;
      const size_t hoff = zoff + size_t(half) * (G * G / 2);
      const int nc = td.cend - td.cbeg;
      const int pair0 = A.batch_pair0[dtile];
      auto issue = [&](int i) {  // thread 0
        const Contrib cc = A.contribs[td.cbeg + i];
        const int sl = i % DS;
        const uint32_t dst = base + uint32_t(sl) * 2u * HB;
        const int rs = (pair0 + cc.slot) % A.ring;
        mbar_arrive_expect_tx(bar + 8u * sl, 2u * HB);
        bulk_load(dst, scratch + size_t(rs) * ng + hoff, HB, bar + 8u * sl);
        bulk_load(dst + HB, src + size_t(cc.partner) * ng + hoff, HB, bar + 8u * sl);
      };
      if (tid == 0) {
        fence_proxy_async_smem();  // earlier items read and wrote these slots through the generic proxy
        for (int i = 0; i < min(DS, nc); ++i) issue(i);
      }
      c64 acc[EPT];
#pragma unroll
      for (int e = 0; e < EPT; ++e) acc[e] = czero<float>();
      bool ok = true;
      for (int i = 0; i < nc; ++i) {
        const int sl = i % DS;
        const Contrib cc = A.contribs[td.cbeg + i];
        const float f = float(occ[cc.occ]);
        const bool got = mbar_wait(bar + 8u * sl, ph[sl] & 1u, TIMEOUT_NS);
        ph[sl]++;
        // a skipped pair (all d = 0) left its ring slot unwritten: never multiply stale data by 0
        if (got && f != 0.f) {
          const c64* sv = reinterpret_cast<const c64*>(sm + sl * 2 * HB);
          const c64* sq = sv + G * G / 2;
#pragma unroll
          for (int e = 0; e < EPT; ++e) {
            c64 a = sv[tid + e * THREADS];
            if (cc.conj) a.im = -a.im;
            acc[e] = acc[e] + cmul(sq[tid + e * THREADS], a) * f;
          }
        }
        if (!__syncthreads_and(got)) {
          ok = false;
          break;
        }
        if (tid == 0 && i + DS < nc) {
          fence_proxy_async_smem();
          issue(i + DS);
        }
      }
      if (!ok) {
        if (tid == 0) atomicOr(A.err, 8);
        break;
      }
      c64* o = out + size_t(td.t) * ng + zoff + half * (G * G / 2) + tid;
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int q = e * THREADS;
        o[q] = td.first ? czero<float>() - acc[e] : o[q] - acc[e];
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        atomicExch(wq, seq + 1);
        atomicAdd(A.cntD + dtile, 1);
      }
      continue;
    }
    u -= nD;
    if (u < nC) {
      // ---------------- C: inverse y/x transforms of planes z0 and z0 + 32 ----------------
      const int p = pC, z0 = u;
      const PairDesc pd = A.pairs[p];
      const int rs = p % A.ring;
      const bool skip = pair_skipped(pd, occ);
      if (tid == 0) {
        const bool ok = wait_count(A.cntB + p, H, A.err, 4);
        if (ok && !skip) {
          fence_proxy_async_global();
          fence_proxy_async_smem();  // earlier items read and wrote these tiles through the generic proxy
          mbar_arrive_expect_tx(bar, TILE_BYTES);
          for (int s = 0; s < 4; ++s) tma_load_4d(base + OFF_A + s * SUB_BYTES, &tm_plane, 16 * s, 0, z0, rs, bar);
          mbar_arrive_expect_tx(bar + 8, TILE_BYTES);
          for (int s = 0; s < 4; ++s)
            tma_load_4d(base + OFF_B + s * SUB_BYTES, &tm_plane, 16 * s, 0, z0 + H, rs, bar + 8);
        }
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) break;
      bool ok = true;
      if (!skip) {
        const int kx = grp;
        c64* gs = reinterpret_cast<c64*>(sm + OFF_A) + grp * 64;
        for (int h = 0; h < 2; ++h) {
          const int z = z0 + h * H;
          const bool got = mbar_wait(bar + 8u * h, ph[h] & 1u, TIMEOUT_NS);
          ph[h]++;
          if (!__syncthreads_and(got)) {
            ok = false;
            break;
          }
          c64 v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q)
            v[q] = *reinterpret_cast<const c64*>(sm + (h ? OFF_B : OFF_A) + sw_off(kx, t + 8 * q));
          __syncthreads();
          fft64_tma(v, t, gs, gpar, tw, true);  // inverse along y: lane t holds y = t + 8k
#pragma unroll
          for (int k = 0; k < 8; ++k) P[pidx(t + 8 * k, kx)] = v[k];
          __syncthreads();
          const int y = grp;
#pragma unroll
          for (int q = 0; q < 8; ++q) v[q] = P[pidx(y, t + 8 * q)];
          fft64_tma(v, t, gs, gpar, tw, true);  // inverse along x: lane t holds x = t + 8k
          c64* o = scratch + size_t(rs) * ng + size_t(z) * G * G + y * G;
#pragma unroll
          for (int k = 0; k < 8; ++k) o[t + 8 * k] = v[k];
        }
      }
      if (!ok) {
        if (tid == 0) atomicOr(A.err, 4);
        break;
      }
      signal_add(A.cntC + A.pair_batch[p], tid);
      continue;
    }
    u -= nC;
    if (u < nB) {
      // ---------------- B: z transform, K(G)/Ng, inverse z of slabs ky0 and ky0 + 32 ----------------
      const int p = pB, ky0 = u;
      const PairDesc pd = A.pairs[p];
      const int rs = p % A.ring;
      const bool skip = pair_skipped(pd, occ);
      if (tid == 0) {
        const bool ok = wait_count(A.cntA + p, G, A.err, 2);
        if (ok && !skip) {
          fence_proxy_async_global();
          fence_proxy_async_smem();
          mbar_arrive_expect_tx(bar, TILE_BYTES);
          for (int s = 0; s < 4; ++s) tma_load_4d(base + OFF_A + s * SUB_BYTES, &tm_slab, 16 * s, ky0, 0, rs, bar);
          mbar_arrive_expect_tx(bar + 8, TILE_BYTES);
          for (int s = 0; s < 4; ++s)
            tma_load_4d(base + OFF_P + s * SUB_BYTES, &tm_slab, 16 * s, ky0 + H, 0, rs, bar + 8);
        }
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) break;
      bool ok = true;
      if (!skip) {
        const int kx = grp;
        c64* gs = reinterpret_cast<c64*>(sm + OFF_B) + grp * 64;
        for (int h = 0; h < 2; ++h) {
          const int ky = ky0 + h * H;
          const uint32_t off = h ? OFF_P : OFF_A;
          float kv[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) kv[k] = ktab[(size_t(t + 8 * k) * G + ky) * G + kx];
          const bool got = mbar_wait(bar + 8u * h, ph[h] & 1u, TIMEOUT_NS);
          ph[h]++;
          if (!__syncthreads_and(got)) {
            ok = false;
            break;
          }
          c64 v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) v[q] = *reinterpret_cast<const c64*>(sm + off + sw_off(kx, t + 8 * q));
          fft64_tma(v, t, gs, gpar, tw, false);
#pragma unroll
          for (int k = 0; k < 8; ++k) v[k] = v[k] * kv[k];
          fft64_tma(v, t, gs, gpar, tw, true);
#pragma unroll
          for (int k = 0; k < 8; ++k) *reinterpret_cast<c64*>(sm + off + sw_off(kx, t + 8 * k)) = v[k];
          fence_proxy_async_smem();
          __syncthreads();
          if (tid == 0) {
            for (int s = 0; s < 4; ++s) tma_store_4d(&tm_slab, 16 * s, ky, 0, rs, base + off + s * SUB_BYTES);
            tma_store_commit();
          }
        }
        if (tid == 0) {
          tma_store_wait_all();  // the slab stores are complete (and their smem free) before the release
          fence_proxy_async_global();
        }
      }
      if (!ok) {
        if (tid == 0) {
          tma_store_wait_all();
          atomicOr(A.err, 2);
        }
        break;
      }
      signal_add(A.cntB + p, tid);
      continue;
    }
    u -= nB;
    {
      // ---------------- A: pair product and x/y transforms of plane z ----------------
      const int p = pA, z = u;
      const PairDesc pd = A.pairs[p];
      const int rs = p % A.ring;
      const bool skip = pair_skipped(pd, occ);
      if (tid == 0) {
        bool ok = true;
        if (p >= A.ring) {  // the last user of this ring slot has been consumed by its tile's D items
          const int b = A.pair_batch[p - A.ring];
          ok = wait_count(A.cntD + b, A.batch_ndone[b], A.err, 1);
        }
        if (ok && !skip) {
          fence_proxy_async_smem();
          mbar_arrive_expect_tx(bar, 2 * TILE_BYTES);
          for (int s = 0; s < 4; ++s) {
            tma_load_4d(base + OFF_A + s * SUB_BYTES, &tm_src, 16 * s, 0, z, pd.i, bar);
            tma_load_4d(base + OFF_B + s * SUB_BYTES, &tm_tgt, 16 * s, 0, z, pd.j, bar);
          }
        }
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) break;
      if (!skip) {
        const bool got = mbar_wait(bar, ph[0] & 1u, TIMEOUT_NS);
        ph[0]++;
        if (!__syncthreads_and(got)) {
          if (tid == 0) atomicOr(A.err, 1);
          break;
        }
        const int x = grp;
        c64 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint32_t o = sw_off(x, t + 8 * q);
          v[q] = cmulc(*reinterpret_cast<const c64*>(sm + OFF_A + o), *reinterpret_cast<const c64*>(sm + OFF_B + o));
        }
        __syncthreads();  // tiles consumed: tile A becomes the group-transpose area
        c64* gs = reinterpret_cast<c64*>(sm + OFF_A) + grp * 64;
        fft64_tma(v, t, gs, gpar, tw, false);  // along y
#pragma unroll
        for (int k = 0; k < 8; ++k) P[pidx(t + 8 * k, x)] = v[k];
        __syncthreads();
        const int ky = grp;
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = P[pidx(ky, t + 8 * q)];
        fft64_tma(v, t, gs, gpar, tw, false);  // along x
        c64* o = scratch + size_t(rs) * ng + size_t(z) * G * G + ky * G;
#pragma unroll
        for (int k = 0; k < 8; ++k) o[t + 8 * k] = v[k];
      }
      signal_add(A.cntA + p, tid);
    }
  }
}

// Host-side tables of one schedule: the pair/tile/target arrays and the wave table, on the device.
struct PersistPlan {
  int P = 0, nbatch = 0, ntgt = 0, nwaves = 0, total = 0, ring = 0, lagB = 0, lagC = 0, lagD = 0, M = 0;
  long long pairs_total = 0;
  void* dev = nullptr;  // one allocation holding every table
  size_t off_pairs, off_pair_batch, off_b_pair0, off_b_ndone, off_b_npairs, off_b_tgt0, off_tgts, off_contribs,
      off_tgt_seq, off_waves;
  ~PersistPlan() { cudaFree(dev); }
};

std::shared_ptr<PersistPlan> make_plan(int N, int M, bool sym, int b, int ring, int lag) {
  PairPlan pp = plan_pairs(N, M, sym, b);
  auto pl = std::make_shared<PersistPlan>();
  pl->P = int(pp.pairs.size());
  pl->nbatch = int(pp.pair_off.size()) - 1;
  pl->ntgt = int(pp.tgts.size());
  pl->M = sym ? N : M;
  pl->lagB = lag;
  pl->lagC = 2 * lag;
  pl->lagD = 3 * lag;
  int bmax = 0;
  for (int k = 0; k < pl->nbatch; ++k) bmax = std::max(bmax, pp.pair_off[k + 1] - pp.pair_off[k]);
  // A(p) waits for the D items of the tile of pair p - R, which the order places before A(p) only if
  // R >= (pairs of a tile) + LD
  pl->ring = std::max(ring, bmax + pl->lagD + 1);
  pl->pairs_total = pl->P;
  std::vector<int> pair_batch(pl->P), b_pair0(pl->nbatch), b_ndone(pl->nbatch), b_npairs(pl->nbatch),
      b_tgt0(pl->nbatch), last_of(pl->nbatch);
  for (int k = 0; k < pl->nbatch; ++k) {
    b_pair0[k] = pp.pair_off[k];
    b_npairs[k] = pp.pair_off[k + 1] - pp.pair_off[k];
    b_tgt0[k] = pp.tgt_off[k];
    b_ndone[k] = (pp.tgt_off[k + 1] - pp.tgt_off[k]) * ZH;
    last_of[k] = pp.pair_off[k + 1] - 1;
    for (int p = pp.pair_off[k]; p < pp.pair_off[k + 1]; ++p) pair_batch[p] = k;
  }
  std::vector<int> tgt_seq(pl->ntgt);
  std::vector<int> seen(pl->M, 0);
  for (int k = 0; k < pl->ntgt; ++k) tgt_seq[k] = seen[pp.tgts[k].t]++;
  // waves: D items of the tile whose last pair is w - LD, then C(w - LC), B(w - LB), A(w)
  std::vector<int> dtile_of_wave(pl->P + pl->lagD, -1);
  for (int k = 0; k < pl->nbatch; ++k) dtile_of_wave[last_of[k] + pl->lagD] = k;
  pl->nwaves = pl->P + pl->lagD;
  std::vector<int2> waves(pl->nwaves + 1);
  long long off = 0;
  for (int w = 0; w < pl->nwaves; ++w) {
    waves[w] = int2{int(off), dtile_of_wave[w]};
    const int d = dtile_of_wave[w];
    if (d >= 0) off += b_ndone[d];
    const int pc = w - pl->lagC, pb = w - pl->lagB;
    if (pc >= 0 && pc < pl->P) off += G / 2;
    if (pb >= 0 && pb < pl->P) off += G / 2;
    if (w < pl->P) off += G;
    if (off > (1ll << 30)) fail(PT_INVALID_ARG, "exchange schedule too large for the persistent 64^3 kernel");
  }
  waves[pl->nwaves] = int2{int(off), -1};
  pl->total = int(off);
  // one device allocation, each table 256-byte aligned
  size_t cur = 0;
  auto place = [&](size_t bytes) {
    const size_t o = cur;
    cur += (bytes + 255) & ~size_t(255);
    return o;
  };
  pl->off_pairs = place(pp.pairs.size() * sizeof(PairDesc));
  pl->off_pair_batch = place(pair_batch.size() * sizeof(int));
  pl->off_b_pair0 = place(b_pair0.size() * sizeof(int));
  pl->off_b_ndone = place(b_ndone.size() * sizeof(int));
  pl->off_b_npairs = place(b_npairs.size() * sizeof(int));
  pl->off_b_tgt0 = place(b_tgt0.size() * sizeof(int));
  pl->off_tgts = place(pp.tgts.size() * sizeof(TargetDesc));
  pl->off_contribs = place(pp.contribs.size() * sizeof(Contrib));
  pl->off_tgt_seq = place(tgt_seq.size() * sizeof(int));
  pl->off_waves = place(waves.size() * sizeof(int2));
  std::vector<unsigned char> h(cur, 0);
  auto put = [&](size_t o, const void* p, size_t bytes) { std::memcpy(h.data() + o, p, bytes); };
  put(pl->off_pairs, pp.pairs.data(), pp.pairs.size() * sizeof(PairDesc));
  put(pl->off_pair_batch, pair_batch.data(), pair_batch.size() * sizeof(int));
  put(pl->off_b_pair0, b_pair0.data(), b_pair0.size() * sizeof(int));
  put(pl->off_b_ndone, b_ndone.data(), b_ndone.size() * sizeof(int));
  put(pl->off_b_npairs, b_npairs.data(), b_npairs.size() * sizeof(int));
  put(pl->off_b_tgt0, b_tgt0.data(), b_tgt0.size() * sizeof(int));
  put(pl->off_tgts, pp.tgts.data(), pp.tgts.size() * sizeof(TargetDesc));
  put(pl->off_contribs, pp.contribs.data(), pp.contribs.size() * sizeof(Contrib));
  put(pl->off_tgt_seq, tgt_seq.data(), tgt_seq.size() * sizeof(int));
  put(pl->off_waves, waves.data(), waves.size() * sizeof(int2));
  PT_CUDA_CHECK(cudaMalloc(&pl->dev, cur));
  PT_CUDA_CHECK(cudaMemcpy(pl->dev, h.data(), cur, cudaMemcpyHostToDevice));
  return pl;
}

}  // namespace

long long exchange64_persist(pt_ctx* ctx, const c64* src, const double* occ, int N, const c64* tgt, int M, bool sym,
                             c64* out, const float* ktab, const c64* tw, cudaStream_t st) {
  constexpr size_t ng = size_t(G) * G * G;
  const int b = std::max(1, std::min(ctx->x64p_tile, std::max(N, M)));
  char key[128];
  snprintf(key, sizeof(key), "x64p:%d:%d:%d:%d:%d:%d", N, M, int(sym), b, ctx->x64p_ring, ctx->x64p_lag);
  std::shared_ptr<PersistPlan> pl;
  auto it = ctx->caches.find(key);
  if (it == ctx->caches.end()) {
    pl = make_plan(N, M, sym, b, ctx->x64p_ring, ctx->x64p_lag);
    ctx->caches[key] = pl;
  } else {
    pl = std::static_pointer_cast<PersistPlan>(it->second);
  }
  const int ring = std::min(pl->ring, std::max(1, pl->P));
  c64* scratch = static_cast<c64*>(ctx->get(ctx->tagged("exchange64p_scratch"), size_t(pl->ring) * ng * sizeof(c64)));
  const size_t ncnt = 1 + 2 * size_t(pl->P) + 2 * size_t(pl->nbatch) + size_t(pl->M) * ZH;
  int* cnt = static_cast<int*>(ctx->get(ctx->tagged("exchange64p_counters"), ncnt * sizeof(int)));
  int* err = static_cast<int*>(ctx->get("exchange_err", sizeof(int)));
  PT_CUDA_CHECK(cudaMemsetAsync(cnt, 0, ncnt * sizeof(int), st));
  if (!ctx->defer_checks) PT_CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st));
  static DeviceOnce once;
  once([] {
    PT_CUDA_CHECK(
        cudaFuncSetAttribute(k_exchange64_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMEM_BYTES)));
  });
  int per_sm = 0;
  PT_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_exchange64_persist, THREADS, SMEM_BYTES));
  if (per_sm < 1) fail(PT_CUDA, "persistent 64^3 exchange kernel cannot be resident");
  const int grid = std::min(per_sm * ctx->num_sms, std::max(1, pl->total));
  const uint64_t strides[3] = {G * 8, G * G * 8, ng * 8};
  const uint32_t plane_box[4] = {16, 64, 1, 1};
  const uint32_t slab_box[4] = {16, 1, 64, 1};
  CUtensorMap tm_src, tm_tgt, tm_plane, tm_slab;
  const uint64_t dsrc[4] = {G, G, G, uint64_t(N)};
  const uint64_t dtgt[4] = {G, G, G, uint64_t(M)};
  const uint64_t dscr[4] = {G, G, G, uint64_t(pl->ring)};
  encode_tmap_4d_u64(&tm_src, src, dsrc, strides, plane_box, CU_TENSOR_MAP_SWIZZLE_128B);
  encode_tmap_4d_u64(&tm_tgt, tgt, dtgt, strides, plane_box, CU_TENSOR_MAP_SWIZZLE_128B);
  encode_tmap_4d_u64(&tm_plane, scratch, dscr, strides, plane_box, CU_TENSOR_MAP_SWIZZLE_128B);
  encode_tmap_4d_u64(&tm_slab, scratch, dscr, strides, slab_box, CU_TENSOR_MAP_SWIZZLE_128B);
  auto* d = static_cast<unsigned char*>(pl->dev);
  PArgs a;
  a.pairs = reinterpret_cast<const PairDesc*>(d + pl->off_pairs);
  a.pair_batch = reinterpret_cast<const int*>(d + pl->off_pair_batch);
  a.batch_pair0 = reinterpret_cast<const int*>(d + pl->off_b_pair0);
  a.batch_ndone = reinterpret_cast<const int*>(d + pl->off_b_ndone);
  a.batch_npairs = reinterpret_cast<const int*>(d + pl->off_b_npairs);
  a.batch_tgt0 = reinterpret_cast<const int*>(d + pl->off_b_tgt0);
  a.tgts = reinterpret_cast<const TargetDesc*>(d + pl->off_tgts);
  a.contribs = reinterpret_cast<const Contrib*>(d + pl->off_contribs);
  a.tgt_seq = reinterpret_cast<const int*>(d + pl->off_tgt_seq);
  a.waves = reinterpret_cast<const int2*>(d + pl->off_waves);
  a.nwaves = pl->nwaves;
  a.total = pl->total;
  a.npairs = pl->P;
  a.ring = ring;
  a.lagB = pl->lagB;
  a.lagC = pl->lagC;
  a.lagD = pl->lagD;
  a.next = cnt;
  a.cntA = cnt + 1;
  a.cntB = a.cntA + pl->P;
  a.cntC = a.cntB + pl->P;
  a.cntD = a.cntC + pl->nbatch;
  a.wseq = a.cntD + pl->nbatch;
  a.err = err;
  // every CTA must be resident at once (they wait on one another): a cooperative launch
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  PT_CUDA_CHECK(cudaLaunchKernelEx(&cfg, k_exchange64_persist, tm_src, tm_tgt, tm_plane, tm_slab, a, src, occ, ktab,
                                   tw, scratch, out));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return pl->pairs_total;
}

}  // namespace pt
