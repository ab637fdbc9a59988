// FP32 pair-FFT exchange for 64^3 grids with TMA staging (Sec. IV-A1, Eq. vxdiag).
//
// Same four pipelined roles as the register/shared-memory kernel (A: pair product + x/y
// transforms of a plane, B: z transform + K + inverse z of a slab, C: inverse y/x transforms
// of a plane, D: occupation-weighted accumulate into the target plane), but every strided
// access to a pair field goes through the tensor-memory accelerator:
//   * plane and slab tiles are fetched with cp.async.bulk.tensor into 128B-swizzled shared
//     tiles (four 16-wide sub-tiles of 128-byte rows); the 16-byte chunk c of row r sits at
//     chunk c ^ (r mod 8), so the column reads of the line transforms (8 lanes on 8 rows of
//     one column, 4 adjacent columns per warp) hit every bank exactly twice per warp;
//   * the z-slab results of pass B go back to the scratch field with TMA stores.
// Row-contiguous traffic (pass A/C results, pass D) stays on plain coalesced loads/stores.
// Each CTA waits on its mbarrier with a %globaltimer deadline; on expiry it sets an error
// word that the host checks after the call, and returns.
#include <algorithm>
#include <cstring>

#include "exchange64_common.cuh"
#include "exchange_sched.h"
#include "fft.cuh"
#include "internal.h"
#include "tma.cuh"

namespace pt {

namespace {

using namespace x64;
constexpr int MAXB = kExchange64MaxTile;         // tile side of the pair schedule on this path
constexpr int MAXP = MAXB * MAXB, MAXT = 2 * MAXB, MAXC = 2 * MAXP;

// The batch descriptors travel in the kernel parameters (constant bank): no dependent global
// load stands between a CTA's start and its first TMA request.
struct Launch {
  int nA, nB, nC, nD;
  int slotA, slotB, slotC, slotD;
  int max_pairs, d_cbeg;
  PairDesc pa[MAXP], pb[MAXP], pc[MAXP];
  TargetDesc td[MAXT];
  Contrib cd[MAXC];
};

__constant__ c64 c_tw64[G];

// FUSED = false: roles A, B, C, D over four slots.  FUSED = true: roles CD, A, B over three slots,
// where a CD CTA owns one target plane and runs C's inverse y/x transforms of each contributing
// pair's plane itself before accumulating (see the CD role below).
template <bool FUSED>
__global__ void __launch_bounds__(THREADS, 2)
    k_exchange64_tma(const __grid_constant__ CUtensorMap tm_src, const __grid_constant__ CUtensorMap tm_tgt,
                     const __grid_constant__ CUtensorMap tm_plane, const __grid_constant__ CUtensorMap tm_slab,
                     const __grid_constant__ Launch L, const c64* __restrict__ src, const double* __restrict__ occ,
                     const float* __restrict__ ktab, c64* __restrict__ scratch, c64* __restrict__ out,
                     int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  c64* P = reinterpret_cast<c64*>(sm + OFF_P);
  c64* tw = reinterpret_cast<c64*>(sm + OFF_TW);
  const uint32_t bar = base + OFF_BAR;
  const int tid = threadIdx.x, grp = tid >> 3, t = tid & 7;
  const int gpar = (grp & 1) << 3;
  constexpr size_t ng = size_t(G) * G * G;
  if (tid < G) tw[tid] = c_tw64[tid];
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 8, 1);   // second tile of the two-item roles B and C
    mbar_init(bar + 16, 1);  // third contribution slot of role D
    fence_mbar_init();
  }
  __syncthreads();
  int bid = blockIdx.x;

  if constexpr (FUSED) {
    if (bid < L.nD) {
      // ---------------- pass CD (one target plane per CTA) ----------------
      // For each contribution (pair slot, partner, occupation, conjugation) of target td at plane z:
      // the pair's plane z after the z transforms arrives by TMA (double-buffered, one contribution
      // ahead), the inverse y and x transforms run here (lane t of group y ends with v[y][t + 8k]),
      // and d * partner * v accumulates in registers.  v_ij never leaves the SM: the C -> D round
      // trip of the four-role pipeline (write and read of every pair field) is gone, at the price of
      // transforming a symmetric pair's plane once for each of its two targets.  Plane-major order:
      // all targets at one z run together, so both targets of a pair read its plane from L2.
      const int nt = L.nD / G;
      const int z = bid / nt;
      const TargetDesc td = L.td[bid % nt];
      __shared__ int s_list[2 * MAXB];
      __shared__ int s_n;
      if (tid == 0) {  // contributions with a nonzero occupation (a skipped pair's slot is stale)
        int n = 0;
        for (int i = td.cbeg; i < td.cend; ++i)
          if (occ[L.cd[i - L.d_cbeg].occ] != 0.0) s_list[n++] = i - L.d_cbeg;
        s_n = n;
      }
      __syncthreads();
      const int n = s_n;
      auto issue = [&](int c) {  // one thread
        const Contrib cc = L.cd[s_list[c]];
        const int orb = L.slotD * L.max_pairs + cc.slot;
        const uint32_t b = uint32_t(c & 1);
        fence_proxy_async_smem();  // the buffer was last read and written through the generic proxy
        mbar_arrive_expect_tx(bar + 8u * b, TILE_BYTES);
        tma_load_5d(base + b * TILE_BYTES, &tm_plane, 0, 0, z, orb, 0, bar + 8u * b);
      };
      if (tid == 0) {
        if (n > 0) issue(0);
        if (n > 1) issue(1);
      }
      c64 acc[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = czero<float>();
      const int y = grp, kx = grp;
      for (int c = 0; c < n; ++c) {
        const uint32_t b = uint32_t(c & 1);
        const bool ok = mbar_wait(bar + 8u * b, uint32_t(c >> 1) & 1u, TIMEOUT_NS);
        if (!__syncthreads_and(ok)) {
          if (tid == 0) atomicOr(err, 16);
          return;
        }
        c64 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = *reinterpret_cast<const c64*>(sm + b * TILE_BYTES + sw_off(kx, t + 8 * q));
        __syncthreads();  // the buffer is consumed: it becomes the group-transpose area
        c64* gs = reinterpret_cast<c64*>(sm + b * TILE_BYTES) + grp * 64;
        fft64_tma(v, t, gs, gpar, tw, true);  // inverse along y: lane t holds y = t + 8k
#pragma unroll
        for (int k = 0; k < 8; ++k) P[pidx(t + 8 * k, kx)] = v[k];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = P[pidx(y, t + 8 * q)];
        fft64_tma(v, t, gs, gpar, tw, true);  // inverse along x: lane t holds x = t + 8k
        const Contrib cc = L.cd[s_list[c]];
        const float f = float(occ[cc.occ]);
        const c64* pp = src + size_t(cc.partner) * ng + size_t(z) * G * G + y * G;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          c64 a = v[k];
          if (cc.conj) a.im = -a.im;
          acc[k] = acc[k] + cmul(pp[t + 8 * k], a) * f;
        }
        __syncthreads();  // the buffer (transpose area) and P are free for the next contribution
        if (tid == 0 && c + 2 < n) issue(c + 2);
      }
      c64* o = out + size_t(td.t) * ng + size_t(z) * G * G + y * G;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int e = t + 8 * k;
        o[e] = td.first ? czero<float>() - acc[k] : o[e] - acc[k];
      }
      return;
    }
    bid -= L.nD;
  }

  if (bid < L.nA) {
    // ---------------- pass A ----------------
    // plane-major order: the CTAs of all pairs of the batch at one z run together, so the source
    // planes shared by the pairs of a tile row or column are read from L2
    const int np = L.nA / G;
    const int z = bid / np, p = bid % np;
    const PairDesc pd = L.pa[p];
    if (tid == 0) {
      mbar_arrive_expect_tx(bar, 2 * TILE_BYTES);
      tma_load_5d(base + OFF_A, &tm_src, 0, 0, z, pd.i, 0, bar);
      tma_load_5d(base + OFF_B, &tm_tgt, 0, 0, z, pd.j, 0, bar);
    }
    const bool skip = pair_skipped(pd, occ);
    if (!mbar_wait(bar, 0, TIMEOUT_NS)) {
      atomicOr(err, 1);
      return;
    }
    if (skip) return;
    const int x = grp;
    c64 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t o = sw_off(x, t + 8 * q);
      v[q] = cmulc(*reinterpret_cast<const c64*>(sm + OFF_A + o), *reinterpret_cast<const c64*>(sm + OFF_B + o));
    }
    __syncthreads();  // tiles consumed: tile A becomes the group-transpose area
    c64* gs = reinterpret_cast<c64*>(sm + OFF_A) + grp * 64;
    fft64_tma(v, t, gs, gpar, tw, false);  // along y: lane t holds ky = t + 8k
#pragma unroll
    for (int k = 0; k < 8; ++k) P[pidx(t + 8 * k, x)] = v[k];
    __syncthreads();
    const int ky = grp;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = P[pidx(ky, t + 8 * q)];
    fft64_tma(v, t, gs, gpar, tw, false);  // along x: lane t holds kx = t + 8k
    c64* o = scratch + (size_t(L.slotA) * L.max_pairs + p) * ng + size_t(z) * G * G + ky * G;
#pragma unroll
    for (int k = 0; k < 8; ++k) o[t + 8 * k] = v[k];
    return;
  }
  bid -= L.nA;
  if (bid < L.nB) {
    // ---------------- pass B (two slabs per CTA: ky and ky + G/2) ----------------
    // Both slab loads are issued at once (the second into the plane-transpose area, which this
    // role does not use), so the second slab's load latency hides behind the first's transforms.
    constexpr int H = G / 2;
    const int ky0 = bid % H, p = bid / H;
    const int kx = grp;
    const PairDesc pd = L.pb[p];
    const int orb = L.slotB * L.max_pairs + p;
    if (tid == 0) {
      mbar_arrive_expect_tx(bar, TILE_BYTES);
      tma_load_5d(base + OFF_A, &tm_slab, 0, ky0, 0, orb, 0, bar);
      mbar_arrive_expect_tx(bar + 8, TILE_BYTES);
      tma_load_5d(base + OFF_P, &tm_slab, 0, ky0 + H, 0, orb, 0, bar + 8);
    }
    const bool skip = pair_skipped(pd, occ);
    c64* gs = reinterpret_cast<c64*>(sm + OFF_B) + grp * 64;
    for (int h = 0; h < 2; ++h) {
      const int ky = ky0 + h * H;
      const uint32_t off = h ? OFF_P : OFF_A;
      float kv[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) kv[k] = ktab[(size_t(t + 8 * k) * G + ky) * G + kx];
      if (!mbar_wait(bar + 8u * h, 0, TIMEOUT_NS)) {
        atomicOr(err, 2);
        return;
      }
      if (skip) continue;  // uniform over the CTA; both loads still land before it exits
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
        tma_store_5d(&tm_slab, 0, ky, 0, orb, 0, base + off);
        tma_store_commit();
      }
    }
    if (tid == 0 && !skip) tma_store_wait_all();
    return;
  }
  bid -= L.nB;
  if constexpr (FUSED) return;
  if (bid < L.nC) {
    // ---------------- pass C (two planes per CTA: z and z + G/2) ----------------
    // The second plane loads into the B tile, unused by this role, while the first is transformed.
    constexpr int H = G / 2;
    const int z0 = bid % H, p = bid / H;
    const PairDesc pd = L.pc[p];
    const int orb = L.slotC * L.max_pairs + p;
    if (tid == 0) {
      mbar_arrive_expect_tx(bar, TILE_BYTES);
      tma_load_5d(base + OFF_A, &tm_plane, 0, 0, z0, orb, 0, bar);
      mbar_arrive_expect_tx(bar + 8, TILE_BYTES);
      tma_load_5d(base + OFF_B, &tm_plane, 0, 0, z0 + H, orb, 0, bar + 8);
    }
    const bool skip = pair_skipped(pd, occ);
    const int kx = grp;
    c64* gs = reinterpret_cast<c64*>(sm + OFF_A) + grp * 64;
    for (int h = 0; h < 2; ++h) {
      const int z = z0 + h * H;
      if (!mbar_wait(bar + 8u * h, 0, TIMEOUT_NS)) {
        atomicOr(err, 4);
        return;
      }
      if (skip) continue;  // uniform over the CTA; both loads still land before it exits
      c64 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        v[q] = *reinterpret_cast<const c64*>(sm + (h ? OFF_B : OFF_A) + sw_off(kx, t + 8 * q));
      // first plane: tile A consumed before it becomes the group-transpose area; second plane:
      // every warp is done with the first plane's transpose areas
      __syncthreads();
      fft64_tma(v, t, gs, gpar, tw, true);  // inverse along y: lane t holds y = t + 8k
#pragma unroll
      for (int k = 0; k < 8; ++k) P[pidx(t + 8 * k, kx)] = v[k];
      __syncthreads();
      const int y = grp;
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = P[pidx(y, t + 8 * q)];
      fft64_tma(v, t, gs, gpar, tw, true);  // inverse along x: lane t holds x = t + 8k
      c64* o = scratch + size_t(orb) * ng + size_t(z) * G * G + y * G;
#pragma unroll
      for (int k = 0; k < 8; ++k) o[t + 8 * k] = v[k];
    }
    return;
  }
  bid -= L.nC;
  {
    // ---------------- pass D (half a plane per CTA) ----------------
    // plane-major order: all targets of the batch at one z run together, so the two targets of a
    // symmetric pair read its v_ij plane close in time (the second read hits L2), as do the
    // partner planes shared by a tile row.  The v_ij and partner half-planes (16 KB each, one
    // contiguous range apiece) stream through a ring of DS shared-memory slots by bulk copies,
    // DS contributions ahead of the arithmetic, so the loads overlap without holding registers.
    const int nt = L.nD / (2 * G);
    const int z = (bid >> 1) / nt, half = bid & 1;
    const TargetDesc td = L.td[(bid >> 1) % nt];
    constexpr int EPT = G * G / (2 * THREADS);
    constexpr uint32_t HB = G * G / 2 * sizeof(c64);  // bytes of a half plane
    constexpr int DS = 3;                             // 3 x 32 KB below the twiddle table
    const int e0 = half * (G * G / 2) + tid;
    const size_t zoff = size_t(z) * G * G;
    const size_t hoff = zoff + size_t(half) * (G * G / 2);
    const int nc = td.cend - td.cbeg;
    auto issue = [&](int i) {  // one thread
      const Contrib cc = L.cd[td.cbeg + i - L.d_cbeg];
      const int sl = i % DS;
      const uint32_t dst = base + uint32_t(sl) * 2u * HB;
      fence_proxy_async_smem();  // the slot's previous contents were read through the generic proxy
      mbar_arrive_expect_tx(bar + 8u * sl, 2u * HB);
      bulk_load(dst, scratch + (size_t(L.slotD) * L.max_pairs + cc.slot) * ng + hoff, HB, bar + 8u * sl);
      bulk_load(dst + HB, src + size_t(cc.partner) * ng + hoff, HB, bar + 8u * sl);
    };
    if (tid == 0)
      for (int i = 0; i < min(DS, nc); ++i) issue(i);
    c64 acc[EPT];
#pragma unroll
    for (int u = 0; u < EPT; ++u) acc[u] = czero<float>();
    for (int i = 0; i < nc; ++i) {
      const int sl = i % DS;
      const Contrib cc = L.cd[td.cbeg + i - L.d_cbeg];
      const float f = float(occ[cc.occ]);
      const bool ok = mbar_wait(bar + 8u * sl, (i / DS) & 1, TIMEOUT_NS);
      // a skipped pair (d = 0) left its scratch slot unwritten: never multiply stale data by 0
      if (ok && f != 0.f) {
        const c64* sv = reinterpret_cast<const c64*>(sm + sl * 2 * HB);
        const c64* sq = sv + G * G / 2;
#pragma unroll
        for (int u = 0; u < EPT; ++u) {
          c64 a = sv[tid + u * THREADS];
          if (cc.conj) a.im = -a.im;
          acc[u] = acc[u] + cmul(sq[tid + u * THREADS], a) * f;
        }
      }
      // every thread is done with slot sl before it is refilled; an expired wait ends the CTA
      // uniformly
      if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicOr(err, 8);
        return;
      }
      if (tid == 0 && i + DS < nc) issue(i + DS);
    }
    c64* o = out + size_t(td.t) * ng + zoff + e0;
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int e = u * THREADS;
      o[e] = td.first ? czero<float>() - acc[u] : o[e] - acc[u];
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    PT_CUDA_CHECK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) fail(PT_CUDA, "cuTensorMapEncodeTiled entry point not found");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

static void encode_tmap_4d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, const uint64_t dims[4],
                          const uint64_t strides_bytes[3], const uint32_t box[4], CUtensorMapSwizzle swizzle) {
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  cuuint64_t d[4] = {dims[0], dims[1], dims[2], dims[3]};
  cuuint64_t s[3] = {strides_bytes[0], strides_bytes[1], strides_bytes[2]};
  cuuint32_t b[4] = {box[0], box[1], box[2], box[3]};
  CUresult r = encode_fn()(map, dt, 4, const_cast<void*>(base), d, s, b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(PT_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(int(r)) + ")");
}

void encode_tmap_4d_f32(CUtensorMap* map, const void* base, const uint64_t dims[4], const uint64_t strides_bytes[3],
                        const uint32_t box[4], CUtensorMapSwizzle swizzle) {
  encode_tmap_4d(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, base, dims, strides_bytes, box, swizzle);
}

void encode_tmap_4d_bf16(CUtensorMap* map, const void* base, const uint64_t dims[4], const uint64_t strides_bytes[3],
                         const uint32_t box[4], CUtensorMapSwizzle swizzle) {
  encode_tmap_4d(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, dims, strides_bytes, box, swizzle);
}

void encode_tmap_5d_u64(CUtensorMap* map, const void* base, const uint64_t dims[5], const uint64_t strides_bytes[4],
                        const uint32_t box[5], CUtensorMapSwizzle swizzle) {
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  cuuint64_t d[5] = {dims[0], dims[1], dims[2], dims[3], dims[4]};
  cuuint64_t s[4] = {strides_bytes[0], strides_bytes[1], strides_bytes[2], strides_bytes[3]};
  cuuint32_t b[5] = {box[0], box[1], box[2], box[3], box[4]};
  CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<void*>(base), d, s, b, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(PT_CUDA, "cuTensorMapEncodeTiled (5-D) failed (" + std::to_string(int(r)) + ")");
}

void encode_tmap_4d_u64(CUtensorMap* map, const void* base, const uint64_t dims[4], const uint64_t strides_bytes[3],
                        const uint32_t box[4], CUtensorMapSwizzle swizzle) {
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  cuuint64_t d[4] = {dims[0], dims[1], dims[2], dims[3]};
  cuuint64_t s[3] = {strides_bytes[0], strides_bytes[1], strides_bytes[2]};
  cuuint32_t b[4] = {box[0], box[1], box[2], box[3]};
  CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<void*>(base), d, s, b, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(PT_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(int(r)) + ")");
}

void exchange64_tma(pt_ctx* ctx, const ScheduleImpl& sch, const c64* src, const double* occ, const c64* tgt, int M,
                    c64* out, const float* ktab, const c64* tw, cudaStream_t st, bool fused) {
  if (sch.B > MAXB) fail(PT_INVALID_ARG, "64^3 exchange schedule tile exceeds the parameter-block capacity");
  constexpr size_t ng = size_t(G) * G * G;
  const int maxp = sch.max_pairs;
  const int ns = fused ? 3 : 4;  // scratch slots: one per role that holds pair fields
  c64* scratch = static_cast<c64*>(ctx->get(ctx->tagged("exchange64_scratch"), size_t(ns) * maxp * ng * sizeof(c64)));
  int* err = static_cast<int*>(ctx->get("exchange_err", sizeof(int)));
  if (!ctx->defer_checks) PT_CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st));  // else zeroed once per batch
  static DeviceOnce once;  // kernel attribute and the constant twiddle table are per device
  once([] {
    PT_CUDA_CHECK(
        cudaFuncSetAttribute(k_exchange64_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    PT_CUDA_CHECK(
        cudaFuncSetAttribute(k_exchange64_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    c64 h[G];
    for (int i = 0; i < G; ++i) {
      const double ang = -2.0 * M_PI * double(i) / double(G);
      h[i] = c64{float(std::cos(ang)), float(std::sin(ang))};
    }
    PT_CUDA_CHECK(cudaMemcpyToSymbol(c_tw64, h, sizeof(h)));
  });
  (void)tw;
  // 5-D views (x mod 16, y, z, field, x / 16) of the [field][z][y][x] complex64 arrays: one copy
  // moves a whole 64 x 64 plane or slab as four 16-column sub-tiles of 128-byte rows (the x / 16
  // dimension, stride 128 B, outermost in the box), the shared-memory layout the line transforms read
  const uint64_t strides[4] = {G * 8, G * G * 8, ng * 8, 16 * 8};
  const uint32_t plane_box[5] = {16, 64, 1, 1, 4};
  const uint32_t slab_box[5] = {16, 1, 64, 1, 4};
  CUtensorMap tm_src, tm_tgt, tm_plane, tm_slab;
  const uint64_t dsrc[5] = {16, G, G, uint64_t(sch.N), 4};
  const uint64_t dtgt[5] = {16, G, G, uint64_t(M), 4};
  const uint64_t dscr[5] = {16, G, G, uint64_t(ns) * maxp, 4};
  encode_tmap_5d_u64(&tm_src, src, dsrc, strides, plane_box, CU_TENSOR_MAP_SWIZZLE_128B);
  encode_tmap_5d_u64(&tm_tgt, tgt, dtgt, strides, plane_box, CU_TENSOR_MAP_SWIZZLE_128B);
  encode_tmap_5d_u64(&tm_plane, scratch, dscr, strides, plane_box, CU_TENSOR_MAP_SWIZZLE_128B);
  encode_tmap_5d_u64(&tm_slab, scratch, dscr, strides, slab_box, CU_TENSOR_MAP_SWIZZLE_128B);
  const int nb = int(sch.pair_off.size()) - 1;
  auto copy_pairs = [&](PairDesc* dst, int batch) {
    const int p0 = sch.pair_off[batch], np = sch.pair_off[batch + 1] - p0;
    std::copy(sch.h_pairs.begin() + p0, sch.h_pairs.begin() + p0 + np, dst);
    return np;
  };
  Launch L;
  // launch k: A of batch k, B of batch k - 1, then C of k - 2 and D of k - 3 (four slots), or the
  // fused CD of batch k - 2 (three slots); the roles of one launch always use distinct slots
  for (int k = 0; k < nb + ns - 1; ++k) {
    std::memset(&L, 0, sizeof(L));
    L.max_pairs = maxp;
    if (k < nb) {
      L.nA = G * copy_pairs(L.pa, k);
      L.slotA = k % ns;
    }
    const int b = k - 1, c = k - 2, d = fused ? k - 2 : k - 3;
    if (b >= 0 && b < nb) {
      L.nB = (G / 2) * copy_pairs(L.pb, b);
      L.slotB = b % ns;
    }
    if (!fused && c >= 0 && c < nb) {
      L.nC = (G / 2) * copy_pairs(L.pc, c);
      L.slotC = c % ns;
    }
    if (d >= 0 && d < nb) {
      const int t0 = sch.tgt_off[d], nt = sch.tgt_off[d + 1] - t0;
      std::copy(sch.h_tgts.begin() + t0, sch.h_tgts.begin() + t0 + nt, L.td);
      L.d_cbeg = sch.h_tgts[t0].cbeg;
      const int cend = sch.h_tgts[t0 + nt - 1].cend;
      if (cend - L.d_cbeg > MAXC || nt > MAXT) fail(PT_INVALID_ARG, "exchange batch exceeds the parameter block");
      for (int q = 0; q < nt; ++q)
        if (sch.h_tgts[t0 + q].cend - sch.h_tgts[t0 + q].cbeg > 2 * MAXB)
          fail(PT_INVALID_ARG, "exchange batch: a target has more contributions than a tile allows");
      std::copy(sch.h_contribs.begin() + L.d_cbeg, sch.h_contribs.begin() + cend, L.cd);
      L.nD = (fused ? G : 2 * G) * nt;
      L.slotD = d % ns;
    }
    const int grid = L.nA + L.nB + L.nC + L.nD;
    if (grid == 0) continue;
    if (fused)
      PT_LAUNCH(k_exchange64_tma<true>, grid, THREADS, SMEM_BYTES, st, tm_src, tm_tgt, tm_plane, tm_slab, L, src, occ,
                ktab, scratch, out, err);
    else
      PT_LAUNCH(k_exchange64_tma<false>, grid, THREADS, SMEM_BYTES, st, tm_src, tm_tgt, tm_plane, tm_slab, L, src,
                occ, ktab, scratch, out, err);
  }
}

}  // namespace pt
