// Gram contractions C = scale * A^H B on the 5th-generation tensor cores (tcgen05, TF32 inputs).
//
// A (N1 orbitals) and B (N2 orbitals) are complex64, orbital-major, so each orbital is a row of
// K' = 2 Ng interleaved floats and both operands are K-major.  For a tile of 64 A-orbitals and
// 64 B-orbitals the MMA operand "A" has 128 rows: rows 0..63 are the A orbitals, rows 64..127 the
// same orbitals multiplied by i, i.e. (-a_im, a_re) pairs.  With B's rows as they are,
//     D[r][c]      = sum_k A_int[r][k] B_int[c][k] = Re (A^H B)[r][c]
//     D[64 + r][c] = sum_k (iA)_int[r][k] B_int[c][k] = Im (A^H B)[r][c]
// so one real M=128, N=64 GEMM yields the complex tile in TMEM.
//
// Warp roles (192 threads): warp 0 issues TMA loads of the A (64 x 32 floats) and B (64 x 32
// floats) tiles straight into the 128B-swizzled MMA operand buffers of a stage; warp 1 allocates
// TMEM and one lane issues tcgen05.mma; warps 2..5 (the converter warpgroup) write the i*A rows
// of the operand (and, in 3xTF32 mode, the FP32 remainders "lo" = x - tf32(x) of A, i*A and B,
// so that hi*hi + hi*lo + lo*hi recovers FP32 accuracy; the raw FP32 values serve as "hi" since
// the tensor core reads only their TF32 bits), then read the TMEM accumulators out every
// `period` stages and add them into Kahan-compensated FP32 registers.  The tensor core's FP32
// accumulation error grows with the number of products summed in TMEM, so a short period keeps
// the result at FP32 accuracy.  The two TMEM accumulators alternate so the tensor cores keep
// running during a readout.  The K range of a tile is split
// over CTAs; each CTA writes an FP64 partial tile and a reduction kernel sums the splits.
// Every mbarrier wait is bounded (%globaltimer); on expiry the CTA records an error, stops its
// loops, waits for its own tensor-core work and frees its TMEM before returning.
#include <algorithm>
#include <cstring>

#include "internal.h"
#include "tma.cuh"

namespace pt {

namespace {

constexpr int TM = 64;          // A orbitals per tile (MMA M = 128 rows: A and iA)
constexpr int TN = 64;          // B orbitals per tile (MMA N)
constexpr int KS = 32;          // floats of K per stage (one 128-byte swizzled row)
constexpr int MAX_STAGES = 8;
constexpr int THREADS = 192;
constexpr uint32_t ROWS_BYTES = 64 * 128;                 // 64 rows of one 128-byte stage row
constexpr uint32_t STAGE_HI = 3 * ROWS_BYTES;             // [raw A | i*A] (MMA A operand) + raw B
constexpr uint32_t STAGE_SPLIT = 6 * ROWS_BYTES;          // + [A lo | i*A lo] + B lo
constexpr uint32_t RING_BYTES = 8 * STAGE_HI;             // 196608: 8 single or 4 split stages
constexpr uint32_t OFF_BAR = RING_BYTES;
constexpr uint32_t SMEM_USED = OFF_BAR + 512;
constexpr uint32_t SMEM_BYTES = SMEM_USED + 1024;
constexpr uint64_t TIMEOUT_NS = 2000000000ull;

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  // K-major, 128B swizzle: start >> 4, LBO unused (1), SBO = 1024 B between 8-row groups,
  // fixed 0b001 at bits 46..48, swizzle mode 2 (128B) at bits 61..63
  uint64_t d = uint64_t((addr >> 4) & 0x3FFFu);
  d |= uint64_t(1) << 16;
  d |= uint64_t(1024 >> 4) << 32;
  d |= uint64_t(1) << 46;
  d |= uint64_t(2) << 61;
  return d;
}

// instruction descriptor: D f32, A/B tf32, K-major both, N = TN, M = 128
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(TN >> 3) << 17) | (uint32_t(128 >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// TF32 part of an FP32 value: sign, exponent and the 10 leading mantissa bits (the tensor core
// reads only these bits of an FP32 operand, so the raw value acts as its own TF32 "hi" part)
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

struct TileArgs {
  int N1, N2;
  int tiles_j;        // number of 64-wide B tiles
  int herm;           // skip tiles below the diagonal
  int stages_total;   // K' / KS (rounded up)
  int stages_per_split;
  int split3;         // 1: 3xTF32, 0: single TF32 product
  int period;         // stages accumulated in TMEM between readouts
};

// Stage ring (each stage 1024-aligned, 128-byte swizzled rows of 32 floats):
//   hi(s)        rows 0..63 raw A (TMA), rows 64..127 i*A (converter)  -> MMA operand A
//   hi(s) + 16K  raw B (TMA)                                           -> MMA operand B
//   hi(s) + 24K  rows 0..63 A lo, rows 64..127 i*A lo (3xTF32 only)
//   hi(s) + 40K  B lo (3xTF32 only)
// The converter copies a chunk of 16 bytes from row r to the same position of row r + 64 (or
// of the lo buffers); rows r and r + 64 share the swizzle phase (r & 7), so the swizzled layout
// carries over unchanged.
__global__ void __launch_bounds__(THREADS, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TileArgs P,
              double* __restrict__ part, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  const int NS = P.split3 ? 4 : 8;
  const uint32_t stage_bytes = P.split3 ? STAGE_SPLIT : STAGE_HI;
  const uint32_t bar0 = base + OFF_BAR;
  auto bar_full = [&](int s) { return bar0 + 8u * s; };
  auto bar_cvt = [&](int s) { return bar0 + 8u * (MAX_STAGES + s); };
  auto bar_empty = [&](int s) { return bar0 + 8u * (2 * MAX_STAGES + s); };
  auto bar_acc_full = [&](int b) { return bar0 + 8u * (3 * MAX_STAGES + b); };
  auto bar_acc_empty = [&](int b) { return bar0 + 8u * (3 * MAX_STAGES + 2 + b); };
  const uint32_t bar_drain = bar0 + 8u * (3 * MAX_STAGES + 4);
  volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(sm + OFF_BAR + 256);
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(sm + OFF_BAR + 264);
  auto hi = [&](int s) { return base + uint32_t(s) * stage_bytes; };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x, split = blockIdx.y;
  const int bi = tile / P.tiles_j, bj = tile % P.tiles_j;
  if (P.herm && bj < bi) return;  // uniform over the CTA, before any barrier or TMEM use
  const int st0 = split * P.stages_per_split;
  const int st1 = min(P.stages_total, st0 + P.stages_per_split);
  const int nst = max(0, st1 - st0);
  const int period = P.period;
  const int nper = (nst + period - 1) / period;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(bar_full(s), 1);
      mbar_init(bar_cvt(s), 128);
      mbar_init(bar_empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_acc_full(b), 1);
      mbar_init(bar_acc_empty(b), 128);
    }
    mbar_init(bar_drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + OFF_BAR + 256),
                 "r"(2 * TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  auto fail_out = [&](int code) {
    atomicOr(err, code);
    *abort_flag = 1;
  };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < nst && !*abort_flag; ++it) {
        const int s = it % NS;
        if (it >= NS && !mbar_wait(bar_empty(s), ((it / NS) - 1) & 1, TIMEOUT_NS)) {
          fail_out(1);
          break;
        }
        mbar_arrive_expect_tx(bar_full(s), 2 * ROWS_BYTES);
        const int k = (st0 + it) * KS;
        tma_load_4d(hi(s), &tmA, k, bi * TM, 0, 0, bar_full(s));
        tma_load_4d(hi(s) + 2 * ROWS_BYTES, &tmB, k, bj * TN, 0, 0, bar_full(s));
        issued = it + 1;
      }
      // loads still in flight must land before the CTA's shared memory is released
      for (int it = max(0, issued - NS); it < issued; ++it)
        if (!mbar_wait(bar_full(it % NS), (it / NS) & 1, TIMEOUT_NS)) atomicOr(err, 128);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      for (int it = 0; it < nst && !*abort_flag; ++it) {
        const int s = it % NS;
        const int per = it / period, b = per & 1;
        if (it % period == 0 && per >= 2 && !mbar_wait(bar_acc_empty(b), ((per / 2) - 1) & 1, TIMEOUT_NS)) {
          fail_out(2);
          break;
        }
        if (!mbar_wait(bar_cvt(s), (it / NS) & 1, TIMEOUT_NS)) {
          fail_out(4);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + uint32_t(b * TN);
        const uint32_t ahi = hi(s), bhi = hi(s) + 2 * ROWS_BYTES;
        const uint32_t alo = hi(s) + 3 * ROWS_BYTES, blo = hi(s) + 5 * ROWS_BYTES;
#pragma unroll
        for (int kk = 0; kk < KS / 8; ++kk) {
          const uint32_t off = uint32_t(kk * 32);
          const uint32_t first = (it % period == 0 && kk == 0) ? 0u : 1u;
          mma_tf32(d, smem_desc_sw128(ahi + off), smem_desc_sw128(bhi + off), first);
          if (P.split3) {
            mma_tf32(d, smem_desc_sw128(ahi + off), smem_desc_sw128(blo + off), 1u);
            mma_tf32(d, smem_desc_sw128(alo + off), smem_desc_sw128(bhi + off), 1u);
          }
        }
        mma_commit(bar_empty(s));
        if (it % period == period - 1 || it == nst - 1) mma_commit(bar_acc_full(b));
      }
      // all issued MMAs complete before TMEM is freed
      mma_commit(bar_drain);
      if (!mbar_wait(bar_drain, 0, TIMEOUT_NS)) atomicOr(err, 256);
    }
  } else {
    // ---------------- converter + readout (warps 2..5) ----------------
    const int ct = tid - 64;  // 0..127
    const int quad = warp & 3;
    const uint32_t lane_base = uint32_t(32 * quad) << 16;
    float sum[TN], comp[TN];
#pragma unroll
    for (int c = 0; c < TN; ++c) sum[c] = comp[c] = 0.f;
    int readouts = 0;
    // waits and aborts are decided per warp (vote), so the .sync.aligned TMEM loads run converged
    auto readout = [&](int per) -> bool {
      const int b = per & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(bar_acc_full(b), (per / 2) & 1, TIMEOUT_NS))) return false;
      tc_fence_after();
#pragma unroll
      for (int c0 = 0; c0 < TN; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + lane_base + uint32_t(b * TN + c0), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float y = v[i] - comp[c0 + i];
          const float t = sum[c0 + i] + y;
          comp[c0 + i] = (t - sum[c0 + i]) - y;
          sum[c0 + i] = t;
        }
      }
      tc_fence_before();
      mbar_arrive(bar_acc_empty(b));
      return true;
    };
    constexpr int LAG = 2;  // read a period out once the converter is LAG stages past its end
    for (int it = 0; it < nst; ++it) {
      if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
      const int s = it % NS;
      if (!__all_sync(0xffffffffu, mbar_wait(bar_full(s), (it / NS) & 1, TIMEOUT_NS))) {
        fail_out(8);
        break;
      }
      unsigned char* st = sm + (hi(s) - base);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        // 64 rows x 8 chunks of 16 bytes per operand; this thread takes chunks ct and ct + 128
        const int q = ct + 128 * u;
        const uint32_t off = uint32_t(q >> 3) * 128u + uint32_t(q & 7) * 16u;
        const float4 v = *reinterpret_cast<const float4*>(st + off);
        const float4 w = *reinterpret_cast<const float4*>(st + 2 * ROWS_BYTES + off);
        const float4 q1 = *reinterpret_cast<const float4*>(st + off + 4096u);
        const float4 w1 = *reinterpret_cast<const float4*>(st + 2 * ROWS_BYTES + off + 4096u);
        // i * (re, im) = (-im, re); the tensor core drops the low mantissa bits itself
        *reinterpret_cast<float4*>(st + ROWS_BYTES + off) = make_float4(-v.y, v.x, -v.w, v.z);
        *reinterpret_cast<float4*>(st + ROWS_BYTES + off + 4096u) = make_float4(-q1.y, q1.x, -q1.w, q1.z);
        if (P.split3) {
          const float4 lo = make_float4(v.x - tf32_hi(v.x), v.y - tf32_hi(v.y), v.z - tf32_hi(v.z),
                                        v.w - tf32_hi(v.w));
          const float4 lo1 = make_float4(q1.x - tf32_hi(q1.x), q1.y - tf32_hi(q1.y), q1.z - tf32_hi(q1.z),
                                         q1.w - tf32_hi(q1.w));
          *reinterpret_cast<float4*>(st + 3 * ROWS_BYTES + off) = lo;
          *reinterpret_cast<float4*>(st + 3 * ROWS_BYTES + off + 4096u) = lo1;
          *reinterpret_cast<float4*>(st + 4 * ROWS_BYTES + off) = make_float4(-lo.y, lo.x, -lo.w, lo.z);
          *reinterpret_cast<float4*>(st + 4 * ROWS_BYTES + off + 4096u) = make_float4(-lo1.y, lo1.x, -lo1.w, lo1.z);
          *reinterpret_cast<float4*>(st + 5 * ROWS_BYTES + off) =
              make_float4(w.x - tf32_hi(w.x), w.y - tf32_hi(w.y), w.z - tf32_hi(w.z), w.w - tf32_hi(w.w));
          *reinterpret_cast<float4*>(st + 5 * ROWS_BYTES + off + 4096u) =
              make_float4(w1.x - tf32_hi(w1.x), w1.y - tf32_hi(w1.y), w1.z - tf32_hi(w1.z), w1.w - tf32_hi(w1.w));
        }
      }
      fence_proxy_async_smem();
      mbar_arrive(bar_cvt(s));
      const int lagged = it - LAG;
      if (lagged >= 0 && (lagged % period == period - 1)) {
        if (!readout(lagged / period)) {
          fail_out(32);
          break;
        }
        ++readouts;
      }
    }
    while (readouts < nper) {
      if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
      if (!readout(readouts)) {
        fail_out(64);
        break;
      }
      ++readouts;
    }
    // FP64 partial: rows 0..63 real part, 64..127 imaginary part of this tile
    const int row = 32 * quad + lane;
    double* out = part + ((size_t(split) * gridDim.x + tile) * 128 + row) * TN;
#pragma unroll
    for (int c = 0; c < TN; ++c) out[c] = double(sum[c]) - double(comp[c]);
  }
  // teardown: every role has left its loop; free TMEM
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TN) : "memory");
  }
}

// C[i][j] = scale * sum_split part[split][tile][row][col]; herm: mirror the tiles not computed
__global__ void k_gram_tc_reduce(const double* __restrict__ part, int nsplit, int ntiles, int tiles_j, int N1, int N2,
                                 double scale, int herm, c128* __restrict__ C) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N1 * N2) return;
  int i = e / N2, j = e % N2;
  bool mirror = false;
  if (herm && (j / TN) < (i / TM)) {
    mirror = true;
    const int t = i;
    i = j;
    j = t;
  }
  const int tile = (i / TM) * tiles_j + (j / TN);
  const int r = i % TM, c = j % TN;
  double re = 0, im = 0;
  for (int s = 0; s < nsplit; ++s) {
    const double* p = part + (size_t(s) * ntiles + tile) * 128 * TN;
    re += p[size_t(r) * TN + c];
    im += p[size_t(TM + r) * TN + c];
  }
  C[e] = mirror ? c128{re * scale, -im * scale} : c128{re * scale, im * scale};
}

}  // namespace

bool gram_tc_applies(const void* A, const void* B, size_t ng) {
  // tensor-map rules: 16-byte aligned bases and row strides (2 Ng floats) a multiple of 16 bytes
  return ng > 0 && ng % 2 == 0 && 2 * ng < (size_t(1) << 31) && reinterpret_cast<uintptr_t>(A) % 16 == 0 &&
         reinterpret_cast<uintptr_t>(B) % 16 == 0;
}

void gram_tc(pt_ctx* ctx, const c64* A, const c64* B, int N1, int N2, size_t ng, double scale, c128* C,
             cudaStream_t st, bool herm, bool split3) {
  if (!gram_tc_applies(A, B, ng)) fail(PT_INVALID_ARG, "tensor-core Gram: operands not TMA-addressable");
  herm = herm && (N1 == N2);
  const int ti = (N1 + TM - 1) / TM, tj = (N2 + TN - 1) / TN;
  const int ntiles = ti * tj;
  const int stages_total = int((2 * ng + KS - 1) / KS);
  const int active = herm ? ti * (ti + 1) / 2 : ntiles;
  // one CTA per SM (the kernel uses ~210 KB of shared memory): split K so that one wave fills the GPU
  int splits = std::max(1, ctx->num_sms / active);
  int sps = (stages_total + splits - 1) / splits;
  splits = (stages_total + sps - 1) / sps;
  double* part = static_cast<double*>(ctx->get("gram_tc_parts", size_t(splits) * ntiles * 128 * TN * sizeof(double)));
  int* err = static_cast<int*>(ctx->get("gram_tc_err", sizeof(int)));
  if (!ctx->tc_err_clean) {
    PT_CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st));
    ctx->tc_err_clean = true;
  }
  static DeviceOnce once;
  once([] { PT_CUDA_CHECK(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)); });
  // 2-D views (as 4-D maps with unit outer dims): K' = 2 Ng floats per orbital row
  CUtensorMap ta, tb;
  const uint64_t da[4] = {2 * ng, uint64_t(N1), 1, 1}, db[4] = {2 * ng, uint64_t(N2), 1, 1};
  const uint64_t sa[3] = {2 * ng * 4, 2 * ng * 4 * uint64_t(N1), 2 * ng * 4 * uint64_t(N1)};
  const uint64_t sb[3] = {2 * ng * 4, 2 * ng * 4 * uint64_t(N2), 2 * ng * 4 * uint64_t(N2)};
  const uint32_t boxa[4] = {KS, TM, 1, 1}, boxb[4] = {KS, TN, 1, 1};
  encode_tmap_4d_f32(&ta, A, da, sa, boxa, CU_TENSOR_MAP_SWIZZLE_128B);
  encode_tmap_4d_f32(&tb, B, db, sb, boxb, CU_TENSOR_MAP_SWIZZLE_128B);
  TileArgs P{N1, N2, tj, herm ? 1 : 0, stages_total, sps, split3 ? 1 : 0, std::max(1, ctx->tc_period)};
  PT_LAUNCH(k_gram_tc, dim3(ntiles, splits), THREADS, SMEM_BYTES, st, ta, tb, P, part, err);
  PT_LAUNCH(k_gram_tc_reduce, (N1 * N2 + 255) / 256, 256, 0, st, part, splits, ntiles, tj, N1, N2, scale,
            herm ? 1 : 0, C);
}

void gram_tc_check(pt_ctx* ctx, cudaStream_t st) {
  if (!ctx->tc_err_clean) return;  // no tensor-core Gram ran since the last check
  int* err = static_cast<int*>(ctx->get("gram_tc_err", sizeof(int)));
  int h = 0;
  PT_CUDA_CHECK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PT_CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st));
  PT_CUDA_CHECK(cudaStreamSynchronize(st));
  if (h) fail(PT_TIMEOUT, "tensor-core Gram: a bounded wait expired on the device (code " + std::to_string(h) + ")");
}

}  // namespace pt
