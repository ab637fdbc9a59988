// Wide-tile Gram contractions on the 5th-generation tensor cores (tcgen05, TF32 inputs):
//   C0 = scale * A^H B0   and, optionally in the same pass,   C1 = scale * A^H B1
// with A, B0, B1 complex64, orbital-major (each orbital a K-major row of K' = 2 Ng interleaved
// floats).  The overlap S = <Phi|Phi> and the subspace matrix <Phi|H Phi> of the PT-IM inner
// iteration (Sec. IV-A2) share their left operand, so one pass computes both.
//
// A tile is one 64-orbital block of A against two 64-orbital B halves: the MMA is M = 128 (rows
// 0..63 the A orbitals, 64..127 the same orbitals times i, giving Re and Im of A^H B in one real
// GEMM, as in the 64 x 64 kernel) by N = 128 (half 0 and half 1, each from B0 or B1).  The wider N
// halves the tensor-core operand traffic and the A-side conversion per product compared with
// N = 64 tiles, and the shared A block is converted once for both halves.  The FP32 accuracy
// comes from three TF32 products hi*hi + hi*lo + lo*hi (the raw FP32 value is its own TF32 "hi";
// "lo" = x - tf32(x) is written by the converter warps).
//
// Warp roles (576 threads): warp 0 issues the TMA loads of a stage (A block, half 0, half 1),
// warp 1 allocates TMEM and one lane issues tcgen05.mma, warps 2..17 (four warpgroups) convert
// the stage (i*A rows and the lo parts) and read the TMEM accumulator out every `period` stages
// into Kahan-compensated FP32 registers, each warpgroup owning 32 of the 128 accumulator
// columns (the TMEM lane quarter of a warp is its index mod 4).  Two TMEM accumulators alternate.
// The K range of every tile is split over CTAs; each CTA writes an FP64 partial tile and a
// reduction kernel sums the splits into C0/C1, mirroring the blocks of a Hermitian product that
// no tile computed.  Every mbarrier wait is bounded (%globaltimer): on expiry the CTA records an
// error, leaves its loops, waits for its own copies and MMAs and frees its TMEM.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tma.cuh"

namespace pt {

namespace {

constexpr int WB = 64;                    // orbitals per A block and per B half
constexpr int WN = 2 * WB;                // MMA N
constexpr int WK = 32;                    // floats of K per stage (one 128-byte swizzled row)
constexpr int W_THREADS = 576;
constexpr int W_CVT = 512;                // converter/readout threads
constexpr int W_MAX_STAGES = 6;
constexpr uint32_t ROWS = 64 * 128;       // 64 rows of one 128-byte stage row
// stage layout: [raw A | i*A] [half 0 | half 1] (MMA "hi" operands), then in 3-product mode
// [A lo | i*A lo] [half 0 lo | half 1 lo]
constexpr uint32_t STAGE_HI = 4 * ROWS;   // 32 KB
constexpr uint32_t STAGE_SPLIT = 8 * ROWS;  // 64 KB
constexpr uint32_t RING = 6 * STAGE_HI;   // 192 KB: 6 single-product or 3 three-product stages
constexpr uint32_t OFF_BAR = RING;
constexpr uint32_t SMEM_BYTES = OFF_BAR + 512 + 1024;
constexpr uint64_t TIMEOUT_NS = 2000000000ull;

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
  // K-major, 128B swizzle: start >> 4, LBO unused (1), SBO = 1024 B between 8-row groups,
  // fixed 0b001 at bits 46..48, swizzle mode 2 (128B) at bits 61..63
  uint64_t d = uint64_t((addr >> 4) & 0x3FFFu);
  d |= uint64_t(1) << 16;
  d |= uint64_t(1024 >> 4) << 32;
  d |= uint64_t(1) << 46;
  d |= uint64_t(2) << 61;
  return d;
}

// instruction descriptor: D f32, A/B tf32, both K-major, N = 128, M = 128
constexpr uint32_t IDESC_W = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(WN >> 3) << 17) | (uint32_t(128 >> 4) << 24);

__device__ __forceinline__ void mma_w(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC_W), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void commit_w(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
// 16-byte shared-memory accesses by 32-bit shared-window address
__device__ __forceinline__ float4 lds128(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts128(uint32_t a, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}
__device__ __forceinline__ float4 lo4(float4 v) {
  return make_float4(v.x - tf32_hi(v.x), v.y - tf32_hi(v.y), v.z - tf32_hi(v.z), v.w - tf32_hi(v.w));
}
__device__ __forceinline__ float4 times_i(float4 v) { return make_float4(-v.y, v.x, -v.w, v.z); }

// one tile: A block r against half 0 = block c0 of B(m0) and half 1 = block c1 of B(m1)
struct WideTile {
  int r, m0, c0, m1, c1;
};

struct WideArgs {
  int stages_total;
  int stages_per_split;
  int split3;
  int period;
};

__global__ void __launch_bounds__(W_THREADS, 1)
    k_gram_tc_wide(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB0,
                   const __grid_constant__ CUtensorMap tmB1, const WideTile* __restrict__ tiles, WideArgs P,
                   double* __restrict__ part, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  const int NS = P.split3 ? 3 : 6;
  const uint32_t stage_bytes = P.split3 ? STAGE_SPLIT : STAGE_HI;
  const uint32_t bar0 = base + OFF_BAR;
  auto bar_full = [&](int s) { return bar0 + 8u * s; };
  auto bar_cvt = [&](int s) { return bar0 + 8u * (W_MAX_STAGES + s); };
  auto bar_empty = [&](int s) { return bar0 + 8u * (2 * W_MAX_STAGES + s); };
  auto bar_acc_full = [&](int b) { return bar0 + 8u * (3 * W_MAX_STAGES + b); };
  auto bar_acc_empty = [&](int b) { return bar0 + 8u * (3 * W_MAX_STAGES + 2 + b); };
  const uint32_t bar_drain = bar0 + 8u * (3 * W_MAX_STAGES + 4);
  volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(sm + OFF_BAR + 256);
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(sm + OFF_BAR + 264);
  auto stg = [&](int s) { return base + uint32_t(s) * stage_bytes; };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x, split = blockIdx.y;
  const int st0 = split * P.stages_per_split;
  const int st1 = min(P.stages_total, st0 + P.stages_per_split);
  const int nst = max(0, st1 - st0);
  const int period = P.period;
  const int nper = (nst + period - 1) / period;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(bar_full(s), 1);
      mbar_init(bar_cvt(s), W_CVT);
      mbar_init(bar_empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_acc_full(b), 1);
      mbar_init(bar_acc_empty(b), W_CVT);
    }
    mbar_init(bar_drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + OFF_BAR + 256),
                 "r"(2 * WN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_holder;
  auto fail_out = [&](int code) {
    atomicOr(err, code);
    *abort_flag = 1;
  };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      const WideTile T = tiles[tile];
      const CUtensorMap* h0 = T.m0 == 1 ? &tmB1 : &tmB0;
      // an absent second half re-reads the first (its columns are never reduced)
      const CUtensorMap* h1 = T.m1 < 0 ? h0 : (T.m1 == 1 ? &tmB1 : &tmB0);
      const int c1 = T.m1 < 0 ? T.c0 : T.c1;
      int issued = 0;
      for (int it = 0; it < nst && !*abort_flag; ++it) {
        const int s = it % NS;
        if (it >= NS && !mbar_wait(bar_empty(s), ((it / NS) - 1) & 1, TIMEOUT_NS)) {
          fail_out(1);
          break;
        }
        mbar_arrive_expect_tx(bar_full(s), 3 * ROWS);
        const int k = (st0 + it) * WK;
        tma_load_4d(stg(s), &tmA, k, T.r * WB, 0, 0, bar_full(s));
        tma_load_4d(stg(s) + 2 * ROWS, h0, k, T.c0 * WB, 0, 0, bar_full(s));
        tma_load_4d(stg(s) + 3 * ROWS, h1, k, c1 * WB, 0, 0, bar_full(s));
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
        fence_after();
        const uint32_t d = tmem + uint32_t(b * WN);
        const uint32_t ahi = stg(s), bhi = stg(s) + 2 * ROWS;
        const uint32_t alo = stg(s) + 4 * ROWS, blo = stg(s) + 6 * ROWS;
#pragma unroll
        for (int kk = 0; kk < WK / 8; ++kk) {
          const uint32_t off = uint32_t(kk * 32);
          const uint32_t first = (it % period == 0 && kk == 0) ? 0u : 1u;
          mma_w(d, desc_sw128(ahi + off), desc_sw128(bhi + off), first);
          if (P.split3) {
            mma_w(d, desc_sw128(ahi + off), desc_sw128(blo + off), 1u);
            mma_w(d, desc_sw128(alo + off), desc_sw128(bhi + off), 1u);
          }
        }
        commit_w(bar_empty(s));
        if (it % period == period - 1 || it == nst - 1) commit_w(bar_acc_full(b));
      }
      // all issued MMAs complete before TMEM is freed
      commit_w(bar_drain);
      if (!mbar_wait(bar_drain, 0, TIMEOUT_NS)) atomicOr(err, 256);
    }
  } else {
    // ---------------- converters + readout (warps 2..17) ----------------
    const int ct = tid - 64;          // 0..511
    const int wg = (warp - 2) >> 2;   // accumulator columns [32 wg, 32 wg + 32)
    const int quad = warp & 3;        // TMEM lane quarter
    const uint32_t lane_base = uint32_t(32 * quad) << 16;
    float sum[32], comp[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) sum[c] = comp[c] = 0.f;
    int readouts = 0;
    // waits and aborts are decided per warp (vote), so the .sync.aligned TMEM loads run converged
    auto readout = [&](int per) -> bool {
      const int b = per & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(bar_acc_full(b), (per / 2) & 1, TIMEOUT_NS))) return false;
      fence_after();
#pragma unroll
      for (int c0 = 0; c0 < 32; c0 += 8) {
        float v[8];
        ld8(tmem + lane_base + uint32_t(b * WN + 32 * wg + c0), v);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float y = v[i] - comp[c0 + i];
          const float t = sum[c0 + i] + y;
          comp[c0 + i] = (t - sum[c0 + i]) - y;
          sum[c0 + i] = t;
        }
      }
      fence_before();
      mbar_arrive(bar_acc_empty(b));
      return true;
    };
    // chunk ct of the A block (64 rows x 8 chunks of 16 bytes) and chunks ct, ct + 512 of the
    // B halves (128 rows); a warp's 32 chunks are 512 contiguous bytes.  Rows r and r + 64 share
    // the swizzle phase (r & 7), so a chunk is written at the same position of the other row.
    const uint32_t offa = uint32_t(ct >> 3) * 128u + uint32_t(ct & 7) * 16u;
    const uint32_t offb0 = offa, offb1 = offa + 64u * 128u;
    constexpr int LAG = 2;  // read a period out once the converters are LAG stages past its end
    for (int it = 0; it < nst; ++it) {
      if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
      const int s = it % NS;
      if (!__all_sync(0xffffffffu, mbar_wait(bar_full(s), (it / NS) & 1, TIMEOUT_NS))) {
        fail_out(8);
        break;
      }
      const uint32_t st = stg(s);
      {
        const float4 a = lds128(st + offa);
        sts128(st + ROWS + offa, times_i(a));
        if (P.split3) {
          const float4 al = lo4(a);
          sts128(st + 4 * ROWS + offa, al);
          sts128(st + 5 * ROWS + offa, times_i(al));
        }
      }
      if (P.split3) {
        sts128(st + 6 * ROWS + offb0, lo4(lds128(st + 2 * ROWS + offb0)));
        sts128(st + 6 * ROWS + offb1, lo4(lds128(st + 2 * ROWS + offb1)));
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
    // FP64 partial: rows 0..63 real part, 64..127 imaginary part; columns 0..63 half 0, 64..127 half 1
    const int row = 32 * quad + lane;
    double* out = part + ((size_t(split) * gridDim.x + tile) * 128 + row) * WN + 32 * wg;
#pragma unroll
    for (int c = 0; c < 32; ++c) out[c] = double(sum[c]) - double(comp[c]);
  }
  // teardown: every role has left its loop; free TMEM
  fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * WN) : "memory");
  }
}

// C_m[i][j] = scale * sum_split part[split][tile][row][col] through a block lookup: entry
// (m, i / 64, j / 64) = tile * 4 + half * 2 + mirror (-1: not computed); a mirrored block is the
// conjugate transpose of block (j / 64, i / 64)
__global__ void k_gram_tc_wide_reduce(const double* __restrict__ part, int nsplit, int ntiles, const int* __restrict__ lut,
                                      int nbi, int nbj, int N1, int N2, double scale, c128* __restrict__ C0,
                                      c128* __restrict__ C1) {
  const size_t n = size_t(N1) * N2;
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int m = int(blockIdx.y);
  if (e >= n) return;
  c128* C = m == 0 ? C0 : C1;
  int i = int(e / N2), j = int(e % N2);
  const int code = lut[(size_t(m) * nbi + i / WB) * nbj + j / WB];
  if (code < 0) return;
  const int tile = code >> 2, half = (code >> 1) & 1, mirror = code & 1;
  if (mirror) {
    const int t = i;
    i = j;
    j = t;
  }
  const int r = i % WB, c = half * WB + j % WB;
  double re = 0, im = 0;
  for (int s = 0; s < nsplit; ++s) {
    const double* p = part + (size_t(s) * ntiles + tile) * 128 * WN;
    re += p[size_t(r) * WN + c];
    im += p[size_t(WB + r) * WN + c];
  }
  C[e] = mirror ? c128{re * scale, -im * scale} : c128{re * scale, im * scale};
}

struct WidePlan {
  int ntiles = 0;
  WideTile* tiles = nullptr;  // device
  int* lut = nullptr;         // device, 2 x nbi x nbj
  ~WidePlan() {
    cudaFree(tiles);
    cudaFree(lut);
  }
};

std::shared_ptr<WidePlan> wide_plan(pt_ctx* ctx, int N1, int N2, bool two, bool herm) {
  char key[96];
  snprintf(key, sizeof(key), "gram_wide:%d:%d:%d:%d", N1, N2, int(two), int(herm));
  auto it = ctx->caches.find(key);
  if (it != ctx->caches.end()) return std::static_pointer_cast<WidePlan>(it->second);
  const int nbi = (N1 + WB - 1) / WB, nbj = (N2 + WB - 1) / WB;
  std::vector<WideTile> tl;
  std::vector<int> lut(size_t(2) * nbi * nbj, -1);
  auto put = [&](int m, int r, int c, int t, int half) {
    lut[(size_t(m) * nbi + r) * nbj + c] = t * 4 + half * 2;
    if (herm && r != c) lut[(size_t(m) * nbi + c) * nbj + r] = t * 4 + half * 2 + 1;
  };
  for (int r = 0; r < nbi; ++r) {
    std::vector<int> cs;
    for (int c = herm ? r : 0; c < nbj; ++c) cs.push_back(c);
    if (two) {
      for (int c : cs) {
        const int t = int(tl.size());
        tl.push_back({r, 0, c, 1, c});
        put(0, r, c, t, 0);
        put(1, r, c, t, 1);
      }
    } else {
      for (size_t k = 0; k < cs.size(); k += 2) {
        const int t = int(tl.size());
        const bool pair = k + 1 < cs.size();
        tl.push_back({r, 0, cs[k], pair ? 0 : -1, pair ? cs[k + 1] : -1});
        put(0, r, cs[k], t, 0);
        if (pair) put(0, r, cs[k + 1], t, 1);
      }
    }
  }
  auto pl = std::make_shared<WidePlan>();
  pl->ntiles = int(tl.size());
  PT_CUDA_CHECK(cudaMalloc(&pl->tiles, tl.size() * sizeof(WideTile)));
  PT_CUDA_CHECK(cudaMemcpy(pl->tiles, tl.data(), tl.size() * sizeof(WideTile), cudaMemcpyHostToDevice));
  PT_CUDA_CHECK(cudaMalloc(&pl->lut, lut.size() * sizeof(int)));
  PT_CUDA_CHECK(cudaMemcpy(pl->lut, lut.data(), lut.size() * sizeof(int), cudaMemcpyHostToDevice));
  ctx->caches[key] = pl;
  return pl;
}

}  // namespace

void gram_tc_wide(pt_ctx* ctx, const c64* A, const c64* B0, c128* C0, const c64* B1, c128* C1, int N1, int N2,
                  size_t ng, double scale, cudaStream_t st, bool herm, bool split3) {
  if (!gram_tc_applies(A, B0, ng) || (B1 && !gram_tc_applies(A, B1, ng)))
    fail(PT_INVALID_ARG, "tensor-core Gram: operands not TMA-addressable");
  herm = herm && (N1 == N2);
  const bool two = B1 != nullptr;
  auto pl = wide_plan(ctx, N1, N2, two, herm);
  const int stages_total = int((2 * ng + WK - 1) / WK);
  // one CTA per SM (~197 KB of shared memory): split K so that one wave fills the GPU
  int splits = std::max(1, ctx->num_sms / pl->ntiles);
  int sps = (stages_total + splits - 1) / splits;
  splits = (stages_total + sps - 1) / sps;
  double* part = static_cast<double*>(
      ctx->get("gram_tc_wide_parts", size_t(splits) * pl->ntiles * 128 * WN * sizeof(double)));
  int* err = static_cast<int*>(ctx->get("gram_tc_err", sizeof(int)));
  if (!ctx->tc_err_clean) {
    PT_CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st));
    ctx->tc_err_clean = true;
  }
  static DeviceOnce once;
  once([] {
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_gram_tc_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  });
  CUtensorMap ta, tb0, tb1;
  const uint64_t da[4] = {2 * ng, uint64_t(N1), 1, 1}, db[4] = {2 * ng, uint64_t(N2), 1, 1};
  const uint64_t sa[3] = {2 * ng * 4, 2 * ng * 4 * uint64_t(N1), 2 * ng * 4 * uint64_t(N1)};
  const uint64_t sb[3] = {2 * ng * 4, 2 * ng * 4 * uint64_t(N2), 2 * ng * 4 * uint64_t(N2)};
  const uint32_t box[4] = {WK, WB, 1, 1};
  encode_tmap_4d_f32(&ta, A, da, sa, box, CU_TENSOR_MAP_SWIZZLE_128B);
  encode_tmap_4d_f32(&tb0, B0, db, sb, box, CU_TENSOR_MAP_SWIZZLE_128B);
  encode_tmap_4d_f32(&tb1, two ? B1 : B0, db, sb, box, CU_TENSOR_MAP_SWIZZLE_128B);
  WideArgs P{stages_total, sps, split3 ? 1 : 0, std::max(1, ctx->tc_period)};
  PT_LAUNCH(k_gram_tc_wide, dim3(pl->ntiles, splits), W_THREADS, SMEM_BYTES, st, ta, tb0, tb1, pl->tiles, P, part,
            err);
  const size_t n = size_t(N1) * N2;
  const int nbi = (N1 + WB - 1) / WB, nbj = (N2 + WB - 1) / WB;
  PT_LAUNCH(k_gram_tc_wide_reduce, dim3(unsigned((n + 255) / 256), two ? 2u : 1u), 256, 0, st, part, splits,
            pl->ntiles, pl->lut, nbi, nbj, N1, N2, scale, C0, C1);
}

}  // namespace pt
