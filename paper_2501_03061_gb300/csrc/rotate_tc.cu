// Orbital rotations out_j = alpha sum_k B[k][j] A_k + sum_t c_t e_t,j on the 5th-generation tensor
// cores (tcgen05, TF32 inputs with a 3-product hi/lo split for FP32 accuracy).
//
// As a real GEMM over grid points r: a row r holds K' = 2 N1 interleaved floats
// (Re A_0(r), Im A_0(r), Re A_1(r), ...), an output row holds (Re out_0(r), Im out_0(r), ...), and
// the real operand B' (2 N2 x K') is built once per call from alpha * B:
//     B'[2j][2k] = Re b,  B'[2j][2k+1] = -Im b,  B'[2j+1][2k] = Im b,  B'[2j+1][2k+1] = Re b
// so that row r of A' times B'^T is row r of the complex product.  One CTA tile is 128 grid
// points x 64 output orbitals (MMA M = 128, N = 128), with all of K' in one TMEM accumulation
// chain that is read out every `period` K stages into FP32 registers.
//
// The orbitals are stored orbital-major (r contiguous for each k), the transpose of the K-major
// operand the tensor core reads, so TMA brings in a [16 orbitals][128 points] block of complex64
// values and a converter warpgroup writes it out as 128 K-major rows of 32 floats (128B swizzle),
// once as the raw values (the tensor core reads their TF32 bits: "hi") and once as the FP32
// remainders x - tf32(x) ("lo").  B' is written once per call as the shared-memory images of
// its stages (for every 128-row block and 32-float K stage, the hi and the lo tile in the 128B
// swizzle the tensor core reads, 32 KB contiguous), so a stage's B operands arrive with one bulk
// copy instead of a tiled load of 2 x 128 rows of 128 bytes.  Products summed per tile:
// hi*hi + hi*lo + lo*hi.
//
// Warp roles (320 threads): warp 0 TMA producer, warp 1 TMEM allocation and MMA issue (one
// lane), warps 2..5 converter, warps 6..9 TMEM readout and the epilogue (alpha is folded into
// B'; the epilogue adds the extra terms and stores complex64).  CTAs are persistent and walk
// the tiles with a grid stride; the two TMEM accumulators alternate between periods, so the
// epilogue of one tile overlaps the MMAs of the next.  Every wait is bounded (%globaltimer); on
// expiry the CTA records an error, leaves its loops, drains its own copies and tensor-core work
// and frees its TMEM.
#include <algorithm>

#include "internal.h"
#include "tma.cuh"

namespace pt {

namespace {

constexpr int RM = 128;                 // grid points per tile (MMA M)
constexpr int RJ = 64;                  // output orbitals per tile (MMA N = 2 RJ real columns)
constexpr int NC = 2 * RJ;              // 128 real output columns
constexpr int KO = 16;                  // orbitals per K stage (32 floats of K')
constexpr int RA = 3;                   // raw A stages
constexpr int RC = 2;                   // converted / B stages
constexpr int THREADS = 320;
constexpr uint32_t RAW_BYTES = KO * RM * 8;          // 16 KB: [16 orbitals][128 points] complex64
constexpr uint32_t OP_BYTES = 128 * 128;             // 16 KB: 128 rows x 32 floats, swizzled
constexpr uint32_t CST_BYTES = 4 * OP_BYTES;         // A hi | A lo | B hi | B lo
constexpr uint32_t OFF_C = 0;                        // converted ring (1024-aligned stages)
constexpr uint32_t OFF_RAW = RC * CST_BYTES;         // 131072
constexpr uint32_t OFF_BAR = OFF_RAW + RA * RAW_BYTES;  // 180224
constexpr uint32_t SMEM_BYTES = OFF_BAR + 256 + 1024;
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

// instruction descriptor: D f32, A/B tf32, K-major both, N = NC, M = RM
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(NC >> 3) << 17) | (uint32_t(RM >> 4) << 24);

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

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

struct RotArgs {
  int N1, N2;
  long long ng;
  int tiles_r, tiles_j, ntiles;
  int stages;          // K stages per tile: ceil(N1 / KO)
  int period;          // stages per TMEM accumulation window
  int split3;
  const float* bp;     // B' stage images: [tiles_j][stages][hi | lo][128 rows x 32 floats, swizzled]
  const c64* e[3];     // epilogue terms (may be null)
  c64 c[3];
  c64* out;
};

// read-only load of one complex64 through the non-coherent path
__device__ __forceinline__ c64 ldg_c64(const c64* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return c64{v.x, v.y};
}

// B'[n'][k'] (npad = tiles_j * 128 rows, kpad = stages * 32 floats), alpha folded in, written as
// stage images: element (n', k') of row block jt = n' / 128, stage s = k' / 32 goes to row
// r = n' % 128, 16-byte chunk (k' % 32) / 4 XOR (r % 8) of the 32 KB block (jt * stages + s),
// the hi part in its first 16 KB and the lo part in its second
__global__ void k_rot_prep_b(const c128* __restrict__ Bm, int ldb, int N1, int N2, c128 alpha, int npad, int kpad,
                             int stages, float* __restrict__ bp) {
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= size_t(npad) * kpad) return;
  const int n = int(e / kpad), kk = int(e % kpad);
  const int j = n >> 1, d = n & 1, k = kk >> 1, c = kk & 1;
  double v = 0.0;
  if (j < N2 && k < N1) {
    const c128 b = cmul(alpha, Bm[size_t(k) * ldb + j]);
    // d = 0 (real output): (Re b, -Im b); d = 1 (imaginary output): (Im b, Re b)
    v = d == 0 ? (c == 0 ? b.re : -b.im) : (c == 0 ? b.im : b.re);
  }
  const float f = float(v);
  const float h = tf32_hi(f);
  const int jt = n / NC, r = n % NC, s = kk / (2 * KO), kq = kk % (2 * KO);
  const size_t blk = size_t(jt * stages + s) * 2 * (NC * 2 * KO);
  const size_t off = size_t(r) * (2 * KO) + size_t((((kq >> 2) ^ (r & 7)) << 2) + (kq & 3));
  bp[blk + off] = h;
  bp[blk + NC * 2 * KO + off] = float(v - double(h));
}

__global__ void __launch_bounds__(THREADS, 1)
    k_rotate_tc(const __grid_constant__ CUtensorMap tmA, RotArgs P, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  const uint32_t bar0 = base + OFF_BAR;
  auto bar_a_full = [&](int s) { return bar0 + 8u * s; };
  auto bar_a_empty = [&](int s) { return bar0 + 8u * (RA + s); };
  auto bar_b_full = [&](int s) { return bar0 + 8u * (2 * RA + s); };
  auto bar_c_full = [&](int s) { return bar0 + 8u * (2 * RA + RC + s); };
  auto bar_c_empty = [&](int s) { return bar0 + 8u * (2 * RA + 2 * RC + s); };
  auto bar_acc_full = [&](int b) { return bar0 + 8u * (2 * RA + 3 * RC + b); };
  auto bar_acc_empty = [&](int b) { return bar0 + 8u * (2 * RA + 3 * RC + 2 + b); };
  const uint32_t bar_drain = bar0 + 8u * (2 * RA + 3 * RC + 4);
  volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(sm + OFF_BAR + 192);
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(sm + OFF_BAR + 200);
  auto a_raw = [&](int s) { return base + OFF_RAW + uint32_t(s) * RAW_BYTES; };
  auto c_ahi = [&](int s) { return base + OFF_C + uint32_t(s) * CST_BYTES; };
  auto c_alo = [&](int s) { return c_ahi(s) + OP_BYTES; };
  auto c_bhi = [&](int s) { return c_ahi(s) + 2 * OP_BYTES; };
  auto c_blo = [&](int s) { return c_ahi(s) + 3 * OP_BYTES; };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...
  const int my_tiles = blockIdx.x < P.ntiles ? (P.ntiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  const int S = P.stages;
  const int nq = my_tiles * S;                     // (tile, stage) steps of this CTA
  const int per_tile = (S + P.period - 1) / P.period;

  if (tid == 0) {
    for (int s = 0; s < RA; ++s) {
      mbar_init(bar_a_full(s), 1);
      mbar_init(bar_a_empty(s), 128);
    }
    for (int s = 0; s < RC; ++s) {
      mbar_init(bar_b_full(s), 1);
      mbar_init(bar_c_full(s), 128);
      mbar_init(bar_c_empty(s), 1);
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
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + OFF_BAR + 192),
                 "r"(2 * NC)
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
  auto tile_of = [&](int q, int& rb, int& jt, int& s) {
    const int t = int(blockIdx.x) + (q / S) * int(gridDim.x);
    rb = t / P.tiles_j;
    jt = t % P.tiles_j;
    s = q % S;
  };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int issued_a = 0, issued_b = 0;
      for (int q = 0; q < nq && !*abort_flag; ++q) {
        int rb, jt, s;
        tile_of(q, rb, jt, s);
        const int sa = q % RA, sc = q % RC;
        if (q >= RA && !mbar_wait(bar_a_empty(sa), ((q / RA) - 1) & 1, TIMEOUT_NS)) {
          fail_out(1);
          break;
        }
        mbar_arrive_expect_tx(bar_a_full(sa), RAW_BYTES);
        tma_load_4d(a_raw(sa), &tmA, rb * RM, s * KO, 0, 0, bar_a_full(sa));
        issued_a = q + 1;
        if (q >= RC && !mbar_wait(bar_c_empty(sc), ((q / RC) - 1) & 1, TIMEOUT_NS)) {
          fail_out(2);
          break;
        }
        mbar_arrive_expect_tx(bar_b_full(sc), 2 * OP_BYTES);
        bulk_load(c_bhi(sc), P.bp + size_t(jt * S + s) * (2 * OP_BYTES / 4), 2 * OP_BYTES, bar_b_full(sc));
        issued_b = q + 1;
      }
      // copies in flight land before the CTA's shared memory is released
      for (int q = max(0, issued_a - RA); q < issued_a; ++q)
        if (!mbar_wait(bar_a_full(q % RA), (q / RA) & 1, TIMEOUT_NS)) atomicOr(err, 128);
      for (int q = max(0, issued_b - RC); q < issued_b; ++q)
        if (!mbar_wait(bar_b_full(q % RC), (q / RC) & 1, TIMEOUT_NS)) atomicOr(err, 128);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int gp = 0;  // global period counter (selects the TMEM accumulator)
      for (int q = 0; q < nq && !*abort_flag; ++q) {
        const int s = q % S, sc = q % RC;
        const int b = gp & 1;
        const bool first = (s % P.period) == 0;
        if (first && gp >= 2 && !mbar_wait(bar_acc_empty(b), ((gp / 2) - 1) & 1, TIMEOUT_NS)) {
          fail_out(4);
          break;
        }
        if (!mbar_wait(bar_b_full(sc), (q / RC) & 1, TIMEOUT_NS) ||
            !mbar_wait(bar_c_full(sc), (q / RC) & 1, TIMEOUT_NS)) {
          fail_out(8);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + uint32_t(b * NC);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t off = uint32_t(kk * 32);
          const uint32_t acc = (first && kk == 0) ? 0u : 1u;
          mma_tf32(d, smem_desc_sw128(c_ahi(sc) + off), smem_desc_sw128(c_bhi(sc) + off), acc);
          if (P.split3) {
            mma_tf32(d, smem_desc_sw128(c_ahi(sc) + off), smem_desc_sw128(c_blo(sc) + off), 1u);
            mma_tf32(d, smem_desc_sw128(c_alo(sc) + off), smem_desc_sw128(c_bhi(sc) + off), 1u);
          }
        }
        mma_commit(bar_c_empty(sc));
        if ((s % P.period) == P.period - 1 || s == S - 1) {
          mma_commit(bar_acc_full(b));
          ++gp;
        }
      }
      mma_commit(bar_drain);
      if (!mbar_wait(bar_drain, 0, TIMEOUT_NS)) atomicOr(err, 256);
    }
  } else if (warp < 6) {
    // ---------------- converter: raw [16][128] complex64 -> K-major swizzled rows ----------------
    const int row = tid - 64;  // 0..127: grid point within the tile
    for (int q = 0; q < nq; ++q) {
      if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
      const int sa = q % RA, sc = q % RC;
      if (!__all_sync(0xffffffffu, mbar_wait(bar_a_full(sa), (q / RA) & 1, TIMEOUT_NS))) {
        fail_out(16);
        break;
      }
      if (q >= RC &&
          !__all_sync(0xffffffffu, mbar_wait(bar_c_empty(sc), ((q / RC) - 1) & 1, TIMEOUT_NS))) {
        fail_out(32);
        break;
      }
      const float2* src = reinterpret_cast<const float2*>(sm + (a_raw(sa) - base));
      float2 v[KO];
#pragma unroll
      for (int k = 0; k < KO; ++k) v[k] = src[k * RM + row];
      mbar_arrive(bar_a_empty(sa));
      unsigned char* hi = sm + (c_ahi(sc) - base) + row * 128;
      unsigned char* lo = sm + (c_alo(sc) - base) + row * 128;
#pragma unroll
      for (int ch = 0; ch < 8; ++ch) {
        const uint32_t pos = uint32_t((ch ^ (row & 7)) * 16);
        const float4 h = make_float4(v[2 * ch].x, v[2 * ch].y, v[2 * ch + 1].x, v[2 * ch + 1].y);
        *reinterpret_cast<float4*>(hi + pos) = h;
        if (P.split3)
          *reinterpret_cast<float4*>(lo + pos) =
              make_float4(h.x - tf32_hi(h.x), h.y - tf32_hi(h.y), h.z - tf32_hi(h.z), h.w - tf32_hi(h.w));
      }
      fence_proxy_async_smem();
      mbar_arrive(bar_c_full(sc));
    }
  } else {
    // ---------------- TMEM readout + epilogue ----------------
    const int quad = warp & 3;
    const int lrow = 32 * quad + lane;
    const uint32_t lane_base = uint32_t(32 * quad) << 16;
    float acc[NC];
    int gp = 0;
    bool ok = true;
    for (int t = 0; t < my_tiles && ok; ++t) {
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = 0.f;
      for (int p = 0; p < per_tile; ++p, ++gp) {
        if (__any_sync(0xffffffffu, *abort_flag != 0)) {
          ok = false;
          break;
        }
        const int b = gp & 1;
        if (!__all_sync(0xffffffffu, mbar_wait(bar_acc_full(b), (gp / 2) & 1, TIMEOUT_NS))) {
          fail_out(64);
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int c0 = 0; c0 < NC; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + lane_base + uint32_t(b * NC + c0), v);
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[c0 + i] += v[i];
        }
        tc_fence_before();
        mbar_arrive(bar_acc_empty(b));
      }
      if (!ok) break;
      const int tl = int(blockIdx.x) + t * int(gridDim.x);
      const int rb = tl / P.tiles_j, jt = tl % P.tiles_j;
      const long long r = (long long)rb * RM + lrow;
      if (r < P.ng) {
        // The terms and the output are distinct per element (a term that is also the output is
        // read before its element is written by the same thread), so the loads of later outputs
        // may be issued ahead of earlier stores: restrict-qualified copies let the compiler batch
        // them instead of paying one memory latency per output.
        const c64* __restrict__ e0 = P.e[0];
        const c64* __restrict__ e1 = P.e[1];
        const c64* __restrict__ e2 = P.e[2];
        c64* __restrict__ op = P.out;
        const int jn = min(RJ, P.N2 - jt * RJ);
        // fully unrolled so that acc[] stays in registers
#pragma unroll
        for (int j0 = 0; j0 < RJ; j0 += 4) {
          c64 tv[3][4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const size_t idx = size_t(jt * RJ + j0 + u) * size_t(P.ng) + size_t(r);
            const bool okj = j0 + u < jn;
            tv[0][u] = (e0 && okj) ? ldg_c64(e0 + idx) : c64{0.f, 0.f};
            tv[1][u] = (e1 && okj) ? ldg_c64(e1 + idx) : c64{0.f, 0.f};
            tv[2][u] = (e2 && okj) ? ldg_c64(e2 + idx) : c64{0.f, 0.f};
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int jj = j0 + u;
            if (jj >= jn) continue;
            const size_t idx = size_t(jt * RJ + jj) * size_t(P.ng) + size_t(r);
            c64 o{acc[2 * jj], acc[2 * jj + 1]};
            o = o + cmul(P.c[0], tv[0][u]) + cmul(P.c[1], tv[1][u]) + cmul(P.c[2], tv[2][u]);
            op[idx] = o;
          }
        }
      }
    }
  }
  // teardown: every role has left its loop; free TMEM
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * NC) : "memory");
  }
}

}  // namespace

bool rotate_tc_applies(const void* A, size_t ng) {
  // tensor-map rules: 16-byte aligned base and orbital stride (Ng complex64) a multiple of 16 bytes
  return ng > 0 && ng % 2 == 0 && ng < (size_t(1) << 31) && reinterpret_cast<uintptr_t>(A) % 16 == 0;
}

void rotate_tc(pt_ctx* ctx, const c64* A, const c128* Bm, int ldb, int N1, int N2, size_t ng, c128 alpha,
               const Term* terms, int nterms, c64* out, cudaStream_t st, bool split3) {
  if (!rotate_tc_applies(A, ng)) fail(PT_INVALID_ARG, "tensor-core rotation: operand not TMA-addressable");
  if (nterms > 3) fail(PT_INVALID_ARG, "tensor-core rotation: at most 3 epilogue terms");
  const int stages = (N1 + KO - 1) / KO;
  const int kpad = stages * 2 * KO;
  const int tiles_j = (N2 + RJ - 1) / RJ;
  const int npad = tiles_j * NC;
  const int tiles_r = int((ng + RM - 1) / RM);
  float* bp = static_cast<float*>(ctx->get("rot_tc_bp", 2 * size_t(npad) * kpad * sizeof(float)));
  int* err = static_cast<int*>(ctx->get("gram_tc_err", sizeof(int)));
  if (!ctx->tc_err_clean) {
    PT_CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st));
    ctx->tc_err_clean = true;
  }
  const size_t nb = size_t(npad) * kpad;
  PT_LAUNCH(k_rot_prep_b, unsigned((nb + 255) / 256), 256, 0, st, Bm, ldb, N1, N2, alpha, npad, kpad, stages, bp);
  static DeviceOnce once;
  once([] { PT_CUDA_CHECK(cudaFuncSetAttribute(k_rotate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)); });
  // A as a [N1][Ng] array of 8-byte elements; box = 128 points x 16 orbitals, no swizzle
  CUtensorMap ta;
  const uint64_t da[4] = {ng, uint64_t(N1), 1, 1};
  const uint64_t sa[3] = {ng * 8, ng * 8 * uint64_t(N1), ng * 8 * uint64_t(N1)};
  const uint32_t boxa[4] = {RM, KO, 1, 1};
  encode_tmap_4d_u64(&ta, A, da, sa, boxa, CU_TENSOR_MAP_SWIZZLE_NONE);
  RotArgs P{};
  P.bp = bp;
  P.N1 = N1;
  P.N2 = N2;
  P.ng = (long long)ng;
  P.tiles_r = tiles_r;
  P.tiles_j = tiles_j;
  P.ntiles = tiles_r * tiles_j;
  P.stages = stages;
  P.period = std::max(1, std::min(ctx->tc_period, stages));
  P.split3 = split3 ? 1 : 0;
  for (int t = 0; t < 3; ++t) {
    P.e[t] = t < nterms ? static_cast<const c64*>(terms[t].x) : nullptr;
    P.c[t] = t < nterms ? c64{float(terms[t].c.re), float(terms[t].c.im)} : c64{0.f, 0.f};
  }
  P.out = out;
  const int grid = std::min(P.ntiles, ctx->num_sms);
  PT_LAUNCH(k_rotate_tc, grid, THREADS, SMEM_BYTES, st, ta, P, err);
}

}  // namespace pt
