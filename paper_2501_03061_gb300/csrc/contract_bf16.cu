// BF16 tensor-core contractions of the FP32 form (the BF16 precision study of the ACE GEMMs):
// the Gram C = scale A^* B and the rotation out_j = alpha sum_k B[k][j] A_k + terms with one BF16
// product per term, FP32 accumulation in TMEM (tcgen05 kind::f16, both operands bf16).
//
// Unlike the TF32 kernels, which convert FP32 tiles in shared memory, the operands are first packed
// into K-major bf16 arrays in HBM (an error-study form, where a pass over the inputs costs little):
//   Gram:     rows [A; iA] per 64-orbital tile (i*(re, im) = (-im, re)), B rows, K' = 2 Ng interleaved;
//   rotation: grid points as rows with K' = 2 N1 interleaved (a transposed copy of A), and the real
//             B' (2 N2 x 2 N1) of the rotation kernel, built from alpha * B.
// The GEMM kernels are then plain warp-specialised tcgen05 loops: one TMA producer warp, one
// MMA-issuing thread, four readout warps (TMEM -> registers every `period` K stages; compensated
// sums in the Gram, FP32 sums plus the fused epilogue in the rotation).  Every mbarrier wait is
// bounded; on expiry the CTA records an error word, drains its copies and MMAs and frees its TMEM.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"
#include "tma.cuh"

namespace pt {

namespace {

constexpr uint64_t TIMEOUT_NS = 2000000000ull;
constexpr int KB = 64;  // bf16 values of K per stage (one 128-byte swizzled row)

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

// instruction descriptor of kind::f16: D f32 (bit 4), A and B bf16 (format 1 at bits 7 and 10),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
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

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  return uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(lo))) |
         (uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(hi))) << 16);
}

// ---------------------------------------------------------------- packing ----
// Gram A operand: row t*128 + o holds orbital t*64 + (o mod 64) (o >= 64: times i), K' = kpad
__global__ void k_pack_gram_a(const c64* __restrict__ A, int N1, size_t ng, size_t kpad, int rows,
                              uint32_t* __restrict__ out) {
  const size_t total = size_t(rows) * (kpad / 2);
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += size_t(gridDim.x) * blockDim.x) {
    const int R = int(e / (kpad / 2));
    const size_t k = e % (kpad / 2);  // complex index along the grid
    const int o = R % 128, orb = (R / 128) * 64 + (o & 63);
    float re = 0.f, im = 0.f;
    if (orb < N1 && k < ng) {
      const c64 v = A[size_t(orb) * ng + k];
      re = v.re;
      im = v.im;
      if (o >= 64) {  // i * (re, im) = (-im, re)
        const float t = re;
        re = -im;
        im = t;
      }
    }
    out[e] = pack_bf16x2(re, im);
  }
}

// plain rows (the Gram's B operand): row j < rows holds orbital j (zero beyond N2)
__global__ void k_pack_rows(const c64* __restrict__ B, int N2, size_t ng, size_t kpad, int rows,
                            uint32_t* __restrict__ out) {
  const size_t total = size_t(rows) * (kpad / 2);
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += size_t(gridDim.x) * blockDim.x) {
    const int j = int(e / (kpad / 2));
    const size_t k = e % (kpad / 2);
    const c64 v = (j < N2 && k < ng) ? B[size_t(j) * ng + k] : c64{0.f, 0.f};
    out[e] = pack_bf16x2(v.re, v.im);
  }
}

// rotation A operand: row r (grid point) holds (Re A_0(r), Im A_0(r), Re A_1(r), ...), kpad/2
// orbitals (zero beyond N1 and beyond Ng); a 32-orbital x 64-point tile transposed through smem
__global__ void __launch_bounds__(256) k_pack_transpose(const c64* __restrict__ A, int N1, size_t ng, int kpad,
                                                        uint32_t* __restrict__ out) {
  __shared__ c64 s[32][65];
  const size_t r0 = size_t(blockIdx.x) * 64;
  const int k0 = blockIdx.y * 32;
  for (int idx = threadIdx.x; idx < 32 * 64; idx += 256) {
    const int kk = idx / 64, p = idx % 64;
    s[kk][p] = (k0 + kk < N1 && r0 + p < ng) ? A[size_t(k0 + kk) * ng + r0 + p] : c64{0.f, 0.f};
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 64 * 32; idx += 256) {
    const int p = idx / 32, kk = idx % 32;
    if (k0 + kk < kpad / 2) out[(r0 + p) * size_t(kpad / 2) + k0 + kk] = pack_bf16x2(s[kk][p].re, s[kk][p].im);
  }
}

// rotation B' (bf16) from alpha * B: B'[2j][2k] = Re b, [2j][2k+1] = -Im b, [2j+1][2k] = Im b, [2j+1][2k+1] = Re b
__global__ void k_pack_rot_b(const c128* __restrict__ Bm, int ldb, int N1, int N2, c128 alpha, int npad, int kpad,
                             uint16_t* __restrict__ out) {
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= size_t(npad) * kpad) return;
  const int n = int(e / kpad), kk = int(e % kpad);
  const int j = n >> 1, d = n & 1, k = kk >> 1, c = kk & 1;
  double v = 0.0;
  if (j < N2 && k < N1) {
    const c128 b = cmul(alpha, Bm[size_t(k) * ldb + j]);
    v = d == 0 ? (c == 0 ? b.re : -b.im) : (c == 0 ? b.im : b.re);
  }
  out[e] = __bfloat16_as_ushort(__float2bfloat16_rn(float(v)));
}

// ---------------------------------------------------------------- Gram ----
constexpr int GS = 8;  // stages
constexpr uint32_t G_A = 128 * 128, G_B = 64 * 128, G_STAGE = G_A + G_B;
constexpr uint32_t G_BAR = GS * G_STAGE;
constexpr uint32_t G_SMEM = G_BAR + 256 + 1024;

struct GramArgs {
  int tiles_j, herm, stages_total, stages_per_split, period;
};

__global__ void __launch_bounds__(192, 1)
    k_gram_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GramArgs P,
                double* __restrict__ part, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  const uint32_t bar0 = base + G_BAR;
  auto bar_full = [&](int s) { return bar0 + 8u * s; };
  auto bar_empty = [&](int s) { return bar0 + 8u * (GS + s); };
  auto bar_acc_full = [&](int b) { return bar0 + 8u * (2 * GS + b); };
  auto bar_acc_empty = [&](int b) { return bar0 + 8u * (2 * GS + 2 + b); };
  const uint32_t bar_drain = bar0 + 8u * (2 * GS + 4);
  volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(sm + G_BAR + 192);
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(sm + G_BAR + 200);
  auto sa = [&](int s) { return base + uint32_t(s) * G_STAGE; };
  auto sb = [&](int s) { return sa(s) + G_A; };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x, split = blockIdx.y;
  const int bi = tile / P.tiles_j, bj = tile % P.tiles_j;
  if (P.herm && bj < bi) return;  // uniform over the CTA, before any barrier or TMEM use
  const int st0 = split * P.stages_per_split;
  const int nst = max(0, min(P.stages_total, st0 + P.stages_per_split) - st0);
  const int period = P.period;
  const int nper = (nst + period - 1) / period;
  constexpr uint32_t IDESC = idesc_bf16(128, 64);

  if (tid == 0) {
    for (int s = 0; s < GS; ++s) {
      mbar_init(bar_full(s), 1);
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
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + G_BAR + 192),
                 "r"(128)
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
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < nst && !*abort_flag; ++it) {
        const int s = it % GS;
        if (it >= GS && !mbar_wait(bar_empty(s), ((it / GS) - 1) & 1, TIMEOUT_NS)) {
          fail_out(1);
          break;
        }
        mbar_arrive_expect_tx(bar_full(s), G_STAGE);
        const int k = (st0 + it) * KB;
        tma_load_4d(sa(s), &tmA, k, bi * 128, 0, 0, bar_full(s));
        tma_load_4d(sb(s), &tmB, k, bj * 64, 0, 0, bar_full(s));
        issued = it + 1;
      }
      for (int it = max(0, issued - GS); it < issued; ++it)
        if (!mbar_wait(bar_full(it % GS), (it / GS) & 1, TIMEOUT_NS)) atomicOr(err, 128);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int it = 0; it < nst && !*abort_flag; ++it) {
        const int s = it % GS;
        const int per = it / period, b = per & 1;
        if (it % period == 0 && per >= 2 && !mbar_wait(bar_acc_empty(b), ((per / 2) - 1) & 1, TIMEOUT_NS)) {
          fail_out(2);
          break;
        }
        if (!mbar_wait(bar_full(s), (it / GS) & 1, TIMEOUT_NS)) {
          fail_out(4);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + uint32_t(b * 64);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t off = uint32_t(kk * 32);
          mma_bf16(d, smem_desc_sw128(sa(s) + off), smem_desc_sw128(sb(s) + off), IDESC,
                   (it % period == 0 && kk == 0) ? 0u : 1u);
        }
        mma_commit(bar_empty(s));
        if (it % period == period - 1 || it == nst - 1) mma_commit(bar_acc_full(b));
      }
      mma_commit(bar_drain);
      if (!mbar_wait(bar_drain, 0, TIMEOUT_NS)) atomicOr(err, 256);
    }
  } else {
    const int quad = warp & 3;
    const uint32_t lane_base = uint32_t(32 * quad) << 16;
    float sum[64], comp[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) sum[c] = comp[c] = 0.f;
    for (int per = 0; per < nper; ++per) {
      if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
      const int b = per & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(bar_acc_full(b), (per / 2) & 1, TIMEOUT_NS))) {
        fail_out(8);
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int c0 = 0; c0 < 64; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + lane_base + uint32_t(b * 64 + c0), v);
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
    }
    const int row = 32 * quad + lane;
    double* out = part + ((size_t(split) * gridDim.x + tile) * 128 + row) * 64;
#pragma unroll
    for (int c = 0; c < 64; ++c) out[c] = double(sum[c]) - double(comp[c]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
  }
}

// C[i][j] = scale * sum_split part (rows 0..63 real, 64..127 imaginary); herm: mirror the lower tiles
__global__ void k_gram_bf16_reduce(const double* __restrict__ part, int nsplit, int ntiles, int tiles_j, int N1,
                                   int N2, double scale, int herm, c128* __restrict__ C) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N1 * N2) return;
  int i = e / N2, j = e % N2;
  bool mirror = false;
  if (herm && (j / 64) < (i / 64)) {
    mirror = true;
    const int t = i;
    i = j;
    j = t;
  }
  const int tile = (i / 64) * tiles_j + (j / 64);
  double re = 0, im = 0;
  for (int s = 0; s < nsplit; ++s) {
    const double* p = part + (size_t(s) * ntiles + tile) * 128 * 64;
    re += p[size_t(i % 64) * 64 + j % 64];
    im += p[size_t(64 + i % 64) * 64 + j % 64];
  }
  C[e] = mirror ? c128{re * scale, -im * scale} : c128{re * scale, im * scale};
}

// ---------------------------------------------------------------- rotation ----
constexpr int RS = 6;  // stages
constexpr uint32_t R_A = 128 * 128, R_B = 128 * 128, R_STAGE = R_A + R_B;
constexpr uint32_t R_BAR = RS * R_STAGE;
constexpr uint32_t R_SMEM = R_BAR + 256 + 1024;

struct RotArgs {
  long long ng;
  int N2, tiles_j, ntiles, stages, period;
  const c64* e[3];
  c64 c[3];
  c64* out;
};

__global__ void __launch_bounds__(192, 1)
    k_rotate_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, RotArgs P,
                  int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  const uint32_t bar0 = base + R_BAR;
  auto bar_full = [&](int s) { return bar0 + 8u * s; };
  auto bar_empty = [&](int s) { return bar0 + 8u * (RS + s); };
  auto bar_acc_full = [&](int b) { return bar0 + 8u * (2 * RS + b); };
  auto bar_acc_empty = [&](int b) { return bar0 + 8u * (2 * RS + 2 + b); };
  const uint32_t bar_drain = bar0 + 8u * (2 * RS + 4);
  volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(sm + R_BAR + 192);
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(sm + R_BAR + 200);
  auto sa = [&](int s) { return base + uint32_t(s) * R_STAGE; };
  auto sb = [&](int s) { return sa(s) + R_A; };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int my_tiles = blockIdx.x < P.ntiles ? (P.ntiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  const int S = P.stages;
  const int nq = my_tiles * S;
  const int per_tile = (S + P.period - 1) / P.period;
  constexpr uint32_t IDESC = idesc_bf16(128, 128);

  if (tid == 0) {
    for (int s = 0; s < RS; ++s) {
      mbar_init(bar_full(s), 1);
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
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + R_BAR + 192),
                 "r"(256)
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
    if (lane == 0) {
      int issued = 0;
      for (int q = 0; q < nq && !*abort_flag; ++q) {
        const int t = int(blockIdx.x) + (q / S) * int(gridDim.x);
        const int rb = t / P.tiles_j, jt = t % P.tiles_j, s = q % S, sl = q % RS;
        if (q >= RS && !mbar_wait(bar_empty(sl), ((q / RS) - 1) & 1, TIMEOUT_NS)) {
          fail_out(1);
          break;
        }
        mbar_arrive_expect_tx(bar_full(sl), R_STAGE);
        tma_load_4d(sa(sl), &tmA, s * KB, rb * 128, 0, 0, bar_full(sl));
        tma_load_4d(sb(sl), &tmB, s * KB, jt * 128, 0, 0, bar_full(sl));
        issued = q + 1;
      }
      for (int q = max(0, issued - RS); q < issued; ++q)
        if (!mbar_wait(bar_full(q % RS), (q / RS) & 1, TIMEOUT_NS)) atomicOr(err, 128);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int gp = 0;
      for (int q = 0; q < nq && !*abort_flag; ++q) {
        const int s = q % S, sl = q % RS;
        const int b = gp & 1;
        const bool first = (s % P.period) == 0;
        if (first && gp >= 2 && !mbar_wait(bar_acc_empty(b), ((gp / 2) - 1) & 1, TIMEOUT_NS)) {
          fail_out(2);
          break;
        }
        if (!mbar_wait(bar_full(sl), (q / RS) & 1, TIMEOUT_NS)) {
          fail_out(4);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + uint32_t(b * 128);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t off = uint32_t(kk * 32);
          mma_bf16(d, smem_desc_sw128(sa(sl) + off), smem_desc_sw128(sb(sl) + off), IDESC,
                   (first && kk == 0) ? 0u : 1u);
        }
        mma_commit(bar_empty(sl));
        if ((s % P.period) == P.period - 1 || s == S - 1) {
          mma_commit(bar_acc_full(b));
          ++gp;
        }
      }
      mma_commit(bar_drain);
      if (!mbar_wait(bar_drain, 0, TIMEOUT_NS)) atomicOr(err, 256);
    }
  } else {
    const int quad = warp & 3;
    const int lrow = 32 * quad + lane;
    const uint32_t lane_base = uint32_t(32 * quad) << 16;
    float acc[128];
    int gp = 0;
    bool ok = true;
    for (int t = 0; t < my_tiles && ok; ++t) {
#pragma unroll
      for (int c = 0; c < 128; ++c) acc[c] = 0.f;
      for (int p = 0; p < per_tile; ++p, ++gp) {
        if (__any_sync(0xffffffffu, *abort_flag != 0)) {
          ok = false;
          break;
        }
        const int b = gp & 1;
        if (!__all_sync(0xffffffffu, mbar_wait(bar_acc_full(b), (gp / 2) & 1, TIMEOUT_NS))) {
          fail_out(8);
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int c0 = 0; c0 < 128; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + lane_base + uint32_t(b * 128 + c0), v);
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[c0 + i] += v[i];
        }
        tc_fence_before();
        mbar_arrive(bar_acc_empty(b));
      }
      if (!ok) break;
      const int tl = int(blockIdx.x) + t * int(gridDim.x);
      const int rb = tl / P.tiles_j, jt = tl % P.tiles_j;
      const long long r = (long long)rb * 128 + lrow;
      if (r < P.ng) {
#pragma unroll
        for (int jj = 0; jj < 64; ++jj) {
          const int j = jt * 64 + jj;
          if (j >= P.N2) continue;
          const size_t idx = size_t(j) * size_t(P.ng) + size_t(r);
          c64 o{acc[2 * jj], acc[2 * jj + 1]};
#pragma unroll
          for (int e = 0; e < 3; ++e)
            if (P.e[e]) o = o + cmul(P.c[e], P.e[e][idx]);
          P.out[idx] = o;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
  }
}

int grid_for(size_t n, int threads, const pt_ctx* ctx) {
  return int(std::max<size_t>(1, std::min<size_t>((n + threads - 1) / threads, size_t(ctx->num_sms) * 16)));
}

}  // namespace

void gram_bf16(pt_ctx* ctx, const c64* A, const c64* B, int N1, int N2, size_t ng, double scale, c128* C,
               cudaStream_t st, bool herm) {
  herm = herm && (N1 == N2) && A == B;
  const int ti = (N1 + 63) / 64, tj = (N2 + 63) / 64, ntiles = ti * tj;
  const int stages_total = int((2 * ng + KB - 1) / KB);
  const size_t kpad = size_t(stages_total) * KB;
  uint32_t* ap = static_cast<uint32_t*>(ctx->get("bf16_gram_a", size_t(ti) * 128 * kpad * 2));
  uint32_t* bp = static_cast<uint32_t*>(ctx->get("bf16_gram_b", size_t(tj) * 64 * kpad * 2));
  PT_LAUNCH(k_pack_gram_a, grid_for(size_t(ti) * 128 * kpad / 2, 256, ctx), 256, 0, st, A, N1, ng, kpad, ti * 128, ap);
  PT_LAUNCH(k_pack_rows, grid_for(size_t(tj) * 64 * kpad / 2, 256, ctx), 256, 0, st, B, N2, ng, kpad, tj * 64, bp);
  const int active = herm ? ti * (ti + 1) / 2 : ntiles;
  int splits = std::max(1, ctx->num_sms / active);
  int sps = (stages_total + splits - 1) / splits;
  splits = (stages_total + sps - 1) / sps;
  double* part = static_cast<double*>(ctx->get("bf16_gram_parts", size_t(splits) * ntiles * 128 * 64 * sizeof(double)));
  int* err = static_cast<int*>(ctx->get("gram_tc_err", sizeof(int)));
  if (!ctx->tc_err_clean) {
    PT_CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st));
    ctx->tc_err_clean = true;
  }
  static DeviceOnce once;
  once([] { PT_CUDA_CHECK(cudaFuncSetAttribute(k_gram_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM)); });
  CUtensorMap ta, tb;
  const uint64_t da[4] = {kpad, uint64_t(ti) * 128, 1, 1}, db[4] = {kpad, uint64_t(tj) * 64, 1, 1};
  const uint64_t sa[3] = {kpad * 2, kpad * 2 * ti * 128, kpad * 2 * ti * 128};
  const uint64_t sb[3] = {kpad * 2, kpad * 2 * tj * 64, kpad * 2 * tj * 64};
  const uint32_t boxa[4] = {KB, 128, 1, 1}, boxb[4] = {KB, 64, 1, 1};
  encode_tmap_4d_bf16(&ta, ap, da, sa, boxa, CU_TENSOR_MAP_SWIZZLE_128B);
  encode_tmap_4d_bf16(&tb, bp, db, sb, boxb, CU_TENSOR_MAP_SWIZZLE_128B);
  GramArgs P{tj, herm ? 1 : 0, stages_total, sps, std::max(1, ctx->tc_period)};
  PT_LAUNCH(k_gram_bf16, dim3(ntiles, splits), 192, G_SMEM, st, ta, tb, P, part, err);
  PT_LAUNCH(k_gram_bf16_reduce, (N1 * N2 + 255) / 256, 256, 0, st, part, splits, ntiles, tj, N1, N2, scale,
            herm ? 1 : 0, C);
}

void rotate_bf16(pt_ctx* ctx, const c64* A, const c128* Bm, int ldb, int N1, int N2, size_t ng, c128 alpha,
                 const Term* terms, int nterms, c64* out, cudaStream_t st) {
  if (nterms > 3) fail(PT_INVALID_ARG, "BF16 rotation: at most 3 epilogue terms");
  const int stages = (2 * N1 + KB - 1) / KB;
  const int kpad = stages * KB;
  const int tiles_j = (N2 + 63) / 64, npad = tiles_j * 128;
  const size_t ngpad = (ng + 127) / 128 * 128;
  uint32_t* at = static_cast<uint32_t*>(ctx->get("bf16_rot_a", ngpad * size_t(kpad) * 2));
  uint16_t* bp = static_cast<uint16_t*>(ctx->get("bf16_rot_b", size_t(npad) * kpad * 2));
  PT_LAUNCH(k_pack_transpose, dim3(unsigned(ngpad / 64), unsigned((kpad / 2 + 31) / 32)), 256, 0, st, A, N1, ng, kpad,
            at);
  const size_t nb = size_t(npad) * kpad;
  PT_LAUNCH(k_pack_rot_b, unsigned((nb + 255) / 256), 256, 0, st, Bm, ldb, N1, N2, alpha, npad, kpad, bp);
  int* err = static_cast<int*>(ctx->get("gram_tc_err", sizeof(int)));
  if (!ctx->tc_err_clean) {
    PT_CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st));
    ctx->tc_err_clean = true;
  }
  static DeviceOnce once;
  once([] { PT_CUDA_CHECK(cudaFuncSetAttribute(k_rotate_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, R_SMEM)); });
  CUtensorMap ta, tb;
  const uint64_t da[4] = {uint64_t(kpad), ngpad, 1, 1}, db[4] = {uint64_t(kpad), uint64_t(npad), 1, 1};
  const uint64_t sa[3] = {uint64_t(kpad) * 2, uint64_t(kpad) * 2 * ngpad, uint64_t(kpad) * 2 * ngpad};
  const uint64_t sb[3] = {uint64_t(kpad) * 2, uint64_t(kpad) * 2 * npad, uint64_t(kpad) * 2 * npad};
  const uint32_t boxa[4] = {KB, 128, 1, 1}, boxb[4] = {KB, 128, 1, 1};
  encode_tmap_4d_bf16(&ta, at, da, sa, boxa, CU_TENSOR_MAP_SWIZZLE_128B);
  encode_tmap_4d_bf16(&tb, bp, db, sb, boxb, CU_TENSOR_MAP_SWIZZLE_128B);
  RotArgs P{};
  P.ng = (long long)ng;
  P.N2 = N2;
  P.tiles_j = tiles_j;
  P.ntiles = int(ngpad / 128) * tiles_j;
  P.stages = stages;
  P.period = std::max(1, std::min(ctx->tc_period, stages));
  for (int t = 0; t < 3; ++t) {
    P.e[t] = t < nterms ? static_cast<const c64*>(terms[t].x) : nullptr;
    P.c[t] = t < nterms ? c64{float(terms[t].c.re), float(terms[t].c.im)} : c64{0.f, 0.f};
  }
  P.out = out;
  PT_LAUNCH(k_rotate_bf16, std::min(P.ntiles, ctx->num_sms), 192, R_SMEM, st, ta, tb, P, err);
}

}  // namespace pt
