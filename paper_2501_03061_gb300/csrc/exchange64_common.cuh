// Pieces shared by the two 64^3 FP32 exchange engines (exchange64_tma.cu: one launch per pipeline
// step; exchange64_persist.cu: one persistent launch per application): the shared-memory layout of
// a CTA, the 128B-swizzled tile addressing of the TMA copies and the 64-point line transform held
// by 8-lane groups (Sec. IV-A1, Eq. vxdiag: the pair FFTs of the exchange).
#pragma once

#include "common.cuh"
#include "fft.cuh"
#include "tma.cuh"

namespace pt {
namespace x64 {

constexpr int G = 64;
constexpr int PITCH = 68;
constexpr int THREADS = 512;
constexpr uint32_t TILE_BYTES = 32768;           // 64 x 64 complex64
constexpr uint32_t SUB_BYTES = 8192;             // 16 columns x 64 rows of 128 B
constexpr uint32_t OFF_A = 0, OFF_B = 32768, OFF_P = 65536;
constexpr uint32_t OFF_TW = OFF_P + G * PITCH * 8;  // 100352
constexpr uint32_t OFF_BAR = OFF_TW + G * 8;        // 100864
constexpr uint32_t SMEM_USED = OFF_BAR + 128;
constexpr uint32_t SMEM_BYTES = SMEM_USED + 1024;   // slack to align the base to 1024 B
constexpr uint64_t TIMEOUT_NS = 2000000000ull;      // 2 s

// byte offset of element (column x, row r) inside a 64 x 64 swizzled tile
__device__ __forceinline__ uint32_t sw_off(int x, int r) {
  const int xx = x & 15;
  return uint32_t(x >> 4) * SUB_BYTES + uint32_t(r) * 128u + uint32_t(((xx >> 1) ^ (r & 7)) << 4) +
         uint32_t((xx & 1) << 3);
}

// element (row, col) of the 64 x 64 plane-transpose buffer: col XOR-swizzled by
// ((row & 7) << 1) ^ ((row & 1) << 3), a bijection of [0, 4096) under which both access patterns of
// the plane passes — column writes (lane t of group g at row t + 8k, column g) and row reads
// (row g, column t + 8q) — reach 16 distinct 8-byte bank slots in every half-warp
__device__ __forceinline__ int pidx(int row, int col) {
  return row * G + (col ^ (((row & 7) << 1) ^ ((row & 1) << 3)));
}

// 64-point transform of the line held by an 8-lane group (lane t holds x[t + 8a]): radix 8,
// twiddles w^{tk} derived in registers, a swizzled group transpose through gs (element e at
// e ^ (8 (g & 1))), radix 8; on return lane t holds X[t + 8k]
__device__ __forceinline__ void fft64_tma(c64 (&v)[8], int t, c64* gs, int gpar, const c64* tw, bool inv) {
  if (inv) dft8<true>(v);
  else dft8<false>(v);
  c64 w1 = tw[t];
  if (inv) w1.im = -w1.im;
  const c64 w2 = cmul(w1, w1), w4 = cmul(w2, w2);
  v[1] = cmul(v[1], w1);
  v[2] = cmul(v[2], w2);
  v[3] = cmul(v[3], cmul(w1, w2));
  v[4] = cmul(v[4], w4);
  v[5] = cmul(v[5], cmul(w1, w4));
  v[6] = cmul(v[6], cmul(w2, w4));
  v[7] = cmul(v[7], cmul(cmul(w1, w2), w4));
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 8; ++k) gs[(k * 8 + (t ^ k)) ^ gpar] = v[k];
  __syncwarp();
#pragma unroll
  for (int s = 0; s < 8; ++s) v[s] = gs[(t * 8 + (s ^ t)) ^ gpar];
  if (inv) dft8<true>(v);
  else dft8<false>(v);
}

}  // namespace x64
}  // namespace pt
