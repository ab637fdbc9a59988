// Compile-time-size Stockham FFT stages on 2-D tiles in shared memory, for cubic grids whose
// side N is known at compile time.
//
// Same algorithm and data movement as the runtime-plan stages of fft.cuh (radices 8, 4, 5, 3, 2;
// threads laid out with the line index fastest so that both tile orientations are free of bank
// conflicts; all reads of a stage finish before its writes, so one buffer serves in place), but
// the radix plan, the butterfly count per thread and every index divisor are template constants:
// the index arithmetic folds into multiplies and shifts and the butterfly loops unroll fully.
#pragma once

#include "fft.cuh"

namespace pt {

struct CPlan {
  int nst;
  int R[8];
  int L[8];
};

// radices 8, 4, 5, 3, 2 in that order; L[s] = product of the radices before stage s
constexpr CPlan make_cplan(int n) {
  CPlan p{0, {0, 0, 0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0, 0, 0}};
  const int rs[5] = {8, 4, 5, 3, 2};
  int L = 1, m = n;
  for (int k = 0; k < 5; ++k) {
    const int r = rs[k];
    while (m % r == 0 && p.nst < 8) {
      p.R[p.nst] = r;
      p.L[p.nst] = L;
      L *= r;
      m /= r;
      ++p.nst;
    }
  }
  return p;
}

// odd row pitch (in elements) of an N x N tile
template <int N>
constexpr int kPitch = (N % 2 == 0) ? N + 1 : N;

// one stage of radix R and span L over NLINES lines; element (line, pos) at buf[line*LS + pos*PS]
template <int R, int L, int N, bool INV, int NT, int NLINES, int LS, int PS, class T>
__device__ __forceinline__ void cstage(cx<T>* buf, const cx<T>* tw) {
  constexpr int NB = N / R;
  constexpr int M = NB / L;
  constexpr int TOTAL = NB * NLINES;
  constexpr int BPT = (TOTAL + NT - 1) / NT;
  const int tid = threadIdx.x;
  cx<T> v[BPT][R];
#pragma unroll
  for (int u = 0; u < BPT; ++u) {
    const int f = tid + u * NT;
    if (TOTAL % NT == 0 || f < TOTAL) {
      const int line = f % NLINES;
      const int b = f / NLINES;
      const int j = b % L;
      const cx<T>* src = buf + line * LS;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        cx<T> x = src[(b + q * NB) * PS];
        if (q > 0 && L > 1) {
          cx<T> w = tw[j * q * M];
          if (INV) w.im = -w.im;
          x = cmul(x, w);
        }
        v[u][q] = x;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < BPT; ++u) {
    const int f = tid + u * NT;
    if (TOTAL % NT == 0 || f < TOTAL) {
      const int line = f % NLINES;
      const int b = f / NLINES;
      const int j = b % L;
      const int k = b / L;
      dft<R, INV>(v[u]);
      cx<T>* dst = buf + line * LS;
#pragma unroll
      for (int p = 0; p < R; ++p) dst[(j + k * L * R + p * L) * PS] = v[u][p];
    }
  }
  __syncthreads();
}

template <int N, bool INV, int NT, int NLINES, int LS, int PS, int S = 0, class T>
__device__ __forceinline__ void cfft_lines(cx<T>* buf, const cx<T>* tw) {
  constexpr CPlan P = make_cplan(N);
  if constexpr (S < P.nst) {
    cstage<P.R[S], P.L[S], N, INV, NT, NLINES, LS, PS>(buf, tw);
    cfft_lines<N, INV, NT, NLINES, LS, PS, S + 1>(buf, tw);
  }
}

// transforms of an N x N tile with rows of pitch kPitch<N>: along the fast axis (within rows)
// and along the slow axis (within columns)
template <int N, bool INV, int NT, class T>
__device__ __forceinline__ void cfft_fast(cx<T>* buf, const cx<T>* tw) {
  cfft_lines<N, INV, NT, N, kPitch<N>, 1>(buf, tw);
}
template <int N, bool INV, int NT, class T>
__device__ __forceinline__ void cfft_slow(cx<T>* buf, const cx<T>* tw) {
  cfft_lines<N, INV, NT, N, 1, kPitch<N>>(buf, tw);
}

// sides with compile-time kernels (cubic grids); others use the runtime-plan kernels
#define PT_FIXED_SIZES(X) X(16) X(20) X(24) X(30) X(32) X(36) X(40) X(48) X(54) X(60) X(64)

inline bool fixed_cubic(const pt_grid& g) {
  if (g.nx != g.ny || g.nx != g.nz) return false;
  switch (g.nx) {
#define PT_CASE(n) case n:
    PT_FIXED_SIZES(PT_CASE)
#undef PT_CASE
    return true;
    default:
      return false;
  }
}

}  // namespace pt
