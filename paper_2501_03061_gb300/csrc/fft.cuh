// Mixed-radix (2,3,4,5,8) Stockham FFT stages on 2-D tiles staged in shared memory.
//
// A tile holds `nlines` lines of length n; element (line, pos) lives at
// buf[line*ls + pos*ps].  Each stage of radix R with span L (product of the
// radices already applied, m = n/(L R)) reads, for butterfly b = j + k L
// (0 <= j < L, 0 <= k < m), the inputs x[b + q n/R] (q < R), multiplies input q
// by w^{j q m} (w = exp(-+2 pi i/n)), takes a radix-R DFT and writes output p to
// y[j + k L R + p L].  Threads are laid out with the LINE index fastest, so a
// warp touches 32 different lines at the same position: stride 1 when the
// transform runs along the slow axis of the tile, stride `pitch` (odd) along
// the fast axis — both free of shared-memory bank conflicts.  All reads of a
// stage complete (barrier) before any write, so one buffer serves in place.
#pragma once

#include "common.cuh"

namespace pt {

constexpr int kMaxDim = 64;   // grid points per axis handled by the tile kernels
constexpr int kMaxStages = 6;

struct AxisPlan {
  int n;
  int nst;
  int R[kMaxStages];
  int L[kMaxStages];
};

struct GridPlan {
  AxisPlan ax[3];  // x, y, z
  int nx, ny, nz;
  int pitch_x;     // odd pitch (>= nx) of a tile whose fast axis is x
};

// host: factor n into radices 8,4,5,3,2 (in that order); returns false if n is not 2,3,5-smooth.
bool make_axis_plan(int n, AxisPlan* ap);
GridPlan make_grid_plan(const pt_grid& g);

// ------------------------------------------------------------------------------------------
// radix-R DFTs in registers; forward uses exp(-2 pi i/R), inverse exp(+2 pi i/R)
// ------------------------------------------------------------------------------------------
template <bool INV, class T>
__device__ __forceinline__ void dft2(cx<T>* a) {
  cx<T> t = a[0] - a[1];
  a[0] = a[0] + a[1];
  a[1] = t;
}

template <bool INV, class T>
__device__ __forceinline__ void dft4(cx<T>& a0, cx<T>& a1, cx<T>& a2, cx<T>& a3) {
  cx<T> s0 = a0 + a2, s1 = a0 - a2, s2 = a1 + a3, s3 = rot90<INV>(a1 - a3);
  a0 = s0 + s2;
  a2 = s0 - s2;
  a1 = s1 + s3;
  a3 = s1 - s3;
}

template <bool INV, class T>
__device__ __forceinline__ void dft3(cx<T>* a) {
  const T h = T(0.86602540378443864676);  // sin(2 pi/3)
  cx<T> s = a[1] + a[2];
  cx<T> d = rot90<INV>(a[1] - a[2]) * h;   // -+ i sin(2pi/3) (a1 - a2)
  cx<T> t = a[0] - s * T(0.5);
  a[0] = a[0] + s;
  a[1] = t + d;
  a[2] = t - d;
}

template <bool INV, class T>
__device__ __forceinline__ void dft5(cx<T>* a) {
  const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);  // cos(2pi/5), cos(4pi/5)
  const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);   // sin(2pi/5), sin(4pi/5)
  cx<T> t1 = a[1] + a[4], t2 = a[2] + a[3];
  cx<T> d1 = a[1] - a[4], d2 = a[2] - a[3];
  cx<T> b1 = a[0] + t1 * c1 + t2 * c2;
  cx<T> b2 = a[0] + t1 * c2 + t2 * c1;
  cx<T> e1 = rot90<INV>(d1 * s1 + d2 * s2);
  cx<T> e2 = rot90<INV>(d1 * s2 - d2 * s1);
  a[0] = a[0] + t1 + t2;
  a[1] = b1 + e1;
  a[4] = b1 - e1;
  a[2] = b2 + e2;
  a[3] = b2 - e2;
}

template <bool INV, class T>
__device__ __forceinline__ void dft8(cx<T>* a) {
  const T r = T(0.70710678118654752440);
  // even/odd radix-4 halves
  cx<T> e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  cx<T> o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // twiddles w8^k, k = 1, 2, 3
  cx<T> t1 = rot90<INV>(o1);                       // (+-i) o1
  o1 = (o1 + t1) * r;                              // (1 -+ i)/sqrt2 * o1
  o2 = rot90<INV>(o2);                             // -+ i
  cx<T> t3 = rot90<INV>(o3);
  o3 = (t3 - o3) * r;                              // (-1 -+ i)/sqrt2 * o3
  a[0] = e0 + o0;
  a[4] = e0 - o0;
  a[1] = e1 + o1;
  a[5] = e1 - o1;
  a[2] = e2 + o2;
  a[6] = e2 - o2;
  a[3] = e3 + o3;
  a[7] = e3 - o3;
}

template <int R, bool INV, class T>
__device__ __forceinline__ void dft(cx<T>* a) {
  if constexpr (R == 2) dft2<INV>(a);
  else if constexpr (R == 3) dft3<INV>(a);
  else if constexpr (R == 4) dft4<INV>(a[0], a[1], a[2], a[3]);
  else if constexpr (R == 5) dft5<INV>(a);
  else dft8<INV>(a);
}

// ------------------------------------------------------------------------------------------
// one Stockham stage over all lines of a tile held in shared memory
// ------------------------------------------------------------------------------------------
template <int R, bool INV, int NT, int MAXELEM, class T>
__device__ __forceinline__ void fft_stage(cx<T>* buf, int n, int L, int nlines, int ls, int ps,
                                          const cx<T>* tw) {
  constexpr int BPT = (MAXELEM / R + NT - 1) / NT;  // butterflies per thread
  const int nb = n / R;
  const int m = nb / L;
  const int total = nb * nlines;
  const int tid = threadIdx.x;
  cx<T> v[BPT][R];
#pragma unroll
  for (int u = 0; u < BPT; ++u) {
    const int f = tid + u * NT;
    if (f < total) {
      const int line = f % nlines;
      const int b = f / nlines;
      const int j = b % L;
      const cx<T>* src = buf + line * ls;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        cx<T> x = src[(b + q * nb) * ps];
        if (q > 0) {
          cx<T> w = tw[j * q * m];
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
    if (f < total) {
      const int line = f % nlines;
      const int b = f / nlines;
      const int j = b % L;
      const int k = b / L;
      dft<R, INV>(v[u]);
      cx<T>* dst = buf + line * ls;
#pragma unroll
      for (int p = 0; p < R; ++p) dst[(j + k * L * R + p * L) * ps] = v[u][p];
    }
  }
  __syncthreads();
}

// All stages of one axis.  MAXELEM bounds nlines*n (tile size in elements).
template <bool INV, int NT, int MAXELEM, class T>
__device__ __forceinline__ void fft_lines(cx<T>* buf, const AxisPlan& ap, int nlines, int ls, int ps,
                                          const cx<T>* tw) {
  for (int s = 0; s < ap.nst; ++s) {
    const int L = ap.L[s];
    switch (ap.R[s]) {
      case 8: fft_stage<8, INV, NT, MAXELEM>(buf, ap.n, L, nlines, ls, ps, tw); break;
      case 4: fft_stage<4, INV, NT, MAXELEM>(buf, ap.n, L, nlines, ls, ps, tw); break;
      case 5: fft_stage<5, INV, NT, MAXELEM>(buf, ap.n, L, nlines, ls, ps, tw); break;
      case 3: fft_stage<3, INV, NT, MAXELEM>(buf, ap.n, L, nlines, ls, ps, tw); break;
      default: fft_stage<2, INV, NT, MAXELEM>(buf, ap.n, L, nlines, ls, ps, tw); break;
    }
  }
}

// ------------------------------------------------------------------------------------------
// device tables for one grid and precision
// ------------------------------------------------------------------------------------------
template <class T>
struct GridTables {
  cx<T>* tw;   // [nx | ny | nz] forward twiddles exp(-2 pi i t/n)
  T* g2;       // [nx | ny | nz] per-axis G_a^2 = (2 pi m_a / L_a)^2
};

struct FftTables {
  pt_grid grid;
  GridPlan plan;
  void* tw = nullptr;   // cx<T>[nx+ny+nz]
  void* g2 = nullptr;   // T[nx+ny+nz]
  void* g2d = nullptr;  // double[nx+ny+nz]
  pt_precision prec;
  ~FftTables();
};

// Tables for (grid, precision) cached in the context.
const FftTables& fft_tables(pt_ctx* ctx, const pt_grid& g, pt_precision prec);
// K(G)/Ng on the whole grid (precision of prec), cached in the context.
const void* kernel_table(pt_ctx* ctx, const pt_grid& g, const pt_kernel& k, pt_precision prec);

// ------------------------------------------------------------------------------------------
// velocity-gauge kinetic factor: 1/2 |G + A|^2 = 1/2 |G|^2 + sum_a m_a c_a + a2h with
// c_a = 2 pi A_a / L_a and a2h = |A|^2 / 2 (m_a the wrapped integer frequency); A = 0 adds 0.0
// ------------------------------------------------------------------------------------------
struct KinField {
  double c[3];
  double a2h;
  int on;  // 0: A = 0, the kinetic factor is 1/2 |G|^2 and no shift is evaluated
};

__host__ __device__ __forceinline__ int wrapped_freq(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

__device__ __forceinline__ double kin_shift(const KinField& f, int x, int y, int z, int nx, int ny, int nz) {
  if (!f.on) return 0.0;
  return (double(wrapped_freq(x, nx)) * f.c[0] + double(wrapped_freq(y, ny)) * f.c[1] +
          double(wrapped_freq(z, nz)) * f.c[2]) + f.a2h;
}

// host: the shift for vector potential A (host double[3], may be null) on grid g
KinField make_kin_field(const pt_grid& g, const double* A);

}  // namespace pt
