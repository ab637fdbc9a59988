// Kinetic preconditioner of the PT-IM inner fixed-point iteration (Algorithm 1, x = T(x) of
// Sec. II-A, solved by Anderson mixing).
//
// Near the fixed point the orbital part of the residual r = T(x) - x responds to a change dPhi of
// the iterate as  -(I + i dt/2 (H - A_jj)) dPhi_j  per orbital column j (the projection term
// Phi_h S^{-1} A of Eq. lisan contributes the shift by the orbital's own energy A_jj = <phi_j|H phi_j>
// on the midpoint).  H is dominated by the kinetic term, diagonal in G, so the map
//     x -> x + M (T(x) - x),   (M r)_j = IFFT[ m_j(G) FFT(r_j) ],
//     m_j(G) = 1 / (1 + i dt/2 (|G + A|^2/2 - Re A_jj))   inside the basis sphere |G|^2/2 <= Ecut,
//     m_j(G) = 1                                           outside,
// has the same fixed points as T (M is invertible) and a much smaller spread of its Jacobian's
// spectrum, so Anderson converges in fewer iterations.  The occupation-matrix part of the residual
// is left alone.  Applied in place to the orbital residual block, in the three FFT passes of the
// Hamiltonian kernels (plane, column with the multiplier, inverse plane), one field per orbital.
#include <algorithm>

#include "fft.cuh"
#include "fft_fixed.cuh"
#include "internal.h"

namespace pt {

namespace {

// m_j(G) * inv_ng for the kinetic factor kin = |G + A|^2/2 of a point inside the sphere
template <class T>
__device__ __forceinline__ cx<T> pc_factor(double kin, double shift, double dt, double inv_ng) {
  const double th = 0.5 * dt * (kin - shift);
  const double s = inv_ng / (1.0 + th * th);
  return cx<T>{T(s), T(-th * s)};  // (1 - i th) / (1 + th^2)
}

// ---------------------------------------------------------------- compile-time cubic sides ----

constexpr int FT = 256;

template <int N, class T>
constexpr size_t pc_tile_bytes() {
  return size_t(N) * kPitch<N> * sizeof(cx<T>);
}

template <int N, class T>
__global__ void __launch_bounds__(FT) k_pc_fwd_plane(const cx<T>* __restrict__ r, int j0, cx<T>* __restrict__ scratch,
                                                     const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = buf + N * kPitch<N>;
  constexpr int PL = N * N;
  constexpr size_t NG = size_t(N) * N * N;
  const int z = blockIdx.x, k = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += FT) tw[t] = twg[t];
  const cx<T>* f = r + size_t(j0 + k) * NG + size_t(z) * PL;
#pragma unroll 8
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int yy = e / N, x = e - yy * N;
    buf[yy * kPitch<N> + x] = f[e];
  }
  __syncthreads();
  cfft_fast<N, false, FT>(buf, tw);
  cfft_slow<N, false, FT>(buf, tw);
  cx<T>* o = scratch + size_t(k) * NG + size_t(z) * PL;
#pragma unroll 8
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int yy = e / N, x = e - yy * N;
    o[e] = buf[yy * kPitch<N> + x];
  }
}

template <int N, class T>
__global__ void __launch_bounds__(FT) k_pc_column(cx<T>* __restrict__ scratch, const double* __restrict__ g2,
                                                  double ecut, KinField kf, double dt, const c128* __restrict__ A,
                                                  int lda, int j0, const cx<T>* __restrict__ twg,
                                                  const unsigned long long* __restrict__ masks) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* ba = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = ba + N * kPitch<N>;
  constexpr size_t NG = size_t(N) * N * N;
  constexpr double inv_ng = 1.0 / double(NG);
  const int yrow = blockIdx.x, k = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += FT) tw[t] = twg[t];
  const double shift = A[size_t(j0 + k) * lda + (j0 + k)].re;
  // FP32 form: the sphere test from the exact FP64 masks, the factor in FP32 from per-axis kinetic
  // terms (M only chooses the iteration path, so FP32 rounding of it leaves the fixed point alone;
  // an FP64 division per grid point would set this pass's time on this part's FP64 pipe)
  __shared__ unsigned long long mrow[N];
  __shared__ float kx[N], kz[N];
  __shared__ float ky;
  if constexpr (sizeof(T) == 4) {
    for (int t = threadIdx.x; t < N; t += FT) {
      mrow[t] = masks[size_t(yrow) * N + t];
      const double w = double(wrapped_freq(t, N));
      kx[t] = float(0.5 * g2[t] + (kf.on ? w * kf.c[0] : 0.0));
      kz[t] = float(0.5 * g2[2 * N + t] + (kf.on ? w * kf.c[2] : 0.0));
    }
    if (threadIdx.x == 0)
      ky = float(0.5 * g2[N + yrow] + (kf.on ? double(wrapped_freq(yrow, N)) * kf.c[1] + kf.a2h : 0.0) - shift);
  }
  cx<T>* fa = scratch + size_t(k) * NG;
#pragma unroll 8
  for (int e = threadIdx.x; e < N * N; e += FT) {
    const int z = e / N, x = e - z * N;
    ba[z * kPitch<N> + x] = fa[(size_t(z) * N + yrow) * N + x];
  }
  __syncthreads();
  cfft_slow<N, false, FT>(ba, tw);
  if constexpr (sizeof(T) == 4) {
    const float hdt = float(0.5 * dt), fng = float(inv_ng);
#pragma unroll 8
    for (int e = threadIdx.x; e < N * N; e += FT) {
      const int z = e / N, x = e - z * N;
      const cx<T> v = ba[z * kPitch<N> + x];
      if ((mrow[x] >> z) & 1ull) {
        // (1 - i th) / (1 + th^2) / Ng with th = dt/2 (|G + A|^2/2 - Re A_kk)
        const float th = hdt * (kx[x] + (ky + kz[z]));
        const float sc = fng / (1.f + th * th);
        ba[z * kPitch<N> + x] = cmul(v, cx<T>{sc, -th * sc});
      } else {
        ba[z * kPitch<N> + x] = v * fng;
      }
    }
  } else {
    // |G|^2 and the sphere test in FP64, as in the Hamiltonian kernels
    const double* g2x = g2;
    const double* g2y = g2 + N;
    const double* g2z = g2 + 2 * N;
#pragma unroll 8
    for (int e = threadIdx.x; e < N * N; e += FT) {
      const int z = e / N, x = e - z * N;
      const double half = 0.5 * (g2x[x] + g2y[yrow] + g2z[z]);
      const cx<T> v = ba[z * kPitch<N> + x];
      ba[z * kPitch<N> + x] = half <= ecut ? cmul(v, pc_factor<T>(half + kin_shift(kf, x, yrow, z, N, N, N), shift,
                                                                   dt, inv_ng))
                                           : v * T(inv_ng);
    }
  }
  __syncthreads();
  cfft_slow<N, true, FT>(ba, tw);
#pragma unroll 8
  for (int e = threadIdx.x; e < N * N; e += FT) {
    const int z = e / N, x = e - z * N;
    fa[(size_t(z) * N + yrow) * N + x] = ba[z * kPitch<N> + x];
  }
}

template <int N, class T>
__global__ void __launch_bounds__(FT) k_pc_inv_plane(const cx<T>* __restrict__ scratch, int j0, cx<T>* __restrict__ out,
                                                     const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = buf + N * kPitch<N>;
  constexpr int PL = N * N;
  constexpr size_t NG = size_t(N) * N * N;
  const int z = blockIdx.x, k = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += FT) tw[t] = twg[t];
  const cx<T>* f = scratch + size_t(k) * NG + size_t(z) * PL;
#pragma unroll 8
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int yy = e / N, x = e - yy * N;
    buf[yy * kPitch<N> + x] = f[e];
  }
  __syncthreads();
  cfft_slow<N, true, FT>(buf, tw);
  cfft_fast<N, true, FT>(buf, tw);
  cx<T>* o = out + size_t(j0 + k) * NG + size_t(z) * PL;
#pragma unroll 8
  for (int e = threadIdx.x; e < PL; e += FT) {
    const int yy = e / N, x = e - yy * N;
    o[e] = buf[yy * kPitch<N> + x];
  }
}

template <int N, class T>
void pc_batch_n(cx<T>* r, int j0, int nb, cx<T>* scratch, const double* g2d, double ecut, KinField kf, double dt,
                const c128* A, int lda, const cx<T>* tw, cudaStream_t st, const unsigned long long* masks) {
  static DeviceOnce once;
  const size_t one = pc_tile_bytes<N, T>() + N * sizeof(cx<T>);
  once([&] {
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pc_fwd_plane<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(one)));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pc_column<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(one)));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pc_inv_plane<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(one)));
  });
  PT_LAUNCH((k_pc_fwd_plane<N, T>), dim3(N, nb), FT, one, st, r, j0, scratch, tw);
  PT_LAUNCH((k_pc_column<N, T>), dim3(N, nb), FT, one, st, scratch, g2d, ecut, kf, dt, A, lda, j0, tw, masks);
  PT_LAUNCH((k_pc_inv_plane<N, T>), dim3(N, nb), FT, one, st, scratch, j0, r, tw);
}

template <class T>
void pc_batch_fixed(int n, cx<T>* r, int j0, int nb, cx<T>* scratch, const double* g2d, double ecut, KinField kf,
                    double dt, const c128* A, int lda, const cx<T>* tw, cudaStream_t st,
                    const unsigned long long* masks) {
  if (sizeof(T) == 4 && !masks) fail(PT_INVALID_ARG, "FP32 column pass without its sphere masks");
  switch (n) {
#define PT_CASE(s)                                                                  \
  case s:                                                                           \
    pc_batch_n<s, T>(r, j0, nb, scratch, g2d, ecut, kf, dt, A, lda, tw, st, masks); \
    return;
    PT_FIXED_SIZES(PT_CASE)
#undef PT_CASE
    default:
      fail(PT_INVALID_ARG, "no compile-time FFT kernels for this grid side");
  }
}

// ---------------------------------------------------------------- any other grid ----

constexpr int NT = 512;
constexpr int MAXE = kMaxDim * kMaxDim;

size_t pc_tile_generic(size_t esize) { return size_t(kMaxDim) * (kMaxDim + 1) * esize; }

template <class T>
__global__ void __launch_bounds__(NT) k_pcg_fwd_plane(GridPlan gp, const cx<T>* __restrict__ r, int j0,
                                                      cx<T>* __restrict__ scratch, const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf = tw + 3 * kMaxDim;
  const int z = blockIdx.x, k = blockIdx.y;
  const int nx = gp.nx, ny = gp.ny, pitch = gp.pitch_x;
  const int plane = nx * ny;
  const size_t ng = size_t(plane) * gp.nz;
  for (int t = threadIdx.x; t < nx + ny + gp.nz; t += NT) tw[t] = twg[t];
  const cx<T>* f = r + size_t(j0 + k) * ng + size_t(z) * plane;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int yy = e / nx, x = e - yy * nx;
    buf[yy * pitch + x] = f[e];
  }
  __syncthreads();
  fft_lines<false, NT, MAXE>(buf, gp.ax[0], ny, pitch, 1, tw);
  fft_lines<false, NT, MAXE>(buf, gp.ax[1], nx, 1, pitch, tw + nx);
  cx<T>* o = scratch + size_t(k) * ng + size_t(z) * plane;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int yy = e / nx, x = e - yy * nx;
    o[e] = buf[yy * pitch + x];
  }
}

template <class T>
__global__ void __launch_bounds__(NT) k_pcg_column(GridPlan gp, cx<T>* __restrict__ scratch,
                                                   const double* __restrict__ g2, double ecut, KinField kf, double dt,
                                                   const c128* __restrict__ A, int lda, int j0,
                                                   const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* ba = tw + 3 * kMaxDim;
  const int yrow = blockIdx.x, k = blockIdx.y;
  const int nx = gp.nx, ny = gp.ny, nz = gp.nz, pitch = gp.pitch_x;
  const size_t ng = size_t(nx) * ny * nz;
  const double inv_ng = 1.0 / double(ng);
  for (int t = threadIdx.x; t < nx + ny + nz; t += NT) tw[t] = twg[t];
  const double shift = A[size_t(j0 + k) * lda + (j0 + k)].re;
  cx<T>* fa = scratch + size_t(k) * ng;
  const int slab = nz * nx;
  for (int e = threadIdx.x; e < slab; e += NT) {
    const int z = e / nx, x = e - z * nx;
    ba[z * pitch + x] = fa[(size_t(z) * ny + yrow) * nx + x];
  }
  __syncthreads();
  fft_lines<false, NT, MAXE>(ba, gp.ax[2], nx, 1, pitch, tw + nx + ny);
  const double* g2x = g2;
  const double* g2y = g2 + nx;
  const double* g2z = g2 + nx + ny;
  for (int e = threadIdx.x; e < slab; e += NT) {
    const int z = e / nx, x = e - z * nx;
    const double half = 0.5 * (g2x[x] + g2y[yrow] + g2z[z]);
    const cx<T> v = ba[z * pitch + x];
    ba[z * pitch + x] = half <= ecut
                            ? cmul(v, pc_factor<T>(half + kin_shift(kf, x, yrow, z, nx, ny, nz), shift, dt, inv_ng))
                            : v * T(inv_ng);
  }
  __syncthreads();
  fft_lines<true, NT, MAXE>(ba, gp.ax[2], nx, 1, pitch, tw + nx + ny);
  for (int e = threadIdx.x; e < slab; e += NT) {
    const int z = e / nx, x = e - z * nx;
    fa[(size_t(z) * ny + yrow) * nx + x] = ba[z * pitch + x];
  }
}

template <class T>
__global__ void __launch_bounds__(NT) k_pcg_inv_plane(GridPlan gp, const cx<T>* __restrict__ scratch, int j0,
                                                      cx<T>* __restrict__ out, const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf = tw + 3 * kMaxDim;
  const int z = blockIdx.x, k = blockIdx.y;
  const int nx = gp.nx, ny = gp.ny, pitch = gp.pitch_x;
  const int plane = nx * ny;
  const size_t ng = size_t(plane) * gp.nz;
  for (int t = threadIdx.x; t < nx + ny + gp.nz; t += NT) tw[t] = twg[t];
  const cx<T>* f = scratch + size_t(k) * ng + size_t(z) * plane;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int yy = e / nx, x = e - yy * nx;
    buf[yy * pitch + x] = f[e];
  }
  __syncthreads();
  fft_lines<true, NT, MAXE>(buf, gp.ax[1], nx, 1, pitch, tw + nx);
  fft_lines<true, NT, MAXE>(buf, gp.ax[0], ny, pitch, 1, tw);
  cx<T>* o = out + size_t(j0 + k) * ng + size_t(z) * plane;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int yy = e / nx, x = e - yy * nx;
    o[e] = buf[yy * pitch + x];
  }
}

template <class T>
void precondition_t(pt_ctx* ctx, cx<T>* r, int N, const c128* A, double dt, double ecut, const pt_grid& g,
                    pt_precision prec, cudaStream_t st, const double* Avec) {
  const KinField kf = make_kin_field(g, Avec);
  const FftTables& ft = fft_tables(ctx, g, prec);
  const size_t ng = ng_of(g);
  const size_t field = ng * sizeof(cx<T>);
  // the Hamiltonian's scratch (two fields per orbital of its batch) holds one field per orbital here
  const size_t budget = exchange_scratch_budget(ctx);
  const int mb = std::min<int>(N, int(std::max<size_t>(1, budget / (2 * field))));
  cx<T>* scratch = static_cast<cx<T>*>(ctx->get("h_scratch", 2 * size_t(mb) * field));
  const int pb = std::min(N, 2 * mb);
  const cx<T>* twg = static_cast<const cx<T>*>(ft.tw);
  const double* g2d = static_cast<const double*>(ft.g2d);
  if (fixed_cubic(g)) {
    const unsigned long long* masks = sizeof(T) == 4 ? sphere_masks(ctx, g, g2d, ecut, st) : nullptr;
    for (int j0 = 0; j0 < N; j0 += pb)
      pc_batch_fixed<T>(g.nx, r, j0, std::min(pb, N - j0), scratch, g2d, ecut, kf, dt, A, N, twg, st, masks);
    return;
  }
  static DeviceOnce once;
  const size_t one = 3 * kMaxDim * sizeof(cx<T>) + pc_tile_generic(sizeof(cx<T>));
  once([&] {
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pcg_fwd_plane<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(one)));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pcg_column<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(one)));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_pcg_inv_plane<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(one)));
  });
  for (int j0 = 0; j0 < N; j0 += pb) {
    const int nb = std::min(pb, N - j0);
    PT_LAUNCH(k_pcg_fwd_plane<T>, dim3(g.nz, nb), NT, one, st, ft.plan, r, j0, scratch, twg);
    PT_LAUNCH(k_pcg_column<T>, dim3(g.ny, nb), NT, one, st, ft.plan, scratch, g2d, ecut, kf, dt, A, N, j0, twg);
    PT_LAUNCH(k_pcg_inv_plane<T>, dim3(g.nz, nb), NT, one, st, ft.plan, scratch, j0, r, twg);
  }
}

}  // namespace

void precondition_residual(pt_ctx* ctx, void* r, int N, const c128* A, double dt, double ecut, const pt_grid& g,
                           pt_precision prec, cudaStream_t st, const double* Avec) {
  if (prec == PT_FP64)
    precondition_t<double>(ctx, static_cast<c128*>(r), N, A, dt, ecut, g, prec, st, Avec);
  else
    precondition_t<float>(ctx, static_cast<c64*>(r), N, A, dt, ecut, g, prec, st, Avec);
}

}  // namespace pt
