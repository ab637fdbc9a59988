// Self-consistent local potential of Eq. 1: rho(r) = spin * P(r, r) with P = Phi sigma Phi^*,
// V_Hxc[rho] = V_H + v_xc, V_H the periodic Hartree potential (Poisson equation in G space with the
// G = 0 term removed by the neutralising background) and v_xc the LDA (Slater exchange plus the
// Perdew-Zunger 1981 fit of the Ceperley-Alder correlation energy of the unpolarised gas).
//
// Density: chi = Phi sigma (the library's rotation, tensor cores in the FP32 forms), then
// rho(r) = spin * Re sum_j chi_j(r) conj(phi_j(r)) in one streaming pass over both blocks
// (2 N Ng complex reads, HBM bound), products in the block's precision and sums in FP64.
// Potential: one FP64 3-D FFT of rho through the generic tile kernels (x/y plane pass, z column
// pass that applies 4 pi/|G|^2 / Ng and transforms back, inverse y/x plane pass), whose last pass
// also evaluates the LDA point by point, adds V_loc and writes the total local potential, with
// per-plane partial sums of the Hartree and xc energies.  All of it is Ng-sized work.
#include <algorithm>

#include "fft.cuh"
#include "internal.h"

namespace pt {

namespace {

constexpr int NT = 512;
constexpr int MAXE = kMaxDim * kMaxDim;
constexpr double kPi = 3.14159265358979323846;

// Perdew-Zunger correlation of the unpolarised gas (rs >= 1: gamma/(1 + beta1 sqrt(rs) + beta2 rs);
// rs < 1: A ln rs + B + C rs ln rs + D rs) and the Slater exchange; v = d(rho eps)/d rho.
__device__ __forceinline__ void lda_point(double rho, double& eps, double& v) {
  if (!(rho > 1e-30)) {
    eps = 0.0;
    v = 0.0;
    return;
  }
  const double ex = -0.75 * cbrt(3.0 * rho / kPi);
  const double rs = cbrt(3.0 / (4.0 * kPi * rho));
  double ec, vc;
  if (rs >= 1.0) {
    const double gamma = -0.1423, b1 = 1.0529, b2 = 0.3334;
    const double s = sqrt(rs);
    const double den = 1.0 + b1 * s + b2 * rs;
    ec = gamma / den;
    vc = ec * (1.0 + (7.0 / 6.0) * b1 * s + (4.0 / 3.0) * b2 * rs) / den;
  } else {
    const double a = 0.0311, b = -0.048, c = 0.0020, d = -0.0116;
    const double l = log(rs);
    ec = a * l + b + c * rs * l + d * rs;
    vc = a * l + (b - a / 3.0) + (2.0 / 3.0) * c * rs * l + (2.0 * d - c) / 3.0 * rs;
  }
  eps = ex + ec;
  v = (4.0 / 3.0) * ex + vc;
}

template <class T>
__global__ void __launch_bounds__(256) k_density(const cx<T>* __restrict__ chi, const cx<T>* __restrict__ phi, int N,
                                                 size_t ng, double spin, double* __restrict__ rho) {
  for (size_t r = size_t(blockIdx.x) * blockDim.x + threadIdx.x; r < ng; r += size_t(gridDim.x) * blockDim.x) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int j = 0;
    for (; j + 4 <= N; j += 4) {
      cx<T> a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = chi[size_t(j + u) * ng + r];
        b[u] = phi[size_t(j + u) * ng + r];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += double(a[u].re * b[u].re + a[u].im * b[u].im);
    }
    for (; j < N; ++j) {
      const cx<T> a = chi[size_t(j) * ng + r], b = phi[size_t(j) * ng + r];
      acc[0] += double(a.re * b.re + a.im * b.im);
    }
    rho[r] = spin * ((acc[0] + acc[1]) + (acc[2] + acc[3]));
  }
}

__global__ void __launch_bounds__(NT) k_hxc_fwd_plane(GridPlan gp, const double* __restrict__ rho,
                                                      c128* __restrict__ scratch, const c128* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  c128* tw = reinterpret_cast<c128*>(smem_raw);
  c128* buf = tw + 3 * kMaxDim;
  const int z = blockIdx.x;
  const int nx = gp.nx, ny = gp.ny, pitch = gp.pitch_x;
  const int plane = nx * ny;
  for (int t = threadIdx.x; t < nx + ny + gp.nz; t += NT) tw[t] = twg[t];
  const double* f = rho + size_t(z) * plane;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int y = e / nx, x = e - y * nx;
    buf[y * pitch + x] = c128{f[e], 0.0};
  }
  __syncthreads();
  fft_lines<false, NT, MAXE>(buf, gp.ax[0], ny, pitch, 1, tw);
  fft_lines<false, NT, MAXE>(buf, gp.ax[1], nx, 1, pitch, tw + nx);
  c128* o = scratch + size_t(z) * plane;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int y = e / nx, x = e - y * nx;
    o[e] = buf[y * pitch + x];
  }
}

__global__ void __launch_bounds__(NT) k_hxc_column(GridPlan gp, c128* __restrict__ scratch,
                                                   const double* __restrict__ g2, double inv_ng,
                                                   const c128* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  c128* tw = reinterpret_cast<c128*>(smem_raw);
  c128* buf = tw + 3 * kMaxDim;
  const int yrow = blockIdx.x;
  const int nx = gp.nx, ny = gp.ny, nz = gp.nz, pitch = gp.pitch_x;
  for (int t = threadIdx.x; t < nx + ny + nz; t += NT) tw[t] = twg[t];
  const int slab = nz * nx;
  for (int e = threadIdx.x; e < slab; e += NT) {
    const int z = e / nx, x = e - z * nx;
    buf[z * pitch + x] = scratch[(size_t(z) * ny + yrow) * nx + x];
  }
  __syncthreads();
  fft_lines<false, NT, MAXE>(buf, gp.ax[2], nx, 1, pitch, tw + nx + ny);
  const double* g2x = g2;
  const double* g2y = g2 + nx;
  const double* g2z = g2 + nx + ny;
  for (int e = threadIdx.x; e < slab; e += NT) {
    const int z = e / nx, x = e - z * nx;
    const double G2 = g2x[x] + g2y[yrow] + g2z[z];
    const double k = G2 > 0.0 ? 4.0 * kPi / G2 * inv_ng : 0.0;
    buf[z * pitch + x] = buf[z * pitch + x] * k;
  }
  __syncthreads();
  fft_lines<true, NT, MAXE>(buf, gp.ax[2], nx, 1, pitch, tw + nx + ny);
  for (int e = threadIdx.x; e < slab; e += NT) {
    const int z = e / nx, x = e - z * nx;
    scratch[(size_t(z) * ny + yrow) * nx + x] = buf[z * pitch + x];
  }
}

// inverse y/x transforms of a plane, LDA, V_loc; optional per-plane energy sums part[2 z + {0, 1}]
__global__ void __launch_bounds__(NT) k_hxc_inv_plane(GridPlan gp, const c128* __restrict__ scratch,
                                                      const double* __restrict__ rho, const double* __restrict__ vloc,
                                                      double* __restrict__ vout, double* __restrict__ part,
                                                      const c128* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  c128* tw = reinterpret_cast<c128*>(smem_raw);
  c128* buf = tw + 3 * kMaxDim;
  __shared__ double red[2][NT / 32];
  const int z = blockIdx.x;
  const int nx = gp.nx, ny = gp.ny, pitch = gp.pitch_x;
  const int plane = nx * ny;
  for (int t = threadIdx.x; t < nx + ny + gp.nz; t += NT) tw[t] = twg[t];
  const c128* f = scratch + size_t(z) * plane;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int y = e / nx, x = e - y * nx;
    buf[y * pitch + x] = f[e];
  }
  __syncthreads();
  fft_lines<true, NT, MAXE>(buf, gp.ax[1], nx, 1, pitch, tw + nx);
  fft_lines<true, NT, MAXE>(buf, gp.ax[0], ny, pitch, 1, tw);
  const size_t off = size_t(z) * plane;
  double eh = 0.0, exc = 0.0;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int y = e / nx, x = e - y * nx;
    const double vh = buf[y * pitch + x].re;
    const double r = rho[off + e];
    double eps, vxc;
    lda_point(r, eps, vxc);
    vout[off + e] = (vloc ? vloc[off + e] : 0.0) + vh + vxc;
    eh += 0.5 * r * vh;
    exc += r * eps;
  }
  if (!part) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    eh += __shfl_xor_sync(0xffffffffu, eh, o);
    exc += __shfl_xor_sync(0xffffffffu, exc, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = eh;
    red[1][w] = exc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < NT / 32; ++k) {
      a += red[0][k];
      b += red[1][k];
    }
    part[2 * z] = a;
    part[2 * z + 1] = b;
  }
}

size_t tile_bytes() { return size_t(kMaxDim) * (kMaxDim + 1) * sizeof(c128) + 3 * kMaxDim * sizeof(c128); }

void set_attrs() {
  static DeviceOnce once;
  once([] {
    const int b = int(tile_bytes());
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_hxc_fwd_plane, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_hxc_column, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_hxc_inv_plane, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
  });
}

}  // namespace

template <class T>
void density(pt_ctx* ctx, const cx<T>* phi, const c128* sigma, int N, size_t ng, double spin, cx<T>* chi,
             double* rho, cudaStream_t st) {
  // chi_j = sum_i sigma_ij phi_i
  rotate<T>(ctx, phi, sigma, N, N, N, ng, c128{1.0, 0.0}, nullptr, 0, chi, st);
  const int blocks = int(std::max<size_t>(1, std::min<size_t>((ng + 255) / 256, size_t(ctx->num_sms) * 16)));
  PT_LAUNCH(k_density<T>, blocks, 256, 0, st, chi, phi, N, ng, spin, rho);
}

template void density<float>(pt_ctx*, const c64*, const c128*, int, size_t, double, c64*, double*, cudaStream_t);
template void density<double>(pt_ctx*, const c128*, const c128*, int, size_t, double, c128*, double*, cudaStream_t);

void hxc_potential(pt_ctx* ctx, const double* rho, const double* vloc, const pt_grid& g, double* v, double* part,
                   cudaStream_t st) {
  const FftTables& ft = fft_tables(ctx, g, PT_FP64);
  const size_t ng = ng_of(g);
  c128* scratch = static_cast<c128*>(ctx->get("hxc_scratch", ng * sizeof(c128)));
  set_attrs();
  const size_t smem = tile_bytes();
  const c128* tw = static_cast<const c128*>(ft.tw);
  PT_LAUNCH(k_hxc_fwd_plane, g.nz, NT, smem, st, ft.plan, rho, scratch, tw);
  PT_LAUNCH(k_hxc_column, g.ny, NT, smem, st, ft.plan, scratch, static_cast<const double*>(ft.g2d),
            1.0 / double(ng), tw);
  PT_LAUNCH(k_hxc_inv_plane, g.nz, NT, smem, st, ft.plan, scratch, rho, vloc, v, part, tw);
}

}  // namespace pt
