// Current of the velocity gauge (the observable that goes with Eq. 1's V_ext(t) as a uniform
// vector potential A): J_a = spin/Omega Re Tr[P (-i d_a + A_a)], P = Phi sigma Phi^*.
//
// With chi_j = sum_i sigma_ij phi_i (the library's rotation) the trace is
// sum_j <phi_j|(-i d_a + A_a) chi_j> = dV/Ng sum_j sum_G (G_a + A_a) conj(phi_j(G)) chi_j(G),
// so batches of (phi_j, chi_j) pairs go through forward x/y plane transforms and a z column pass
// that multiplies the two spectra and reduces (G_a + A_a) Re(conj(phi) chi) over its slab into
// FP64 per-block partials, summed on the host.  An observable evaluated once per step: the
// generic tile kernels (any 2.3.5-smooth grid up to 64 per axis) serve every size.
#include <algorithm>
#include <vector>

#include "fft.cuh"
#include "internal.h"

namespace pt {

namespace {

constexpr int NT = 512;
constexpr int MAXE = kMaxDim * kMaxDim;

// item k of the batch: phi_{j0+k/2} (k even) or chi_{j0+k/2} (k odd)
template <class T>
__global__ void __launch_bounds__(NT) k_cur_fwd_plane(GridPlan gp, const cx<T>* __restrict__ phi,
                                                      const cx<T>* __restrict__ chi, int j0,
                                                      cx<T>* __restrict__ scratch, const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf = tw + 3 * kMaxDim;
  const int z = blockIdx.x, k = blockIdx.y;
  const int nx = gp.nx, ny = gp.ny, pitch = gp.pitch_x;
  const int plane = nx * ny;
  const size_t ng = size_t(plane) * gp.nz;
  for (int t = threadIdx.x; t < nx + ny + gp.nz; t += NT) tw[t] = twg[t];
  const cx<T>* f = ((k & 1) ? chi : phi) + size_t(j0 + (k >> 1)) * ng + size_t(z) * plane;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int y = e / nx, x = e - y * nx;
    buf[y * pitch + x] = f[e];
  }
  __syncthreads();
  fft_lines<false, NT, MAXE>(buf, gp.ax[0], ny, pitch, 1, tw);
  fft_lines<false, NT, MAXE>(buf, gp.ax[1], nx, 1, pitch, tw + nx);
  cx<T>* o = scratch + size_t(k) * ng + size_t(z) * plane;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int y = e / nx, x = e - y * nx;
    o[e] = buf[y * pitch + x];
  }
}

// z transforms of both fields of pair j on slab yrow, then the (G + A)-weighted overlap of their
// spectra: part[((j * ny) + yrow) * 3 + a]
template <class T>
__global__ void __launch_bounds__(NT) k_cur_column(GridPlan gp, const cx<T>* __restrict__ scratch, double3 gstep,
                                                   double3 A, double* __restrict__ part,
                                                   const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* ba = tw + 3 * kMaxDim;
  cx<T>* bb = ba + kMaxDim * (kMaxDim + 1);
  __shared__ double red[3][NT / 32];
  const int yrow = blockIdx.x, j = blockIdx.y;
  const int nx = gp.nx, ny = gp.ny, nz = gp.nz, pitch = gp.pitch_x;
  const size_t ng = size_t(nx) * ny * nz;
  for (int t = threadIdx.x; t < nx + ny + nz; t += NT) tw[t] = twg[t];
  const cx<T>* fa = scratch + size_t(2 * j) * ng;
  const cx<T>* fb = fa + ng;
  const int slab = nz * nx;
  for (int e = threadIdx.x; e < slab; e += NT) {
    const int z = e / nx, x = e - z * nx;
    const size_t gi = (size_t(z) * ny + yrow) * nx + x;
    ba[z * pitch + x] = fa[gi];
    bb[z * pitch + x] = fb[gi];
  }
  __syncthreads();
  fft_lines<false, NT, MAXE>(ba, gp.ax[2], nx, 1, pitch, tw + nx + ny);
  fft_lines<false, NT, MAXE>(bb, gp.ax[2], nx, 1, pitch, tw + nx + ny);
  const double gy = double(wrapped_freq(yrow, ny)) * gstep.y + A.y;
  double s[3] = {0.0, 0.0, 0.0};
  for (int e = threadIdx.x; e < slab; e += NT) {
    const int z = e / nx, x = e - z * nx;
    const cx<T> a = ba[z * pitch + x], b = bb[z * pitch + x];
    const double w = double(a.re) * double(b.re) + double(a.im) * double(b.im);  // Re(conj(a) b)
    s[0] += (double(wrapped_freq(x, nx)) * gstep.x + A.x) * w;
    s[1] += gy * w;
    s[2] += (double(wrapped_freq(z, nz)) * gstep.z + A.z) * w;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[a] += __shfl_xor_sync(0xffffffffu, s[a], o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int a = 0; a < 3; ++a) red[a][w] = s[a];
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int k = 0; k < NT / 32; ++k) t += red[threadIdx.x][k];
    part[(size_t(j) * ny + yrow) * 3 + threadIdx.x] = t;
  }
}

template <class T>
void current_t(pt_ctx* ctx, const cx<T>* phi, const c128* sigma, int N, const pt_grid& g, pt_precision prec,
               const double* A, double spin, double* J, cudaStream_t st) {
  const FftTables& ft = fft_tables(ctx, g, prec);
  const size_t ng = ng_of(g);
  const size_t field = ng * sizeof(cx<T>);
  cx<T>* chi = static_cast<cx<T>*>(ctx->get("current_chi", size_t(N) * field));
  rotate<T>(ctx, phi, sigma, N, N, N, ng, c128{1.0, 0.0}, nullptr, 0, chi, st);
  const int mb = int(std::max<size_t>(1, std::min<size_t>(size_t(N), exchange_scratch_budget(ctx) / (2 * field))));
  cx<T>* scratch = static_cast<cx<T>*>(ctx->get("current_scratch", 2 * size_t(mb) * field));
  double* part = static_cast<double*>(ctx->get("current_part", size_t(mb) * g.ny * 3 * sizeof(double)));
  const size_t tile = size_t(kMaxDim) * (kMaxDim + 1) * sizeof(cx<T>);
  const size_t one = 3 * kMaxDim * sizeof(cx<T>) + tile;
  const size_t two = one + tile;
  static DeviceOnce once;
  once([&] {
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_cur_fwd_plane<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(one)));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_cur_column<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(two)));
  });
  const double two_pi = 6.283185307179586476925286766559;
  const double3 gstep = make_double3(two_pi / g.L[0], two_pi / g.L[1], two_pi / g.L[2]);
  const double3 av = A ? make_double3(A[0], A[1], A[2]) : make_double3(0.0, 0.0, 0.0);
  const cx<T>* twg = static_cast<const cx<T>*>(ft.tw);
  double acc[3] = {0.0, 0.0, 0.0};
  std::vector<double> h(size_t(mb) * g.ny * 3);
  for (int j0 = 0; j0 < N; j0 += mb) {
    const int nb = std::min(mb, N - j0);
    PT_LAUNCH(k_cur_fwd_plane<T>, dim3(g.nz, 2 * nb), NT, one, st, ft.plan, phi, chi, j0, scratch, twg);
    PT_LAUNCH(k_cur_column<T>, dim3(g.ny, nb), NT, two, st, ft.plan, scratch, gstep, av, part, twg);
    const size_t cnt = size_t(nb) * g.ny * 3;
    PT_CUDA_CHECK(cudaMemcpyAsync(h.data(), part, cnt * sizeof(double), cudaMemcpyDeviceToHost, st));
    PT_CUDA_CHECK(cudaStreamSynchronize(st));
    for (size_t k = 0; k < cnt; ++k) acc[k % 3] += h[k];
  }
  // spin/Omega * dV/Ng = spin/Ng^2
  const double f = spin / (double(ng) * double(ng));
  for (int a = 0; a < 3; ++a) J[a] = f * acc[a];
}

}  // namespace

void current(pt_ctx* ctx, const void* phi, const c128* sigma, int N, const pt_grid& g, pt_precision prec,
             const double* A, double spin, double* J, cudaStream_t st) {
  if (prec == PT_FP64)
    current_t<double>(ctx, static_cast<const c128*>(phi), sigma, N, g, prec, A, spin, J, st);
  else
    current_t<float>(ctx, static_cast<const c64*>(phi), sigma, N, g, prec, A, spin, J, st);
}

}  // namespace pt
