// H psi = P_sph[ 1/2 (-i grad + A)^2 psi + V_loc psi + alpha V_x psi ]   (Eq. 1; V_ext(t) as the
// uniform vector potential A of the velocity gauge, V_Hxc inside V_loc).
//
// With y = V_loc psi + alpha X (X = V_ACE psi or V_x psi, computed by the caller):
//   out = IFFT( mask(G) * ( |G + A|^2/2 * FFT(psi) + FFT(y) ) / Ng ),  mask = [|G|^2/2 <= Ecut]
// (the basis sphere does not move with A).
// The three FFT passes follow the exchange kernels: x/y plane transforms of both
// fields, one column kernel that transforms both along z, combines them in G space
// and transforms back along z, and an inverse plane pass that writes the result.
#include <algorithm>

#include "fft.cuh"
#include "fft_fixed.cuh"
#include "internal.h"

namespace pt {

// compile-time-size passes for cubic grids (hamiltonian_fixed.cu)
template <class T>
void apply_h_batch_fixed(int n, const cx<T>* psi, const T* vloc, const cx<T>* X, double alpha, int j0, int nb,
                         cx<T>* scratch, const double* g2d, double ecut, KinField kf, const cx<T>* tw, cx<T>* out,
                         cudaStream_t st, const unsigned long long* masks);

namespace {

__global__ void k_sphere_masks(const double* __restrict__ g2, int n, double ecut, unsigned long long* __restrict__ m) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int y = e / n, x = e % n;
  unsigned long long bits = 0;
  for (int z = 0; z < n; ++z)
    if (0.5 * (g2[x] + g2[n + y] + g2[2 * n + z]) <= ecut) bits |= 1ull << z;
  m[e] = bits;
}

// V_loc in the orbital precision (the FP32 passes multiply by the FP32-rounded value either way)
__global__ void k_to_float(const double* __restrict__ a, size_t n, float* __restrict__ b) {
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x)
    b[e] = float(a[e]);
}

struct SphereMasks {
  unsigned long long* d = nullptr;
  ~SphereMasks() { cudaFree(d); }
};

constexpr int NT = 512;
constexpr int MAXE = kMaxDim * kMaxDim;

// item k of the batch: field psi_{j0+k/2} (k even) or y_{j0+k/2} (k odd)
template <class T>
__global__ void __launch_bounds__(NT) k_h_fwd_plane(GridPlan gp, const cx<T>* __restrict__ psi,
                                                    const double* __restrict__ vloc, const cx<T>* __restrict__ X,
                                                    T alpha, int j0, cx<T>* __restrict__ scratch,
                                                    const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf = tw + 3 * kMaxDim;
  const int z = blockIdx.x, k = blockIdx.y;
  const int nx = gp.nx, ny = gp.ny, pitch = gp.pitch_x;
  const int plane = nx * ny;
  const size_t ng = size_t(plane) * gp.nz;
  for (int t = threadIdx.x; t < nx + ny + gp.nz; t += NT) tw[t] = twg[t];
  const size_t off = size_t(j0 + (k >> 1)) * ng + size_t(z) * plane;
  const cx<T>* f = psi + off;
  if (k & 1) {  // y = V_loc psi + alpha X
    const double* v = vloc + size_t(z) * plane;
    const cx<T>* xx = X ? X + off : nullptr;
    for (int e = threadIdx.x; e < plane; e += NT) {
      const int yy = e / nx, x = e - yy * nx;
      cx<T> val = f[e] * T(v[e]);
      if (xx) val = val + xx[e] * alpha;
      buf[yy * pitch + x] = val;
    }
  } else {
    for (int e = threadIdx.x; e < plane; e += NT) {
      const int yy = e / nx, x = e - yy * nx;
      buf[yy * pitch + x] = f[e];
    }
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
__global__ void __launch_bounds__(NT) k_h_column(GridPlan gp, cx<T>* __restrict__ scratch,
                                                 const double* __restrict__ g2, double ecut, KinField kf, T inv_ng,
                                                 const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* ba = tw + 3 * kMaxDim;
  cx<T>* bb = ba + kMaxDim * (kMaxDim + 1);
  const int yrow = blockIdx.x, j = blockIdx.y;
  const int nx = gp.nx, ny = gp.ny, nz = gp.nz, pitch = gp.pitch_x;
  const size_t ng = size_t(nx) * ny * nz;
  for (int t = threadIdx.x; t < nx + ny + nz; t += NT) tw[t] = twg[t];
  cx<T>* fa = scratch + size_t(2 * j) * ng;
  cx<T>* fb = fa + ng;
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
  // |G|^2 and the sphere test in FP64 so that the cutoff boundary does not depend on the precision
  const double* g2x = g2;
  const double* g2y = g2 + nx;
  const double* g2z = g2 + nx + ny;
  for (int e = threadIdx.x; e < slab; e += NT) {
    const int z = e / nx, x = e - z * nx;
    const double half = 0.5 * (g2x[x] + g2y[yrow] + g2z[z]);
    cx<T> v = czero<T>();
    if (half <= ecut) {
      const double kin = half + kin_shift(kf, x, yrow, z, nx, ny, nz);  // 1/2 |G + A|^2
      v = (ba[z * pitch + x] * T(kin) + bb[z * pitch + x]) * inv_ng;
    }
    ba[z * pitch + x] = v;
  }
  __syncthreads();
  fft_lines<true, NT, MAXE>(ba, gp.ax[2], nx, 1, pitch, tw + nx + ny);
  for (int e = threadIdx.x; e < slab; e += NT) {
    const int z = e / nx, x = e - z * nx;
    fa[(size_t(z) * ny + yrow) * nx + x] = ba[z * pitch + x];
  }
}

template <class T>
__global__ void __launch_bounds__(NT) k_h_inv_plane(GridPlan gp, const cx<T>* __restrict__ scratch, int j0,
                                                    cx<T>* __restrict__ out, const cx<T>* __restrict__ twg) {
  extern __shared__ unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf = tw + 3 * kMaxDim;
  const int z = blockIdx.x, j = blockIdx.y;
  const int nx = gp.nx, ny = gp.ny, pitch = gp.pitch_x;
  const int plane = nx * ny;
  const size_t ng = size_t(plane) * gp.nz;
  for (int t = threadIdx.x; t < nx + ny + gp.nz; t += NT) tw[t] = twg[t];
  const cx<T>* f = scratch + size_t(2 * j) * ng + size_t(z) * plane;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int yy = e / nx, x = e - yy * nx;
    buf[yy * pitch + x] = f[e];
  }
  __syncthreads();
  fft_lines<true, NT, MAXE>(buf, gp.ax[1], nx, 1, pitch, tw + nx);
  fft_lines<true, NT, MAXE>(buf, gp.ax[0], ny, pitch, 1, tw);
  cx<T>* o = out + size_t(j0 + j) * ng + size_t(z) * plane;
  for (int e = threadIdx.x; e < plane; e += NT) {
    const int yy = e / nx, x = e - yy * nx;
    o[e] = buf[yy * pitch + x];
  }
}

size_t tile_bytes(size_t esize) { return size_t(kMaxDim) * (kMaxDim + 1) * esize; }

template <class T>
void set_attrs() {
  static DeviceOnce once;
  once([] {
    const int one = int(3 * kMaxDim * sizeof(cx<T>) + tile_bytes(sizeof(cx<T>)));
    const int two = int(3 * kMaxDim * sizeof(cx<T>) + 2 * tile_bytes(sizeof(cx<T>)));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_h_fwd_plane<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, one));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_h_inv_plane<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, one));
    PT_CUDA_CHECK(cudaFuncSetAttribute(k_h_column<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, two));
  });
}

template <class T>
void apply_h_t(pt_ctx* ctx, const cx<T>* psi, int M, cx<T>* out, const double* vloc, const cx<T>* X, double alpha,
               double ecut, const pt_grid& g, pt_precision prec, cudaStream_t st, const double* A) {
  const KinField kf = make_kin_field(g, A);
  const FftTables& ft = fft_tables(ctx, g, prec);
  const size_t ng = ng_of(g);
  const size_t field = ng * sizeof(cx<T>);
  const size_t budget = exchange_scratch_budget(ctx);
  int mb = int(std::max<size_t>(1, budget / (2 * field)));
  mb = std::min(mb, M);
  cx<T>* scratch = static_cast<cx<T>*>(ctx->get("h_scratch", 2 * size_t(mb) * field));
  if (fixed_cubic(g)) {
    const unsigned long long* masks = nullptr;
    const T* vl = nullptr;
    if constexpr (sizeof(T) == 4) {
      masks = sphere_masks(ctx, g, static_cast<const double*>(ft.g2d), ecut, st);
      float* v32 = static_cast<float*>(ctx->get("h_vloc32", ng * sizeof(float)));
      PT_LAUNCH(k_to_float, int(std::min<size_t>((ng + 255) / 256, size_t(ctx->num_sms) * 8)), 256, 0, st, vloc, ng,
                v32);
      vl = v32;
    } else {
      vl = vloc;
    }
    for (int j0 = 0; j0 < M; j0 += mb)
      apply_h_batch_fixed<T>(g.nx, psi, vl, X, alpha, j0, std::min(mb, M - j0), scratch,
                             static_cast<const double*>(ft.g2d), ecut, kf, static_cast<const cx<T>*>(ft.tw), out, st,
                             masks);
    return;
  }
  set_attrs<T>();
  const size_t one = 3 * kMaxDim * sizeof(cx<T>) + tile_bytes(sizeof(cx<T>));
  const size_t two = one + tile_bytes(sizeof(cx<T>));
  const cx<T>* twg = static_cast<const cx<T>*>(ft.tw);
  for (int j0 = 0; j0 < M; j0 += mb) {
    const int nb = std::min(mb, M - j0);
    PT_LAUNCH(k_h_fwd_plane<T>, dim3(g.nz, 2 * nb), NT, one, st, ft.plan, psi, vloc, X, T(alpha), j0, scratch,
              twg);
    PT_LAUNCH(k_h_column<T>, dim3(g.ny, nb), NT, two, st, ft.plan, scratch, static_cast<const double*>(ft.g2d), ecut,
              kf, T(1.0 / double(ng)), twg);
    PT_LAUNCH(k_h_inv_plane<T>, dim3(g.nz, nb), NT, one, st, ft.plan, scratch, j0, out, twg);
  }
}

}  // namespace

void apply_h(pt_ctx* ctx, const void* psi, int M, void* out, const double* vloc, const void* X, double alpha,
             double ecut, const pt_grid& g, pt_precision prec, cudaStream_t st, const double* A) {
  if (prec == PT_FP64)
    apply_h_t<double>(ctx, static_cast<const c128*>(psi), M, static_cast<c128*>(out), vloc,
                      static_cast<const c128*>(X), alpha, ecut, g, prec, st, A);
  else
    apply_h_t<float>(ctx, static_cast<const c64*>(psi), M, static_cast<c64*>(out), vloc, static_cast<const c64*>(X),
                     alpha, ecut, g, prec, st, A);
}

const unsigned long long* sphere_masks(pt_ctx* ctx, const pt_grid& g, const double* g2d, double ecut,
                                       cudaStream_t st) {
  if (g.nx != g.ny || g.nx != g.nz || g.nx > 64) fail(PT_INVALID_ARG, "sphere masks: cubic grids of side <= 64");
  char key[160];
  snprintf(key, sizeof(key), "sphere_masks:%d:%.17g:%.17g:%.17g:%.17g", g.nx, g.L[0], g.L[1], g.L[2], ecut);
  auto it = ctx->caches.find(key);
  if (it != ctx->caches.end()) return std::static_pointer_cast<SphereMasks>(it->second)->d;
  auto sm = std::make_shared<SphereMasks>();
  const int n = g.nx;
  PT_CUDA_CHECK(cudaMalloc(&sm->d, size_t(n) * n * sizeof(unsigned long long)));
  PT_LAUNCH(k_sphere_masks, (n * n + 255) / 256, 256, 0, st, g2d, n, ecut, sm->d);
  ctx->caches[key] = sm;
  return sm->d;
}

KinField make_kin_field(const pt_grid& g, const double* A) {
  KinField f{{0.0, 0.0, 0.0}, 0.0, 0};
  if (!A || (A[0] == 0.0 && A[1] == 0.0 && A[2] == 0.0)) return f;
  f.on = 1;
  const double two_pi = 6.283185307179586476925286766559;
  for (int a = 0; a < 3; ++a) f.c[a] = two_pi * A[a] / g.L[a];
  f.a2h = 0.5 * (A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
  return f;
}

}  // namespace pt
