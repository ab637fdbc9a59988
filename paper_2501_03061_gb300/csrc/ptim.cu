// One PT-IM(-ACE) time step (Alg. 1; Eqs. n+1/2, p_tilde, lisan, x=tx; the double SCF loop of Sec. IV-A2).
//
// Unknowns x = (Phi_{n+1}, sigma_{n+1}), initial guess (Phi_n, sigma_n).  Fixed-point map, with
// midpoints Phi_h = (Phi + Phi_n)/2 and sigma_h = (sigma + sigma_n)/2:
//     T_Phi   = Phi_n   - i dt (H Phi_h - Phi_h S^{-1} A),   S = <Phi_h|Phi_h>,  A = <Phi_h|H Phi_h>
//     T_sigma = sigma_n - i dt (A sigma_h - sigma_h A)
// Outer loop: diagonalise sigma_h (FP64 Jacobi), phit = Phi_h Q, W = (V_x phit) Q^*, ACE from
// (Phi_h, W).  Inner loop: Anderson mixing (type II, real coefficients, depth <= 20, history on
// the device) on x = T(x) with the ACE frozen; the relative residual is reduced in FP64 and read
// by the host each iteration.  The outer loop stops when the midpoint the ACE was built on moved
// by less than tol.  Finally Loewdin: Phi <- Phi S^{-1/2}, sigma <- S^{1/2} sigma S^{1/2}, then
// sigma <- (sigma + sigma^*)/2.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace pt {

namespace {

constexpr int kMaxDepth = 20;

// names of the phases (the order of pt_ptim_stats.phase_ms), also the NVTX range names
const char* const kPhaseNames[12] = {"ptim/exchange",      "ptim/ace_build", "ptim/ace_apply", "ptim/apply_H",
                                     "ptim/subspace_gemm", "ptim/subspace_nxn", "ptim/sigma_eig", "ptim/sigma_rot",
                                     "ptim/commutator",    "ptim/anderson",  "ptim/loewdin",   "ptim/hxc"};

// CUDA events around the phases of a step, summed per phase once the step has synchronised; each
// phase is also an NVTX range on the host thread
class PhaseTimer {
 public:
  explicit PhaseTimer(cudaStream_t st) : st_(st) {}
  ~PhaseTimer() {
    if (open_) trace_pop();  // a phase left by an error
    for (auto& r : recs_) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
  }
  void begin(int phase) {
    Rec r{phase, nullptr, nullptr};
    check_cuda(cudaEventCreate(&r.a), "cudaEventCreate");
    check_cuda(cudaEventCreate(&r.b), "cudaEventCreate");
    check_cuda(cudaEventRecord(r.a, st_), "cudaEventRecord");
    recs_.push_back(r);
    trace_push(kPhaseNames[phase]);
    open_ = true;
  }
  void end() {
    check_cuda(cudaEventRecord(recs_.back().b, st_), "cudaEventRecord");
    if (open_) trace_pop();
    open_ = false;
  }
  // the stream must have been synchronised
  void sum(double* ms) const {
    for (const auto& r : recs_) {
      float t = 0.f;
      check_cuda(cudaEventElapsedTime(&t, r.a, r.b), "cudaEventElapsedTime");
      ms[r.phase] += t;
    }
  }

 private:
  struct Rec {
    int phase;
    cudaEvent_t a, b;
  };
  cudaStream_t st_;
  std::vector<Rec> recs_;
  bool open_ = false;
};
enum { PH_EXCH = 0, PH_ACE_BUILD, PH_ACE_APPLY, PH_H, PH_SUB, PH_SUBNN, PH_EIG, PH_ROT, PH_COMM, PH_AND, PH_LOEW, PH_HXC };

// out[0] = max |A_e - B_e|^2 over the entries (squared: no FP64 square root per entry), as the
// bit pattern of a non-negative double, whose integer order is its numeric order (out zeroed first)
__global__ void __launch_bounds__(256) k_maxabs2_diff(const c128* __restrict__ A, const c128* __restrict__ B, int n,
                                                      unsigned long long* __restrict__ out) {
  double m = 0;
  for (int e = blockIdx.x * 256 + threadIdx.x; e < n; e += gridDim.x * 256) {
    const double dr = A[e].re - B[e].re, di = A[e].im - B[e].im;
    m = fmax(m, dr * dr + di * di);
  }
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ double s[8];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int w = 0; w < 8; ++w) r = fmax(r, s[w]);
    if (!(r == r)) r = __longlong_as_double(0x7ff0000000000000ll);  // NaN counts as +inf
    atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(r)));
  }
}

// out[0] = max over entries of |sigma_ij - sigma_00 delta_ij| + |Im sigma_00|: zero exactly when
// sigma = c I with c real (a pure state up to normalisation); out[1] = Re sigma_00
__global__ void k_pure_check(const c128* __restrict__ sig, int N, double* __restrict__ out) {
  const c128 c = sig[0];
  double m = fabs(c.im);
  const int n2 = N * N;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    const int i = e / N, j = e - i * N;
    const double dr = sig[e].re - (i == j ? c.re : 0.0), di = sig[e].im - (i == j ? c.im : 0.0);
    m = fmax(m, fabs(dr) + fabs(di));
  }
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ double s[32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) r = fmax(r, s[w]);
    out[0] = r;
    out[1] = c.re;
  }
}

// Fingerprint of a state (phi, sigma): the wrapping 64-bit sum over elements e of a mixed hash of
// (e, bit pattern of element e).  Integer arithmetic only, so it is exact and independent of the
// reduction order; any change of a bit of any element changes it except with probability ~2^-64.
// Stage 1: one partial per block; stage 2 (one block) sums the partials.
constexpr int FP_BLOCKS = 256;
__device__ __forceinline__ uint64_t fp_mix(uint64_t h) {  // splitmix64 finaliser (Steele, Lea, Flood 2014)
  h ^= h >> 30;
  h *= 0xBF58476D1CE4E5B9ull;
  h ^= h >> 27;
  h *= 0x94D049BB133111EBull;
  h ^= h >> 31;
  return h;
}
__device__ __forceinline__ uint64_t fp_bits(float re, float im) {
  return (uint64_t(__float_as_uint(re)) << 32) | __float_as_uint(im);
}
__device__ __forceinline__ uint64_t fp_bits(double re, double im) {
  return fp_mix(uint64_t(__double_as_longlong(re))) ^ uint64_t(__double_as_longlong(im));
}
template <class T>
__global__ void __launch_bounds__(256) k_fingerprint(const cx<T>* __restrict__ a, size_t n,
                                                     unsigned long long* __restrict__ part) {
  unsigned long long s = 0;
  for (size_t e = size_t(blockIdx.x) * 256 + threadIdx.x; e < n; e += size_t(FP_BLOCKS) * 256) {
    const cx<T> v = a[e];
    s += fp_mix(fp_bits(v.re, v.im) ^ (uint64_t(e) * 0x9E3779B97F4A7C15ull));
  }
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ unsigned long long sh[8];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long r = 0;
    for (int w = 0; w < 8; ++w) r += sh[w];
    part[blockIdx.x] = r;
  }
}
__global__ void k_fingerprint_sum(const unsigned long long* __restrict__ part, unsigned long long* __restrict__ out) {
  if (threadIdx.x == 0) {
    unsigned long long r = 0;
    for (int b = 0; b < FP_BLOCKS; ++b) r += part[b];
    out[0] = r;
  }
}

// ||S - I||_F^2 in a fixed order: one partial per block, then one block adds the partials
constexpr int SD_BLOCKS = 64;
__global__ void __launch_bounds__(256) k_sdev_part(const c128* __restrict__ S, int N, double* __restrict__ part) {
  double s = 0.0;
  const int nn = N * N;
  for (int e = blockIdx.x * 256 + threadIdx.x; e < nn; e += SD_BLOCKS * 256) {
    c128 v = S[e];
    if (e / N == e % N) v.re -= 1.0;
    s += v.re * v.re + v.im * v.im;
  }
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double sh[8];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < 8; ++w) r += sh[w];
    part[blockIdx.x] = r;
  }
}
__global__ void k_sdev_sum(const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int b = 0; b < SD_BLOCKS; ++b) r += part[b];
    out[0] = r;
  }
}

// out = M - M^*: the commutator A sigma - sigma A of two Hermitian matrices from M = A sigma alone
// (sigma A = (A sigma)^*), exactly anti-Hermitian
__global__ void k_minus_adjoint(const c128* __restrict__ M, int N, c128* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const int i = e / N, j = e - i * N;
  const c128 a = M[e], b = M[size_t(j) * N + i];
  out[e] = c128{a.re - b.re, a.im + b.im};
}

// N x N conversions of the mixed-precision S^{-1} A
__global__ void k_to_c64(const c128* __restrict__ a, int n, c64* __restrict__ b) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) b[e] = c64{float(a[e].re), float(a[e].im)};
}
__global__ void k_to_c128(const c64* __restrict__ a, int n, c128* __restrict__ b) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) b[e] = c128{double(a[e].re), double(a[e].im)};
}
__global__ void k_add_c64(c128* __restrict__ x, const c64* __restrict__ c, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) x[e] = c128{x[e].re + double(c[e].re), x[e].im + double(c[e].im)};
}
// flag = 1 when ||c||_F > tol ||x||_F (the last refinement correction against the solution): one
// partial pair per block, then one thread adds them in order
__global__ void __launch_bounds__(256) k_corr_part(const c64* __restrict__ c, const c128* __restrict__ x, int n,
                                                   double* __restrict__ part) {
  float sc = 0.f, sx = 0.f;
  for (int e = blockIdx.x * 256 + threadIdx.x; e < n; e += SD_BLOCKS * 256) {
    sc += c[e].re * c[e].re + c[e].im * c[e].im;
    const float xr = float(x[e].re), xi = float(x[e].im);
    sx += xr * xr + xi * xi;
  }
  for (int o = 16; o; o >>= 1) {
    sc += __shfl_down_sync(0xffffffffu, sc, o);
    sx += __shfl_down_sync(0xffffffffu, sx, o);
  }
  __shared__ float red[2][8];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sc;
    red[1][threadIdx.x >> 5] = sx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < 8; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}
__global__ void k_corr_flag(const double* __restrict__ part, double tol, int* __restrict__ flag) {
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < SD_BLOCKS; ++k) {
      a += part[2 * k];
      b += part[2 * k + 1];
    }
    flag[0] = (a > tol * tol * b || !(a == a)) ? 1 : 0;
  }
}

__global__ void k_fill(double* __restrict__ d, int n, const double* __restrict__ v) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) d[e] = v[0];
}

// sum_i d_i Re <phit_i|V phit_i> * dV   (one block per orbital, FP64 block reduction)
template <class T>
__global__ void k_weighted_diag(const cx<T>* __restrict__ a, const cx<T>* __restrict__ b, const double* __restrict__ d,
                                size_t ng, double dV, double* __restrict__ out) {
  const int i = blockIdx.x;
  const cx<T>* x = a + size_t(i) * ng;
  const cx<T>* y = b + size_t(i) * ng;
  double s = 0;
  if constexpr (sizeof(T) == 4) {
    float sf = 0.f, cf = 0.f;  // compensated FP32 sum per thread, FP64 across threads
    for (size_t e = threadIdx.x; e < ng; e += blockDim.x) {
      const cx<T> u = x[e], v = y[e];
      const float yv = (u.re * v.re + u.im * v.im) - cf;
      const float t = sf + yv;
      cf = (t - sf) - yv;
      sf = t;
    }
    s = double(sf) - double(cf);
  } else {
    for (size_t e = threadIdx.x; e < ng; e += blockDim.x) {
      const cx<T> u = x[e], v = y[e];
      s += double(u.re * v.re + u.im * v.im);
    }
  }
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) r += sh[w];
    out[i] = r * dV * d[i];
  }
}

template <class T>
__global__ void k_diff(cx<T>* out, const cx<T>* a, const cx<T>* b, size_t n) {
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x)
    out[e] = a[e] - b[e];
}

// How S^{-1} A is formed for the overlap S = I + E of the midpoint block.  With e = ||E||_F (an
// upper bound of ||E||_2), the Neumann series sum_{k=0..K} (-E)^k A in Horner form (K products)
// is off by at most e^{K+1}/(1-e) relative, and the product (I - E)(I + E^2)(I + E^4)...(I + E^{2^J}),
// which equals (I - E^{2^{J+1}}) (I + E)^{-1}, by e^{2^{J+1}}/(1-e) (2J+1 products).  A form is
// usable when that bound is at the FP64 rounding level; the Cholesky route (factor, triangular
// inverse, two products) costs about as much as kSinvCholCost products on this part, whose FP64
// pipe runs the serial pivot chain slowly.  mode 1 takes the cheapest usable form, mode 2 the product
// form whenever usable, mode 0 always the Cholesky route.
enum SinvKind { kSinvChol = 0, kSinvHorner = 1, kSinvProduct = 2, kSinvMixed = 3 };
struct SinvPlan {
  SinvKind kind;
  int terms;  // K (Horner) or J (product)
};
constexpr double kSinvTol = 1e-17;
constexpr int kMixedPasses = 2;      // FP64 refinement passes of the mixed-precision route
constexpr double kMixedCheck = 1e-10;  // largest last correction, relative, that the route accepts
constexpr int kSinvCholCost = 10;
SinvPlan sinv_plan(double e, int mode) {
  if (mode == 0 || !(e < 0.25)) return {kSinvChol, 0};
  const double bound = kSinvTol * (1.0 - e);
  int K = 0;
  double p = e;  // e^{K+1}
  while (p > bound && K < kSinvCholCost) {
    p *= e;
    ++K;
  }
  int J = 0;
  double q = e * e;  // e^{2^{J+1}}
  while (q > bound && 2 * J + 1 < kSinvCholCost) {
    q *= q;
    ++J;
  }
  const bool horner_ok = p <= bound, product_ok = q <= bound;
  if (mode == 2) return product_ok ? SinvPlan{kSinvProduct, J} : SinvPlan{kSinvChol, 0};
  if (horner_ok && (!product_ok || K <= 2 * J + 1)) return {kSinvHorner, K};
  if (product_ok) return {kSinvProduct, J};
  return {kSinvChol, 0};
}

template <class T>
struct Seg {
  cx<T>* phi;
  c128* sig;
};

template <class T>
struct Step {
  pt_ctx* ctx;
  int N;
  size_t ng;      // grid points
  size_t nv;      // length of an orbital vector: ng, or npad plane-wave coefficients
  size_t n1, n2;  // N nv orbital entries, N^2 sigma entries
  double dV;
  pt_grid g;
  pt_kernel k;
  pt_precision prec;
  pt_ptim_params p;
  cudaStream_t st;
  int blocks;

  void* buf(const char* name, size_t bytes) { return ctx->get(name, bytes); }

  // ||a||^2 and ||b||^2 (weight dV on the orbital segment, 1 on sigma) in one pass and one synchronisation
  void norm2_pair(const cx<T>* aphi, const c128* asig, const cx<T>* bphi, const c128* bsig, double* ra, double* rb) {
    double* dev = static_cast<double*>(buf("ptim_norm", 2 * sizeof(double)));
    sqnorms<T>(ctx, aphi, asig, bphi, bsig, n1, n2, dV, 1.0, dev, st);
    double h[2] = {0, 0};
    PT_CUDA_CHECK(cudaMemcpyAsync(h, dev, sizeof(h), cudaMemcpyDeviceToHost, st));
    PT_CUDA_CHECK(cudaStreamSynchronize(st));
    *ra = h[0];
    *rb = h[1];
  }

  void midpoint(cx<T>* phih, c128* sigh, const cx<T>* phi, const cx<T>* phin, const c128* sig, const c128* sign) {
    Term t[2] = {{phi, c128{0.5, 0}}, {phin, c128{0.5, 0}}};
    lincomb<T>(ctx, phih, n1, t, 2, st);
    Term s[2] = {{sig, c128{0.5, 0}}, {sign, c128{0.5, 0}}};
    lincomb<double>(ctx, sigh, n2, s, 2, st);
  }
};

template <class T>
pt_status ptim_step_t(pt_ctx* ctx, cx<T>* phi, c128* sig, int N, const double* vloc, const pt_grid& g,
                      const pt_kernel& kern, const pt_ptim_params& P, pt_precision prec, pt_ptim_stats* stats,
                      cudaStream_t st) {
  // Plane-wave basis (option ptim_pw): on cubic grids with compile-time FFTs the orbital blocks of
  // the step live as their coefficients in the Ecut sphere, the basis the orbitals are expanded in
  // (a unitary transform: every inner product and so every iterate is that of the grid form), when
  // the input lies in the sphere to the rounding of the transform; the caller's real-space block is
  // read at the start and written at the end
  cx<T>* const phi_io = phi;
  const PwBasis* pwb = nullptr;
  if (ctx->ptim_pw && pw_applies(g)) {
    const PwBasis& b = pw_basis(ctx, g, P.ecut, st);
    cx<T>* c = static_cast<cx<T>*>(ctx->get("ptim_phipw", size_t(N) * b.npad * sizeof(cx<T>)));
    const double outside = pw_from_grid<T>(ctx, b, phi, N, c, st, true);
    if (outside <= (prec == PT_FP64 ? 1e-24 : 1e-10)) {  // fraction of sum |phi|^2 outside the sphere
      pwb = &b;
      phi = c;
    }
  }
  const size_t nv = pwb ? pwb->npad : ng_of(g);
  Step<T> S{ctx, N, ng_of(g), nv, nv * N, size_t(N) * N, dv_of(g), g, kern, prec, P, st, 0};
  // a step that fails part-way (non-finite input, a failed factorisation) may leave a basis that is
  // not unitary in "ptim_Q": the context's next step must not warm-start its eigensolves from it
  struct WarmStartGuard {
    pt_ctx* c;
    bool done;
    ~WarmStartGuard() {
      if (!done) c->ptim_q_n = 0;
    }
  } warm_guard{ctx, false};
  const size_t fb = S.n1 * sizeof(cx<T>);
  const size_t mb = S.n2 * sizeof(c128);
  const int depth = std::max(1, std::min(P.anderson_depth, kMaxDepth));
  auto F = [&](const char* n) { return static_cast<cx<T>*>(S.buf(n, fb)); };
  auto Mx = [&](const char* n) { return static_cast<c128*>(S.buf(n, mb)); };
  cx<T>* phin = F("ptim_phin");
  cx<T>* phih = F("ptim_phih");
  cx<T>* phit = F("ptim_phit");
  cx<T>* vphit = F("ptim_vphit");
  cx<T>* W = F("ptim_W");
  cx<T>* xi = F("ptim_xi");
  cx<T>* X = F("ptim_X");
  cx<T>* Hphi = F("ptim_Hphi");
  cx<T>* rphi_buf[2] = {F("ptim_rphi0"), F("ptim_rphi1")};  // residuals of consecutive iterations
  cx<T>* aphi = F("ptim_anchor_phi");
  cx<T>* dxp_phi = F("ptim_dxpend_phi");
  c128* sign = Mx("ptim_sign");
  c128* sigh = Mx("ptim_sigh");
  c128* asig = Mx("ptim_anchor_sig");
  c128* Q = Mx("ptim_Q");
  c128* QH = Mx("ptim_QH");
  c128* A = Mx("ptim_A");
  c128* Sm = Mx("ptim_S");
  c128* Sn = Mx("ptim_Sn");
  c128* Lc = Mx("ptim_L");
  c128* Li = Mx("ptim_Linv");
  c128* T1 = Mx("ptim_T1");
  // real-space blocks of the plane-wave form (the exchange's input and output, the density's)
  cx<T>* R0 = pwb ? static_cast<cx<T>*>(S.buf("ptim_real0", S.ng * N * sizeof(cx<T>))) : nullptr;
  cx<T>* R1 = pwb ? static_cast<cx<T>*>(S.buf("ptim_real1", S.ng * N * sizeof(cx<T>))) : nullptr;
  c128* Tc = Mx("ptim_Tcomm");  // the sigma commutator, computed on a side stream
  c128* Tcm = Mx("ptim_Tcomm_half");  // A sigma_h, its half
  c128* SinvA = Mx("ptim_SinvA");
  c128* rsig_buf[2] = {Mx("ptim_rsig0"), Mx("ptim_rsig1")};
  c128* dxp_sig = Mx("ptim_dxpend_sig");
  double* d = static_cast<double*>(S.buf("ptim_d", N * sizeof(double)));
  double* dsc = static_cast<double*>(S.buf("ptim_dscratch", (2 * N + 64) * sizeof(double)));
  int* info = static_cast<int*>(S.buf("ptim_info", sizeof(int)));
  // partial sums of the N x N checks: ||S - I||_F (SD_BLOCKS + 1), the refinement check (2 SD_BLOCKS)
  double* sdp = static_cast<double*>(S.buf("ptim_sdev", (2 * SD_BLOCKS + 2) * sizeof(double)));
  // FP32 N x N work matrices and flags of the mixed-precision S^{-1} A
  auto M32 = [&](const char* n) { return static_cast<c64*>(S.buf(n, S.n2 * sizeof(c64))); };
  c64 *s32 = M32("ptim_s32"), *l32 = M32("ptim_l32"), *li32 = M32("ptim_li32"), *si32 = M32("ptim_si32");
  c64 *r32 = M32("ptim_r32"), *c32 = M32("ptim_c32");
  int* info32 = static_cast<int*>(S.buf("ptim_info32", 2 * sizeof(int)));
  int* mixflag = info32 + 1;
  bool mixed_ok = true;
  // Anderson history ring: dR and Z = dX + beta dR per slot, for both segments
  std::vector<cx<T>*> Zp(depth), dRp(depth);
  std::vector<c128*> Zs(depth), dRs(depth);
  for (int a = 0; a < depth; ++a) {
    char nm[64];
    snprintf(nm, sizeof(nm), "ptim_Z_phi_%d", a);
    Zp[a] = F(nm);
    snprintf(nm, sizeof(nm), "ptim_dR_phi_%d", a);
    dRp[a] = F(nm);
    snprintf(nm, sizeof(nm), "ptim_Z_sig_%d", a);
    Zs[a] = Mx(nm);
    snprintf(nm, sizeof(nm), "ptim_dR_sig_%d", a);
    dRs[a] = Mx(nm);
  }
  double* Gd = static_cast<double*>(S.buf("ptim_G", kMaxDepth * kMaxDepth * sizeof(double)));
  double* Gp = static_cast<double*>(S.buf("ptim_Gpacked", kMaxDepth * kMaxDepth * sizeof(double)));
  double* dots = static_cast<double*>(S.buf("ptim_dots", (2 * kMaxDepth + 2) * sizeof(double)));
  double* rhs = static_cast<double*>(S.buf("ptim_rhs", kMaxDepth * sizeof(double)));
  double* gamma = static_cast<double*>(S.buf("ptim_gamma", kMaxDepth * sizeof(double)));
  int* idx_d = static_cast<int*>(S.buf("ptim_idx", 2 * kMaxDepth * sizeof(int)));
  // self-consistent V_Hxc: midpoint density and the total local potential V_loc + V_Hxc[rho_h]
  double* rho = P.hxc ? static_cast<double*>(S.buf("ptim_rho", S.ng * sizeof(double))) : nullptr;
  double* vtot = P.hxc ? static_cast<double*>(S.buf("ptim_vtot", S.ng * sizeof(double))) : nullptr;
  double* hxc_part = P.hxc ? static_cast<double*>(S.buf("ptim_hxc_part", 2 * size_t(g.nz) * sizeof(double))) : nullptr;
  // E(t_n) from the first inner iteration, whose midpoint is (Phi_n, sigma_n) and whose exchange
  // operator is exact on it: spin Re Tr[sigma_n A_0] holds the exchange energy twice and, with
  // V_Hxc, int rho V_Hxc in place of E_H + E_xc (host copies of A_0, sigma_n and the V_Hxc fields)
  std::vector<c128> e_A, e_sig;
  std::vector<double> e_rho, e_vt, e_vl, e_part;
  double ex0 = NAN;

  PT_CUDA_CHECK(cudaMemcpyAsync(phin, phi, fb, cudaMemcpyDeviceToDevice, st));
  PT_CUDA_CHECK(cudaMemcpyAsync(sign, sig, mb, cudaMemcpyDeviceToDevice, st));
  // the iteration updates (phi, sig) in place: a step that ends in an error (not PT_NOT_CONVERGED,
  // which returns normally with its last iterate) copies the input state back from (phin, sign)
  struct RestoreGuard {
    void *phi, *sig;
    const void *phin, *sign;
    size_t fb, mb;
    cudaStream_t st;
    bool armed;
    ~RestoreGuard() {
      if (!armed) return;
      cudaMemcpyAsync(phi, phin, fb, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(sig, sign, mb, cudaMemcpyDeviceToDevice, st);
      cudaStreamSynchronize(st);
    }
  } restore{phi, sig, phin, sign, fb, mb, st, true};
  gram<T>(ctx, phin, phin, N, N, S.nv, S.dV, Sn, st);
  // Pure state (sigma_n = c I, Eq. pure_vx): sigma_h stays c I, its eigenbasis is any basis, the
  // commutator [A, c I] vanishes, so the eigensolve, the rotations into and out of the eigenbasis
  // and the commutator are skipped; Algorithm 1's final step then orthonormalises Phi and keeps
  // sigma = c I (the general step's S^{1/2} sigma S^{1/2} differs from c I by c (S - I), at the
  // level of the orthonormality error)
  bool pure = false;
  {
    PT_LAUNCH(k_pure_check, 1, 1024, 0, st, sign, N, dsc);
    double h[2] = {1.0, 0.0};
    PT_CUDA_CHECK(cudaMemcpyAsync(h, dsc, sizeof(h), cudaMemcpyDeviceToHost, st));
    PT_CUDA_CHECK(cudaStreamSynchronize(st));
    pure = h[0] == 0.0;
    if (pure) PT_LAUNCH(k_fill, std::max(1, (N + 255) / 256), 256, 0, st, d, N, dsc + 1);  // d_i = c
  }
  // Warm start of the ACE operator (option ptim_ace_warm): when this step's input is exactly the
  // output of the context's previous step (same sizes, grid, kernel and precision, equal fingerprint
  // of (phi, sigma)), "ptim_xi" still holds that step's last ACE operator, built at a midpoint near
  // this step's first one.  The first outer pass then solves its loose inner problem with it instead
  // of paying an exchange application; the operators this step builds, the anchors they define and
  // the stopping test are unchanged, so the fixed point is the same.
  char warm_key[256];
  snprintf(warm_key, sizeof(warm_key), "%d:%d:%d:%d:%.17g:%.17g:%.17g:%d:%.17g:%.17g:%d:%zu", N, g.nx, g.ny, g.nz,
           g.L[0], g.L[1], g.L[2], kern.type, kern.mu, kern.g0, int(prec), pwb ? pwb->npad : size_t(0));
  auto* fpd = static_cast<unsigned long long*>(
      S.buf("ptim_fingerprint", (2 * FP_BLOCKS + 2) * sizeof(unsigned long long)));
  // of the caller's real-space blocks (a round trip through the plane-wave coefficients is not exact)
  auto fingerprint = [&](const cx<T>* ph, const c128* sg, unsigned long long out[2]) {
    PT_LAUNCH(k_fingerprint<T>, FP_BLOCKS, 256, 0, st, ph, S.ng * N, fpd);
    PT_LAUNCH(k_fingerprint_sum, 1, 32, 0, st, fpd, fpd + 2 * FP_BLOCKS);
    PT_LAUNCH(k_fingerprint<double>, FP_BLOCKS, 256, 0, st, sg, S.n2, fpd + FP_BLOCKS);
    PT_LAUNCH(k_fingerprint_sum, 1, 32, 0, st, fpd + FP_BLOCKS, fpd + 2 * FP_BLOCKS + 1);
    PT_CUDA_CHECK(cudaMemcpyAsync(out, fpd + 2 * FP_BLOCKS, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    PT_CUDA_CHECK(cudaStreamSynchronize(st));
  };
  bool ace_warm = false;
  if (ctx->ptim_ace_warm && P.use_ace && ctx->ptim_warm_valid && ctx->ptim_warm_key == warm_key) {
    unsigned long long f[2];
    fingerprint(phi_io, sign, f);
    ace_warm = f[0] == ctx->ptim_warm_fp[0] && f[1] == ctx->ptim_warm_fp[1];
  }
  ctx->ptim_warm_valid = false;  // "ptim_xi" is about to change; valid again only after a finished step

  pt_ptim_stats stv;
  std::memset(&stv, 0, sizeof(stv));
  stv.residual = NAN;
  PhaseTimer tm(st);
  bool converged = false, inner_conv = false, have_anchor = false;
  const int nthreads = 256;
  const int sblocks = std::max(1, std::min<int>(ctx->num_sms * 8, int((S.n1 + nthreads - 1) / nthreads)));
  const int sblocks2 = std::max(1, int((S.n2 + nthreads - 1) / nthreads));

  // event pairs bracketing each exchange application (read once the step has synchronised)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  struct EvGuard {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& v;
    ~EvGuard() {
      for (auto& e : v) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
      }
    }
  } ev_guard{ev};
  // The sigma commutator [A, sigma_h] needs only A: it runs on a side stream while the overlap is
  // factorised (the FP64 Cholesky chain keeps a few CTAs busy at a time) and joins before r_sigma
  if (ctx->side_streams.empty()) {
    cudaStream_t s2 = nullptr;
    PT_CUDA_CHECK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    ctx->side_streams.push_back(s2);
  }
  cudaStream_t side = ctx->side_streams[0];
  cudaEvent_t comm_ev[2] = {nullptr, nullptr};
  for (auto& e : comm_ev) PT_CUDA_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  struct CommEvGuard {
    cudaEvent_t* e;
    ~CommEvGuard() {
      cudaEventDestroy(e[0]);
      cudaEventDestroy(e[1]);
    }
  } comm_guard{comm_ev};
  // V_x[P_h] Phi_h through the sigma_h eigenbasis: (V_x phit) Q^*, phit = Phi_h Q
  // sigma_h changes little between outer iterations and between steps: eigensolves start from the
  // last basis the context holds (any unitary start is correct; a near one converges in a sweep or two)
  auto exchange_on_midpoint = [&](cx<T>* out, bool energy) {
    if (pure) {  // phit = Phi_h, d_i = c: V_x Phi_h directly, no eigenbasis
      tm.begin(PH_EXCH);
      std::pair<cudaEvent_t, cudaEvent_t> e;
      PT_CUDA_CHECK(cudaEventCreate(&e.first));
      PT_CUDA_CHECK(cudaEventCreate(&e.second));
      ev.push_back(e);
      const cx<T>* src = phih;
      if (pwb) {  // the exchange works on real-space fields
        pw_to_grid<T>(ctx, *pwb, phih, N, R0, st);
        src = R0;
      }
      PT_CUDA_CHECK(cudaEventRecord(e.first, st));
      stv.pair_ffts += exchange(ctx, src, d, N, nullptr, N, pwb ? R1 : out, g, kern, prec, st);
      PT_CUDA_CHECK(cudaEventRecord(e.second, st));
      if (pwb) pw_from_grid<T>(ctx, *pwb, R1, N, out, st);
      tm.end();
      stv.exchange_calls++;
      if (energy) {
        PT_LAUNCH(k_weighted_diag<T>, N, 256, 0, st, phih, out, d, S.nv, S.dV, dsc);
        std::vector<double> h(N);
        PT_CUDA_CHECK(cudaMemcpyAsync(h.data(), dsc, N * sizeof(double), cudaMemcpyDeviceToHost, st));
        PT_CUDA_CHECK(cudaStreamSynchronize(st));
        double en = 0;
        for (double v : h) en += v;
        stv.exch_energy = P.spin * 0.5 * P.alpha * en;
      }
      return;
    }
    tm.begin(PH_EIG);
    const bool warm = ctx->ptim_q_n == N;
    ctx->ptim_q_n = 0;  // Q is being rewritten
    // FP32 forms: sigma_h = Q diag(d) Q^* to 1e-9 relative, two orders below the rounding of the
    // FP32 exchange it feeds (~1e-7); the FP64 form runs Jacobi to its rounding floor
    stv.eig_sweeps += heev(ctx, sigh, N, Q, d, st, 30, warm ? Q : nullptr, prec == PT_FP64 ? 0.0 : 1e-9);
    ctx->ptim_q_n = N;
    tm.end();
    tm.begin(PH_ROT);
    rotate<T>(ctx, phih, Q, N, N, N, S.nv, c128{1, 0}, nullptr, 0, phit, st);
    tm.end();
    tm.begin(PH_EXCH);
    std::pair<cudaEvent_t, cudaEvent_t> e;
    PT_CUDA_CHECK(cudaEventCreate(&e.first));
    PT_CUDA_CHECK(cudaEventCreate(&e.second));
    ev.push_back(e);
    const cx<T>* src = phit;
    if (pwb) {  // the exchange works on real-space fields
      pw_to_grid<T>(ctx, *pwb, phit, N, R0, st);
      src = R0;
    }
    PT_CUDA_CHECK(cudaEventRecord(e.first, st));
    stv.pair_ffts += exchange(ctx, src, d, N, nullptr, N, pwb ? R1 : vphit, g, kern, prec, st);
    PT_CUDA_CHECK(cudaEventRecord(e.second, st));
    if (pwb) pw_from_grid<T>(ctx, *pwb, R1, N, vphit, st);
    tm.end();
    stv.exchange_calls++;
    if (energy) {
      PT_LAUNCH(k_weighted_diag<T>, N, 256, 0, st, phit, vphit, d, S.nv, S.dV, dsc);
      std::vector<double> h(N);
      PT_CUDA_CHECK(cudaMemcpyAsync(h.data(), dsc, N * sizeof(double), cudaMemcpyDeviceToHost, st));
      PT_CUDA_CHECK(cudaStreamSynchronize(st));
      double e = 0;
      for (double v : h) e += v;
      stv.exch_energy = P.spin * 0.5 * P.alpha * e;
    }
    tm.begin(PH_ROT);
    conj_transpose(Q, N, QH, st);
    rotate<T>(ctx, vphit, QH, N, N, N, S.nv, c128{1, 0}, nullptr, 0, out, st);
    tm.end();
  };

  // Inner tolerance per outer iteration.  While the midpoint the ACE operator is built on still
  // moves by a relative Delta between outer iterations, the inner fixed point of that operator is
  // only needed to kappa * Delta (at most `inner_cap`, at least tol); the step converges only when
  // the midpoint has settled to tol AND the last inner loop met tol itself.  kappa = 0 keeps tol
  // throughout.
  const double kappa = ctx->ptim_inner_kappa, cap = ctx->ptim_inner_cap;
  double inner_tol = P.tol;
  // relative distance of the midpoint (phih, sigh) from the anchor (aphi, asig) the operator was
  // built on; the difference goes to W and T1 (free outside the build and the commutator), so the
  // anchor itself is kept
  auto anchor_distance = [&]() {
    PT_LAUNCH(k_diff<T>, sblocks, nthreads, 0, st, W, phih, aphi, S.n1);
    PT_LAUNCH(k_diff<double>, sblocks2, nthreads, 0, st, T1, sigh, asig, S.n2);
    double ch = 0, nr = 0;
    S.norm2_pair(W, T1, phih, sigh, &ch, &nr);
    return std::sqrt(ch / nr);
  };
  const int max_outer = P.use_ace ? P.max_outer : 1;
  int aces = 0;
  for (int outer = 0; outer < max_outer && !converged; ++outer) {
    S.midpoint(phih, sigh, phi, phin, sig, sign);
    if (P.use_ace) {
      bool rebuild = true;
      if (have_anchor) {
        const double delta = anchor_distance();
        if (delta < P.tol) {
          if (inner_conv) {
            converged = true;
            break;
          }
          // the operator is exact to tol on this midpoint: finish the inner solve with it (the anchor
          // stays where the operator was built, so the next check measures the distance to it)
          rebuild = false;
          inner_tol = P.tol;
        } else {
          inner_tol = kappa > 0.0 ? std::max(P.tol, std::min(cap, kappa * delta)) : P.tol;
        }
      } else {
        inner_tol = kappa > 0.0 ? std::max(P.tol, cap) : P.tol;
        // warm start: a pre-pass with the previous step's operator; no anchor is set, so the next
        // outer iteration builds this step's first operator at the improved midpoint
        if (outer == 0 && ace_warm) rebuild = false;
      }
      if (rebuild) {
        PT_CUDA_CHECK(cudaMemcpyAsync(aphi, phih, fb, cudaMemcpyDeviceToDevice, st));
        PT_CUDA_CHECK(cudaMemcpyAsync(asig, sigh, mb, cudaMemcpyDeviceToDevice, st));
        have_anchor = true;
        stv.outer = ++aces;
        exchange_on_midpoint(W, true);
        tm.begin(PH_ACE_BUILD);
        ace_from_w(ctx, W, phih, N, g, prec, xi, st, pwb ? S.nv : 0);
        tm.end();
      }
    } else {
      stv.outer = 1;
    }
    // ---- inner Anderson loop ----
    inner_conv = false;
    const int pass = stv.passes++;
    int next_slot = 0;
    std::vector<int> order;  // active history slots, oldest first
    for (int inner = 0; inner < P.max_inner; ++inner) {
      stv.inner++;
      if (pass < 16) stv.pass_inner[pass]++;
      const bool first = stv.inner == 1;
      cx<T>* rphi = rphi_buf[inner & 1];
      c128* rsig = rsig_buf[inner & 1];
      S.midpoint(phih, sigh, phi, phin, sig, sign);
      const double* vh = vloc;
      if (P.hxc) {
        // H_{n+1/2} = H[P_{n+1/2}] (Eq. p_tilde): rho_h = spin P_h(r, r); X is free until the
        // exchange term below, so it holds chi = Phi_h sigma_h
        tm.begin(PH_HXC);
        if (pwb) {
          pw_to_grid<T>(ctx, *pwb, phih, N, R0, st);
          density<T>(ctx, R0, sigh, N, S.ng, P.spin, R1, rho, st);
        } else {
          density<T>(ctx, phih, sigh, N, S.ng, P.spin, X, rho, st);
        }
        hxc_potential(ctx, rho, vloc, g, vtot, first ? hxc_part : nullptr, st);
        tm.end();
        vh = vtot;
      }
      if (P.use_ace) {
        tm.begin(PH_ACE_APPLY);
        ace_apply(ctx, xi, N, phih, N, X, g, prec, st, pwb ? S.nv : 0);
        tm.end();
      } else {
        exchange_on_midpoint(X, inner == 0);
      }
      if (first) ex0 = stv.exch_energy;
      tm.begin(PH_H);
      if (pwb)
        pw_apply_h<T>(ctx, *pwb, phih, N, Hphi, vh, X, P.alpha, P.A, st);
      else
        apply_h(ctx, phih, N, Hphi, vh, X, P.alpha, P.ecut, g, prec, st, P.A);
      tm.end();
      tm.begin(PH_SUB);
      // A = <Phi_h|H Phi_h> and S = <Phi_h|Phi_h> are Hermitian: upper tiles only, mirrored
      gram2<T>(ctx, phih, Hphi, A, phih, Sm, N, N, S.nv, S.dV, st, true);
      if (first) {
        e_A.resize(S.n2);
        e_sig.resize(S.n2);
        PT_CUDA_CHECK(cudaMemcpyAsync(e_A.data(), A, mb, cudaMemcpyDeviceToHost, st));
        PT_CUDA_CHECK(cudaMemcpyAsync(e_sig.data(), sign, mb, cudaMemcpyDeviceToHost, st));
        if (P.hxc) {
          e_rho.resize(S.ng);
          e_vt.resize(S.ng);
          e_vl.resize(S.ng);
          e_part.resize(2 * size_t(g.nz));
          PT_CUDA_CHECK(cudaMemcpyAsync(e_rho.data(), rho, S.ng * sizeof(double), cudaMemcpyDeviceToHost, st));
          PT_CUDA_CHECK(cudaMemcpyAsync(e_vt.data(), vtot, S.ng * sizeof(double), cudaMemcpyDeviceToHost, st));
          PT_CUDA_CHECK(cudaMemcpyAsync(e_vl.data(), vloc, S.ng * sizeof(double), cudaMemcpyDeviceToHost, st));
          PT_CUDA_CHECK(cudaMemcpyAsync(e_part.data(), hxc_part, e_part.size() * sizeof(double),
                                        cudaMemcpyDeviceToHost, st));
        }
      }
      tm.end();
      if (!pure) {
        PT_CUDA_CHECK(cudaEventRecord(comm_ev[0], st));
        PT_CUDA_CHECK(cudaStreamWaitEvent(side, comm_ev[0], 0));
        // A sigma_h - sigma_h A = M - M^* with M = A sigma_h (both Hermitian): one product
        zgemm('N', 'N', N, N, N, c128{1, 0}, A, N, sigh, N, c128{0, 0}, Tcm, N, side);
        PT_LAUNCH(k_minus_adjoint, (N * N + 255) / 256, 256, 0, side, Tcm, N, Tc);
        PT_CUDA_CHECK(cudaEventRecord(comm_ev[1], side));
      }
      tm.begin(PH_SUBNN);
      SinvPlan plan{kSinvChol, 0};
      const bool mixed = ctx->ptim_sinv_mixed && mixed_ok;
      if (mixed) {  // FP32 factor of S for the mixed-precision route, before the synchronisation
        PT_LAUNCH(k_to_c64, (N * N + 255) / 256, 256, 0, st, Sm, N * N, s32);
        cholesky<float>(ctx, s32, N, l32, info32, st);
      }
      if (ctx->ptim_sinv_series || mixed) {
        double e2 = NAN;
        int h_info32 = 1;
        if (ctx->ptim_sinv_series) {
          PT_LAUNCH(k_sdev_part, SD_BLOCKS, 256, 0, st, Sm, N, sdp);
          PT_LAUNCH(k_sdev_sum, 1, 32, 0, st, sdp, sdp + SD_BLOCKS);
          PT_CUDA_CHECK(cudaMemcpyAsync(&e2, sdp + SD_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, st));
        }
        if (mixed) PT_CUDA_CHECK(cudaMemcpyAsync(&h_info32, info32, sizeof(int), cudaMemcpyDeviceToHost, st));
        PT_CUDA_CHECK(cudaStreamSynchronize(st));
        if (ctx->ptim_sinv_series) {
          const double e = std::sqrt(e2);
          if (!(e <= stv.s_dev_max)) stv.s_dev_max = e;
          plan = sinv_plan(e, ctx->ptim_sinv_series);
        }
        if (plan.kind == kSinvChol && mixed && h_info32 == 0) plan = SinvPlan{kSinvMixed, kMixedPasses};
      }
      stv.sinv_path[plan.kind]++;
      if (plan.kind == kSinvMixed) {
        // S^{-1} A from the FP32 factor S32 = L32 L32^*, refined in FP64 (iterative refinement):
        // X = S32^{-1} A, then X <- X + S32^{-1} (A - S X) with the residual in FP64; each pass
        // multiplies the error by ~kappa(S) eps_32, the last correction is checked against X
        const int nn = N * N, nb = (N * N + 255) / 256;
        const c64 one32{1.f, 0.f}, zero32{0.f, 0.f};
        tri_inv_lower<float>(ctx, l32, N, li32, st);
        gemm<float>('C', 'N', N, N, N, one32, li32, N, li32, N, zero32, si32, N, si32, N, st);  // S32^{-1}
        PT_LAUNCH(k_to_c64, nb, 256, 0, st, A, nn, r32);
        gemm<float>('N', 'N', N, N, N, one32, si32, N, r32, N, zero32, c32, N, c32, N, st);
        PT_LAUNCH(k_to_c128, nb, 256, 0, st, c32, nn, SinvA);
        for (int pass = 0; pass < plan.terms; ++pass) {
          zgemm_add('N', 'N', N, N, N, c128{-1, 0}, Sm, N, SinvA, N, c128{1, 0}, A, N, T1, N, st);  // A - S X
          PT_LAUNCH(k_to_c64, nb, 256, 0, st, T1, nn, r32);
          gemm<float>('N', 'N', N, N, N, one32, si32, N, r32, N, zero32, c32, N, c32, N, st);
          PT_LAUNCH(k_add_c64, nb, 256, 0, st, SinvA, c32, nn);
        }
        PT_LAUNCH(k_corr_part, SD_BLOCKS, 256, 0, st, c32, SinvA, nn, sdp);
        PT_LAUNCH(k_corr_flag, 1, 32, 0, st, sdp, kMixedCheck, mixflag);
        PT_CUDA_CHECK(cudaMemsetAsync(info, 0, sizeof(int), st));
      } else if (plan.kind == kSinvChol) {
        // S^{-1} A = L^{-*} (L^{-1} A)
        cholesky(ctx, Sm, N, Lc, info, st);
        tri_inv_lower(ctx, Lc, N, Li, st);
        zgemm('N', 'N', N, N, N, c128{1, 0}, Li, N, A, N, c128{0, 0}, T1, N, st);
        zgemm('C', 'N', N, N, N, c128{1, 0}, Li, N, T1, N, c128{0, 0}, SinvA, N, st);
      } else {
        PT_CUDA_CHECK(cudaMemsetAsync(info, 0, sizeof(int), st));
        add_diagonal(Sm, N, -1.0, st);  // E = S - I
        // every product writes a fresh buffer (T1 and SinvA in turn, the last one SinvA)
        const int writes = plan.kind == kSinvHorner ? plan.terms : plan.terms + 1;
        int w = 0;
        auto next_out = [&]() {
          ++w;
          return ((writes - w) & 1) ? T1 : SinvA;
        };
        const c128* y = A;
        if (writes == 0) PT_CUDA_CHECK(cudaMemcpyAsync(SinvA, A, mb, cudaMemcpyDeviceToDevice, st));  // E = 0
        if (plan.kind == kSinvHorner) {
          for (int k = 0; k < plan.terms; ++k) {  // y <- A - E y
            c128* o = next_out();
            zgemm_add('N', 'N', N, N, N, c128{-1, 0}, Sm, N, y, N, c128{1, 0}, A, N, o, N, st);
            y = o;
          }
        } else {
          c128* o = next_out();  // y <- (I - E) A
          zgemm_add('N', 'N', N, N, N, c128{-1, 0}, Sm, N, A, N, c128{1, 0}, A, N, o, N, st);
          y = o;
          c128* Pw = Sm;  // E^{2^j}
          c128* Pn = Li;
          for (int j = 1; j <= plan.terms; ++j) {
            zgemm('N', 'N', N, N, N, c128{1, 0}, Pw, N, Pw, N, c128{0, 0}, Pn, N, st);
            std::swap(Pw, Pn);
            o = next_out();  // y <- (I + E^{2^j}) y
            zgemm_add('N', 'N', N, N, N, c128{1, 0}, Pw, N, y, N, c128{1, 0}, y, N, o, N, st);
            y = o;
          }
        }
      }
      tm.end();
      tm.begin(PH_SUB);
      // r_Phi = Phi_n - i dt (H Phi_h - Phi_h S^{-1}A) - Phi
      Term tr[3] = {{Hphi, c128{0, -P.dt}}, {phin, c128{1, 0}}, {phi, c128{-1, 0}}};
      rotate<T>(ctx, phih, SinvA, N, N, N, S.nv, c128{0, P.dt}, tr, 3, rphi, st);
      tm.end();
      tm.begin(PH_COMM);
      // r_sigma = sigma_n - i dt (A sigma_h - sigma_h A) - sigma  (the commutator is 0 in a pure state)
      if (pure) {
        PT_CUDA_CHECK(cudaMemsetAsync(Tc, 0, mb, st));
      } else {
        PT_CUDA_CHECK(cudaStreamWaitEvent(st, comm_ev[1], 0));
      }
      Term ts[3] = {{sign, c128{1, 0}}, {Tc, c128{0, -P.dt}}, {sig, c128{-1, 0}}};
      lincomb<double>(ctx, rsig, S.n2, ts, 3, st);
      tm.end();
      tm.begin(PH_AND);
      int h_info = 0, h_mix = 0;
      PT_CUDA_CHECK(cudaMemcpyAsync(&h_info, info, sizeof(int), cudaMemcpyDeviceToHost, st));
      if (plan.kind == kSinvMixed) PT_CUDA_CHECK(cudaMemcpyAsync(&h_mix, mixflag, sizeof(int), cudaMemcpyDeviceToHost, st));
      double rr = 0, xx = 0;
      S.norm2_pair(rphi, rsig, phi, sig, &rr, &xx);  // synchronises st
      if (h_mix) {  // refinement too slow for this S (kappa(S) eps_32 not small): FP64 Cholesky from now on
        mixed_ok = false;
        stv.sinv_mixed_fallback = 1;
      }
      if (first) {
        double tr = 0.0;  // Re Tr[sigma_n A_0] = Re sum_ij sigma_ij A_ji
        for (int i = 0; i < N; ++i)
          for (int j = 0; j < N; ++j) {
            const c128 sv = e_sig[size_t(i) * N + j], av = e_A[size_t(j) * N + i];
            tr += sv.re * av.re - sv.im * av.im;
          }
        double e = P.spin * tr - ex0;
        if (P.hxc) {
          double eh = 0.0, exc = 0.0, rv = 0.0;
          for (int z = 0; z < g.nz; ++z) {
            eh += e_part[2 * size_t(z)];
            exc += e_part[2 * size_t(z) + 1];
          }
          for (size_t r = 0; r < S.ng; ++r) rv += e_rho[r] * (e_vt[r] - e_vl[r]);
          e += S.dV * (eh + exc - rv);
        }
        // with a warm-started operator the first iteration's exchange is not exact at (Phi_n, sigma_n)
        stv.total_energy = ace_warm ? NAN : e;
      }
      if (h_info) fail(PT_NOT_PD, "PT-IM: overlap of the midpoint orbitals is not positive definite");
      const double res = std::sqrt(rr / xx);
      stv.residual = res;
      if (!std::isfinite(res)) fail(PT_NONFINITE, "PT-IM residual is not finite");
      if (res < inner_tol) {
        const bool at_tol = res < P.tol;
        // Loose tolerance met.  When the midpoint is still within tol of the anchor, the outer
        // check that follows would keep the operator and finish the inner solve to tol: do that
        // here, going on from this iteration's residual instead of recomputing it in a new loop
        if (!at_tol && P.use_ace && have_anchor && anchor_distance() < P.tol) {
          inner_tol = P.tol;
        } else {
          tm.end();
          inner_conv = at_tol;
          break;
        }
      }
      // kinetic preconditioning: Anderson then solves x = x + M (T(x) - x), same fixed point
      if (ctx->ptim_precond) {
        if (pwb)
          pw_precondition<T>(ctx, *pwb, rphi, N, A, P.dt, P.A, st);
        else
          precondition_residual(ctx, rphi, N, A, P.dt, P.ecut, g, prec, st, P.A);
      }
      // ---- Anderson (type II, real coefficients) ----
      int m = 0;
      if (inner > 0) {
        const int slot = next_slot;
        next_slot = (next_slot + 1) % depth;
        order.erase(std::remove(order.begin(), order.end(), slot), order.end());
        const std::vector<int> others = order;
        order.push_back(slot);
        m = int(order.size());
        const int mo = int(others.size());
        AndersonSeg<T> a1{};
        a1.rk = rphi;
        a1.rprev = rphi_buf[(inner + 1) & 1];
        a1.dxp = dxp_phi;
        a1.dRs = dRp[slot];
        a1.Zs = Zp[slot];
        a1.n = S.n1;
        AndersonSeg<double> a2{};
        a2.rk = rsig;
        a2.rprev = rsig_buf[(inner + 1) & 1];
        a2.dxp = dxp_sig;
        a2.dRs = dRs[slot];
        a2.Zs = Zs[slot];
        a2.n = S.n2;
        for (int o = 0; o < mo; ++o) {
          a1.dR[o] = dRp[others[o]];
          a2.dR[o] = dRs[others[o]];
        }
        anderson_prepare<T>(ctx, a1, a2, mo, P.anderson_beta, S.dV, dots, st);
        int hidx[2 * kMaxDepth];
        for (int o = 0; o < mo; ++o) hidx[o] = others[o];
        for (int p = 0; p < m; ++p) hidx[kMaxDepth + p] = order[p];
        PT_CUDA_CHECK(cudaMemcpyAsync(idx_d, hidx, sizeof(hidx), cudaMemcpyHostToDevice, st));
        anderson_gram(Gd, dots, slot, idx_d, mo, idx_d + kMaxDepth, m, Gp, rhs, st);
        small_solve(Gp, rhs, m, 1e-14, gamma, st);
      }
      std::vector<const cx<T>*> zp(m);
      std::vector<const c128*> zs(m);
      for (int p = 0; p < m; ++p) {
        zp[p] = Zp[order[p]];
        zs[p] = Zs[order[p]];
      }
      anderson_update<T>(ctx, phi, rphi, zp.data(), m, gamma, P.anderson_beta, dxp_phi, S.n1, st);
      anderson_update<double>(ctx, sig, rsig, zs.data(), m, gamma, P.anderson_beta, dxp_sig, S.n2, st);
      tm.end();
    }
    if (!P.use_ace && inner_conv) converged = true;
  }
  // ---- final orthonormalisation and conjugate symmetrisation ----
  tm.begin(PH_LOEW);
  gram<T>(ctx, phi, phi, N, N, S.nv, S.dV, Sm, st);
  auto* dmax = reinterpret_cast<unsigned long long*>(dsc);
  PT_CUDA_CHECK(cudaMemsetAsync(dmax, 0, 2 * sizeof(unsigned long long), st));
  const int mblocks = std::max(1, std::min(SD_BLOCKS, int((S.n2 + 255) / 256)));
  PT_LAUNCH(k_maxabs2_diff, mblocks, 256, 0, st, Sm, Sn, int(S.n2), dmax);
  set_identity(T1, N, st);
  PT_LAUNCH(k_maxabs2_diff, mblocks, 256, 0, st, Sm, T1, int(S.n2), dmax + 1);
  double devs[2] = {0, 0};
  PT_CUDA_CHECK(cudaMemcpyAsync(devs, dsc, sizeof(devs), cudaMemcpyDeviceToHost, st));
  PT_CUDA_CHECK(cudaStreamSynchronize(st));
  devs[0] = std::sqrt(devs[0]);  // the kernels keep squares
  devs[1] = std::sqrt(devs[1]);
  stv.orth_error = devs[0];
  PT_CUDA_CHECK(cudaMemsetAsync(info, 0, sizeof(int), st));
  const double sdev = devs[1];  // max |S - I|
  if (sdev < 0.05) {
    // S close to I: coupled Newton-Schulz  T = (3I - Z Y)/2, Y <- Y T, Z <- T Z,  Y -> S^{1/2}, Z -> S^{-1/2}
    c128* Y = Lc;   // S^{1/2}
    c128* Z = A;    // S^{-1/2}
    PT_CUDA_CHECK(cudaMemcpyAsync(Y, Sm, mb, cudaMemcpyDeviceToDevice, st));
    set_identity(Z, N, st);
    const int iters = sdev < 1e-6 ? 3 : (sdev < 1e-3 ? 4 : 6);
    for (int it = 0; it < iters; ++it) {
      zgemm('N', 'N', N, N, N, c128{-0.5, 0}, Z, N, Y, N, c128{0, 0}, T1, N, st);
      add_diagonal(T1, N, 1.5, st);  // T = 1.5 I - 0.5 Z Y
      zgemm('N', 'N', N, N, N, c128{1, 0}, Y, N, T1, N, c128{0, 0}, SinvA, N, st);
      std::swap(Y, SinvA);
      zgemm('N', 'N', N, N, N, c128{1, 0}, T1, N, Z, N, c128{0, 0}, SinvA, N, st);
      std::swap(Z, SinvA);
    }
    if (Z != A) PT_CUDA_CHECK(cudaMemcpyAsync(A, Z, mb, cudaMemcpyDeviceToDevice, st));
    if (Y != Lc) PT_CUDA_CHECK(cudaMemcpyAsync(Lc, Y, mb, cudaMemcpyDeviceToDevice, st));
  } else {
    // Q receives the eigenvectors of S, not of sigma: ptim_q_n stays 0 so that the next step's
    // sigma eigensolve starts cold instead of from this unrelated basis
    ctx->ptim_q_n = 0;
    heev(ctx, Sm, N, Q, d, st);
    scale_cols_pow(Q, d, N, -0.5, T1, info, st);
    zgemm('N', 'C', N, N, N, c128{1, 0}, T1, N, Q, N, c128{0, 0}, A, N, st);   // S^{-1/2}
    scale_cols_pow(Q, d, N, 0.5, T1, info, st);
    zgemm('N', 'C', N, N, N, c128{1, 0}, T1, N, Q, N, c128{0, 0}, Lc, N, st);  // S^{1/2}
    // a non-positive eigenvalue of S is reported before phi and sigma are overwritten, so a step
    // that fails here leaves the caller's (Phi_n, sigma_n) as they were
    int s_info = 0;
    PT_CUDA_CHECK(cudaMemcpyAsync(&s_info, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    PT_CUDA_CHECK(cudaStreamSynchronize(st));
    if (s_info) fail(PT_NOT_PD, "PT-IM: final overlap matrix is not positive definite");
  }
  rotate<T>(ctx, phi, A, N, N, N, S.nv, c128{1, 0}, nullptr, 0, rphi_buf[0], st);
  PT_CUDA_CHECK(cudaMemcpyAsync(phi, rphi_buf[0], fb, cudaMemcpyDeviceToDevice, st));
  if (pwb) pw_to_grid<T>(ctx, *pwb, phi, N, phi_io, st);
  if (pure) {
    PT_CUDA_CHECK(cudaMemcpyAsync(sig, sign, mb, cudaMemcpyDeviceToDevice, st));  // sigma stays c I
  } else {
    zgemm('N', 'N', N, N, N, c128{1, 0}, Lc, N, sig, N, c128{0, 0}, T1, N, st);
    zgemm('N', 'N', N, N, N, c128{1, 0}, T1, N, Lc, N, c128{0, 0}, sig, N, st);
    conj_transpose(sig, N, T1, st);
    Term th[2] = {{sig, c128{0.5, 0}}, {T1, c128{0.5, 0}}};
    lincomb<double>(ctx, sig, S.n2, th, 2, st);
  }
  tm.end();
  int h_info = 0;
  PT_CUDA_CHECK(cudaMemcpyAsync(&h_info, info, sizeof(int), cudaMemcpyDeviceToHost, st));
  PT_CUDA_CHECK(cudaStreamSynchronize(st));
  if (h_info) fail(PT_NOT_PD, "PT-IM: final overlap matrix is not positive definite");
  tm.sum(stv.phase_ms);
  for (auto& e : ev) {
    float ms = 0.f;
    PT_CUDA_CHECK(cudaEventElapsedTime(&ms, e.first, e.second));
    stv.exchange_ms += ms;
  }
  stv.converged = converged ? 1 : 0;
  stv.pure_state = pure ? 1 : 0;
  stv.ace_warm = ace_warm ? 1 : 0;
  stv.plane_waves = pwb ? int(pwb->npw) : 0;
  if (ctx->ptim_ace_warm && P.use_ace && stv.outer > 0) {
    fingerprint(phi_io, sig, ctx->ptim_warm_fp);
    ctx->ptim_warm_key = warm_key;
    ctx->ptim_warm_valid = true;
  }
  if (stats) *stats = stv;
  warm_guard.done = true;
  restore.armed = false;
  return converged ? PT_OK : PT_NOT_CONVERGED;
}

}  // namespace

pt_status ptim_step(pt_ctx* ctx, void* phi, void* sigma, int N, const double* vloc, const pt_grid& g,
                    const pt_kernel& k, const pt_ptim_params& P, pt_precision prec, pt_ptim_stats* stats,
                    cudaStream_t st) {
  if (prec == PT_FP64)
    return ptim_step_t<double>(ctx, static_cast<c128*>(phi), static_cast<c128*>(sigma), N, vloc, g, k, P, prec,
                               stats, st);
  return ptim_step_t<float>(ctx, static_cast<c64*>(phi), static_cast<c128*>(sigma), N, vloc, g, k, P, prec, stats,
                            st);
}

}  // namespace pt
