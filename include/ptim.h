/*
 * ptim.h — C ABI of the GB300 library for the hot path of finite-temperature
 * PT-IM real-time TDDFT with a hybrid functional (arXiv 2501.03061).
 *
 * The library applies the occupation-weighted screened Fock exchange operator
 * to a block of orbitals, builds and applies its adaptively compressed (ACE)
 * form, applies the Hamiltonian, and takes one PT-IM(-ACE) time step.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Grid: nx*ny*nz points (each dimension 2..64 and 2,3,5-smooth) on an
 *    orthorhombic cell Lx*Ly*Lz (bohr).  Ng = nx*ny*nz, dV = Lx*Ly*Lz/Ng.
 *  - Orbital blocks are complex, interleaved (re, im), ORBITAL-MAJOR: orbital
 *    j, point (x,y,z) sits at element j*Ng + (z*ny + y)*nx + x.  The element
 *    type is double2 (complex128) for PT_FP64 and float2 (complex64) for the
 *    FP32 precisions.  Buffers start on a 16-byte boundary.
 *  - N x N matrices (sigma, Q, ...) are complex128, row-major: a[i*N + j],
 *    also on a 16-byte boundary.
 *  - Orbital counts (N, M, N1, N2) are 1..PT_MAX_ORBITALS; others return
 *    PT_INVALID_ARG.
 *  - Inner product <a|b> = dV * sum_r conj(a(r)) b(r).
 *  - All pointers passed in are DEVICE pointers unless stated otherwise.  The
 *    caller owns every buffer it passes; the library never frees caller memory
 *    and never keeps a caller pointer past the call.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream) unless its comment says it synchronises.  Errors are
 *    returned as pt_status; nothing is thrown across the ABI.  After an error,
 *    pt_last_error(ctx) gives a one-line description.
 *  - A pt_ctx is not thread-safe: use one context per host thread.
 */
#ifndef PTIM_H
#define PTIM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int pt_status;
enum {
  PT_OK = 0,
  PT_INVALID_ARG = 1,    /* bad size, null pointer, misaligned buffer, unsupported grid */
  PT_OOM = 2,            /* device allocation failed or the context's HBM budget is exceeded */
  PT_NOT_PD = 3,         /* Cholesky met a non-positive pivot (ACE: -M not positive definite) */
  PT_NOT_CONVERGED = 4,  /* PT-IM iteration caps reached before the tolerance */
  PT_NONFINITE = 5,      /* a NaN/Inf appeared in a residual or a small dense factorisation */
  PT_TIMEOUT = 6,        /* a bounded device-side wait ran out */
  PT_CUDA = 7,           /* a CUDA runtime error; see pt_last_error */
  PT_UNSUPPORTED = 8     /* valid request that this build does not implement */
};

/* Largest orbital count a call accepts (N x N matrices are indexed with 32-bit products). */
#define PT_MAX_ORBITALS 32768

/* Orthorhombic periodic cell sampled on an nx*ny*nz grid. */
typedef struct {
  int nx, ny, nz;
  double L[3];
} pt_grid;

/* Fourier-space interaction K(G) of V_x(r,r') = -P(r,r') K(r,r') (Sec. II-B, Eq. 1).
 *   type 0: Coulomb 4*pi/|G|^2, with K(0) = g0 (use 0).
 *   type 1: erfc-screened Coulomb 4*pi/|G|^2 * (1 - exp(-|G|^2/(4 mu^2))),
 *           K(0) = g0 if g0 is finite, else the analytic limit pi/mu^2 (pass NaN).
 * G = 2*pi*m/L with m wrapped to [-n/2, n/2). */
typedef struct {
  int type;
  double mu;
  double g0;
} pt_kernel;

typedef enum {
  PT_FP64 = 0,          /* every step in FP64 (the plain FP64 form) */
  PT_FP32 = 1,          /* pair products, FFTs and Ng-long contractions in FP32;
                           N x N factorisations, residuals and Loewdin in FP64 */
  PT_FP32_TC_TF32 = 2,  /* as PT_FP32 with the Gram/rotation contractions as one TF32 tensor-core product */
  PT_FP32_TC_BF16 = 3   /* as PT_FP32 with the Gram/rotation contractions as one BF16 tensor-core
                           product (operands rounded to bf16, FP32 accumulation); an error-study
                           form: the pair products and FFTs of the exchange run as in PT_FP32 */
} pt_precision;

typedef struct pt_ctx pt_ctx;
typedef struct pt_ace pt_ace;

/* ---- context --------------------------------------------------------------------------- */

/* Create a context on CUDA `device`.  hbm_budget caps the bytes of device
 * workspace the context may hold (0 = 90% of the device's free memory at
 * creation).  The context owns its workspace, cached FFT/kernel tables and
 * pair schedules.  Synchronises the device. */
pt_status pt_create(pt_ctx** ctx, int device, size_t hbm_budget);
/* Free the context and all workspace it owns (synchronises). */
void pt_destroy(pt_ctx* ctx);
/* One-line description of the last error of this context ("" if none). */
const char* pt_last_error(const pt_ctx* ctx);
/* Bytes of device workspace currently held by the context. */
size_t pt_workspace_bytes(const pt_ctx* ctx);
/* Release cached workspace (synchronises). */
pt_status pt_trim(pt_ctx* ctx);
/* Set a tuning option of the context.  Keys (besides "graphs" and "autotune" of the batched
 * exchange, 0 or 1):
 *   "ptim_inner_kappa", "ptim_inner_cap"  the PT-IM step solves the inner fixed point of an
 *                    outer iteration to max(tol, min(cap, kappa * Delta)), Delta the relative move
 *                    of the midpoint since the last ACE anchor (cap alone in the first outer
 *                    iteration); the step still converges only when the midpoint has settled to
 *                    tol and the last inner loop met tol.  Defaults 0.1 and 1e-2; kappa = 0 uses
 *                    tol throughout.
 *   "ptim_precond"   1: the inner Anderson iteration of pt_ptim_step works on the kinetically
 *                    preconditioned map x -> x + M (T(x) - x), M acting on each orbital column j of
 *                    the residual as 1/(1 + i dt/2 (|G + A|^2/2 - Re <phi_j|H phi_j>)) in Fourier space
 *                    inside the basis sphere (identity outside, sigma untouched).  M is invertible, so
 *                    the fixed point (the step's result) is unchanged; the iteration needs fewer
 *                    steps (64^3 grid, N = 320, orbital blocks on the grid: 39 inner iterations per
 *                    step against 46-47).
 *                    Default 1; 0: plain Anderson on T(x) - x.
 *   "ptim_ace_warm"  1: when a step's input (phi, sigma) is exactly the output of the context's
 *                    previous step (same sizes, grid, kernel, precision; checked by a fingerprint),
 *                    its first outer pass solves its loose inner problem with that step's last ACE
 *                    operator instead of building one, saving an exchange application; the operators
 *                    the step builds and its stopping test are unchanged (64^3 grid, N = 320: 3 ACE
 *                    builds per step against 4).  total_energy is NaN for such steps.  Default 1.
 *   "ptim_pw"        1 (default): on cubic grids of side <= 64 with compile-time FFT kernels, the
 *                    step holds its orbital blocks (iterates, residuals, Anderson history, ACE
 *                    operator) as their coefficients at the plane waves |G|^2/2 <= ecut of the
 *                    unitary FFT (the orbital basis of Sec. VI), entering real space only for the
 *                    local potential, the exchange and the density.  Inner products and so every
 *                    iterate equal those of the grid form; it applies when the input phi lies in
 *                    the sphere (the part of sum |phi|^2 outside it at most 1e-24 in PT_FP64, 1e-10
 *                    otherwise: the rounding of the transform), else the step runs on the grid.
 *                    The output phi is the real-space field of the final coefficients.  0: always
 *                    on the grid.
 *   "ptim_sinv_series"  how the inner iteration forms S^{-1} A, S = <Phi_h|Phi_h> = I + E the
 *                    overlap of the midpoint block.  1 (default): with e = ||E||_F < 1/4, the cheaper
 *                    of the Neumann series sum_{k<=K} (-E)^k A (K products, error <= e^{K+1}/(1-e))
 *                    and the product (I - E)(I + E^2)...(I + E^{2^J}) A (2J+1 products, error
 *                    <= e^{2^{J+1}}/(1-e)) that reaches 1e-17 relative, unless the Cholesky route
 *                    is cheaper; 2: the product form wherever it applies; 0: always S = L L^* and
 *                    S^{-1} A = L^{-*} (L^{-1} A).  The forms agree to FP64 rounding; the series
 *                    costs one synchronisation per inner iteration to read e.
 *   "ptim_sinv_mixed"  1 (default): where no series form applies, S^{-1} A comes from an FP32
 *                    Cholesky factor of S refined in FP64: X = S32^{-1} A, then twice X <- X +
 *                    S32^{-1} (A - S X) with the residual A - S X in FP64 (each pass multiplies the
 *                    error by ~kappa(S) eps_32); a last correction above 1e-10 of X, or an FP32
 *                    factorisation that fails, sends the step to the FP64 Cholesky route.  0: the
 *                    FP64 Cholesky route (S = L L^*, S^{-1} A = L^{-*} (L^{-1} A)).
 *   "scratch_bytes"  bytes of pair/orbital fields one FFT batch may hold (default 512 MiB: the
 *                    cost per pair falls with the pair tile even past L2 residency, 4-10% from
 *                    48 MiB to 512 MiB; smaller values give more, smaller batches).
 *   "exchange64_scratch_bytes"  the same for the 64^3 FP32 exchange pipeline (default 512 MiB:
 *                    16 x 16 pair tiles, the largest its parameter block holds), which keeps four
 *                    such batches in flight.
 *   "tc_gram"        1: in the PT_FP32 form, run the Gram contractions (A^H B over the grid) on
 *                    the tensor cores with a 3-product TF32 split (hi*hi + hi*lo + lo*hi) that
 *                    keeps FP32-level accuracy; 0 (default): CUDA cores.
 *   "tc_period"      K stages of 32 floats the tensor-core Gram accumulates in TMEM between
 *                    readouts into compensated registers (1..64, default 2).
 *   "tc_gram_wide"   1 (default): tensor-core Grams with more than 64 right-hand orbitals use
 *                    64 x 128 tiles, and the PT-IM step computes <Phi|H Phi> and <Phi|Phi> in
 *                    one pass over Phi; 0: 64 x 64 tiles, one Gram at a time. */
pt_status pt_set_option(pt_ctx* ctx, const char* key, double value);

/* ---- Fock exchange (Sec. IV-A1, Eq. vxdiag; Alg. 2 with sigma diagonalised) ------------ */

/* out_j = (V_x tgt_j)(r) = - sum_i occ_i src_i(r) * IFFT[ K(G) * FFT[ conj(src_i) tgt_j ] ](r)
 * for j = 0..M-1, i = 0..N-1 (forward FFT unnormalised, inverse divided by Ng).
 *   src  Ng x N orbitals phit_i in the basis that diagonalises sigma (Eq. diag_sigma)
 *   occ  N doubles d_i (the eigenvalues of sigma); pairs with occ_i == 0 are skipped
 *   tgt  Ng x M orbitals, or NULL to use tgt = src (then M must equal N and the
 *        kernel's symmetry v_ji = conj(v_ij) halves the FFT work)
 *   out  Ng x M, overwritten; must not alias src or tgt.
 * The result carries no mixing fraction alpha.  Precisions: PT_FP64 or any FP32 form. */
pt_status pt_apply_exchange(pt_ctx* ctx, const void* src, const double* occ, int N,
                            const void* tgt, int M, void* out,
                            const pt_grid* grid, const pt_kernel* kernel,
                            pt_precision prec, void* stream);

/* The same operator for a general (non-diagonal) occupation matrix, evaluated as Algorithm 2's
 * undiagonalised triple loop (Sec. III-B; Sec. II-B Eq. mixed_vx):
 *   out_j = - sum_{k,i} sigma[i][k] phi_i(r) * IFFT[ K(G) * FFT[ conj(phi_k) tgt_j ] ](r)
 * for j < M, i, k < N, with the pair FFT of (k, j) recomputed for every i (N*N*M pair FFTs, the
 * baseline that the diagonalisation of Sec. IV-A1 replaces by N*M).  Kept as the comparison
 * form: pt_apply_exchange on phit = phi Q with d = eig(sigma) gives the same result.
 *   phi    Ng x N orbitals (any basis); sigma: N x N complex128 device matrix, row-major, used as
 *          given (not symmetrised, no entry skipped)
 *   tgt    Ng x M orbitals or NULL (tgt = phi, M = N); out: Ng x M, overwritten, no aliasing.
 * *pair_ffts (optional, host) receives N*N*M.  Precisions: PT_FP64 or any FP32 form (the pair
 * products and FFTs in FP32).  Asynchronous on `stream`. */
pt_status pt_apply_exchange_mixed(pt_ctx* ctx, const void* phi, const void* sigma, int N, const void* tgt, int M,
                                  void* out, const pt_grid* grid, const pt_kernel* kernel, pt_precision prec,
                                  long long* pair_ffts, void* stream);

/* Allocation-free variant of pt_apply_exchange (no counterpart in the paper: it exists for
 * callers that cannot allocate device memory while they run — an application whose own pool
 * allocator owns the whole device memory, or a latency-critical loop that cannot afford the
 * device synchronisation of cudaMalloc/cudaFree).  Same arguments and result as
 * pt_apply_exchange, but no context: every buffer beyond the caller's inputs and outputs lives
 * in static device arrays of this library (32 MiB pair scratch, a 64^3 kernel table, small
 * schedule tables) that every GPU loading the library holds until the process exits.  Limits:
 * N, M <= 1024 and grids of at most 64^3 points (the regular grid rules apply); larger requests
 * return PT_INVALID_ARG.  The arrays (about 34 MiB) become resident when the CUDA runtime loads
 * this library's device code on a GPU, which under lazy module loading can happen inside the
 * first call: a caller that hands all free device memory to its own pool should make one call
 * before doing so.  The first call on a device (with that device current) also looks up the
 * device addresses of those arrays; make that first call before any stream capture begins.  All
 * calls share the arrays and the last call's contents stay in them: calls that overlap on the
 * GPU (other streams or host threads) race.  Uses the generic (non-TMA) exchange kernels.  Other
 * status codes as pt_apply_exchange. */
pt_status pt_apply_exchange_noalloc(const void* src, const double* occ, int N, const void* tgt, int M, void* out,
                                    const pt_grid* grid, const pt_kernel* kernel, pt_precision prec, void* stream);

/* One item of a batched exchange call: out = V_x tgt for its own orbitals, grid and kernel
 * (fields as in pt_apply_exchange; tgt NULL means tgt = src and M = N). */
typedef struct {
  const void* src;
  const double* occ;
  int N;
  const void* tgt;
  int M;
  void* out;
  pt_grid grid;
  pt_kernel kernel;
} pt_exchange_item;

/* Batched exchange: `count` independent V_x applications (different orbital counts, grids and
 * kernels) in one call, in the given precision, in item order on `stream`.  The pair-tile size
 * of each grid is chosen by timing a few candidates the first time the grid is seen (option
 * "autotune", default 1).  The first call with a given item set (the same buffers and sizes)
 * runs eagerly and records the batch into a CUDA graph; later calls with the same item set
 * replay the graph as one launch (option "graphs", default 1).  pt_trim drops the graphs.
 * Synchronises `stream` once at the end to read the kernels' error word (PT_TIMEOUT if a
 * bounded wait expired).  *pair_ffts (optional) receives the pair FFTs of the batch and
 * *graph_nodes (optional) the node count of the graph that ran (0: eager).  No counterpart
 * in the paper, which treats one system at a time: this is the batched serving form. */
pt_status pt_apply_exchange_batched(pt_ctx* ctx, const pt_exchange_item* items, int count, pt_precision prec,
                                    long long* pair_ffts, size_t* graph_nodes, void* stream);

/* ---- adaptively compressed exchange (Sec. IV-A2, Eq. vx_ace; Lin's construction) -------- */

/* Build the ACE operator of V_x[P] on span(phi), P = sum_i occ_i phi_i phi_i^*:
 *   W = V_x phi (with src = tgt = phi),  M = <phi|W>,  -M = L L^* (FP64 Cholesky),
 *   xi = W L^{-*},  so that V_ACE = -xi xi^* (dV inner product) and V_ACE phi = W.
 *   phi  Ng x N orbitals in the sigma-diagonal basis; occ N doubles (device).
 * On success *ace holds a library-owned object with xi (Ng x N, precision prec).
 * Returns PT_NOT_PD if -M is not positive definite (e.g. negative occupations). */
pt_status pt_build_ace(pt_ctx* ctx, const void* phi, const double* occ, int N,
                       const pt_grid* grid, const pt_kernel* kernel, pt_precision prec,
                       pt_ace** ace, void* stream);
/* Same construction from a given W = V_x phi (for phi not in the sigma-diagonal basis). */
pt_status pt_build_ace_from(pt_ctx* ctx, const void* W, const void* phi, int N,
                            const pt_grid* grid, pt_precision prec, pt_ace** ace, void* stream);
/* out = V_ACE psi = - xi (xi^* psi):  out_j = - sum_k xi_k <xi_k|psi_j>, j = 0..M-1.
 * psi, out: Ng x M in the ACE's precision; out must not alias psi. */
pt_status pt_apply_ace(pt_ctx* ctx, const pt_ace* ace, const void* psi, int M, void* out, void* stream);
/* Copy xi (Ng x N, the ACE's precision) into a caller buffer. */
pt_status pt_ace_get_xi(const pt_ace* ace, void* xi_out, void* stream);
void pt_ace_destroy(pt_ace* ace);

/* ---- overlaps (the Gram contractions of ACE's M = <phi|W> and of PT-IM's S = <phi|phi>) -- */

/* C[i][j] = dV * sum_r conj(A_i(r)) B_j(r), i < N1, j < N2: the dV-weighted inner products
 * of two orbital blocks, e.g. M = Phi^* W of the ACE construction (Sec. IV-A2) or the overlap
 * S of the Loewdin orthonormalisation.  A: Ng x N1 and B: Ng x N2 orbitals (device, orbital-
 * major, precision prec); C: N1 x N2 complex128 (device, row-major).  In PT_FP32 the
 * contraction runs on CUDA cores with compensated sums unless the "tc_gram" option selects the
 * 3-product TF32 tensor-core form; PT_FP32_TC_TF32 runs one TF32 product (about 1e-3 relative
 * error per term, for error studies).  Asynchronous on `stream`, except that the tensor-core
 * forms synchronise once to read the kernel's error word (PT_TIMEOUT if a bounded wait expired). */
pt_status pt_overlap(pt_ctx* ctx, const void* A, int N1, const void* B, int N2, const pt_grid* grid,
                     pt_precision prec, void* C, void* stream);

/* out_j = sum_k B[k][j] A_k, j < N2: the rotation of an orbital block by an N1 x N2 matrix, e.g.
 * phit = Phi Q into the sigma eigenbasis (Eq. vxdiag) or xi = W L^{-*} of the ACE construction.
 * A: Ng x N1 orbitals, out: Ng x N2 orbitals (device, orbital-major, precision prec; out must
 * not overlap A); B: N1 x N2 complex128 (device, row-major).  Engines as for pt_overlap. */
pt_status pt_rotate(pt_ctx* ctx, const void* A, int N1, const void* B, int N2, const pt_grid* grid,
                    pt_precision prec, void* out, void* stream);

/* ---- Hamiltonian (Eq. 1) ----------------------------------------------------------------- */

/* out = P_sph[ 1/2 (-i grad + A)^2 psi + vloc * psi + alpha * V_ACE psi ], the projection
 * P_sph keeping the plane waves with |G|^2/2 <= ecut (the sphere does not move with A).
 * ace may be NULL (no exchange term).  vloc: Ng doubles (device; V_ext's scalar part and
 * V_Hxc, frozen or from pt_hxc_potential).  A: NULL (no field) or a host array of 3 doubles,
 * the uniform vector potential of the velocity gauge (V_ext(t) of Eq. 1 for a field
 * E(t) = -dA/dt).  psi/out Ng x M, out != psi. */
pt_status pt_apply_H(pt_ctx* ctx, const void* psi, int M, void* out, const double* vloc,
                     const pt_ace* ace, double alpha, double ecut, const double* A, const pt_grid* grid,
                     pt_precision prec, void* stream);

/* The velocity-gauge current J_a = spin/Omega Re Tr[P (-i d_a + A_a)], P = Phi sigma Phi^*
 * (Tr[P O] = sum_ij sigma_ij <phi_j|O phi_i>; the electric current density of electrons is -J).
 * phi: Ng x N device orbitals (precision prec, 16-byte aligned); sigma: N x N complex128 device;
 * A: NULL or host double[3]; J: host double[3].  Synchronises the stream. */
pt_status pt_current(pt_ctx* ctx, const void* phi, const void* sigma, int N, const pt_grid* grid, pt_precision prec,
                     const double* A, double spin, double* J, void* stream);

/* ---- self-consistent local potential (Eq. 1: V_Hxc[P]) ------------------------------------ */

/* rho(r) = spin * P(r, r) = spin * Re sum_ij sigma_ij phi_i(r) conj(phi_j(r)) for the density
 * matrix P = Phi sigma Phi^* (Sec. II-A, Eq. mix_P).  phi: Ng x N orbital-major, precision prec
 * (16-byte aligned); sigma: N x N complex128 row-major (Hermitian); rho: Ng doubles.  All device
 * pointers.  The FP32 forms form chi = Phi sigma with the library's rotation (tensor cores when
 * enabled) and sum the products in FP64.  Workspace: one Ng x N block held by the context. */
pt_status pt_density(pt_ctx* ctx, const void* phi, const void* sigma, int N, const pt_grid* grid, pt_precision prec,
                     double spin, double* rho, void* stream);

/* v = vloc + V_H[rho] + v_xc(rho), all FP64 (Eq. 1's V_Hxc; the paper does not name its local
 * functional: this is the LDA).  V_H(G) = 4 pi rho(G)/|G|^2 with V_H(G = 0) = 0 (neutralising
 * background); v_xc = d(rho eps_xc)/d rho with Slater exchange and the Perdew-Zunger (1981)
 * correlation of the unpolarised gas; eps = v = 0 where rho <= 1e-30.  rho, vloc, v: Ng doubles
 * on the device (vloc may be NULL: zero; v must not alias rho).  energies: NULL or a host array
 * of 2 that receives (E_H, E_xc) = (1/2 int rho V_H, int rho eps_xc) in Ha; with energies the
 * call synchronises the stream. */
pt_status pt_hxc_potential(pt_ctx* ctx, const double* rho, const double* vloc, const pt_grid* grid, double* v,
                           double* energies, void* stream);

/* ---- occupation matrix (Sec. IV-A1, Eq. diag_sigma) -------------------------------------- */

/* sigma = Q diag(d) Q^* for Hermitian sigma (its Hermitian part is used), FP64
 * parallel Jacobi on the GPU.  d ascending.  sigma, Q: N x N complex128 row-major;
 * d: N doubles.  All device pointers.  Synchronises the stream (sweep convergence test). */
pt_status pt_diag_occupations(pt_ctx* ctx, const void* sigma, int N, void* Q, double* d, void* stream);

/* ---- one PT-IM time step (Alg. 1; Eqs. n+1/2, p_tilde, lisan; Sec. IV-A2 double loop) --- */

typedef struct {
  double dt;             /* time step (au) */
  double alpha;          /* exchange mixing fraction (0.25 for HSE-like functionals) */
  double ecut;           /* plane-wave cutoff (Ha) of the projection P_sph and of the orbital basis, > 0 */
  double tol;            /* relative residual of x = T(x), and of the ACE anchor change */
  int max_outer;         /* outer (ACE rebuild) iterations */
  int max_inner;         /* inner Anderson iterations per outer iteration */
  int anderson_depth;    /* mixing history (<= 20) */
  double anderson_beta;  /* mixing parameter */
  int use_ace;           /* 1: PT-IM-ACE double loop; 0: V_x applied exactly every iteration */
  double spin;           /* electrons per orbital: spin factor of the reported energies and of
                            rho = spin * P(r, r) (2 = closed shell) */
  int hxc;               /* 0: the local potential is vloc alone (V_ext + V_Hxc frozen);
                            1: vloc + V_Hxc[rho_{n+1/2}] rebuilt from the midpoint density in
                            every inner iteration (Eq. 1 with Eq. p_tilde; see pt_hxc_potential) */
  double A[3];           /* V_ext(t) as a uniform vector potential (velocity gauge, bohr^-1): the
                            value A(t_n + dt/2) at the step's midpoint time (Eq. p_tilde's
                            H(t_{n+1/2}, P)), supplied by the caller; {0, 0, 0}: no field */
} pt_ptim_params;

typedef struct {
  int outer, inner;         /* iterations taken */
  double residual;          /* last relative residual of the inner loop */
  double exch_energy;       /* spin*(alpha/2) Tr[P V_x[P]] at the last ACE anchor (Ha) */
  double orth_error;        /* max |Phi^*Phi - Phi_n^*Phi_n| before the final orthonormalisation */
  int converged;            /* 1 when both loops met tol */
  long long pair_ffts;      /* pair FFTs executed (counting a symmetric pair once) */
  int exchange_calls;       /* V_x applications */
  double exchange_ms;       /* device time of those applications (CUDA events on the stream) */
  /* device time per phase (CUDA events on the stream):
     0 exchange, 1 ACE build (Gram, Cholesky, xi), 2 ACE apply, 3 H application,
     4 subspace contractions (A, S, projection), 5 subspace N x N (Cholesky, inverse, S^{-1}A),
     6 sigma diagonalisation, 7 rotations into/out of the sigma eigenbasis, 8 sigma commutator,
     9 Anderson mixing and residual norms, 10 final Loewdin orthonormalisation,
     11 V_Hxc (midpoint density, Hartree FFT, LDA; params.hxc = 1) */
  double phase_ms[12];
  int eig_sweeps;           /* Jacobi sweeps of the sigma eigensolves (phase 6) */
  double total_energy;      /* E(t_n) of the input state (Ha): spin Tr[P_n (-Lap/2 + V_loc)] + E_x
                               (+ E_H + E_xc with params.hxc; the kinetic term carries params.A),
                               from the first iteration, where the midpoint is (Phi_n, sigma_n) */
  int pure_state;           /* 1 when sigma_n = c I exactly (c real): the pure-state path ran (Eq.
                               pure_vx: no sigma eigensolve, rotation or commutator; sigma_{n+1} = c I) */
  int ace_warm;             /* 1 when the first outer pass used the previous step's ACE operator
                               (option "ptim_ace_warm"); total_energy is then NaN */
  int passes;               /* inner loops run: one per ACE operator built, plus the warm-started
                               first pass and any pass that kept the operator to finish at tol */
  int pass_inner[16];       /* inner iterations of each of the first 16 passes */
  int sinv_path[4];         /* inner iterations whose S^{-1} A took [0] the FP64 Cholesky route, [1] the
                               Neumann series in E = S - I, [2] the product form (option
                               "ptim_sinv_series"), [3] the FP32 factor refined in FP64 (option
                               "ptim_sinv_mixed") */
  int sinv_mixed_fallback;  /* 1 when the refinement converged too slowly and the step went on with
                               the FP64 Cholesky route */
  double s_dev_max;         /* largest ||S - I||_F of the midpoint overlaps met (0 with the option off) */
  int plane_waves;          /* plane waves of the Ecut sphere the step held its orbitals in (option
                               "ptim_pw"); 0 when it ran on the grid */
} pt_ptim_stats;

/* One PT-IM(-ACE) step from (phi, sigma) = (Phi_n, sigma_n) to (Phi_{n+1}, sigma_{n+1}),
 * both updated in place.  phi: Ng x N (precision prec); sigma: N x N complex128;
 * vloc: Ng doubles.  Returns PT_NOT_CONVERGED (with the last iterate stored) when the
 * caps are reached.  On any other error status (a non-finite residual, a failed factorisation,
 * an expired device wait) phi and sigma are restored to their input values before the call
 * returns, unless the CUDA context itself has failed (PT_CUDA), after which their contents are
 * unspecified.  Synchronises the stream once per inner iteration (residual test). */
pt_status pt_ptim_step(pt_ctx* ctx, void* phi, void* sigma, int N, const double* vloc,
                       const pt_grid* grid, const pt_kernel* kernel, const pt_ptim_params* params,
                       pt_precision prec, pt_ptim_stats* stats, void* stream);

/* Upper bound of the device workspace (bytes) that pt_ptim_step with these sizes makes a fresh
 * context allocate: the orbital blocks of the step, the Anderson ring of `anderson_depth`
 * entries, FFT/exchange scratch at the context's default batch size, and the N x N matrices.
 * Used by a serving loop to admit requests by HBM footprint.  Pure host arithmetic. */
size_t pt_ptim_footprint(int N, const pt_grid* grid, pt_precision prec, int anderson_depth);

/* ---- small helpers used by the binding and tests ------------------------------------------ */

/* Library version string and the GPU architecture it was compiled for. */
const char* pt_version(void);
/* Number of this library's kernel launches issued so far by the calling process. */
long long pt_kernel_launches(void);

/* FP32 and FP64 FMA throughput of the context's device in TFLOP/s (host outputs): every SM runs
 * eight CTAs of 256 threads, each thread eight independent register FMA chains, timed with CUDA
 * events on `stream` after a warm-up (tens of ms).  The CUDA-core roofline denominators for
 * kernels bound by FP32 or FP64 arithmetic.  Synchronises the stream. */
pt_status pt_alu_peaks(pt_ctx* ctx, double* fp32_tflops, double* fp64_tflops, void* stream);

/* Self-test of the bounded device waits (no counterpart in the paper).  One CTA waits on a
 * shared-memory mbarrier through the same deadline-bounded wait the TMA and tensor-core
 * pipelines use.  arrive = 1: the barrier completes and the call returns PT_OK.  arrive = 0:
 * nothing ever arrives, the wait gives up after timeout_s (0 < timeout_s <= 2), the kernel
 * records the expiry and returns, and the call returns PT_TIMEOUT with the context still usable
 * (the path every pipeline takes when a copy or a peer role never completes).  Synchronises the
 * stream.  PT_INVALID_ARG for a NULL context, arrive not 0 or 1, or timeout_s out of range. */
pt_status pt_selftest_wait(pt_ctx* ctx, int arrive, double timeout_s, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PTIM_H */
