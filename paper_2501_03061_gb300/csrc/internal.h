// Declarations shared between the translation units of the library (not part of the ABI).
#pragma once

#include "common.cuh"

namespace pt {

// linear-combination term: coefficient c times the orbital block x (precision of the call)
struct Term {
  const void* x;
  c128 c;
};

// ---- exchange (exchange.cu) ----
// largest pair-tile side of the 64^3 TMA pipeline (its batch descriptors travel in the kernel
// parameters: 16 bytes x (5 B^2 + 2 B) of the 32 KB parameter space)
constexpr int kExchange64MaxTile = 16;
// the 64^3 FP32 exchange engines apply (exchange.cu)
bool exchange64_applies(const pt_grid& g);
size_t exchange_scratch_budget(const pt_ctx* ctx);
// W = V_x tgt (tgt == nullptr: tgt = src, symmetric pairs).  Returns the number of pair FFTs.
long long exchange(pt_ctx* ctx, const void* src, const double* occ, int N, const void* tgt, int M, void* out,
                   const pt_grid& g, const pt_kernel& k, pt_precision prec, cudaStream_t st);
// Algorithm 2's undiagonalised triple loop (N * N * M pair FFTs): out_j = -sum_ik sigma_ik phi_i v_kj
long long exchange_mixed(pt_ctx* ctx, const void* phi, const c128* sigma, int N, const void* tgt, int M, void* out,
                         const pt_grid& g, const pt_kernel& k, pt_precision prec, cudaStream_t st);

// ---- batched exchange (batched.cu): autotuned pair tiles, replay from captured CUDA graphs ----
long long exchange_batched(pt_ctx* ctx, const pt_exchange_item* items, int count, pt_precision prec,
                           cudaStream_t st, size_t* graph_nodes);
void exchange_check(pt_ctx* ctx, cudaStream_t st);

// ---- contractions over the grid (blas.cu) ----
template <class T>
void gram(pt_ctx* ctx, const cx<T>* A, const cx<T>* B, int N1, int N2, size_t ng, double scale, c128* C,
          cudaStream_t st, bool herm = false);
// C0 = scale A^H B0 and C1 = scale A^H B1 (one pass over A on the tensor-core path, two Grams otherwise)
template <class T>
void gram2(pt_ctx* ctx, const cx<T>* A, const cx<T>* B0, c128* C0, const cx<T>* B1, c128* C1, int N1, int N2,
           size_t ng, double scale, cudaStream_t st, bool herm = false);
template <class T>
void rotate(pt_ctx* ctx, const cx<T>* A, const c128* Bm, int ldb, int N1, int N2, size_t ng, c128 alpha,
            const Term* terms, int nterms, cx<T>* out, cudaStream_t st);
template <class T>
void lincomb(pt_ctx* ctx, cx<T>* out, size_t n, const Term* terms, int nterms, cudaStream_t st);
template <class T>
void potential_apply(pt_ctx* ctx, cx<T>* out, const cx<T>* psi, const double* v, size_t ng, int M, const cx<T>* X,
                     double a, cudaStream_t st);
// out[0] = w1 ||a0||^2 + w2 ||s0||^2, out[1] = w1 ||a1||^2 + w2 ||s1||^2 (device doubles)
template <class T>
void sqnorms(pt_ctx* ctx, const cx<T>* a0, const c128* s0, const cx<T>* a1, const c128* s1, size_t n1, size_t n2,
             double w1, double w2, double* out, cudaStream_t st);


// ---- tensor-core Gram (gram_tc.cu) ----
void gram_tc(pt_ctx* ctx, const c64* A, const c64* B, int N1, int N2, size_t ng, double scale, c128* C,
             cudaStream_t st, bool herm, bool split3);
void gram_tc_check(pt_ctx* ctx, cudaStream_t st);  // raises PT_TIMEOUT if a bounded wait expired
// 64 x 128 tiles (gram_tc_wide.cu): C0 = scale A^H B0 and, when B1 is not NULL, C1 = scale A^H B1
void gram_tc_wide(pt_ctx* ctx, const c64* A, const c64* B0, c128* C0, const c64* B1, c128* C1, int N1, int N2,
                  size_t ng, double scale, cudaStream_t st, bool herm, bool split3);
bool gram_tc_applies(const void* A, const void* B, size_t ng);

// ---- tensor-core rotation (rotate_tc.cu): out = alpha A Bm + sum_t c_t x_t (complex64 orbitals) ----
void rotate_tc(pt_ctx* ctx, const c64* A, const c128* Bm, int ldb, int N1, int N2, size_t ng, c128 alpha,
               const Term* terms, int nterms, c64* out, cudaStream_t st, bool split3);
bool rotate_tc_applies(const void* A, size_t ng);

// ---- self-consistent local potential (hxc.cu) ----
// rho = spin * Re sum_ij sigma_ij phi_i conj(phi_j) (chi: Ng x N scratch of the block's precision)
template <class T>
void density(pt_ctx* ctx, const cx<T>* phi, const c128* sigma, int N, size_t ng, double spin, cx<T>* chi,
             double* rho, cudaStream_t st);
// v = vloc (may be null) + V_H[rho] + v_xc(rho); part (may be null): 2 nz per-plane sums (E_H, E_xc) / dV
void hxc_potential(pt_ctx* ctx, const double* rho, const double* vloc, const pt_grid& g, double* v, double* part,
                   cudaStream_t st);

// ---- BF16 tensor-core contractions (contract_bf16.cu): operands packed to bf16, FP32 accumulation ----
void gram_bf16(pt_ctx* ctx, const c64* A, const c64* B, int N1, int N2, size_t ng, double scale, c128* C,
               cudaStream_t st, bool herm);
void rotate_bf16(pt_ctx* ctx, const c64* A, const c128* Bm, int ldb, int N1, int N2, size_t ng, c128 alpha,
                 const Term* terms, int nterms, c64* out, cudaStream_t st);

// ---- FP64 N x N (dense.cu) ----
void zgemm(char opA, char opB, int m, int n, int k, c128 alpha, const c128* A, int lda, const c128* B, int ldb,
           c128 beta, c128* C, int ldc, cudaStream_t st);
void zgemm_add(char opA, char opB, int m, int n, int k, c128 alpha, const c128* A, int lda, const c128* B, int ldb,
               c128 beta, const c128* D, int ldd, c128* C, int ldc, cudaStream_t st);
// S (Hermitian part used) = Q diag(d) Q^*, ascending d.  Synchronises st once per sweep.
// Q0 (optional): an orthonormal basis that nearly diagonalises S (warm start); may alias Q.
// rel_tol (optional): also stop once the off-diagonal Frobenius norm of Q^* S Q is at most
// rel_tol * ||S||_F, which bounds ||S - Q diag(d) Q^*||_F (0: run to the FP64 rounding floor).
// Returns the number of Jacobi sweeps run.
int heev(pt_ctx* ctx, const c128* S, int N, c128* Q, double* d, cudaStream_t st, int max_sweeps = 30,
         const c128* Q0 = nullptr, double rel_tol = 0.0);
// A (overwritten) = L L^* ; L written to a separate buffer; *info = k+1 on a bad pivot k.
template <class T>
void cholesky(pt_ctx* ctx, cx<T>* A, int N, cx<T>* L, int* info, cudaStream_t st);
// X = L^{-1} for the factor of the preceding cholesky(ctx, ...) of the same precision (uses its
// diagonal-block inverses)
template <class T>
void tri_inv_lower(pt_ctx* ctx, const cx<T>* L, int N, cx<T>* X, cudaStream_t st);
// C = alpha op(A) op(B) + beta D in the precision of T (op in {N, C, T}; D may be C)
template <class T>
void gemm(char opA, char opB, int m, int n, int k, cx<T> alpha, const cx<T>* A, int lda, const cx<T>* B, int ldb,
          cx<T> beta, const cx<T>* D, int ldd, cx<T>* C, int ldc, cudaStream_t st);
void scale_cols_pow(const c128* U, const double* lam, int N, double power, c128* out, int* info, cudaStream_t st);
void small_solve(const double* G, const double* rhs, int m, double reg, double* x, cudaStream_t st);
void set_identity(c128* A, int N, cudaStream_t st);
void add_diagonal(c128* A, int N, double v, cudaStream_t st);

// ---- Anderson mixing (anderson.cu) ----
template <class T>
struct AndersonSeg {
  const cx<T>* rk;     // current residual
  const cx<T>* rprev;  // previous residual
  const cx<T>* dxp;    // x_k - x_{k-1} from the last update
  cx<T>* dRs;          // new history entry dR_s (written)
  cx<T>* Zs;           // new history entry Z_s = dX + beta dR_s (written)
  const cx<T>* dR[20]; // the other entries' dR, in the caller's order
  size_t n;
};
// dots: for each other entry o: <dR_o, dR_s>, <dR_o, r_k>; then <dR_s, dR_s>, <dR_s, r_k>
// (orbital segment weighted by w_phi, sigma segment by 1)
template <class T>
void anderson_prepare(pt_ctx* ctx, const AndersonSeg<T>& phi, const AndersonSeg<double>& sig, int mo, double beta,
                      double w_phi, double* dots, cudaStream_t st);
void anderson_gram(double* G, const double* dots, int s, const int* others_d, int mo, const int* order_d, int m,
                   double* Gp, double* rhs, cudaStream_t st);
// x += beta r - sum_a gamma_a Z_a;  dxp = that increment
template <class T>
void anderson_update(pt_ctx* ctx, cx<T>* x, const cx<T>* r, const cx<T>* const* Z, int m, const double* gamma,
                     double beta, cx<T>* dxp, size_t n, cudaStream_t st);

// ---- Hamiltonian (hamiltonian.cu) ----
// sphere masks of the compile-time column passes (cubic grids of side n <= 64): bit z of
// mask[y * n + x] is set when 0.5 (g2[x] + g2[n + y] + g2[2n + z]) <= ecut, the FP64 test of the
// basis sphere, evaluated once per (grid, ecut) and kept in the context
const unsigned long long* sphere_masks(pt_ctx* ctx, const pt_grid& g, const double* g2d, double ecut,
                                       cudaStream_t st);
// out = P_sph[ -1/2 Lap psi + y ],  y = vloc*psi + alpha*X (X may be null)
// A: vector potential of the velocity-gauge field (host double[3]; null = no field)
void apply_h(pt_ctx* ctx, const void* psi, int M, void* out, const double* vloc, const void* X, double alpha,
             double ecut, const pt_grid& g, pt_precision prec, cudaStream_t st, const double* A = nullptr);
// in place on the orbital residual r (Ng x N): r_j <- IFFT[m_j(G) FFT(r_j)] with
// m_j = 1/(1 + i dt/2 (|G + A|^2/2 - Re A_jj)) inside the sphere |G|^2/2 <= ecut, 1 outside;
// A: N x N device matrix <Phi_h|H Phi_h>; Avec: vector potential (host double[3] or null)
void precondition_residual(pt_ctx* ctx, void* r, int N, const c128* A, double dt, double ecut, const pt_grid& g,
                           pt_precision prec, cudaStream_t st, const double* Avec);
// J_a = spin/Omega Re sum_ij sigma_ij <phi_j|(-i d_a + A_a) phi_i> (host J[3]; synchronises st)
void current(pt_ctx* ctx, const void* phi, const c128* sigma, int N, const pt_grid& g, pt_precision prec,
             const double* A, double spin, double* J, cudaStream_t st);

void conj_transpose(const c128* A, int N, c128* B, cudaStream_t st);

// ---- plane-wave basis of the Ecut sphere (pw.cu; cubic grids of side <= 64) ----
// Orbitals as unitary-FFT coefficients at the plane waves |G|^2/2 <= ecut, each vector npad long
// (npw coefficients, zero padding); inner products over the grid equal those over the coefficients.
struct PwBasis {
  pt_grid grid;
  double ecut;
  size_t npw, npad;
  const unsigned long long* masks;  // bit z of masks[y n + x]: (x, y, z) in the sphere
  const int* col_off;               // index of the first plane wave of column (y, x)
  const int* xyz;                   // plane wave -> x | y << 8 | z << 16 (-1 on the padding)
  const int* yact;                  // the y rows that hold sphere points (ny_act of them)
  int ny_act;
  unsigned long long ymask;         // bit y: row y holds sphere points
  std::shared_ptr<void> tables;     // owner of col_off and xyz
};
bool pw_applies(const pt_grid& g);
const PwBasis& pw_basis(pt_ctx* ctx, const pt_grid& g, double ecut, cudaStream_t st);
// c = coefficients of the M real-space fields phi (projection onto the sphere); with check, returns
// the part of sum |phi|^2 outside the sphere as a fraction of the whole (synchronises st), else 0
template <class T>
double pw_from_grid(pt_ctx* ctx, const PwBasis& b, const cx<T>* phi, int M, cx<T>* c, cudaStream_t st,
                    bool check = false);
// phi = the M real-space fields of the coefficient vectors c
template <class T>
void pw_to_grid(pt_ctx* ctx, const PwBasis& b, const cx<T>* c, int M, cx<T>* phi, cudaStream_t st);
// out = coefficients of P_sph[1/2 (-i grad + A)^2 psi + vloc psi] + alpha X for coefficient vectors c
// (X: coefficient vectors or null; Avec: vector potential, host double[3] or null)
template <class T>
void pw_apply_h(pt_ctx* ctx, const PwBasis& b, const cx<T>* c, int M, cx<T>* out, const double* vloc, const cx<T>* X,
                double alpha, const double* Avec, cudaStream_t st);
// r_j(G) <- r_j(G) / (1 + i dt/2 (|G + A|^2/2 - Re A_jj)) (the kinetic preconditioner, diagonal here)
template <class T>
void pw_precondition(pt_ctx* ctx, const PwBasis& b, cx<T>* r, int M, const c128* A, double dt, const double* Avec,
                     cudaStream_t st);

// ---- PT-IM step (ptim.cu) ----
pt_status ptim_step(pt_ctx* ctx, void* phi, void* sigma, int N, const double* vloc, const pt_grid& g,
                    const pt_kernel& k, const pt_ptim_params& P, pt_precision prec, pt_ptim_stats* stats,
                    cudaStream_t st);

// ---- ACE (ace.cu) ----
// xi from (phi, W): M = <phi|W>, -M = L L^*, xi = W L^{-*}.  Synchronises st (pivot check).
// nvec: length of each vector when they are not grid fields (plane-wave coefficient vectors; 0:
// the grid's Ng); the inner products keep the grid's dV either way.
void ace_from_w(pt_ctx* ctx, const void* W, const void* phi, int N, const pt_grid& g, pt_precision prec, void* xi,
                cudaStream_t st, size_t nvec = 0);
// out = -xi (xi^* psi)  (+ beta*out0 is not supported: out is overwritten)
void ace_apply(pt_ctx* ctx, const void* xi, int N, const void* psi, int M, void* out, const pt_grid& g,
               pt_precision prec, cudaStream_t st, size_t nvec = 0);

// ---- FMA throughput of the device (peaks.cu), TFLOP/s; synchronises st ----
void alu_peaks(pt_ctx* ctx, double* fp32_tflops, double* fp64_tflops, cudaStream_t st);

// ---- bounded-wait self-test (selftest.cu): PT_TIMEOUT when arrive = 0; synchronises st ----
void wait_selftest(pt_ctx* ctx, int arrive, double timeout_s, cudaStream_t st);

}  // namespace pt
