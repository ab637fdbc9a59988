"""FP64 CPU oracle for the finite-temperature PT-IM hybrid-functional hot path.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
statement of what the GPU library computes.  Only the test suite, the smoke
check and the benchmark's CPU-baseline leg may import it; the library never
does, and it shares no code, table or constant with the CUDA path.

Everything is complex128/float64 numpy.  numpy's FFT (forward unnormalised,
inverse divided by Ng) and LAPACK (eigh, cholesky, solve) serve as library
primitives; nothing is blocked, fused or reordered beyond the equations.

Array layouts (same as the library's C ABI):
  orbitals     (N, nz, ny, nx) complex, orbital-major, x fastest
  sigma        (N, N) complex, sigma[i, j] = sigma_ij
  occupations  (N,) float
  potential    (nz, ny, nx) float

Notation: Ng = nx ny nz, Omega = Lx Ly Lz, dV = Omega/Ng,
<a|b> = dV sum_r conj(a(r)) b(r).

Readings of places where the paper is silent or garbled are stated beside the
code that takes them (kernel value at G = 0, spin factor, sphere projection,
ACE sign convention, Anderson details, stopping rule, orthonormalisation).

Parity status per function: every public function here is pinned by the
`-m "not gpu"` tests (direct convolution, plane-wave closed forms, Hermiticity,
ACE identity, triple-sum vs diagonalised exchange, PT-IM invariants, the
Cayley closed form, stationary states, energy conservation and an RK4
cross-check; for V_Hxc: the Hartree potential of cosine densities, the Slater
constant, the Perdew-Zunger high-density limit and branch continuity, potentials
as derivatives of their energies, and PT-IM with V_Hxc[rho(t)] against RK4; for
the velocity-gauge field: plane-wave eigenvalues 1/2 |G + A|^2, the Cayley
closed form under a constant field, the current of plane waves, and PT-IM with
A(t_{n+1/2}) against RK4 with A(t)).  The Anderson trajectory itself (iteration counts, the exact
stop point) is parity unpinned: only converged states are compared.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FFT_AXES = (1, 2, 3)


# ----------------------------------------------------------------------------------------
# Grid, kernel, inner products
# ----------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    Lx: float
    Ly: float
    Lz: float

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ng(self):
        return self.nx * self.ny * self.nz

    @property
    def volume(self):
        return self.Lx * self.Ly * self.Lz

    @property
    def dV(self):
        return self.volume / self.ng


def grid_of(cell) -> Grid:
    """Grid from anything with .n = (nx, ny, nz) and .L = (Lx, Ly, Lz)."""
    return Grid(int(cell.n[0]), int(cell.n[1]), int(cell.n[2]),
                float(cell.L[0]), float(cell.L[1]), float(cell.L[2]))


def _wrapped(n):
    # m in [-n/2, n/2): 0, 1, ..., ceil(n/2)-1, -floor(n/2), ..., -1
    m = np.arange(n)
    return np.where(m < (n + 1) // 2, m, m - n)


def g_squared(g: Grid) -> np.ndarray:
    """|G|^2 on the grid, G = 2 pi m / L with m wrapped to [-n/2, n/2)."""
    gx = 2 * np.pi * _wrapped(g.nx) / g.Lx
    gy = 2 * np.pi * _wrapped(g.ny) / g.Ly
    gz = 2 * np.pi * _wrapped(g.nz) / g.Lz
    return gz[:, None, None] ** 2 + gy[None, :, None] ** 2 + gx[None, None, :] ** 2


def exchange_kernel(g: Grid, ktype: int = 1, mu: float = 0.106, g0: float | None = None) -> np.ndarray:
    """Fourier-space interaction K(G) of V_x(r,r') = -P(r,r') K(r,r') (Sec. II-B, Eq. 1).

    ktype 0: bare Coulomb 4 pi/|G|^2, K(0) = 0 unless g0 is given.
    ktype 1: erfc-screened Coulomb 4 pi/|G|^2 (1 - exp(-|G|^2/(4 mu^2))), K(0) = pi/mu^2,
             the |G| -> 0 limit (the paper states only that K may be screened).
    """
    g2 = g_squared(g)
    K = np.zeros_like(g2)
    nz = g2 > 0
    if ktype == 0:
        K[nz] = 4 * np.pi / g2[nz]
        K[~nz] = 0.0 if g0 is None else g0
    elif ktype == 1:
        K[nz] = 4 * np.pi / g2[nz] * (1.0 - np.exp(-g2[nz] / (4 * mu * mu)))
        K[~nz] = np.pi / (mu * mu) if g0 is None else g0
    else:
        raise ValueError("unknown kernel type")
    return K


def overlap(a: np.ndarray, b: np.ndarray, dV: float) -> np.ndarray:
    """Matrix of inner products  O[i, j] = <a_i|b_j> = dV sum_r conj(a_i) b_j."""
    A = a.reshape(a.shape[0], -1)
    B = b.reshape(b.shape[0], -1)
    return dV * (A.conj() @ B.T)


def rotate(phi: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """Columns of Phi Q:  out_j = sum_k Q[k, j] phi_k  (Phi stored orbital-major)."""
    P = phi.reshape(phi.shape[0], -1)
    return (Q.T @ P).reshape((Q.shape[1],) + phi.shape[1:])


# ----------------------------------------------------------------------------------------
# Fock exchange (Sec. II-B Eqs. pure_vx / mixed_vx; Sec. IV-A1 Eqs. diag_sigma, p_diag, vxdiag)
# ----------------------------------------------------------------------------------------

def pair_potential(phi_i: np.ndarray, phi_j: np.ndarray, K: np.ndarray) -> np.ndarray:
    """v_ij(r) = int K(r - r') conj(phi_i(r')) phi_j(r') dr' on the periodic cell.

    With numpy's convention ifftn(K * fftn(rho)) equals dV sum_r' k(r - r') rho(r')
    where k(r) = (1/Omega) sum_G K(G) e^{iG.r}, i.e. the integral above.
    Pair densities are formed on the wavefunction grid (no de-aliasing).
    """
    rho = np.conj(phi_i) * phi_j
    return np.fft.ifftn(K * np.fft.fftn(rho))


def apply_exchange(src: np.ndarray, occ: np.ndarray, tgt: np.ndarray, K: np.ndarray) -> np.ndarray:
    """(V_x tgt_j)(r) = - sum_i d_i src_i(r) v_ij(r),  v_ij from conj(src_i) tgt_j  (Eq. vxdiag).

    src are the orbitals in the basis that diagonalises sigma, occ = d.  The
    result carries no mixing fraction alpha (alpha multiplies V_x only in H).
    Eq. vxdiag carries the minus sign; the listing of the baseline loop (Alg. 2)
    accumulates with a plus, and the equation is followed here.
    All N*M pairs are formed explicitly; d_i = 0 terms are still computed.
    """
    out = np.zeros_like(tgt, dtype=np.complex128)
    for j in range(tgt.shape[0]):
        acc = np.zeros(tgt.shape[1:], dtype=np.complex128)
        for i in range(src.shape[0]):
            acc += occ[i] * src[i] * pair_potential(src[i], tgt[j], K)
        out[j] = -acc
    return out


def apply_exchange_mixed(phi: np.ndarray, sigma: np.ndarray, tgt: np.ndarray, K: np.ndarray) -> np.ndarray:
    """(V_x[P] tgt_j)(r) = - sum_{i,k} sigma_ik phi_i(r) int K conj(phi_k) tgt_j   (Eq. mixed_vx).

    The N^3 triple sum of the undiagonalised mixed-state exchange; small N only.
    """
    out = np.zeros_like(tgt, dtype=np.complex128)
    N = phi.shape[0]
    for j in range(tgt.shape[0]):
        acc = np.zeros(tgt.shape[1:], dtype=np.complex128)
        for k in range(N):
            v = pair_potential(phi[k], tgt[j], K)
            for i in range(N):
                if sigma[i, k] != 0:
                    acc += sigma[i, k] * phi[i] * v
        out[j] = -acc
    return out


def diagonalize_occupations(sigma: np.ndarray):
    """sigma = Q diag(d) Q^*  (Eq. diag_sigma); ascending d, Hermitian part of sigma."""
    h = 0.5 * (sigma + sigma.conj().T)
    d, Q = np.linalg.eigh(h)
    return Q, d


def apply_exchange_sigma(phi: np.ndarray, sigma: np.ndarray, tgt: np.ndarray, K: np.ndarray) -> np.ndarray:
    """V_x[Phi sigma Phi^*] tgt through the diagonalised form (Eqs. diag_sigma, p_diag, vxdiag)."""
    Q, d = diagonalize_occupations(sigma)
    phit = rotate(phi, Q)
    return apply_exchange(phit, d, tgt, K)


def exchange_energy(phi: np.ndarray, sigma: np.ndarray, K: np.ndarray, dV: float,
                    alpha: float = 0.25, spin: float = 2.0) -> float:
    """E_x = spin * (alpha/2) * Tr[P V_x[P]] = spin*(alpha/2) sum_i d_i <phit_i|V_x phit_i>.

    spin = 2 (closed shell; the paper omits spin degeneracy, Sec. II-A).
    """
    Q, d = diagonalize_occupations(sigma)
    phit = rotate(phi, Q)
    vx = apply_exchange(phit, d, phit, K)
    return float(spin * 0.5 * alpha * np.real(np.sum(d * np.diag(overlap(phit, vx, dV)))))


def exchange_energy_pairs(phit: np.ndarray, d: np.ndarray, K: np.ndarray, dV: float, rows=None) -> float:
    """Sum over pairs of E_x / (spin alpha/2) = sum_i d_i <phit_i|V_x phit_i>, by Parseval.

    With rho_ij = conj(phit_i) phit_j, <phit_i|V_x phit_i> = -sum_j d_j dV sum_r conj(rho_ji) v_ji, and
    sum_r conj(rho) ifftn(K fftn(rho)) = (1/Ng) sum_G K(G) |fftn(rho)(G)|^2, so
        sum_i d_i <phit_i|V_x phit_i> = -(dV/Ng) sum_{i,j} d_i d_j sum_G K(G) |fftn(rho_ij)(G)|^2,
    one forward FFT per unordered pair (|rho_ji^| and |rho_ij^| sum the same K-weighted squares, K
    being even).  `rows` restricts i to a subset (the pairs i <= j with i in rows), so that callers
    can split the sum; the full sum is rows = all i.  Same value as exchange_energy / (spin alpha/2)
    for sigma = diag(d) in the basis phit (Sec. IV-A1, Eq. vxdiag; the energy of Sec. II-B).
    """
    N = phit.shape[0]
    ng = int(np.prod(phit.shape[1:]))
    rows = range(N) if rows is None else rows
    s = 0.0
    for i in rows:
        for j in range(i, N):
            rh = np.fft.fftn(np.conj(phit[i]) * phit[j])
            w = 1.0 if i == j else 2.0
            s += w * d[i] * d[j] * float(np.sum(K * (rh.real ** 2 + rh.imag ** 2)))
    return -dV / ng * s


# ----------------------------------------------------------------------------------------
# Adaptively compressed exchange (Sec. IV-A2, Eq. vx_ace; construction of Lin 2016)
# ----------------------------------------------------------------------------------------

def build_ace(phi: np.ndarray, W: np.ndarray, dV: float) -> np.ndarray:
    """xi such that V_ACE = -xi xi^* (with the dV inner product) satisfies V_ACE phi = W.

    W = V_x phi;  M = <phi|W> (Hermitian, negative definite);  -M = L L^*
    (lower Cholesky);  xi = W L^{-*}.  The printed Eq. vx_ace drops the
    conjugate and mixes indices; this is the construction of the cited ACE
    reference.
    """
    M = overlap(phi, W, dV)
    M = 0.5 * (M + M.conj().T)
    L = np.linalg.cholesky(-M)
    # xi = W L^{-*}: rows of the (N, Ng) array transform with L^{-1} conjugated
    Wm = W.reshape(W.shape[0], -1)
    Linv = np.linalg.inv(L)
    xi = (Linv.conj() @ Wm)  # xi_k = sum_j conj(Linv[k, j]) W_j
    return xi.reshape(W.shape)


def apply_ace(xi: np.ndarray, psi: np.ndarray, dV: float) -> np.ndarray:
    """V_ACE psi = - xi (xi^* psi):  out_j = - sum_k xi_k <xi_k|psi_j>."""
    C = overlap(xi, psi, dV)  # (Nxi, M)
    return -rotate(xi, C)


# ----------------------------------------------------------------------------------------
# Hamiltonian (Eq. 1):  H = -1/2 Laplacian + V_loc + alpha V_x, projected on |G|^2/2 <= Ecut
# ----------------------------------------------------------------------------------------

def sphere_mask(g: Grid, ecut: float) -> np.ndarray:
    """1 on the plane waves with |G|^2/2 <= Ecut, 0 elsewhere (the plane-wave basis)."""
    return (0.5 * g_squared(g) <= ecut).astype(np.float64)


def g_vectors(g: Grid):
    """(Gx, Gy, Gz) on the grid, each broadcast to (nz, ny, nx); G = 2 pi m / L, m wrapped."""
    gx = 2 * np.pi * _wrapped(g.nx) / g.Lx
    gy = 2 * np.pi * _wrapped(g.ny) / g.Ly
    gz = 2 * np.pi * _wrapped(g.nz) / g.Lz
    shape = (g.nz, g.ny, g.nx)
    return (np.broadcast_to(gx[None, None, :], shape), np.broadcast_to(gy[None, :, None], shape),
            np.broadcast_to(gz[:, None, None], shape))


def kinetic_factor(g: Grid, A=None) -> np.ndarray:
    """1/2 |G + A|^2: the kinetic operator 1/2 (-i grad + A)^2 of the velocity gauge in G space
    (Eq. 1's V_ext(t) for a spatially uniform field E(t) = -dA/dt in a periodic cell; A = 0 is the
    field-free 1/2 |G|^2)."""
    if A is None or not np.any(A):
        return 0.5 * g_squared(g)
    G = g_vectors(g)
    return 0.5 * sum((G[a] + A[a]) ** 2 for a in range(3))


def apply_kinetic_local(phi: np.ndarray, vloc: np.ndarray, g: Grid, A=None) -> np.ndarray:
    """(1/2 (-i grad + A)^2 + V_loc) phi without projection: kinetic by FFT, potential pointwise."""
    kin = np.fft.ifftn(kinetic_factor(g, A) * np.fft.fftn(phi, axes=FFT_AXES), axes=FFT_AXES)
    return kin + vloc[None] * phi


def project_sphere(psi: np.ndarray, g: Grid, ecut: float) -> np.ndarray:
    """P_sph psi: drop the plane waves outside the Ecut sphere."""
    mask = sphere_mask(g, ecut)
    return np.fft.ifftn(mask * np.fft.fftn(psi, axes=FFT_AXES), axes=FFT_AXES)


def apply_H(phi: np.ndarray, vloc: np.ndarray, g: Grid, ecut: float, alpha: float, vx_phi: np.ndarray,
            A=None) -> np.ndarray:
    """H phi = P_sph[ 1/2 (-i grad + A)^2 phi + V_loc phi + alpha V_x phi ]   (Eq. 1).

    vx_phi is V_x phi computed by the caller (exactly or through ACE).  The
    projection onto the Ecut sphere keeps the propagation in the plane-wave
    basis of the paper (Ecut = 10 Ha; the sphere is the field-free |G|^2/2 <=
    Ecut, the basis does not move with A); pair densities inside V_x are not
    masked.  A: the uniform vector potential of V_ext(t) (None: no field).  V_x
    needs no field term: as a functional of P it is gauge covariant.
    """
    y = apply_kinetic_local(phi, vloc, g, A) + alpha * vx_phi
    return project_sphere(y, g, ecut)


# ----------------------------------------------------------------------------------------
# Self-consistent local potential V_Hxc[rho] (Eq. 1): Hartree by the periodic Poisson
# equation, exchange-correlation in the local density approximation
# ----------------------------------------------------------------------------------------

def hartree_potential(rho: np.ndarray, g: Grid) -> np.ndarray:
    """V_H solving -Lap V_H = 4 pi (rho - mean rho) on the periodic cell.

    V_H(G) = 4 pi rho(G) / |G|^2 for G != 0 and V_H(0) = 0: the G = 0 term of a periodic cell
    is cancelled by the neutralising background (the paper does not state it; this is the
    standard plane-wave reading).
    """
    g2 = g_squared(g)
    rg = np.fft.fftn(rho)
    vg = np.zeros_like(rg)
    nz = g2 > 0
    vg[nz] = 4 * np.pi * rg[nz] / g2[nz]
    return np.fft.ifftn(vg).real


# Perdew-Zunger (Phys. Rev. B 23, 5048 (1981)) fit of the Ceperley-Alder correlation energy
# of the unpolarised electron gas, per electron, as a function of rs = (3/(4 pi rho))^(1/3)
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334   # rs >= 1
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116  # rs < 1
RHO_FLOOR = 1e-30  # below this density (and for rounding-negative densities) eps = v = 0


def lda_xc(rho: np.ndarray):
    """(eps_xc, v_xc) per point of the LDA: Slater exchange + Perdew-Zunger correlation.

    eps_x = -(3/4) (3 rho / pi)^(1/3),  v_x = d(rho eps_x)/d rho = (4/3) eps_x.
    eps_c from the two Perdew-Zunger branches; v_c = eps_c - (rs/3) d eps_c / d rs.
    The paper's hybrid functional is not named beyond its screened exchange; the local part
    here is the LDA (the semilocal part of HSE-type functionals is PBE, a gradient correction
    that this reading leaves out).
    """
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    m = rho > RHO_FLOOR
    r = rho[m]
    ex = -0.75 * np.cbrt(3.0 * r / np.pi)
    vx = 4.0 / 3.0 * ex
    rs = np.cbrt(3.0 / (4.0 * np.pi * r))
    ec = np.empty_like(r)
    vc = np.empty_like(r)
    hi = rs >= 1.0
    s = np.sqrt(rs[hi])
    den = 1.0 + PZ_BETA1 * s + PZ_BETA2 * rs[hi]
    ec[hi] = PZ_GAMMA / den
    vc[hi] = ec[hi] * (1.0 + 7.0 / 6.0 * PZ_BETA1 * s + 4.0 / 3.0 * PZ_BETA2 * rs[hi]) / den
    lo = ~hi
    x = rs[lo]
    lnx = np.log(x)
    ec[lo] = PZ_A * lnx + PZ_B + PZ_C * x * lnx + PZ_D * x
    vc[lo] = PZ_A * lnx + (PZ_B - PZ_A / 3.0) + 2.0 / 3.0 * PZ_C * x * lnx + (2.0 * PZ_D - PZ_C) / 3.0 * x
    eps[m] = ex + ec
    v[m] = vx + vc
    return eps, v


def hxc_potential(rho: np.ndarray, g: Grid) -> np.ndarray:
    """V_Hxc[rho] = V_H[rho] + v_xc(rho)."""
    return hartree_potential(rho, g) + lda_xc(rho)[1]


def hxc_energy(rho: np.ndarray, g: Grid) -> tuple[float, float]:
    """(E_H, E_xc) = (1/2 int rho V_H, int rho eps_xc); V_Hxc is their functional derivative."""
    eh = 0.5 * g.dV * float(np.sum(rho * hartree_potential(rho, g)))
    exc = g.dV * float(np.sum(rho * lda_xc(rho)[0]))
    return eh, exc


# ----------------------------------------------------------------------------------------
# PT-IM time step (Sec. II-A Eqs. PTIM, n+1/2, p_tilde, lisan, x=tx; Alg. 1; Sec. IV-A2 double loop)
# ----------------------------------------------------------------------------------------

@dataclasses.dataclass
class PtimParams:
    dt: float = 0.5
    alpha: float = 0.25
    ecut: float = 10.0
    tol: float = 1e-13           # relative residual of x = T(x) (inner) and midpoint change (outer)
    max_outer: int = 30
    max_inner: int = 200
    anderson_depth: int = 20      # maximum mixing dimension (Sec. VI)
    anderson_beta: float = 1.0
    use_ace: bool = True
    hxc: bool = False             # V_Hxc[rho_h] from the midpoint density in every iteration
    spin: float = 2.0             # electrons per orbital in rho = spin * P(r, r)
    A: tuple = (0.0, 0.0, 0.0)    # vector potential A(t_{n+1/2}) of V_ext at the step's midpoint time


@dataclasses.dataclass
class PtimStats:
    outer: int = 0
    inner: int = 0
    residual: float = float("nan")
    converged: bool = False
    orth_error: float = float("nan")  # max |Phi^* Phi - I| before the final orthonormalisation


def _norm2(phi, sigma, dV):
    # Euclidean norm of x = (Phi, sigma) with weight dV on the orbital entries
    return float(dV * np.vdot(phi, phi).real + np.vdot(sigma, sigma).real)


class _Anderson:
    """Type-II Anderson mixing with real coefficients on x = (Phi, sigma).

    x_{k+1} = x_k + beta r_k - (dX + beta dR) gamma,  gamma = argmin || r_k - dR gamma ||
    with the real inner product Re<.,.> (dV-weighted on Phi).  Real gamma keeps
    Hermitian sigma iterates Hermitian.  History is reset with each outer
    iteration because the fixed-point map changes with the ACE operator.
    """

    def __init__(self, depth, beta, dV):
        self.depth, self.beta, self.dV = depth, beta, dV
        self.dX, self.dR = [], []
        self.x_prev = self.r_prev = None

    def _vec(self, phi, sigma):
        return np.concatenate([math.sqrt(self.dV) * phi.ravel(), sigma.ravel()])

    def step(self, x, r):
        beta = self.beta
        if self.x_prev is not None:
            self.dX.append(x - self.x_prev)
            self.dR.append(r - self.r_prev)
            if len(self.dX) > self.depth:
                self.dX.pop(0)
                self.dR.pop(0)
        self.x_prev, self.r_prev = x.copy(), r.copy()
        xn = x + beta * r
        if self.dR:
            R = np.stack(self.dR, axis=1)
            Rr = np.concatenate([R.real, R.imag])
            rr = np.concatenate([r.real, r.imag])
            gamma, *_ = np.linalg.lstsq(Rr, rr, rcond=None)
            X = np.stack(self.dX, axis=1)
            xn = xn - (X + beta * R) @ gamma
        return xn


def ptim_step(phi_n: np.ndarray, sigma_n: np.ndarray, vloc: np.ndarray, g: Grid, K: np.ndarray,
              p: PtimParams | None = None):
    """One PT-IM (or PT-IM-ACE) step (Alg. 1 with the double SCF loop of Sec. IV-A2).

    Unknowns x = (Phi_{n+1}, sigma_{n+1}); midpoints (Eq. n+1/2); the fixed-point
    map (Eq. lisan, read with balanced parentheses):
        T_Phi   = Phi_n   - i dt (I - Pt) H Phi_h,   Pt = Phi_h S^{-1} Phi_h^*,  S = Phi_h^* Phi_h
        T_sigma = sigma_n - i dt [A, sigma_h],        A = Phi_h^* H Phi_h
    with H = H(t_{n+1/2}, P_h), P_h = Phi_h sigma_h Phi_h^* (Eq. p_tilde): the time enters through
    p.A = A(t_{n+1/2}), the caller's vector potential at the midpoint time; with p.hxc the local potential
    is V_loc + V_Hxc[spin * P_h(r, r)], else V_loc alone (V_ext + V_Hxc frozen).  Initial guess:
    x = (Phi_n, sigma_n).  Outer loop: diagonalise sigma_h, W = V_x[P_h] Phi_h,
    ACE from (Phi_h, W).  Inner loop: Anderson on x = T(x) with the ACE frozen
    (or V_x applied exactly when use_ace is False).  Outer stop: the midpoint
    the ACE was built on changed by less than tol.  Finally Phi is made
    orthonormal (Loewdin, Phi <- Phi S^{-1/2}, with sigma <- S^{1/2} sigma S^{1/2}
    so P is unchanged) and sigma conjugate-symmetrised.

    Returns (phi_{n+1}, sigma_{n+1}, stats).
    """
    p = p or PtimParams()
    dV = g.dV
    N = phi_n.shape[0]
    phi, sigma = phi_n.copy(), sigma_n.copy()
    stats = PtimStats()
    anchor = None
    for outer in range(p.max_outer):
        stats.outer = outer + 1
        phi_h = 0.5 * (phi + phi_n)
        sig_h = 0.5 * (sigma + sigma_n)
        if anchor is not None:
            dphi = phi_h - anchor[0]
            dsig = sig_h - anchor[1]
            change = math.sqrt(_norm2(dphi, dsig, dV) / _norm2(phi_h, sig_h, dV))
            if change < p.tol and inner_converged:
                stats.converged = True
                stats.outer = outer
                break
        anchor = (phi_h.copy(), sig_h.copy())
        Q, d = diagonalize_occupations(sig_h)
        phit = rotate(phi_h, Q)
        if p.use_ace:
            W = rotate(apply_exchange(phit, d, phit, K), Q.conj().T)  # (V_x phit) Q^*
            xi = build_ace(phi_h, W, dV)
            exch = lambda psi, sh: apply_ace(xi, psi, dV)  # noqa: E731
        else:
            # exact PT-IM: H_{n+1/2} = H[P_{n+1/2}] is rebuilt from the current midpoint
            def exch(psi, sh):
                Qh, dh = diagonalize_occupations(sh)
                pt = rotate(psi, Qh)
                return rotate(apply_exchange(pt, dh, pt, K), Qh.conj().T)

        mixer = _Anderson(p.anderson_depth, p.anderson_beta, dV)
        inner_converged = False
        for inner in range(p.max_inner):
            stats.inner += 1
            phi_h = 0.5 * (phi + phi_n)
            sig_h = 0.5 * (sigma + sigma_n)
            v = vloc
            if p.hxc:  # H_{n+1/2} = H[P_{n+1/2}] (Eq. p_tilde): V_Hxc from rho of the midpoint
                v = vloc + hxc_potential(p.spin * density(phi_h, sig_h).real, g)
            Hphi = apply_H(phi_h, v, g, p.ecut, p.alpha, exch(phi_h, sig_h), np.asarray(p.A, dtype=float))
            A = overlap(phi_h, Hphi, dV)
            S = overlap(phi_h, phi_h, dV)
            SinvA = np.linalg.solve(S, A)
            T_phi = phi_n - 1j * p.dt * (Hphi - rotate(phi_h, SinvA))
            T_sig = sigma_n - 1j * p.dt * (A @ sig_h - sig_h @ A)
            r_phi, r_sig = T_phi - phi, T_sig - sigma
            res = math.sqrt(_norm2(r_phi, r_sig, dV) / _norm2(phi, sigma, dV))
            stats.residual = res
            if res < p.tol:
                inner_converged = True
                break
            x = mixer._vec(phi, sigma)
            r = mixer._vec(r_phi, r_sig)
            xn = mixer.step(x, r)
            phi = (xn[: phi.size] / math.sqrt(dV)).reshape(phi.shape)
            sigma = xn[phi.size:].reshape(sigma.shape)
        if not p.use_ace and inner_converged:
            stats.converged = True
            break
    # Final orthonormalisation and conjugate symmetrisation (Algorithm 1, end of the step)
    S = overlap(phi, phi, dV)
    stats.orth_error = float(np.abs(S - overlap(phi_n, phi_n, dV)).max())
    S = 0.5 * (S + S.conj().T)
    lam, U = np.linalg.eigh(S)
    S_mhalf = (U * lam ** -0.5) @ U.conj().T
    S_half = (U * lam ** 0.5) @ U.conj().T
    phi = rotate(phi, S_mhalf)
    sigma = S_half @ sigma @ S_half
    sigma = 0.5 * (sigma + sigma.conj().T)
    return phi, sigma, stats


# ----------------------------------------------------------------------------------------
# Observables used by the tests
# ----------------------------------------------------------------------------------------

def density(phi: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """rho(r) = sum_ij phi_i(r) sigma_ij conj(phi_j(r))  (Sec. III-C item 1; real for Hermitian sigma)."""
    P = phi.reshape(phi.shape[0], -1)
    return np.einsum("ir,ij,jr->r", P, sigma, P.conj()).reshape(phi.shape[1:])


def current(phi: np.ndarray, sigma: np.ndarray, g: Grid, A=None, spin: float = 2.0) -> np.ndarray:
    """Cell-averaged velocity density J = (spin/Omega) Re Tr[P (-i grad + A)], P = Phi sigma Phi^*.

    Tr[P O] = sum_ij sigma_ij <phi_j|O phi_i>; -i grad is G in Fourier space.  This is the
    observable of a velocity-gauge run (the electric current is -J for electrons of charge -1).
    """
    A = np.zeros(3) if A is None else np.asarray(A, dtype=float)
    G = g_vectors(g)
    fphi = np.fft.fftn(phi, axes=FFT_AXES)
    out = np.zeros(3)
    for a in range(3):
        dphi = np.fft.ifftn((G[a] + A[a])[None] * fphi, axes=FFT_AXES)  # (-i d_a + A_a) phi_i
        B = overlap(phi, dphi, g.dV)  # B[j, i] = <phi_j|(-i d_a + A_a) phi_i>
        out[a] = spin / g.volume * float(np.real(np.sum(sigma * B.T)))
    return out


def total_energy(phi: np.ndarray, sigma: np.ndarray, vloc: np.ndarray, g: Grid, K: np.ndarray,
                 ecut: float, alpha: float = 0.25, spin: float = 2.0, hxc: bool = False, A=None) -> float:
    """E = spin * Tr[P (-1/2 Lap + V_loc)] + spin*(alpha/2) Tr[P V_x[P]] (+ E_H + E_xc), P = Phi sigma Phi^*.

    Tr[P O] = sum_ij sigma_ij <phi_j|O phi_i>.  The energy whose functional
    derivative is spin*H for the Hamiltonian used here (with hxc, rho = spin P(r, r)).
    """
    hphi = project_sphere(apply_kinetic_local(phi, vloc, g, A), g, ecut)
    B = overlap(phi, hphi, g.dV)  # B[j, i] = <phi_j|h phi_i>
    e_one = spin * np.real(np.sum(sigma * B.T))
    e = e_one + exchange_energy(phi, sigma, K, g.dV, alpha, spin)
    if hxc:
        e += sum(hxc_energy(spin * density(phi, sigma).real, g))
    return float(e)
