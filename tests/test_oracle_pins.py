"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test compares the oracle with something that is not the oracle: an
O(Ng^2) real-space convolution, closed forms for plane waves, operator
identities, exact invariants of the implicit midpoint rule, a dense
diagonalisation of a tiny Hamiltonian, and an explicit RK4 integration of the
same ODE at a 100x smaller step (the paper's accuracy methodology, Sec. VII-A).
Orthorhombic grids with distinct nx, ny, nz are used where an axis mix-up
could otherwise hide.
"""
import math

import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth


def rand_orbitals(rng, g, N, scale=1.0):
    a = rng.standard_normal((N,) + g.shape) + 1j * rng.standard_normal((N,) + g.shape)
    return scale * a / math.sqrt(g.volume)


def ortho_grid():
    return O.Grid(6, 8, 10, 7.0, 9.0, 11.0)


# --------------------------------------------------------------------------------------
# p1: FFT convolution == direct real-space convolution with k(r) from an explicit DFT sum
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("ktype", [0, 1])
@pytest.mark.parametrize("shape", [(6, 8, 10), (8, 8, 8)])
def test_pair_potential_matches_direct_convolution(ktype, shape):
    nx, ny, nz = shape
    g = O.Grid(nx, ny, nz, 7.0, 9.0, 11.0)
    rng = np.random.default_rng(1)
    a, b = rand_orbitals(rng, g, 2)
    K = O.exchange_kernel(g, ktype, 0.35)
    v = O.pair_potential(a, b, K)
    # k(r) = (1/Omega) sum_G K(G) exp(i G.r), explicit sum over every grid G
    mx = np.arange(nx); mx = np.where(mx < (nx + 1) // 2, mx, mx - nx)
    my = np.arange(ny); my = np.where(my < (ny + 1) // 2, my, my - ny)
    mz = np.arange(nz); mz = np.where(mz < (nz + 1) // 2, mz, mz - nz)
    # K values indexed independently of the oracle's table: recompute from |G|^2
    Gx, Gy, Gz = 2 * np.pi * mx / g.Lx, 2 * np.pi * my / g.Ly, 2 * np.pi * mz / g.Lz
    X = np.arange(nx) * g.Lx / nx
    Y = np.arange(ny) * g.Ly / ny
    Z = np.arange(nz) * g.Lz / nz
    k = np.zeros((nz, ny, nx), dtype=complex)
    mu = 0.35
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                G2 = Gx[ix] ** 2 + Gy[iy] ** 2 + Gz[iz] ** 2
                if G2 == 0:
                    Kg = 0.0 if ktype == 0 else math.pi / mu ** 2
                elif ktype == 0:
                    Kg = 4 * math.pi / G2
                else:
                    Kg = 4 * math.pi / G2 * (1 - math.exp(-G2 / (4 * mu * mu)))
                k += Kg * np.exp(1j * (Gz[iz] * Z[:, None, None] + Gy[iy] * Y[None, :, None] + Gx[ix] * X[None, None, :]))
    k /= g.volume
    rho = np.conj(a) * b
    direct = np.zeros_like(rho)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                # k(r - r') for every r', periodic
                kk = k[np.ix_((z - np.arange(nz)) % nz, (y - np.arange(ny)) % ny, (x - np.arange(nx)) % nx)]
                direct[z, y, x] = g.dV * np.sum(kk * rho)
    assert np.abs(direct - v).max() < 1e-12 * np.abs(v).max()


# --------------------------------------------------------------------------------------
# p2: plane-wave closed forms
# --------------------------------------------------------------------------------------

def _wrap(m, n):
    m = m % n
    return m if m < (n + 1) // 2 else m - n


def _Kclosed(g, dm, mu, ktype=1):
    mx, my, mz = (_wrap(dm[0], g.nx), _wrap(dm[1], g.ny), _wrap(dm[2], g.nz))
    G2 = (2 * np.pi * mx / g.Lx) ** 2 + (2 * np.pi * my / g.Ly) ** 2 + (2 * np.pi * mz / g.Lz) ** 2
    if G2 == 0:
        return math.pi / mu ** 2 if ktype == 1 else 0.0
    base = 4 * math.pi / G2
    return base if ktype == 0 else base * (1 - math.exp(-G2 / (4 * mu * mu)))


PW_FREQS = [(0, 0, 0), (1, 0, 0), (0, -1, 2), (2, 3, -1), (-3, 1, 4)]


@pytest.mark.parametrize("ktype", [0, 1])
def test_exchange_of_plane_waves_closed_form(ktype):
    g = ortho_grid()
    cell = synth.Cell((g.nx, g.ny, g.nz), (g.Lx, g.Ly, g.Lz))
    phi = synth.plane_wave_orbitals(cell, PW_FREQS)
    d = np.array([1.0, 0.7, 0.3, 0.05, 0.9])
    mu = 0.4
    K = O.exchange_kernel(g, ktype, mu)
    vx = O.apply_exchange(phi, d, phi, K)
    for j, Gj in enumerate(PW_FREQS):
        lam = -sum(d[i] * _Kclosed(g, np.subtract(Gj, Gi), mu, ktype) for i, Gi in enumerate(PW_FREQS)) / g.volume
        assert np.abs(vx[j] - lam * phi[j]).max() < 1e-12 * np.abs(lam * phi[j]).max()
    # exchange energy E_x = -(spin alpha / 2 Omega) sum_ij d_i d_j K(G_j - G_i)
    Ex = O.exchange_energy(phi, np.diag(d).astype(complex), K, g.dV, alpha=0.25, spin=2.0)
    ref = -(2 * 0.25 / (2 * g.volume)) * sum(
        d[i] * d[j] * _Kclosed(g, np.subtract(PW_FREQS[j], PW_FREQS[i]), mu, ktype)
        for i in range(5) for j in range(5))
    assert abs(Ex - ref) < 1e-12 * abs(ref)


@pytest.mark.parametrize("ktype", [0, 1])
def test_exchange_energy_by_pairs_plane_waves_closed_form(ktype):
    """The one-FFT-per-pair (Parseval) energy route: plane waves give
    sum_i d_i <phi_i|V_x phi_i> = -(1/Omega) sum_ij d_i d_j K(G_j - G_i) exactly."""
    g = ortho_grid()
    cell = synth.Cell((g.nx, g.ny, g.nz), (g.Lx, g.Ly, g.Lz))
    phi = synth.plane_wave_orbitals(cell, PW_FREQS)
    d = np.array([1.0, 0.7, 0.3, 0.05, 0.9])
    mu = 0.4
    K = O.exchange_kernel(g, ktype, mu)
    s = O.exchange_energy_pairs(phi, d, K, g.dV)
    ref = -sum(d[i] * d[j] * _Kclosed(g, np.subtract(PW_FREQS[j], PW_FREQS[i]), mu, ktype)
               for i in range(5) for j in range(5)) / g.volume
    assert abs(s - ref) < 1e-12 * abs(ref)


def test_exchange_energy_by_pairs_matches_the_exchange_route():
    """Random (non-orthogonal, complex) orbitals on an orthorhombic grid: the Parseval route equals
    sum_i d_i <phi_i|V_x phi_i> through apply_exchange (forward and inverse FFTs per ordered
    pair), and splitting the rows i sums to the whole."""
    g = ortho_grid()
    rng = np.random.default_rng(12)
    phi = rand_orbitals(rng, g, 5)
    d = np.array([0.9, 0.0, 0.4, 1.0, 0.15])
    K = O.exchange_kernel(g, 1, 0.3)
    vx = O.apply_exchange(phi, d, phi, K)
    ref = float(np.real(np.sum(d * np.diag(O.overlap(phi, vx, g.dV)))))
    s = O.exchange_energy_pairs(phi, d, K, g.dV)
    assert abs(s - ref) < 1e-12 * abs(ref)
    parts = O.exchange_energy_pairs(phi, d, K, g.dV, rows=[0, 3]) + O.exchange_energy_pairs(phi, d, K, g.dV,
                                                                                            rows=[1, 2, 4])
    assert abs(parts - s) < 1e-13 * abs(s)
    # and the spin alpha/2 scaled value is the oracle's exchange energy of sigma = diag(d)
    Ex = O.exchange_energy(phi, np.diag(d).astype(complex), K, g.dV, alpha=0.25, spin=2.0)
    assert abs(2 * 0.125 * s - Ex) < 1e-12 * abs(Ex)


def test_mixed_exchange_of_plane_waves_closed_form():
    """Full sigma: V_x phi_j = -(1/Omega^{3/2}) sum_ik sigma_ik K(G_j-G_k) e^{i(G_i+G_j-G_k).r}."""
    g = ortho_grid()
    cell = synth.Cell((g.nx, g.ny, g.nz), (g.Lx, g.Ly, g.Lz))
    freqs = PW_FREQS[:4]
    phi = synth.plane_wave_orbitals(cell, freqs)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    sigma = 0.5 * (A + A.conj().T)
    mu = 0.4
    K = O.exchange_kernel(g, 1, mu)
    vx = O.apply_exchange_mixed(phi, sigma, phi, K)
    X = np.arange(g.nx) / g.nx
    Y = np.arange(g.ny) / g.ny
    Z = np.arange(g.nz) / g.nz
    for j, Gj in enumerate(freqs):
        ref = np.zeros(g.shape, dtype=complex)
        for i, Gi in enumerate(freqs):
            for k, Gk in enumerate(freqs):
                m = np.add(np.subtract(Gi, Gk), Gj)
                ph = 2j * np.pi * (m[2] * Z[:, None, None] + m[1] * Y[None, :, None] + m[0] * X[None, None, :])
                ref += sigma[i, k] * _Kclosed(g, np.subtract(Gj, Gk), mu) * np.exp(ph)
        ref *= -1.0 / g.volume ** 1.5
        assert np.abs(vx[j] - ref).max() < 1e-12 * np.abs(ref).max()


# --------------------------------------------------------------------------------------
# p3: Hermiticity and sign of V_x
# --------------------------------------------------------------------------------------

def test_exchange_is_hermitian_negative_semidefinite():
    g = ortho_grid()
    rng = np.random.default_rng(5)
    src = rand_orbitals(rng, g, 5)
    d = rng.uniform(0, 1, 5)
    K = O.exchange_kernel(g, 1, 0.3)
    assert K.min() > 0
    ab = rand_orbitals(rng, g, 4)
    vab = O.apply_exchange(src, d, ab, K)
    M = O.overlap(ab, vab, g.dV)
    assert np.abs(M - M.conj().T).max() < 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.conj().T)).max() < 1e-12 * np.abs(M).max()
    assert np.all(np.real(np.diag(M)) < 0)


# --------------------------------------------------------------------------------------
# p4: ACE identity V_ACE Phi = V_x Phi, V_ACE Hermitian and negative semidefinite
# --------------------------------------------------------------------------------------

def test_ace_reproduces_exchange_on_its_orbitals():
    g = ortho_grid()
    rng = np.random.default_rng(9)
    src = rand_orbitals(rng, g, 4)
    d = rng.uniform(0.1, 1, 4)
    K = O.exchange_kernel(g, 1, 0.3)
    phi = rand_orbitals(rng, g, 4)  # not orthonormal on purpose
    W = O.apply_exchange(src, d, phi, K)
    xi = O.build_ace(phi, W, g.dV)
    out = O.apply_ace(xi, phi, g.dV)
    assert np.abs(out - W).max() < 1e-12 * np.abs(W).max()
    psi = rand_orbitals(rng, g, 3)
    C = O.overlap(psi, O.apply_ace(xi, psi, g.dV), g.dV)
    assert np.abs(C - C.conj().T).max() < 1e-12 * np.abs(C).max()
    assert np.linalg.eigvalsh(0.5 * (C + C.conj().T)).max() < 1e-12 * np.abs(C).max()


# --------------------------------------------------------------------------------------
# p5: triple sum (mixed states) == diagonalised double sum
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("N", [4, 5])
def test_diagonalised_exchange_equals_triple_sum(N):
    g = ortho_grid()
    rng = np.random.default_rng(20 + N)
    phi = rand_orbitals(rng, g, N)
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    sigma = 0.3 * (A + A.conj().T)
    K = O.exchange_kernel(g, 1, 0.3)
    tgt = rand_orbitals(rng, g, 3)
    a = O.apply_exchange_mixed(phi, sigma, tgt, K)
    b = O.apply_exchange_sigma(phi, sigma, tgt, K)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
    Q, dd = O.diagonalize_occupations(sigma)
    assert np.abs(Q @ np.diag(dd) @ Q.conj().T - sigma).max() < 1e-13 * np.abs(sigma).max()
    assert np.all(np.diff(dd) >= 0)


# --------------------------------------------------------------------------------------
# PT-IM step pins (p6-p10)
# --------------------------------------------------------------------------------------

def small_workload(n=10, N=4, seed=11, kT=0.05):
    w = synth.small_cell(seed, n, 8.0, N, kT=kT, ecut=6.0)
    return w, O.grid_of(w.cell)


def test_ptim_quadratic_invariants():
    """Implicit midpoint conserves Phi^*Phi, tr sigma and tr sigma^2 at the fixed point (p6)."""
    w, g = small_workload()
    K = O.exchange_kernel(g, 1, 0.106)
    rng = np.random.default_rng(2)
    sig0 = np.diag(w.occ).astype(complex)
    sig0[0, 1] = sig0[1, 0] = 0.05  # off-diagonal coherence
    sig0[2, 3] = 0.03j
    sig0[3, 2] = -0.03j
    p = O.PtimParams(tol=1e-13, dt=0.5)
    phi1, sig1, st = O.ptim_step(w.phi, sig0, w.vloc, g, K, p)
    assert st.converged
    assert st.orth_error < 1e-11
    assert abs(np.trace(sig1) - np.trace(sig0)) < 1e-11
    assert abs(np.trace(sig1 @ sig1) - np.trace(sig0 @ sig0)) < 1e-11
    assert np.abs(sig1 - sig1.conj().T).max() < 1e-14
    assert np.abs(O.overlap(phi1, phi1, g.dV) - np.eye(w.N)).max() < 1e-13
    assert np.abs(phi1 - w.phi).max() > 1e-3  # it actually moved
    del rng


def test_ptim_free_electron_cayley_closed_form():
    """alpha = 0, V = 0, plane waves: Phi fixed, sigma_ij -> sigma_ij (1 - i dt w/2)/(1 + i dt w/2) (p7)."""
    g = O.Grid(8, 8, 8, 9.0, 9.0, 9.0)
    cell = synth.Cell((8, 8, 8), (9.0,) * 3)
    freqs = [(0, 0, 0), (1, 0, 0), (0, 1, 1), (1, -1, 0)]
    phi = synth.plane_wave_orbitals(cell, freqs)
    rng = np.random.default_rng(4)
    A = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    sigma = 0.1 * (A + A.conj().T) + np.diag([0.9, 0.6, 0.3, 0.1])
    K = O.exchange_kernel(g, 1, 0.106)
    dt = 0.7
    p = O.PtimParams(tol=1e-14, dt=dt, alpha=0.0, ecut=50.0)
    phi1, sig1, st = O.ptim_step(phi, sigma, np.zeros(g.shape), g, K, p)
    assert st.converged
    eps = np.array([0.5 * sum((2 * np.pi * m / 9.0) ** 2 for m in f) for f in freqs])
    w = eps[:, None] - eps[None, :]
    ref = sigma * (1 - 0.5j * dt * w) / (1 + 0.5j * dt * w)
    assert np.abs(sig1 - ref).max() < 1e-12
    assert np.abs(phi1 - phi).max() < 1e-12 * np.abs(phi).max()


def test_ptim_plane_waves_with_exchange_are_stationary():
    """alpha != 0, diagonal sigma, plane waves: every term of H is diagonal, the step is the identity (p7)."""
    g = O.Grid(8, 8, 8, 9.0, 9.0, 9.0)
    cell = synth.Cell((8, 8, 8), (9.0,) * 3)
    phi = synth.plane_wave_orbitals(cell, [(0, 0, 0), (1, 0, 0), (0, 0, -1)])
    sigma = np.diag([1.0, 0.5, 0.25]).astype(complex)
    K = O.exchange_kernel(g, 1, 0.106)
    p = O.PtimParams(tol=1e-14, dt=0.5, alpha=0.25, ecut=50.0)
    phi1, sig1, st = O.ptim_step(phi, sigma, np.zeros(g.shape), g, K, p)
    assert np.abs(sig1 - sigma).max() < 1e-13
    assert np.abs(phi1 - phi).max() < 1e-12 * np.abs(phi).max()


def test_ptim_eigenstates_are_stationary():
    """alpha = 0, V_loc != 0: exact eigenvectors of the projected H with diagonal sigma do not move (p8)."""
    g = O.Grid(8, 8, 8, 8.0, 8.0, 8.0)
    cell = synth.Cell((8, 8, 8), (8.0,) * 3)
    rng = np.random.default_rng(6)
    v = synth.gaussian_wells(cell, synth.silicon_like_sites(rng, 8, 8.0), depth=1.0, width=1.0)
    ecut = 3.0
    # dense H in the plane-wave basis of the Ecut sphere, independent of the oracle's FFT path
    m = [np.where(np.arange(n) < (n + 1) // 2, np.arange(n), np.arange(n) - n) for n in (8, 8, 8)]
    basis = [(mx, my, mz) for mz in m[2] for my in m[1] for mx in m[0]
             if 0.5 * ((2 * np.pi / 8.0) ** 2) * (mx * mx + my * my + mz * mz) <= ecut]
    X = np.arange(8) / 8
    vhat = {}
    def vq(q):  # (1/Ng) sum_r V(r) e^{-i q.r}, aliased onto the grid
        q = tuple(int(c) % 8 for c in q)
        if q not in vhat:
            ph = np.exp(-2j * np.pi * (q[2] * X[:, None, None] + q[1] * X[None, :, None] + q[0] * X[None, None, :]))
            vhat[q] = np.sum(v * ph) / 512
        return vhat[q]
    nb = len(basis)
    H = np.zeros((nb, nb), dtype=complex)
    for a, Ga in enumerate(basis):
        H[a, a] += 0.5 * (2 * np.pi / 8.0) ** 2 * sum(c * c for c in Ga)
        for b, Gb in enumerate(basis):
            H[a, b] += vq(np.subtract(Ga, Gb))
    e, C = np.linalg.eigh(H)
    N = 4
    freqs = basis
    pw = synth.plane_wave_orbitals(cell, freqs)
    phi = np.einsum("ga,gzyx->azyx", C[:, :N], pw)
    sigma = np.diag([1.0, 0.8, 0.4, 0.1]).astype(complex)
    K = O.exchange_kernel(g, 1, 0.106)
    p = O.PtimParams(tol=1e-14, dt=0.5, alpha=0.0, ecut=ecut)
    phi1, sig1, st = O.ptim_step(phi, sigma, v, g, K, p)
    assert np.abs(sig1 - sigma).max() < 1e-12
    assert np.abs(phi1 - phi).max() < 1e-11 * np.abs(phi).max()


def _pt_rhs(phi, sigma, vloc, g, K, ecut, alpha):
    """Right-hand side of the PT gauge ODE (Eq. PTIM): (-i (I - Pt) H Phi, -i [Phi^* H Phi, sigma])."""
    vx = O.apply_exchange_sigma(phi, sigma, phi, K) if alpha else 0 * phi
    Hphi = O.apply_H(phi, vloc, g, ecut, alpha, vx)
    A = O.overlap(phi, Hphi, g.dV)
    S = O.overlap(phi, phi, g.dV)
    R = Hphi - O.rotate(phi, np.linalg.solve(S, A))
    return -1j * R, -1j * (A @ sigma - sigma @ A)


def _rk4(phi, sigma, vloc, g, K, ecut, alpha, T, steps):
    h = T / steps
    for _ in range(steps):
        k1 = _pt_rhs(phi, sigma, vloc, g, K, ecut, alpha)
        k2 = _pt_rhs(phi + 0.5 * h * k1[0], sigma + 0.5 * h * k1[1], vloc, g, K, ecut, alpha)
        k3 = _pt_rhs(phi + 0.5 * h * k2[0], sigma + 0.5 * h * k2[1], vloc, g, K, ecut, alpha)
        k4 = _pt_rhs(phi + h * k3[0], sigma + h * k3[1], vloc, g, K, ecut, alpha)
        phi = phi + h / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        sigma = sigma + h / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
    return phi, sigma


@pytest.mark.slow
def test_ptim_matches_rk4_and_is_second_order():
    """One PT-IM step vs RK4 at dt/100 on the same ODE: local error O(dt^3) (p9, Sec. VII-A)."""
    w = synth.small_cell(31, 8, 7.0, 3, kT=0.05, ecut=4.0)
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, 0.106)
    sig0 = np.diag(w.occ).astype(complex)
    sig0[0, 2] = sig0[2, 0] = 0.04
    errs = []
    for dt in (0.4, 0.2):
        p = O.PtimParams(tol=1e-14, dt=dt, use_ace=False, ecut=4.0)
        phi1, sig1, st = O.ptim_step(w.phi, sig0, w.vloc, g, K, p)
        assert st.converged
        phir, sigr = _rk4(w.phi, sig0, w.vloc, g, K, 4.0, 0.25, dt, 100)
        # gauge-invariant comparison through the density matrix P = Phi sigma Phi^*
        P1 = np.einsum("ir,ij,js->rs", phi1.reshape(3, -1), sig1, phi1.reshape(3, -1).conj())
        Pr = np.einsum("ir,ij,js->rs", phir.reshape(3, -1), sigr, phir.reshape(3, -1).conj())
        errs.append(np.abs(P1 - Pr).max() / np.abs(Pr).max())
        assert np.abs(sig1 - sigr).max() < 50 * dt ** 3
    ratio = errs[0] / errs[1]
    assert 5.0 < ratio < 11.0, (errs, ratio)


@pytest.mark.slow
def test_ptim_energy_drift_is_second_order():
    """Field-free total energy stays bounded and its drift falls ~4x when dt halves (p9)."""
    w = synth.small_cell(41, 8, 7.0, 3, kT=0.05, ecut=4.0)
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, 0.106)
    sig0 = np.diag(w.occ).astype(complex)
    sig0[0, 1] = sig0[1, 0] = 0.05
    E0 = O.total_energy(w.phi, sig0, w.vloc, g, K, 4.0)
    drifts = []
    for dt, steps in ((0.4, 5), (0.2, 10)):
        phi, sig = w.phi, sig0
        worst = 0.0
        p = O.PtimParams(tol=1e-13, dt=dt, ecut=4.0)
        for _ in range(steps):
            phi, sig, st = O.ptim_step(phi, sig, w.vloc, g, K, p)
            assert st.converged
            worst = max(worst, abs(O.total_energy(phi, sig, w.vloc, g, K, 4.0) - E0))
        drifts.append(worst)
    assert drifts[0] < 1e-2 * abs(E0)
    assert 2.5 < drifts[0] / drifts[1] < 6.0, drifts


def test_ptim_ace_and_exact_share_the_fixed_point():
    """PT-IM-ACE and PT-IM with V_x applied exactly converge to the same step (p10)."""
    w, g = small_workload(n=10, N=4, seed=13)
    K = O.exchange_kernel(g, 1, 0.106)
    sig0 = np.diag(w.occ).astype(complex)
    sig0[1, 2] = sig0[2, 1] = 0.02
    a = O.ptim_step(w.phi, sig0, w.vloc, g, K, O.PtimParams(tol=1e-13))
    b = O.ptim_step(w.phi, sig0, w.vloc, g, K, O.PtimParams(tol=1e-13, use_ace=False))
    assert a[2].converged and b[2].converged
    assert np.abs(a[0] - b[0]).max() < 1e-11 * np.abs(a[0]).max()
    assert np.abs(a[1] - b[1]).max() < 1e-11


def test_kernel_small_g_limit_and_coulomb_zero():
    g = O.Grid(4, 4, 4, 1e5, 1e5, 1e5)  # tiny |G|: screened kernel approaches pi/mu^2
    K = O.exchange_kernel(g, 1, 0.5)
    assert abs(K.ravel()[1] - math.pi / 0.25) < 1e-3 * math.pi / 0.25
    assert K.ravel()[0] == math.pi / 0.25
    assert O.exchange_kernel(g, 0).ravel()[0] == 0.0
