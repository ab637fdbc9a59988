"""Pins of the oracle's self-consistent local potential V_Hxc[rho] (Eq. 1) and of the PT-IM
step that uses it.

Facts used (none is the oracle restated): the Hartree potential of a cosine density is a cosine
scaled by 4 pi/|G|^2; the Slater exchange energy of the uniform gas is -0.458165/rs Ha per
electron; the Perdew-Zunger fit's high-density coefficient is the Gell-Mann-Brueckner
(1 - ln 2)/pi^2 and its two branches meet with a continuous slope at rs = 1; a potential is the
derivative of its energy (checked by central differences); the density integrates to the number
of electrons; and a PT-IM step with V_Hxc[rho(t)] is a second-order integrator of the same
ODE integrated by RK4 at a 100x smaller step (the paper's accuracy methodology, Sec. VII-A).
"""
import math

import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth


def ortho_grid():
    return O.Grid(6, 8, 10, 7.0, 9.0, 11.0)


def rs_to_rho(rs):
    return 3.0 / (4.0 * math.pi * rs ** 3)


# --------------------------------------------------------------------------------------
# Hartree
# --------------------------------------------------------------------------------------

def test_hartree_of_cosine_densities_closed_form():
    """rho = rho0 + sum_k a_k cos(G_k.r + t_k) -> V_H = sum_k a_k 4 pi/|G_k|^2 cos(G_k.r + t_k)."""
    g = ortho_grid()
    z, y, x = np.meshgrid(np.arange(g.nz) * g.Lz / g.nz, np.arange(g.ny) * g.Ly / g.ny,
                          np.arange(g.nx) * g.Lx / g.nx, indexing="ij")
    modes = [((1, 0, 0), 0.3, 0.1), ((0, 2, 0), -0.2, 1.0), ((0, 0, 3), 0.15, -0.5), ((2, -1, 1), 0.05, 2.0)]
    rho = np.full(g.shape, 0.7)
    ref = np.zeros(g.shape)
    for (mx, my, mz), a, t in modes:
        G = np.array([2 * math.pi * mx / g.Lx, 2 * math.pi * my / g.Ly, 2 * math.pi * mz / g.Lz])
        phase = G[0] * x + G[1] * y + G[2] * z + t
        rho += a * np.cos(phase)
        ref += a * 4 * math.pi / float(G @ G) * np.cos(phase)
    v = O.hartree_potential(rho, g)
    assert np.abs(v - ref).max() < 1e-12 * np.abs(ref).max()
    # a uniform density has no Hartree potential (neutralising background)
    assert np.abs(O.hartree_potential(np.full(g.shape, 0.3), g)).max() < 1e-14


# --------------------------------------------------------------------------------------
# LDA
# --------------------------------------------------------------------------------------

def test_slater_exchange_of_the_uniform_gas():
    """eps_x = -0.458165/rs Ha (textbook value of -(3/4)(9/(4 pi^2))^(1/3)); v_x = 4/3 eps_x."""
    for rs in (0.3, 1.0, 2.0, 5.0):
        rho = rs_to_rho(rs)
        # correlation alone, from the fit, subtracted to isolate exchange
        eps, v = O.lda_xc(np.array([rho]))
        if rs >= 1:
            s = math.sqrt(rs)
            ec = O.PZ_GAMMA / (1 + O.PZ_BETA1 * s + O.PZ_BETA2 * rs)
        else:
            ec = O.PZ_A * math.log(rs) + O.PZ_B + O.PZ_C * rs * math.log(rs) + O.PZ_D * rs
        assert abs((eps[0] - ec) * rs + 0.458165) < 2e-6


def test_pz_high_density_limit_and_branch_continuity():
    """A = (1 - ln 2)/pi^2 (Gell-Mann-Brueckner), and both eps_c and d eps_c/d rs continuous at rs = 1."""
    assert abs(O.PZ_A - (1 - math.log(2)) / math.pi ** 2) < 2e-5
    below = O.lda_xc(np.array([rs_to_rho(1 - 1e-9)]))
    above = O.lda_xc(np.array([rs_to_rho(1 + 1e-9)]))
    assert abs(below[0][0] - above[0][0]) < 5e-5  # the published fit joins to about 3e-5 Ha
    assert abs(below[1][0] - above[1][0]) < 5e-5
    # slopes of the two branches at rs = 1
    lo = O.PZ_A + O.PZ_C + O.PZ_D
    hi = -O.PZ_GAMMA * (O.PZ_BETA1 / 2 + O.PZ_BETA2) / (1 + O.PZ_BETA1 + O.PZ_BETA2) ** 2
    assert abs(lo - hi) < 1e-4


@pytest.mark.parametrize("rs", [0.05, 0.4, 0.99, 1.01, 2.5, 8.0, 40.0])
def test_vxc_is_the_derivative_of_rho_eps(rs):
    """v_xc(rho) = d(rho eps_xc)/d rho (fourth-order central difference in log rho)."""
    rho = rs_to_rho(rs)
    h = 1e-3

    def f(r):
        return r * O.lda_xc(np.array([r]))[0][0]

    d = (-f(rho * math.exp(2 * h)) + 8 * f(rho * math.exp(h)) - 8 * f(rho * math.exp(-h))
         + f(rho * math.exp(-2 * h))) / (12 * h * rho)
    v = O.lda_xc(np.array([rho]))[1][0]
    assert abs(d - v) < 1e-8 * max(1.0, abs(v))


def test_zero_and_negative_densities_give_zero():
    eps, v = O.lda_xc(np.array([0.0, -1e-12, 1e-40]))
    assert np.all(eps == 0) and np.all(v == 0)


# --------------------------------------------------------------------------------------
# V_Hxc as the functional derivative of E_H + E_xc; the density
# --------------------------------------------------------------------------------------

def test_hxc_potential_is_the_functional_derivative():
    g = ortho_grid()
    rng = np.random.default_rng(7)
    rho = 0.02 + 0.015 * rng.random(g.shape)
    drho = rng.standard_normal(g.shape) * 1e-3
    h = 1e-3

    def E(r):
        return sum(O.hxc_energy(r, g))

    dE = (E(rho + h * drho) - E(rho - h * drho)) / (2 * h)
    lin = g.dV * float(np.sum(O.hxc_potential(rho, g) * drho))
    assert abs(dE - lin) < 1e-7 * abs(lin)


def test_density_integrates_to_trace_and_matches_diagonal_form():
    w = synth.small_cell(5, 10, 8.0, 5, kT=0.05, ecut=6.0)
    g = O.grid_of(w.cell)
    sig = np.diag(w.occ).astype(complex)
    sig[0, 3] = 0.04 + 0.01j
    sig[3, 0] = np.conj(sig[0, 3])
    rho = O.density(w.phi, sig)
    assert np.abs(rho.imag).max() < 1e-14 * np.abs(rho).max()
    assert abs(g.dV * rho.real.sum() - np.trace(sig).real) < 1e-12
    Q, d = O.diagonalize_occupations(sig)
    pt = O.rotate(w.phi, Q)
    assert np.abs(rho.real - np.einsum("k,kzyx->zyx", d, np.abs(pt) ** 2)).max() < 1e-12 * np.abs(rho).max()


# --------------------------------------------------------------------------------------
# PT-IM with V_Hxc[rho(t)]
# --------------------------------------------------------------------------------------

def _rhs_hxc(phi, sigma, vloc, g, K, ecut, alpha, spin):
    v = vloc + O.hxc_potential(spin * O.density(phi, sigma).real, g)
    vx = O.apply_exchange_sigma(phi, sigma, phi, K)
    Hphi = O.apply_H(phi, v, g, ecut, alpha, vx)
    A = O.overlap(phi, Hphi, g.dV)
    S = O.overlap(phi, phi, g.dV)
    R = Hphi - O.rotate(phi, np.linalg.solve(S, A))
    return -1j * R, -1j * (A @ sigma - sigma @ A)


def _rk4_hxc(phi, sigma, vloc, g, K, ecut, alpha, spin, T, steps):
    h = T / steps
    for _ in range(steps):
        k1 = _rhs_hxc(phi, sigma, vloc, g, K, ecut, alpha, spin)
        k2 = _rhs_hxc(phi + 0.5 * h * k1[0], sigma + 0.5 * h * k1[1], vloc, g, K, ecut, alpha, spin)
        k3 = _rhs_hxc(phi + 0.5 * h * k2[0], sigma + 0.5 * h * k2[1], vloc, g, K, ecut, alpha, spin)
        k4 = _rhs_hxc(phi + h * k3[0], sigma + h * k3[1], vloc, g, K, ecut, alpha, spin)
        phi = phi + h / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        sigma = sigma + h / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
    return phi, sigma


def _hxc_workload():
    w = synth.small_cell(33, 8, 7.0, 3, kT=0.05, ecut=4.0)
    g = O.grid_of(w.cell)
    sig0 = np.diag(w.occ).astype(complex)
    sig0[0, 2] = sig0[2, 0] = 0.04
    return w, g, O.exchange_kernel(g, 1, 0.106), sig0


def test_ptim_hxc_invariants_and_ace_fixed_point():
    """With V_Hxc: Phi^*Phi, tr sigma, tr sigma^2 conserved; ACE and exact V_x share the fixed point;
    and the step differs from the frozen-potential step (the density term acts)."""
    w, g, K, sig0 = _hxc_workload()
    a = O.ptim_step(w.phi, sig0, w.vloc, g, K, O.PtimParams(tol=1e-13, ecut=4.0, hxc=True))
    b = O.ptim_step(w.phi, sig0, w.vloc, g, K, O.PtimParams(tol=1e-13, ecut=4.0, hxc=True, use_ace=False))
    c = O.ptim_step(w.phi, sig0, w.vloc, g, K, O.PtimParams(tol=1e-13, ecut=4.0))
    assert a[2].converged and b[2].converged
    phi1, sig1 = a[0], a[1]
    assert abs(np.trace(sig1) - np.trace(sig0)) < 1e-11
    assert abs(np.trace(sig1 @ sig1) - np.trace(sig0 @ sig0)) < 1e-11
    assert np.abs(O.overlap(phi1, phi1, g.dV) - np.eye(3)).max() < 1e-13
    assert np.abs(a[0] - b[0]).max() < 1e-11 * np.abs(a[0]).max()
    assert np.abs(a[1] - b[1]).max() < 1e-11
    Pa = np.einsum("ir,ij,js->rs", a[0].reshape(3, -1), a[1], a[0].reshape(3, -1).conj())
    Pc = np.einsum("ir,ij,js->rs", c[0].reshape(3, -1), c[1], c[0].reshape(3, -1).conj())
    assert np.abs(Pa - Pc).max() > 1e-4 * np.abs(Pc).max()


@pytest.mark.slow
def test_ptim_hxc_matches_rk4_and_is_second_order():
    """One PT-IM step with V_Hxc[rho(t)] vs RK4 at dt/100: local error O(dt^3) (ratio ~8 per halving).

    Evaluating the density anywhere but at the midpoint would make the step first order."""
    w, g, K, sig0 = _hxc_workload()
    errs = []
    for dt in (0.4, 0.2):
        p = O.PtimParams(tol=1e-14, dt=dt, use_ace=False, ecut=4.0, hxc=True)
        phi1, sig1, st = O.ptim_step(w.phi, sig0, w.vloc, g, K, p)
        assert st.converged
        phir, sigr = _rk4_hxc(w.phi, sig0, w.vloc, g, K, 4.0, 0.25, 2.0, dt, 100)
        P1 = np.einsum("ir,ij,js->rs", phi1.reshape(3, -1), sig1, phi1.reshape(3, -1).conj())
        Pr = np.einsum("ir,ij,js->rs", phir.reshape(3, -1), sigr, phir.reshape(3, -1).conj())
        errs.append(np.abs(P1 - Pr).max() / np.abs(Pr).max())
    ratio = errs[0] / errs[1]
    assert 5.0 < ratio < 11.0, (errs, ratio)


@pytest.mark.slow
def test_ptim_hxc_energy_drift_is_second_order():
    """E = E_kin+loc + E_H + E_xc + E_x stays bounded; its drift falls ~4x when dt halves."""
    w, g, K, sig0 = _hxc_workload()
    E0 = O.total_energy(w.phi, sig0, w.vloc, g, K, 4.0, hxc=True)
    drifts = []
    for dt, steps in ((0.4, 5), (0.2, 10)):
        phi, sig = w.phi, sig0
        worst = 0.0
        p = O.PtimParams(tol=1e-13, dt=dt, ecut=4.0, hxc=True)
        for _ in range(steps):
            phi, sig, st = O.ptim_step(phi, sig, w.vloc, g, K, p)
            assert st.converged
            worst = max(worst, abs(O.total_energy(phi, sig, w.vloc, g, K, 4.0, hxc=True) - E0))
        drifts.append(worst)
    assert drifts[0] < 1e-2 * abs(E0)
    assert 2.5 < drifts[0] / drifts[1] < 6.0, drifts
