"""Pins of the oracle's time-dependent external field (Eq. 1's V_ext(t), velocity gauge) and of
the current observable.

Facts used: a plane wave e^{iG.r} is an eigenfunction of 1/2 (-i grad + A)^2 with eigenvalue
1/2 |G + A|^2 (computed here from the integer frequencies and the cell lengths); free plane waves
under a constant field evolve by the Cayley factor of their eigenvalue differences (implicit
midpoint rule); the current of plane-wave occupations is spin/Omega sum_k sigma_kk (G_k + A)
with no contribution from coherences between different plane waves; and the PT-IM step with
the field taken at the midpoint time is a second-order integrator of the ODE with A(t), checked
against RK4 at a 100x smaller step.
"""
import math

import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth

L3 = (7.0, 8.0, 9.5)
SHAPE = (8, 10, 12)  # (nx, ny, nz)


def cell_grid():
    cell = synth.Cell(SHAPE, L3)
    return cell, O.grid_of(cell)


def eig(m, A):
    """1/2 |G + A|^2 for integer frequencies m = (mx, my, mz) on the L3 cell."""
    return 0.5 * sum((2 * math.pi * m[a] / L3[a] + A[a]) ** 2 for a in range(3))


FREQS = [(0, 0, 0), (1, 0, 0), (0, -1, 2), (1, 1, -1)]
A0 = np.array([0.31, -0.17, 0.08])


def test_plane_waves_are_eigenfunctions_with_field():
    cell, g = cell_grid()
    phi = synth.plane_wave_orbitals(cell, FREQS)
    h = O.apply_H(phi, np.zeros(g.shape), g, 50.0, 0.0, 0 * phi, A0)
    for k, m in enumerate(FREQS):
        assert np.abs(h[k] - eig(m, A0) * phi[k]).max() < 1e-12 * np.abs(phi[k]).max()


def test_cayley_closed_form_with_constant_field():
    """alpha = 0, V = 0: Phi fixed, sigma_ij -> sigma_ij (1 - i dt w_ij/2)/(1 + i dt w_ij/2) with
    w_ij = 1/2|G_i + A|^2 - 1/2|G_j + A|^2."""
    cell, g = cell_grid()
    phi = synth.plane_wave_orbitals(cell, FREQS)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    sigma = 0.02 * (X + X.conj().T) + np.diag([0.9, 0.6, 0.3, 0.15])
    assert np.linalg.eigvalsh(sigma).min() > 0  # occupations stay a density matrix (ACE needs M < 0)
    dt = 0.6
    p = O.PtimParams(tol=1e-14, dt=dt, alpha=0.0, ecut=50.0, A=tuple(A0))
    phi1, sig1, st = O.ptim_step(phi, sigma, np.zeros(g.shape), g, O.exchange_kernel(g, 1, 0.106), p)
    assert st.converged
    e = np.array([eig(m, A0) for m in FREQS])
    w = e[:, None] - e[None, :]
    assert np.abs(sig1 - sigma * (1 - 0.5j * dt * w) / (1 + 0.5j * dt * w)).max() < 1e-12
    assert np.abs(phi1 - phi).max() < 1e-12 * np.abs(phi).max()


def test_current_of_plane_waves():
    cell, g = cell_grid()
    phi = synth.plane_wave_orbitals(cell, FREQS)
    sigma = np.diag([0.9, 0.6, 0.3, 0.1]).astype(complex)
    sigma[0, 2] = sigma[2, 0] = 0.05  # coherence between different plane waves: no current
    vol = L3[0] * L3[1] * L3[2]
    for A in (np.zeros(3), A0):
        ref = np.zeros(3)
        for k, m in enumerate(FREQS):
            ref += sigma[k, k].real * np.array([2 * math.pi * m[a] / L3[a] + A[a] for a in range(3)])
        ref *= 2.0 / vol
        assert np.abs(O.current(phi, sigma, g, A, spin=2.0) - ref).max() < 1e-13


def test_current_is_the_field_derivative_of_the_energy():
    """Omega J_a = dE/dA_a (d/dA of 1/2 (-i grad + A)^2 is -i d_a + A_a): central differences of
    the total energy for band-limited orbitals and a complex Hermitian sigma."""
    w = synth.small_cell(19, 10, 8.0, 4, kT=0.05, ecut=5.0)
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, 0.106)
    sig = np.diag(w.occ).astype(complex)
    sig[0, 3] = 0.05 + 0.02j
    sig[3, 0] = np.conj(sig[0, 3])
    A = np.array([0.2, -0.1, 0.05])
    J = O.current(w.phi, sig, g, A)
    h = 1e-4
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        dE = (O.total_energy(w.phi, sig, w.vloc, g, K, 5.0, A=A + e)
              - O.total_energy(w.phi, sig, w.vloc, g, K, 5.0, A=A - e)) / (2 * h)
        assert abs(g.volume * J[a] - dE) < 1e-7 * max(1.0, abs(dE))


def _pulse(t, T=4.0, amp=0.4, w=0.9):
    """A smooth vector potential that is zero at t = 0."""
    return amp * math.sin(math.pi * t / T) ** 2 * math.sin(w * t) * np.array([1.0, 0.5, -0.3])


def _rhs(phi, sigma, vloc, g, K, ecut, alpha, A):
    vx = O.apply_exchange_sigma(phi, sigma, phi, K)
    Hphi = O.apply_H(phi, vloc, g, ecut, alpha, vx, A)
    Am = O.overlap(phi, Hphi, g.dV)
    S = O.overlap(phi, phi, g.dV)
    R = Hphi - O.rotate(phi, np.linalg.solve(S, Am))
    return -1j * R, -1j * (Am @ sigma - sigma @ Am)


def _rk4(phi, sigma, vloc, g, K, ecut, alpha, t0, T, steps):
    h = T / steps
    t = t0
    for _ in range(steps):
        k1 = _rhs(phi, sigma, vloc, g, K, ecut, alpha, _pulse(t))
        k2 = _rhs(phi + 0.5 * h * k1[0], sigma + 0.5 * h * k1[1], vloc, g, K, ecut, alpha, _pulse(t + 0.5 * h))
        k3 = _rhs(phi + 0.5 * h * k2[0], sigma + 0.5 * h * k2[1], vloc, g, K, ecut, alpha, _pulse(t + 0.5 * h))
        k4 = _rhs(phi + h * k3[0], sigma + h * k3[1], vloc, g, K, ecut, alpha, _pulse(t + h))
        phi = phi + h / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        sigma = sigma + h / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
        t += h
    return phi, sigma


@pytest.mark.slow
def test_ptim_with_field_at_midpoint_time_is_second_order():
    """One step from t0 = 1.0 with A(t0 + dt/2) vs RK4 with A(t) at dt/100: local error O(dt^3);
    the field taken at t0 instead is only first order (the error ratio per halving falls to ~4)."""
    w = synth.small_cell(37, 8, 7.0, 3, kT=0.05, ecut=4.0)
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, 0.106)
    sig0 = np.diag(w.occ).astype(complex)
    sig0[0, 1] = sig0[1, 0] = 0.04
    t0 = 1.0

    def err(dt, t_field):
        p = O.PtimParams(tol=1e-14, dt=dt, use_ace=False, ecut=4.0, A=tuple(_pulse(t_field)))
        phi1, sig1, st = O.ptim_step(w.phi, sig0, w.vloc, g, K, p)
        assert st.converged
        phir, sigr = _rk4(w.phi, sig0, w.vloc, g, K, 4.0, 0.25, t0, dt, 100)
        P1 = np.einsum("ir,ij,js->rs", phi1.reshape(3, -1), sig1, phi1.reshape(3, -1).conj())
        Pr = np.einsum("ir,ij,js->rs", phir.reshape(3, -1), sigr, phir.reshape(3, -1).conj())
        return np.abs(P1 - Pr).max() / np.abs(Pr).max()

    mid = [err(dt, t0 + dt / 2) for dt in (0.4, 0.2)]
    assert 5.0 < mid[0] / mid[1] < 11.0, mid
    start = [err(dt, t0) for dt in (0.4, 0.2)]
    assert start[0] / start[1] < 6.0 and start[1] > 3 * mid[1], (start, mid)
