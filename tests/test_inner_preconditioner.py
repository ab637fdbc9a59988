"""The kinetic preconditioner proposed for the PT-IM inner iteration, restated with the oracle's
routines on the CPU: Anderson on the preconditioned map x -> x + M (T(x) - x), where M acts on each
orbital column j of the residual as [1 + i dt/2 (1/2|G|^2 - A_jj)]^{-1} in Fourier space inside
the Ecut sphere (A = <Phi_h|H Phi_h>, sigma left alone), reaches the oracle's fixed point in fewer
inner iterations than plain Anderson.  This pins the behaviour a device implementation of the
preconditioner must reproduce (same fixed point, fewer iterations); the unshifted form
(A_jj = 0) is shown to be worse, which is why the shift is part of it."""
import math

import numpy as np

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth


def step(phi_n, sigma_n, vloc, g, K, p, shift=None):
    """The oracle's PT-IM-ACE step (full-tolerance inner loops) with an optional preconditioner:
    shift None = plain Anderson, True = per-orbital shift A_jj, False = no shift."""
    dV = g.dV
    kin = O.kinetic_factor(g)
    inside = O.sphere_mask(g, p.ecut) > 0
    phi, sigma = phi_n.copy(), sigma_n.copy()
    anchor, inner_converged, inner_total = None, False, 0
    for _ in range(p.max_outer):
        phi_h, sig_h = 0.5 * (phi + phi_n), 0.5 * (sigma + sigma_n)
        if anchor is not None:
            move = math.sqrt(O._norm2(phi_h - anchor[0], sig_h - anchor[1], dV) / O._norm2(phi_h, sig_h, dV))
            if move < p.tol and inner_converged:
                break
        anchor = (phi_h.copy(), sig_h.copy())
        Q, d = O.diagonalize_occupations(sig_h)
        phit = O.rotate(phi_h, Q)
        xi = O.build_ace(phi_h, O.rotate(O.apply_exchange(phit, d, phit, K), Q.conj().T), dV)
        mixer = O._Anderson(p.anderson_depth, p.anderson_beta, dV)
        inner_converged = False
        for _ in range(p.max_inner):
            inner_total += 1
            phi_h, sig_h = 0.5 * (phi + phi_n), 0.5 * (sigma + sigma_n)
            hphi = O.apply_H(phi_h, vloc, g, p.ecut, p.alpha, O.apply_ace(xi, phi_h, dV))
            A = O.overlap(phi_h, hphi, dV)
            S = O.overlap(phi_h, phi_h, dV)
            r_phi = phi_n - 1j * p.dt * (hphi - O.rotate(phi_h, np.linalg.solve(S, A))) - phi
            r_sig = sigma_n - 1j * p.dt * (A @ sig_h - sig_h @ A) - sigma
            if math.sqrt(O._norm2(r_phi, r_sig, dV) / O._norm2(phi, sigma, dV)) < p.tol:
                inner_converged = True
                break
            if shift is not None:
                s = np.real(np.diag(A)) if shift else np.zeros(A.shape[0])
                m = 1.0 / (1.0 + 0.5j * p.dt * (kin[None] - s[:, None, None, None]))
                m = np.where(inside[None], m, 1.0)
                r_phi = np.fft.ifftn(m * np.fft.fftn(r_phi, axes=(1, 2, 3)), axes=(1, 2, 3))
            xn = mixer.step(mixer._vec(phi, sigma), mixer._vec(r_phi, r_sig))
            phi = (xn[: phi.size] / math.sqrt(dV)).reshape(phi.shape)
            sigma = xn[phi.size:].reshape(sigma.shape)
    return phi, sigma, inner_total


def test_shifted_kinetic_preconditioner_same_fixed_point_fewer_iterations():
    w = synth.small_cell(1, 16, 10.26, 16, kT=0.02, ecut=10.0)
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    p = O.PtimParams(tol=1e-6, ecut=10.0)
    plain = step(w.phi, w.sigma, w.vloc, g, K, p)
    shifted = step(w.phi, w.sigma, w.vloc, g, K, p, shift=True)
    ref = O.ptim_step(w.phi, w.sigma, w.vloc, g, K, O.PtimParams(tol=1e-12, ecut=10.0))
    for phi, sig, _ in (plain, shifted):
        assert np.linalg.norm(phi - ref[0]) / np.linalg.norm(ref[0]) <= 1e-5
        assert np.abs(sig - ref[1]).max() <= 1e-5
    assert shifted[2] <= 0.7 * plain[2], (plain[2], shifted[2])


def test_unshifted_kinetic_preconditioner_is_slower():
    """Without the orbital's own energy the preconditioner mis-scales the residual of every orbital
    (band-limited orbitals carry several hartree of kinetic energy) and the iteration slows down."""
    w = synth.small_cell(1, 12, 8.0, 8, kT=0.02, ecut=10.0)
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    p = O.PtimParams(tol=1e-6, ecut=10.0, max_inner=300)
    plain = step(w.phi, w.sigma, w.vloc, g, K, p)
    unshifted = step(w.phi, w.sigma, w.vloc, g, K, p, shift=False)
    assert unshifted[2] > plain[2], (plain[2], unshifted[2])
