"""The identities the plane-wave form of the PT-IM step rests on, checked with the oracle on small
cells (no GPU): with c(G) = FFT(phi)(G)/sqrt(Ng) at the plane waves of the Ecut sphere,
  * inner products with the grid's dV are the same sums over the coefficients (Parseval);
  * for an orbital in the sphere, the coefficients of H phi (Eq. 1, projected on the sphere) are
    1/2 |G + A|^2 c + the sphere part of FFT(V_loc phi)/sqrt(Ng) + alpha times those of V_x phi;
  * the kinetic preconditioner of the inner iteration is a multiply by
    1/(1 + i dt/2 (1/2 |G + A|^2 - e_j)) of the coefficients;
  * the oracle's step maps orbitals in the sphere to orbitals in the sphere, so the coefficients
    hold every iterate exactly.
The library's GPU test compares its plane-wave step with its grid step; these pin the algebra."""
import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth


def coefficients(phi, inside):
    """Unitary-FFT coefficients of the fields phi (N, nz, ny, nx) at the sphere points."""
    ng = phi[0].size
    return np.fft.fftn(phi, axes=(1, 2, 3)).reshape(phi.shape[0], -1)[:, inside] / np.sqrt(ng)


@pytest.fixture(scope="module")
def cell():
    w = synth.small_cell(71, 12, 7.0, 6, kT=0.05, ecut=6.0)
    g = O.grid_of(w.cell)
    inside = O.sphere_mask(g, 6.0).ravel() > 0
    return w, g, inside


def test_inner_products_are_sums_over_the_coefficients(cell):
    w, g, inside = cell
    c = coefficients(w.phi, inside)
    S_grid = O.overlap(w.phi, w.phi, g.dV)
    S_pw = g.dV * c.conj() @ c.T
    assert np.abs(S_pw - S_grid).max() < 1e-12
    assert np.abs(S_grid - np.eye(w.phi.shape[0])).max() < 1e-12  # orthonormal orbitals


@pytest.mark.parametrize("A", [None, (0.21, -0.13, 0.07)])
def test_hamiltonian_in_coefficients(cell, A):
    w, g, inside = cell
    rng = np.random.default_rng(5)
    vx = rng.standard_normal(w.phi.shape) + 1j * rng.standard_normal(w.phi.shape)  # any V_x phi
    alpha = 0.25
    H_grid = O.apply_H(w.phi, w.vloc, g, 6.0, alpha, vx, A=None if A is None else np.array(A))
    c = coefficients(w.phi, inside)
    kin = O.kinetic_factor(g, None if A is None else np.array(A)).ravel()[inside]
    H_pw = kin[None] * c + coefficients(w.vloc[None] * w.phi, inside) + alpha * coefficients(vx, inside)
    ref = coefficients(H_grid, inside)
    assert np.abs(H_pw - ref).max() < 1e-12 * np.abs(ref).max()
    # and H phi has nothing outside the sphere
    spec = np.fft.fftn(H_grid, axes=(1, 2, 3)).reshape(w.phi.shape[0], -1)
    assert np.abs(spec[:, ~inside]).max() < 1e-12 * np.abs(spec).max()


def test_preconditioner_is_diagonal_in_coefficients(cell):
    w, g, inside = cell
    rng = np.random.default_rng(6)
    N = w.phi.shape[0]
    r = O.project_sphere(rng.standard_normal(w.phi.shape) + 1j * rng.standard_normal(w.phi.shape), g, 6.0)
    e = rng.uniform(-1.0, 3.0, N)  # orbital energies Re A_jj
    dt = 0.5
    kin = O.kinetic_factor(g)
    # the grid form: each orbital's FFT times m_j inside the sphere, identity outside, back
    m = 1.0 / (1.0 + 0.5j * dt * (kin[None] - e[:, None, None, None]))
    mask = O.sphere_mask(g, 6.0)[None] > 0
    R = np.fft.fftn(r, axes=(1, 2, 3))
    Mr = np.fft.ifftn(np.where(mask, m * R, R), axes=(1, 2, 3))
    diag = 1.0 / (1.0 + 0.5j * dt * (kin.ravel()[inside][None] - e[:, None]))
    assert np.abs(diag * coefficients(r, inside) - coefficients(Mr, inside)).max() < 1e-12


def test_oracle_step_keeps_orbitals_in_the_sphere(cell):
    w, g, inside = cell
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    phi, sigma, st = O.ptim_step(w.phi, w.sigma, w.vloc, g, K, O.PtimParams(ecut=6.0, tol=1e-11))
    assert st.converged
    spec = np.fft.fftn(phi, axes=(1, 2, 3)).reshape(phi.shape[0], -1)
    assert np.abs(spec[:, ~inside]).max() < 1e-11 * np.abs(spec).max()
