"""Degenerate occupation matrices in the PT-IM step, against the oracle: the pure state sigma = I
and sigma = I/2 (every eigenvalue equal, so the eigenbasis is arbitrary and only basis-independent
results are compared; such steps take the pure-state path: no eigensolve or commutator, sigma stays
c I) and a diagonal sigma with exactly empty
orbitals (pairs of two empty orbitals are skipped by the exchange)."""
import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


SIGMAS = {
    "pure": np.eye(6, dtype=np.complex128),
    "pure_half": 0.5 * np.eye(6, dtype=np.complex128),
    "empty_orbitals": np.diag([1.0, 1.0, 0.9, 0.0, 0.0, 0.0]).astype(np.complex128),
}


@pytest.fixture(scope="module")
def refs():
    w = synth.small_cell(41, 12, 8.0, 6, kT=0.05, ecut=6.0)
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    out = {}
    for name, sig in SIGMAS.items():
        phi1, sig1, st = O.ptim_step(w.phi, sig, w.vloc, g, K, O.PtimParams(tol=1e-12, ecut=6.0))
        assert st.converged
        out[name] = (phi1, sig1)
    return w, out


@pytest.mark.parametrize("name", list(SIGMAS))
@pytest.mark.parametrize("precision,tc_gram,tol,bar", [("fp64", 0, 1e-12, 1e-10), ("fp32", 1, 2e-6, 5e-5)])
def test_degenerate_sigma_step_matches_oracle(ctx, refs, name, precision, tc_gram, tol, bar):
    w, out = refs
    phi1, sig1 = out[name]
    dt = np.complex128 if precision == "fp64" else np.complex64
    phi = torch.from_numpy(w.phi.astype(dt)).cuda()
    sigma = torch.from_numpy(SIGMAS[name].copy()).cuda()
    ctx.set_option("tc_gram", tc_gram)
    try:
        st = ctx.ptim_step(phi, sigma, torch.from_numpy(w.vloc).cuda(), cell=w.cell, kernel=w.kernel,
                           precision=precision, dt=0.5, ecut=6.0, tol=tol)
    finally:
        ctx.set_option("tc_gram", 0)
    assert st["converged"]
    s = sigma.cpu().numpy()
    # basis-independent comparison: the density matrix P = Phi sigma Phi^* on the grid
    p = phi.cpu().numpy().astype(np.complex128).reshape(6, -1)
    r = phi1.reshape(6, -1)
    P = np.einsum("ir,ij,js->rs", p, s, p.conj())
    R = np.einsum("ir,ij,js->rs", r, sig1, r.conj())
    assert rel(P, R) <= bar
    assert np.abs(s - sig1).max() <= bar
    if name.startswith("pure"):
        # sigma_n = c I takes the pure-state path (Eq. pure_vx): no eigensolve, sigma stays c I
        assert st["pure_state"] and st["eig_sweeps"] == 0 and st["phase_ms"]["sigma_eig"] == 0.0
        assert np.abs(s - SIGMAS[name]).max() == 0.0
    else:
        assert not st["pure_state"]
