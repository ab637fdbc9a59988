"""GPU parity of the velocity-gauge external field (Eq. 1's V_ext(t) as a uniform vector potential
A) and of the current observable, through the C ABI, against the FP64 oracle.

Tolerances: H with the field as the field-free H parity (FP64 1e-11, FP32 1e-5 relative); the
current to 1e-11 (FP64) and 1e-5 (FP32) of the sum of |terms| it is made of (spin/Omega
sum_j sum_G |G + A| |phi_j(G)| |chi_j(G)|); PT-IM steps as the field-free step parity.
"""
import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A0 = (0.31, -0.17, 0.08)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,L", [((24, 24, 24), (9.0, 9.0, 9.0)), ((9, 10, 12), (5.0, 5.5, 6.5))])
def test_apply_H_with_field_matches_oracle(ctx, precision, shape, L):
    """Compile-time kernels (cubic 24^3) and generic kernels (9 x 10 x 12), no exchange term."""
    rng = np.random.default_rng(501)
    cell = synth.Cell(shape, L)
    g = O.grid_of(cell)
    psi = synth.random_orbitals(rng, cell, 7, ecut=4.0)
    v = rng.standard_normal(g.shape) * 0.2
    ref = O.apply_H(psi, v, g, 4.0, 0.0, 0 * psi, np.array(A0))
    dt = np.complex128 if precision == "fp64" else np.complex64
    out = ctx.apply_H(dev(psi.astype(dt)), dev(v), None, 0.0, 4.0, cell=cell, precision=precision, A=A0)
    assert rel(out.cpu().numpy().astype(np.complex128), ref) <= (1e-11 if precision == "fp64" else 1e-5)
    # the field changes H by (G.A + |A|^2/2) inside the sphere: a real difference
    free = O.apply_H(psi, v, g, 4.0, 0.0, 0 * psi)
    assert rel(free, ref) > 1e-3


def _current_scale(phi, sig, g, A, spin):
    G = O.g_vectors(g)
    f = np.fft.fftn(phi, axes=(1, 2, 3))
    chi = np.fft.fftn(O.rotate(phi, sig), axes=(1, 2, 3))
    w = np.sum(np.abs(f) * np.abs(chi), axis=0)
    return np.array([spin / g.ng ** 2 * np.sum(np.abs(G[a] + A[a]) * w) for a in range(3)])


@pytest.mark.parametrize("mode", ["fp64", "fp32", "fp32_tc"])
@pytest.mark.parametrize("shape", [(9, 10, 12), (32, 32, 32)])
def test_current_matches_oracle(ctx, mode, shape):
    rng = np.random.default_rng(502)
    cell = synth.Cell(shape, (6.0, 6.5, 7.0))
    g = O.grid_of(cell)
    N = 40
    phi = synth.random_orbitals(rng, cell, N, ecut=4.0)
    sig = np.diag(np.linspace(1.0, 0.05, N)).astype(complex)
    X = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    sig += 0.01 * (X + X.conj().T)
    prec = "fp32" if mode == "fp32_tc" else mode
    ph = phi if prec == "fp64" else phi.astype(np.complex64)
    p64 = ph.astype(np.complex128)
    for A in (None, A0):
        ref = O.current(p64, sig, g, None if A is None else np.array(A))
        ctx.set_option("tc_gram", 1 if mode == "fp32_tc" else 0)
        try:
            J = ctx.current(dev(ph), dev(sig), cell=cell, precision=prec, A=A)
        finally:
            ctx.set_option("tc_gram", 0)
        scale = _current_scale(p64, sig, g, np.zeros(3) if A is None else np.array(A), 2.0)
        assert np.all(np.abs(J - ref) <= (1e-11 if prec == "fp64" else 1e-5) * scale), (J, ref, scale)


def _case():
    w = synth.small_cell(23, 12, 8.0, 6, kT=0.05, ecut=6.0)
    sig = np.diag(w.occ).astype(np.complex128)
    sig[0, 1] = sig[1, 0] = 0.03
    sig[2, 4] = 0.02j
    sig[4, 2] = -0.02j
    return w, sig


@pytest.fixture(scope="module")
def ref_field():
    w, sig = _case()
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    out = {}
    for hxc in (False, True):
        phi1, sig1, st = O.ptim_step(w.phi, sig, w.vloc, g, K, O.PtimParams(tol=1e-12, ecut=6.0, A=A0, hxc=hxc))
        assert st.converged
        out[hxc] = (phi1, sig1)
    return out


@pytest.mark.parametrize("hxc", [False, True])
def test_ptim_step_with_field_fp64_matches_oracle(ctx, ref_field, hxc):
    w, sig = _case()
    phi, sigma = dev(w.phi), dev(sig)
    st = ctx.ptim_step(phi, sigma, dev(w.vloc), cell=w.cell, kernel=w.kernel, precision="fp64", dt=0.5,
                       ecut=6.0, tol=1e-12, A=A0, hxc=hxc)
    assert st["converged"]
    assert rel(phi.cpu().numpy(), ref_field[hxc][0]) <= 1e-10
    assert np.abs(sigma.cpu().numpy() - ref_field[hxc][1]).max() <= 1e-10


def test_ptim_step_with_field_fp32_matches_oracle(ctx, ref_field):
    w, sig = _case()
    phi, sigma = dev(w.phi.astype(np.complex64)), dev(sig)
    ctx.set_option("tc_gram", 1)
    try:
        st = ctx.ptim_step(phi, sigma, dev(w.vloc), cell=w.cell, kernel=w.kernel, precision="fp32", dt=0.5,
                           ecut=6.0, tol=2e-6, A=A0)
    finally:
        ctx.set_option("tc_gram", 0)
    assert st["converged"]
    assert rel(phi.cpu().numpy().astype(np.complex128), ref_field[False][0]) <= 5e-5
    assert np.abs(sigma.cpu().numpy() - ref_field[False][1]).max() <= 5e-5
