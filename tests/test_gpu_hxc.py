"""GPU parity of the self-consistent local potential (Eq. 1's V_Hxc[P]) through the C ABI:
the density rho = spin P(r, r), the Hartree + LDA potential with its energies, and PT-IM steps
that rebuild V_Hxc from the midpoint density, against the FP64 oracle on the same inputs.

Tolerances: FP64 results to 1e-11 relative (FFT rounding); the FP32 density element-wise within
2e-6 of spin * sum_ij |sigma_ij| |phi_i| |phi_j| (FP32 products and the rotation chi = Phi sigma,
summed in FP64); PT-IM steps as the frozen-potential step parity (FP64 1e-10, FP32 5e-5).
"""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def hermitian_sigma(rng, occ, coh=0.03):
    N = len(occ)
    s = np.diag(occ).astype(np.complex128)
    c = coh * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) / np.sqrt(N)
    return s + 0.5 * (c + c.conj().T)


@pytest.mark.parametrize("mode", ["fp64", "fp32", "fp32_tc"])
@pytest.mark.parametrize("shape", [(9, 10, 12), (24, 24, 24)])
def test_density_matches_oracle(ctx, mode, shape):
    """N = 70 (ragged rotation tiles), non-diagonal Hermitian sigma, ragged and cubic grids."""
    rng = np.random.default_rng(401)
    cell = synth.Cell(shape, (6.0, 6.5, 7.0))
    phi = synth.random_orbitals(rng, cell, 70, ecut=4.0)
    sig = hermitian_sigma(rng, np.linspace(1.0, 0.02, 70))
    prec = "fp32" if mode == "fp32_tc" else mode
    ph = phi if prec == "fp64" else phi.astype(np.complex64)
    ctx.set_option("tc_gram", 1 if mode == "fp32_tc" else 0)
    try:
        rho = ctx.density(dev(ph), dev(sig), cell=cell, precision=prec, spin=2.0).cpu().numpy()
    finally:
        ctx.set_option("tc_gram", 0)
    p64 = ph.astype(np.complex128)
    ref = 2.0 * O.density(p64, sig).real
    if prec == "fp64":
        assert np.abs(rho - ref).max() <= 1e-12 * np.abs(ref).max()
    else:
        a = np.abs(p64).reshape(70, -1)
        scale = 2.0 * np.einsum("ir,ij,jr->r", a, np.abs(sig), a).reshape(ref.shape)
        assert np.all(np.abs(rho - ref) <= 2e-6 * scale), float((np.abs(rho - ref) / scale).max())
    assert abs(O.grid_of(cell).dV * rho.sum() - 2.0 * np.trace(sig).real) < 1e-4


@pytest.mark.parametrize("shape,L", [((9, 10, 12), (5.0, 5.5, 6.0)), ((32, 32, 32), (12.0, 12.0, 12.0))])
def test_hxc_potential_and_energies_match_oracle(ctx, shape, L):
    """Densities spanning both Perdew-Zunger branches (rs from ~0.3 to ~20), exact zeros and
    rounding-negative points (eps = v = 0 there), with and without V_loc."""
    rng = np.random.default_rng(402)
    cell = synth.Cell(shape, L)
    g = O.grid_of(cell)
    rho = np.exp(rng.uniform(np.log(3e-5), np.log(8.0), size=g.shape))
    flat = rho.reshape(-1)
    flat[:7] = 0.0
    flat[7:11] = -1e-13
    vloc = rng.standard_normal(g.shape) * 0.3
    ref = vloc + O.hxc_potential(rho, g)
    eh, exc = O.hxc_energy(rho, g)
    v, (geh, gexc) = ctx.hxc_potential(dev(rho), dev(vloc), cell=cell, energies=True)
    v = v.cpu().numpy()
    assert np.abs(v - ref).max() <= 1e-11 * np.abs(ref).max()
    assert abs(geh - eh) <= 1e-11 * abs(eh)
    assert abs(gexc - exc) <= 1e-11 * abs(exc)
    v0 = ctx.hxc_potential(dev(rho), None, cell=cell).cpu().numpy()
    assert np.abs(v0 - (ref - vloc)).max() <= 1e-11 * np.abs(ref).max()


def test_hxc_rejects_aliasing(ctx):
    from paper_2501_03061_gb300 import _lib as L
    from paper_2501_03061_gb300 import api
    cell = synth.cubic(8, 5.0)
    r = torch.ones((8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(api.PtimError) as ei:
        ctx.hxc_potential(r, cell=cell, out=r)
    assert ei.value.status == L.PT_INVALID_ARG


# ---------------------------------------------------------------------------- PT-IM with V_Hxc ----

def _case():
    w = synth.small_cell(23, 12, 8.0, 6, kT=0.05, ecut=6.0)
    sig = np.diag(w.occ).astype(np.complex128)
    sig[0, 1] = sig[1, 0] = 0.03
    sig[2, 4] = 0.02j
    sig[4, 2] = -0.02j
    return w, sig


@pytest.fixture(scope="module")
def ref_hxc():
    w, sig = _case()
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    phi1, sig1, st = O.ptim_step(w.phi, sig, w.vloc, g, K, O.PtimParams(tol=1e-12, ecut=6.0, hxc=True))
    assert st.converged
    return phi1, sig1


@pytest.mark.parametrize("use_ace", [True, False])
def test_ptim_step_hxc_fp64_matches_oracle(ctx, ref_hxc, use_ace):
    w, sig = _case()
    phi, sigma = dev(w.phi), dev(sig)
    st = ctx.ptim_step(phi, sigma, dev(w.vloc), cell=w.cell, kernel=w.kernel, precision="fp64", dt=0.5,
                       ecut=6.0, tol=1e-12, use_ace=use_ace, hxc=True)
    assert st["converged"]
    assert rel(phi.cpu().numpy(), ref_hxc[0]) <= 1e-10
    assert np.abs(sigma.cpu().numpy() - ref_hxc[1]).max() <= 1e-10
    assert st["phase_ms"]["hxc"] > 0.0


@pytest.mark.parametrize("tc_gram", [0, 1])
def test_ptim_step_hxc_fp32_matches_oracle(ctx, ref_hxc, tc_gram):
    w, sig = _case()
    phi, sigma = dev(w.phi.astype(np.complex64)), dev(sig)
    ctx.set_option("tc_gram", tc_gram)
    try:
        st = ctx.ptim_step(phi, sigma, dev(w.vloc), cell=w.cell, kernel=w.kernel, precision="fp32", dt=0.5,
                           ecut=6.0, tol=2e-6, hxc=True)
    finally:
        ctx.set_option("tc_gram", 0)
    assert st["converged"]
    assert rel(phi.cpu().numpy().astype(np.complex128), ref_hxc[0]) <= 5e-5
    assert np.abs(sigma.cpu().numpy() - ref_hxc[1]).max() <= 5e-5


def test_density_64cubed_N320_sampled(ctx):
    """Full size (64^3, N = 320, FP32 with tensor-core rotation): sampled points against the
    definition rho(r) = spin sum_ij sigma_ij phi_i(r) conj(phi_j(r)) evaluated point by point."""
    rng = np.random.default_rng(403)
    cell = synth.cubic(64, 20.5)
    N = 320
    shp = (N,) + tuple(cell.n[::-1])
    phi = np.empty(shp, dtype=np.complex64)
    phi.real = rng.standard_normal(shp, dtype=np.float32) / 90.0
    phi.imag = rng.standard_normal(shp, dtype=np.float32) / 90.0
    sig = hermitian_sigma(rng, synth.fermi_dirac_occupations(N, 0.02), coh=0.01)
    ctx.set_option("tc_gram", 1)
    try:
        rho = ctx.density(dev(phi), dev(sig), cell=cell, precision="fp32").cpu().numpy().reshape(-1)
    finally:
        ctx.set_option("tc_gram", 0)
    P = phi.reshape(N, -1)
    for r in rng.integers(0, P.shape[1], size=48):
        col = P[:, r].astype(np.complex128)
        ref = 2.0 * np.real(col @ sig @ col.conj())
        scale = 2.0 * np.abs(col) @ np.abs(sig) @ np.abs(col)
        assert abs(rho[r] - ref) <= 2e-6 * scale
