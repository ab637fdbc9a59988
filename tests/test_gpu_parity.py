"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded inputs.

Tolerances: FP64 form ||dV_x Psi||_F/||V_x Psi||_F <= 1e-11; FP32 form <= 1e-5 on V_x Psi and
<= 1e-6 Ha/atom on the exchange energy, both against FP64.
"""

import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 1e-5


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


@pytest.fixture(scope="module")
def w24():
    return synth.exchange_small()


@pytest.fixture(scope="module")
def oracle24(w24):
    g = O.grid_of(w24.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    return O.apply_exchange(w24.phi, w24.occ, w24.phi, K)


# ---------------------------------------------------------------------------- exchange ----

def test_exchange_fp64_24cubed_N16(ctx, w24, oracle24):
    out = ctx.apply_exchange(dev(w24.phi), dev(w24.occ), cell=w24.cell, kernel=w24.kernel, precision="fp64")
    assert rel(out.cpu().numpy(), oracle24) <= FP64_TOL


def test_exchange_fp32_24cubed_N16_and_energy(ctx, w24, oracle24):
    phi32 = dev(w24.phi.astype(np.complex64))
    out = ctx.apply_exchange(phi32, dev(w24.occ), cell=w24.cell, kernel=w24.kernel, precision="fp32")
    got = out.cpu().numpy().astype(np.complex128)
    assert rel(got, oracle24) <= FP32_TOL
    # E_x = spin*(alpha/2) sum_i d_i <phi_i|V_x phi_i>, per atom
    g = O.grid_of(w24.cell)
    ex_gpu = 2 * 0.125 * float(np.real(np.sum(w24.occ * np.diag(O.overlap(w24.phi, got, g.dV)))))
    ex_ref = 2 * 0.125 * float(np.real(np.sum(w24.occ * np.diag(O.overlap(w24.phi, oracle24, g.dV)))))
    assert abs(ex_gpu - ex_ref) / w24.natoms <= 1e-6


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_exchange_general_targets_ragged_multibatch(ctx, precision):
    """tgt != src, orthorhombic 20x24x30 grid, N=7 sources, M=5 targets, tiny batches (ragged tail)."""
    rng = np.random.default_rng(17)
    cell = synth.Cell((20, 24, 30), (7.5, 9.0, 11.0))
    src = synth.random_orbitals(rng, cell, 7, ecut=6.0)
    tgt = synth.random_orbitals(rng, cell, 5, ecut=6.0)
    occ = np.array([1.0, 0.9, 0.0, 0.5, 0.25, 0.0, 0.05])  # exact zeros are skipped
    g = O.grid_of(cell)
    K = O.exchange_kernel(g, 1, 0.2)
    ref = O.apply_exchange(src, occ, tgt, K)
    dt = np.complex128 if precision == "fp64" else np.complex64
    field = g.ng * (16 if precision == "fp64" else 8)
    ctx.set_option("scratch_bytes", 4 * field)  # batches of 2x2 pairs
    try:
        out = ctx.apply_exchange(dev(src.astype(dt)), dev(occ), dev(tgt.astype(dt)), cell=cell,
                                 kernel={"type": 1, "mu": 0.2}, precision=precision)
    finally:
        ctx.set_option("scratch_bytes", 512 << 20)
    assert rel(out.cpu().numpy().astype(np.complex128), ref) <= (FP64_TOL if precision == "fp64" else FP32_TOL)


@pytest.mark.parametrize("n,N", [(30, 9), (36, 5), (40, 4), (45, 3), (54, 3), (60, 2)])
def test_exchange_fp64_radix_mix(ctx, n, N):
    """Every radix path (2,3,4,5,8 and 9=3x3 chains) against the oracle, symmetric pairs, several batches."""
    rng = np.random.default_rng(n)
    cell = synth.cubic(n, 0.32 * n)
    phi = synth.random_orbitals(rng, cell, N, ecut=4.0)
    occ = np.linspace(1.0, 0.1, N)
    g = O.grid_of(cell)
    ref = O.apply_exchange(phi, occ, phi, O.exchange_kernel(g, 1, 0.106))
    ctx.set_option("scratch_bytes", 3 * g.ng * 16)
    try:
        out = ctx.apply_exchange(dev(phi), dev(occ), cell=cell, kernel={"type": 1, "mu": 0.106}, precision="fp64")
    finally:
        ctx.set_option("scratch_bytes", 512 << 20)
    assert rel(out.cpu().numpy(), ref) <= FP64_TOL


def test_exchange_coulomb_kernel_fp64(ctx):
    rng = np.random.default_rng(3)
    cell = synth.Cell((12, 16, 20), (6.0, 8.0, 10.0))
    phi = synth.random_orbitals(rng, cell, 4, ecut=5.0)
    occ = np.array([1.0, 0.6, 0.3, 0.1])
    g = O.grid_of(cell)
    ref = O.apply_exchange(phi, occ, phi, O.exchange_kernel(g, 0))
    out = ctx.apply_exchange(dev(phi), dev(occ), cell=cell, kernel={"type": 0, "mu": 0.0, "g0": 0.0},
                             precision="fp64")
    assert rel(out.cpu().numpy(), ref) <= FP64_TOL


def test_exchange_single_orbital_and_all_zero(ctx):
    cell = synth.cubic(8, 5.0)
    rng = np.random.default_rng(1)
    phi = synth.random_orbitals(rng, cell, 1, ecut=8.0)
    g = O.grid_of(cell)
    ref = O.apply_exchange(phi, np.array([0.7]), phi, O.exchange_kernel(g, 1, 0.3))
    out = ctx.apply_exchange(dev(phi), dev(np.array([0.7])), cell=cell, kernel={"type": 1, "mu": 0.3})
    assert rel(out.cpu().numpy(), ref) <= FP64_TOL
    out0 = ctx.apply_exchange(dev(phi), dev(np.array([0.0])), cell=cell, kernel={"type": 1, "mu": 0.3})
    assert float(out0.abs().max()) == 0.0


def test_exchange_rejects_bad_grid(ctx):
    from paper_2501_03061_gb300.api import PtimError
    cell = synth.cubic(14, 5.0)  # 14 = 2*7 is not 2,3,5-smooth
    phi = torch.zeros((2, 14, 14, 14), dtype=torch.complex128, device="cuda")
    with pytest.raises(PtimError, match="PT_INVALID_ARG"):
        ctx.apply_exchange(phi, torch.ones(2, dtype=torch.float64), cell=cell)


def test_exchange_sampled_targets_at_64cubed_N320(ctx):
    """Full-size workload (64^3, N=320, FP32, the benchmark's launch configuration): sampled targets vs oracle."""
    w = synth.ptim_cell128()
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    out = ctx.apply_exchange(dev(w.phi.astype(np.complex64)), dev(w.occ), cell=w.cell, kernel=w.kernel,
                             precision="fp32")
    got = out.cpu().numpy()
    for j in (0, 131, 319):
        ref = O.apply_exchange(w.phi, w.occ, w.phi[j:j + 1], K)[0]
        assert rel(got[j].astype(np.complex128), ref) <= FP32_TOL, j


# ---------------------------------------------------------------------------- sigma eig ----

@pytest.mark.parametrize("N", [1, 2, 7, 16, 33])
def test_diag_occupations(ctx, N):
    rng = np.random.default_rng(N)
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    sigma = 0.25 * (A + A.conj().T) + np.diag(np.linspace(0, 1, N))
    Q, d = ctx.diag_occupations(dev(sigma))
    Q, d = Q.cpu().numpy(), d.cpu().numpy()
    assert np.abs(Q @ np.diag(d) @ Q.conj().T - sigma).max() <= 1e-13 * max(1.0, np.abs(sigma).max()) * N
    assert np.abs(Q.conj().T @ Q - np.eye(N)).max() <= 1e-13 * N
    assert np.abs(d - np.linalg.eigvalsh(sigma)).max() <= 1e-13 * N


@pytest.mark.parametrize("N", [64, 320])
def test_diag_occupations_fermi_dirac_clustered(ctx, N):
    """Many nearly equal occupations (f ~ 1): the backward error stays at FP64 level."""
    f = synth.fermi_dirac_occupations(N, 0.002)
    rng = np.random.default_rng(0)
    Qr, _ = np.linalg.qr(rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    sigma = Qr @ np.diag(f) @ Qr.conj().T
    Q, d = ctx.diag_occupations(dev(sigma))
    Q, d = Q.cpu().numpy(), d.cpu().numpy()
    assert np.abs(Q @ np.diag(d) @ Q.conj().T - sigma).max() <= 1e-13 * max(1.0, N / 64)
    assert np.abs(Q.conj().T @ Q - np.eye(N)).max() <= 1e-13 * max(1.0, N / 64)
    assert np.abs(np.sort(f) - d).max() <= 1e-13 * max(1.0, N / 64)


# ---------------------------------------------------------------------------- ACE ----

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ace_matches_oracle(ctx, w24, oracle24, precision):
    g = O.grid_of(w24.cell)
    dt = np.complex128 if precision == "fp64" else np.complex64
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    phi = dev(w24.phi.astype(dt))
    ace = ctx.build_ace(phi, dev(w24.occ), cell=w24.cell, kernel=w24.kernel, precision=precision)
    xi_ref = O.build_ace(w24.phi, oracle24, g.dV)
    assert rel(ace.xi().cpu().numpy().astype(np.complex128), xi_ref) <= tol
    # V_ACE phi = V_x phi
    out = ctx.apply_ace(ace, phi)
    assert rel(out.cpu().numpy().astype(np.complex128), oracle24) <= tol
    # on other vectors, against the oracle's V_ACE
    rng = np.random.default_rng(5)
    psi = synth.random_orbitals(rng, w24.cell, 5)
    ref = O.apply_ace(xi_ref, psi, g.dV)
    out = ctx.apply_ace(ace, dev(psi.astype(dt)))
    assert rel(out.cpu().numpy().astype(np.complex128), ref) <= tol
    ace.close()


def test_ace_rejects_negative_occupations(ctx, w24):
    from paper_2501_03061_gb300.api import PtimError
    occ = -np.abs(w24.occ)  # makes -M negative definite
    with pytest.raises(PtimError, match="PT_NOT_PD"):
        ctx.build_ace(dev(w24.phi), dev(occ), cell=w24.cell, kernel=w24.kernel)


# ---------------------------------------------------------------------------- H ----

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_apply_H_matches_oracle(ctx, w24, oracle24, precision):
    g = O.grid_of(w24.cell)
    dt = np.complex128 if precision == "fp64" else np.complex64
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    ace = ctx.build_ace(dev(w24.phi.astype(dt)), dev(w24.occ), cell=w24.cell, kernel=w24.kernel, precision=precision)
    xi_ref = O.build_ace(w24.phi, oracle24, g.dV)
    rng = np.random.default_rng(8)
    psi = synth.random_orbitals(rng, w24.cell, 6)
    ref = O.apply_H(psi, w24.vloc, g, 10.0, 0.25, O.apply_ace(xi_ref, psi, g.dV))
    out = ctx.apply_H(dev(psi.astype(dt)), dev(w24.vloc), ace, 0.25, 10.0, cell=w24.cell, precision=precision)
    assert rel(out.cpu().numpy().astype(np.complex128), ref) <= tol
    ace.close()


def test_apply_H_without_exchange_orthorhombic(ctx):
    rng = np.random.default_rng(2)
    cell = synth.Cell((16, 20, 24), (6.0, 7.5, 9.0))
    psi = synth.random_orbitals(rng, cell, 3, ecut=12.0)
    v = synth.gaussian_wells(cell, np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]]))
    g = O.grid_of(cell)
    ref = O.apply_H(psi, v, g, 6.0, 0.0, 0 * psi)
    out = ctx.apply_H(dev(psi), dev(v), None, 0.0, 6.0, cell=cell, precision="fp64")
    assert rel(out.cpu().numpy(), ref) <= FP64_TOL


# ---------------------------------------------------------------------------- PT-IM step ----

def _ptim_case():
    w = synth.small_cell(23, 12, 8.0, 6, kT=0.05, ecut=6.0)
    sig = np.diag(w.occ).astype(np.complex128)
    sig[0, 1] = sig[1, 0] = 0.03
    sig[2, 4] = 0.02j
    sig[4, 2] = -0.02j
    return w, sig


@pytest.fixture(scope="module")
def ptim_ref():
    w, sig = _ptim_case()
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    phi1, sig1, st = O.ptim_step(w.phi, sig, w.vloc, g, K, O.PtimParams(tol=1e-12, ecut=6.0))
    assert st.converged
    return phi1, sig1


@pytest.mark.parametrize("use_ace", [True, False])
def test_ptim_step_fp64_matches_oracle(ctx, ptim_ref, use_ace):
    w, sig = _ptim_case()
    phi = dev(w.phi)
    sigma = dev(sig)
    st = ctx.ptim_step(phi, sigma, dev(w.vloc), cell=w.cell, kernel=w.kernel, precision="fp64", dt=0.5,
                       ecut=6.0, tol=1e-12, use_ace=use_ace)
    assert st["converged"]
    assert rel(phi.cpu().numpy(), ptim_ref[0]) <= 1e-10
    assert np.abs(sigma.cpu().numpy() - ptim_ref[1]).max() <= 1e-10
    assert st["orth_error"] <= 1e-10


@pytest.mark.parametrize("tc_gram", [0, 1])
def test_ptim_step_fp32_matches_oracle(ctx, ptim_ref, tc_gram):
    """FP32 orbitals, FP64 N x N algebra: the step agrees with the FP64 oracle to FP32 accuracy,
    with the Gram contractions on CUDA cores or on tensor cores (3-product TF32)."""
    w, sig = _ptim_case()
    phi = dev(w.phi.astype(np.complex64))
    sigma = dev(sig)
    ctx.set_option("tc_gram", tc_gram)
    try:
        st = ctx.ptim_step(phi, sigma, dev(w.vloc), cell=w.cell, kernel=w.kernel, precision="fp32", dt=0.5,
                           ecut=6.0, tol=2e-6)
    finally:
        ctx.set_option("tc_gram", 0)
    assert st["converged"]
    assert rel(phi.cpu().numpy().astype(np.complex128), ptim_ref[0]) <= 5e-5
    assert np.abs(sigma.cpu().numpy() - ptim_ref[1]).max() <= 5e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("sym", [True, False])
@pytest.mark.parametrize("tile", [2, 6, 10])
def test_exchange_64cubed_specialised_path(ctx, precision, sym, tile):
    """The 64^3 kernels (pipelined plane/column/plane/accumulate roles in FP32) against the oracle:
    several batches of 2x2, 6x6 or 10x10 pair tiles (10: the largest the parameter block holds),
    ragged at the edge (N = 7, 13 or 23), an exact-zero occupation (skipped pairs), separate
    targets."""
    rng = np.random.default_rng(64 + sym + 10 * tile)
    cell = synth.cubic(64, 20.5)
    n = {2: 7, 6: 13, 10: 23}[tile]
    src = synth.random_orbitals(rng, cell, n)
    tgt = src if sym else synth.random_orbitals(rng, cell, {2: 3, 6: 8, 10: 12}[tile])
    occ = np.linspace(1.0, 0.05, n)
    occ[1] = 0.0
    g = O.grid_of(cell)
    ref = O.apply_exchange(src, occ, tgt, O.exchange_kernel(g, 1, synth.SCREENED_MU))
    dt = np.complex128 if precision == "fp64" else np.complex64
    ctx.set_option("scratch_bytes", tile * tile * g.ng * 16)
    ctx.set_option("exchange64_scratch_bytes", tile * tile * g.ng * 8)
    try:
        out = ctx.apply_exchange(dev(src.astype(dt)), dev(occ), None if sym else dev(tgt.astype(dt)), cell=cell,
                                 kernel={"type": 1, "mu": synth.SCREENED_MU}, precision=precision)
    finally:
        ctx.set_option("scratch_bytes", 512 << 20)
        ctx.set_option("exchange64_scratch_bytes", 512 << 20)
    assert rel(out.cpu().numpy().astype(np.complex128), ref) <= (FP64_TOL if precision == "fp64" else FP32_TOL)


@pytest.fixture(scope="module")
def ref_N66():
    w = synth.small_cell(29, 10, 9.0, 66, kT=0.05, ecut=12.0)
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    phi1, sig1, st = O.ptim_step(w.phi, w.sigma, w.vloc, g, K, O.PtimParams(tol=1e-9, ecut=12.0))
    assert st.converged
    return w, phi1, sig1


@pytest.mark.parametrize("tc_gram", [0, 1])
def test_ptim_step_fp32_multitile_N66(ctx, ref_N66, tc_gram):
    """N = 66 spans two 64-wide Gram tiles (Hermitian mirror of A and S) and several exchange batches."""
    w, phi1, sig1 = ref_N66
    phi = dev(w.phi.astype(np.complex64))
    sigma = dev(w.sigma)
    ctx.set_option("tc_gram", tc_gram)
    try:
        s = ctx.ptim_step(phi, sigma, dev(w.vloc), cell=w.cell, kernel=w.kernel, precision="fp32", dt=0.5,
                          ecut=12.0, tol=2e-6)
    finally:
        ctx.set_option("tc_gram", 0)
    assert s["converged"]
    assert rel(phi.cpu().numpy().astype(np.complex128), phi1) <= 5e-5
    assert np.abs(sigma.cpu().numpy() - sig1).max() <= 5e-5
