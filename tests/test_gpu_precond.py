"""The kinetically preconditioned inner iteration of the PT-IM step (context option
"ptim_precond") against the FP64 oracle: the preconditioner changes only how Anderson approaches
the fixed point x = T(x) of Algorithm 1 (Sec. II-A, Eqs. lisan and x=tx), so the step must land on
the oracle's (Phi_{n+1}, sigma_{n+1}) — in FP64 to 1e-10, in FP32 to FP32 accuracy, with the exact
exchange, with V_Hxc rebuilt from the midpoint density, with a velocity-gauge field, on a
non-cubic grid (the runtime-plan FFT kernels) — and it must do so in fewer inner iterations than
plain Anderson on the same cell.
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


def _case():
    w = synth.small_cell(23, 12, 8.0, 6, kT=0.05, ecut=6.0)
    sig = np.diag(w.occ).astype(np.complex128)
    sig[0, 1] = sig[1, 0] = 0.03
    sig[2, 4] = 0.02j
    sig[4, 2] = -0.02j
    return w, sig


@pytest.fixture(scope="module")
def refs():
    w, sig = _case()
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    out = {}
    for name, kw in (("plain", {}), ("hxc", {"hxc": True}), ("field", {"A": A0})):
        phi1, sig1, st = O.ptim_step(w.phi, sig, w.vloc, g, K, O.PtimParams(tol=1e-12, ecut=6.0, **kw))
        assert st.converged
        out[name] = (phi1, sig1)
    return out


def step(ctx, w, sig, precision, precond, **kw):
    dt = np.complex128 if precision == "fp64" else np.complex64
    phi, sigma = dev(w.phi.astype(dt)), dev(sig)
    ctx.set_option("ptim_precond", precond)
    try:
        st = ctx.ptim_step(phi, sigma, dev(w.vloc), cell=w.cell, kernel=w.kernel, precision=precision, dt=0.5,
                           **kw)
    finally:
        ctx.set_option("ptim_precond", 1)  # the library's default
    return st, phi.cpu().numpy().astype(np.complex128), sigma.cpu().numpy()


@pytest.mark.parametrize("case,kw", [("plain", {}), ("plain", {"use_ace": False}), ("hxc", {"hxc": True}),
                                     ("field", {"A": A0})])
def test_preconditioned_step_fp64_matches_oracle(ctx, refs, case, kw):
    w, sig = _case()
    st, phi, sigma = step(ctx, w, sig, "fp64", 1, ecut=6.0, tol=1e-12, **kw)
    assert st["converged"]
    assert rel(phi, refs[case][0]) <= 1e-10
    assert np.abs(sigma - refs[case][1]).max() <= 1e-10


@pytest.mark.parametrize("tc_gram", [0, 1])
def test_preconditioned_step_fp32_matches_oracle(ctx, refs, tc_gram):
    w, sig = _case()
    ctx.set_option("tc_gram", tc_gram)
    try:
        st, phi, sigma = step(ctx, w, sig, "fp32", 1, ecut=6.0, tol=2e-6)
    finally:
        ctx.set_option("tc_gram", 0)
    assert st["converged"]
    assert rel(phi, refs["plain"][0]) <= 5e-5
    assert np.abs(sigma - refs["plain"][1]).max() <= 5e-5


def test_preconditioned_step_non_cubic_grid(ctx):
    """A 12 x 15 x 10 cell runs the runtime-plan FFT kernels of the preconditioner."""
    rng = np.random.default_rng(41)
    cell = synth.Cell((12, 15, 10), (7.2, 9.0, 6.0))
    N = 5
    phi0 = synth.random_orbitals(rng, cell, N, ecut=6.0)
    occ = synth.fermi_dirac_occupations(N, 0.05)
    sig = np.diag(occ).astype(np.complex128)
    sig[0, 2] = 0.02 + 0.01j
    sig[2, 0] = 0.02 - 0.01j
    vloc = synth.gaussian_wells(cell, np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 1.5]]))
    g = O.grid_of(cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    phi1, sig1, st = O.ptim_step(phi0, sig, vloc, g, K, O.PtimParams(tol=1e-12, ecut=6.0))
    assert st.converged
    w = synth.Workload("noncubic", cell, phi0, occ, sig, vloc, 8, {"type": 1, "mu": synth.SCREENED_MU}, {})
    got, phi, sigma = step(ctx, w, sig, "fp64", 1, ecut=6.0, tol=1e-12)
    assert got["converged"]
    assert rel(phi, phi1) <= 1e-10
    assert np.abs(sigma - sig1).max() <= 1e-10


def test_preconditioner_takes_fewer_inner_iterations(ctx):
    """16^3 cell at the benchmark's grid spacing class (L = 10.26 bohr, Ecut 10 Ha, N = 16), tol 1e-6:
    the preconditioned step converges to the same state in fewer inner iterations."""
    w = synth.small_cell(1, 16, 10.26, 16, kT=0.02, ecut=10.0)
    plain, p0, s0 = step(ctx, w, w.sigma, "fp64", 0, ecut=10.0, tol=1e-6)
    pre, p1, s1 = step(ctx, w, w.sigma, "fp64", 1, ecut=10.0, tol=1e-6)
    print(f"inner iterations: plain {plain['inner']} (ACE builds {plain['outer']}), preconditioned "
          f"{pre['inner']} (ACE builds {pre['outer']})")
    assert plain["converged"] and pre["converged"]
    assert rel(p1, p0) <= 2e-5
    assert pre["inner"] <= 0.85 * plain["inner"], (plain["inner"], pre["inner"])
