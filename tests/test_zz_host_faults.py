"""Faults injected on the host, none of which faults, traps or hangs the GPU: an impossible
tolerance (PT_NOT_CONVERGED, with the statistics and the last iterate), and a non-finite entry in
the orbitals or in the occupation matrix (an error status, PT_NONFINITE or PT_NOT_PD from the first
check or factorisation the NaN reaches; the caller's orbitals and occupation matrix come back
unchanged).  After each, the same context takes a valid step that matches the oracle: a failed step
leaves nothing behind that the next one starts from."""
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


def case():
    w = synth.small_cell(23, 12, 8.0, 6, kT=0.05, ecut=6.0)
    sig = np.diag(w.occ).astype(np.complex128)
    sig[0, 1] = sig[1, 0] = 0.03
    sig[2, 4] = 0.02j
    sig[4, 2] = -0.02j
    return w, sig


@pytest.fixture(scope="module")
def ref():
    w, sig = case()
    g = O.grid_of(w.cell)
    phi1, sig1, st = O.ptim_step(w.phi, sig, w.vloc, g, O.exchange_kernel(g, 1, synth.SCREENED_MU),
                                 O.PtimParams(tol=1e-12, ecut=6.0))
    assert st.converged
    return phi1, sig1


def valid_step(ctx, ref, precision):
    w, sig = case()
    dt = np.complex128 if precision == "fp64" else np.complex64
    phi = torch.from_numpy(w.phi.astype(dt)).cuda()
    sigma = torch.from_numpy(sig).cuda()
    st = ctx.ptim_step(phi, sigma, torch.from_numpy(w.vloc).cuda(), cell=w.cell, kernel=w.kernel,
                       precision=precision, dt=0.5, ecut=6.0, tol=1e-12 if precision == "fp64" else 2e-6)
    bar = 1e-10 if precision == "fp64" else 5e-5
    assert st["converged"]
    got = phi.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref[0]) / np.linalg.norm(ref[0]) <= bar
    assert np.abs(sigma.cpu().numpy() - ref[1]).max() <= bar


def test_impossible_tolerance_reports_not_converged(ctx, ref):
    w, sig = case()
    phi = torch.from_numpy(w.phi).cuda()
    sigma = torch.from_numpy(sig).cuda()
    st = ctx.ptim_step(phi, sigma, torch.from_numpy(w.vloc).cuda(), cell=w.cell, kernel=w.kernel,
                       precision="fp64", dt=0.5, ecut=6.0, tol=1e-300, max_outer=2, max_inner=3,
                       allow_unconverged=True)
    assert st["status"] == "PT_NOT_CONVERGED" and not st["converged"]
    assert 1 <= st["inner"] <= 6 and np.isfinite(st["residual"])
    assert torch.isfinite(phi.abs()).all() and torch.isfinite(sigma.abs()).all()
    valid_step(ctx, ref, "fp64")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("where", ["phi", "sigma"])
def test_non_finite_input_is_an_error_and_the_context_recovers(ctx, ref, where, precision):
    from paper_2501_03061_gb300 import _lib as L
    from paper_2501_03061_gb300 import api
    w, sig = case()
    ph = w.phi.astype(np.complex128 if precision == "fp64" else np.complex64)
    if where == "phi":
        ph[0, 1, 2, 3] = np.nan
    else:
        sig[0, 1] = sig[1, 0] = np.nan
    phi = torch.from_numpy(ph).cuda()
    sigma = torch.from_numpy(sig).cuda()
    with pytest.raises(api.PtimError) as ei:
        ctx.ptim_step(phi, sigma, torch.from_numpy(w.vloc).cuda(), cell=w.cell, kernel=w.kernel,
                      precision=precision, dt=0.5, ecut=6.0, tol=1e-10)
    assert ei.value.status in (L.PT_NONFINITE, L.PT_NOT_PD), str(ei.value)
    # the failed step hands the caller's input back unchanged (NaN entries compared as NaN)
    np.testing.assert_array_equal(phi.cpu().numpy(), ph)
    np.testing.assert_array_equal(sigma.cpu().numpy(), sig)
    valid_step(ctx, ref, precision)
