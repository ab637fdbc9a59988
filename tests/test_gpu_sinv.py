"""S^{-1} A inside the PT-IM inner iteration (context option ptim_sinv_series): the Neumann series
and the product form in E = S - I against the Cholesky route.  All three give S^{-1} A to FP64
rounding, so a step lands on the same state with each, to its tolerance; the step statistics
show which route each inner iteration took."""
import numpy as np
import pytest

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


def step(ctx, w, mode, precision, tol, dt=0.1, mixed=0):
    ctype = np.complex128 if precision == "fp64" else np.complex64
    phi = torch.from_numpy(w.phi.astype(ctype)).cuda()
    sigma = torch.from_numpy(w.sigma.copy()).cuda()
    ctx.set_option("ptim_sinv_series", mode)
    ctx.set_option("ptim_sinv_mixed", mixed)
    try:
        st = ctx.ptim_step(phi, sigma, torch.from_numpy(w.vloc).cuda(), cell=w.cell, kernel=w.kernel,
                           precision=precision, dt=dt, ecut=10.0, tol=tol)
    finally:
        ctx.set_option("ptim_sinv_series", 1)  # the library's defaults
        ctx.set_option("ptim_sinv_mixed", 1)
    return phi.cpu().numpy().astype(np.complex128), sigma.cpu().numpy(), st


@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-11, 1e-9), ("fp32", 1e-6, 2e-5)])
def test_series_forms_match_the_cholesky_route(ctx, precision, tol, bar):
    """dt = 0.1: the midpoint overlaps of this cell come within the series' reach (||S - I||_F < 1/4)
    in some inner iterations; the others take the Cholesky route in every mode."""
    w = synth.small_cell(31, 16, 10.0, 12, kT=0.05, ecut=10.0)
    ref = step(ctx, w, 0, precision, tol)
    assert ref[2]["sinv_path"] == [ref[2]["inner"], 0, 0, 0] and ref[2]["s_dev_max"] == 0.0
    for mode in (1, 2):
        phi, sigma, st = step(ctx, w, mode, precision, tol)
        assert st["converged"]
        assert sum(st["sinv_path"]) == st["inner"]
        assert st["s_dev_max"] > 0.0
        if mode == 1:
            assert st["sinv_path"][1] + st["sinv_path"][2] >= 1
        else:
            assert st["sinv_path"][1] == 0 and st["sinv_path"][2] >= 1
        ep = np.linalg.norm(phi - ref[0]) / np.linalg.norm(ref[0])
        es = np.linalg.norm(sigma - ref[1]) / np.linalg.norm(ref[1])
        print(precision, "mode", mode, "paths", st["sinv_path"], "max ||S-I||_F %.3g" % st["s_dev_max"],
              "phi %.2e sigma %.2e" % (ep, es))
        assert ep < bar and es < bar


@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-11, 1e-9), ("fp32", 1e-6, 2e-5)])
def test_mixed_precision_route_matches_the_fp64_cholesky_route(ctx, precision, tol, bar):
    """dt = 0.5: the midpoint overlaps are beyond the series' reach, so with the option on every
    inner iteration takes the FP32 factor refined in FP64."""
    w = synth.small_cell(33, 16, 10.0, 12, kT=0.05, ecut=10.0)
    ref = step(ctx, w, 0, precision, tol, dt=0.5, mixed=0)
    phi, sigma, st = step(ctx, w, 0, precision, tol, dt=0.5, mixed=1)
    assert ref[2]["sinv_path"] == [ref[2]["inner"], 0, 0, 0]
    assert st["sinv_path"] == [0, 0, 0, st["inner"]] and not st["sinv_mixed_fallback"]
    ep = np.linalg.norm(phi - ref[0]) / np.linalg.norm(ref[0])
    es = np.linalg.norm(sigma - ref[1]) / np.linalg.norm(ref[1])
    print(precision, "mixed route: inner", st["inner"], "against", ref[2]["inner"], "phi %.2e sigma %.2e" % (ep, es))
    assert ep < bar and es < bar


def test_option_values(ctx):
    for bad in (-1, 3, 0.5):
        with pytest.raises(Exception):
            ctx.set_option("ptim_sinv_series", bad)
