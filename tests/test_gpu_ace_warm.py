"""The warm-started ACE operator of chained PT-IM steps (context option ptim_ace_warm): the first
outer pass of a step whose input is the previous step's output reuses that step's last ACE operator.
Only the iteration path changes (Algorithm 1's fixed point x = T(x) and the stopping test are the
same), so a chain of steps lands on the same states as the same chain without it, to the
tolerance; a step whose input differs from the last output (another state, a perturbed state, a
trimmed context) builds its own operator."""
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


def chain(ctx, w, precision, warm, steps, tol):
    dt = np.complex128 if precision == "fp64" else np.complex64
    phi = torch.from_numpy(w.phi.astype(dt)).cuda()
    sigma = torch.from_numpy(w.sigma.copy()).cuda()
    vloc = torch.from_numpy(w.vloc).cuda()
    ctx.set_option("ptim_ace_warm", warm)
    ctx.trim()  # no operator from an earlier test
    stats = []
    try:
        for _ in range(steps):
            stats.append(ctx.ptim_step(phi, sigma, vloc, cell=w.cell, kernel=w.kernel, precision=precision, dt=0.5,
                                       ecut=10.0, tol=tol))
    finally:
        ctx.set_option("ptim_ace_warm", 1)  # the library's default
    return phi.cpu().numpy().astype(np.complex128), sigma.cpu().numpy(), stats


@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-11, 1e-9), ("fp32", 1e-6, 2e-5)])
def test_warm_chain_matches_cold_chain(ctx, precision, tol, bar):
    w = synth.small_cell(77, 16, 10.26, 16, kT=0.02, ecut=10.0)
    p0, s0, st0 = chain(ctx, w, precision, 0, 3, tol)
    p1, s1, st1 = chain(ctx, w, precision, 1, 3, tol)
    assert all(x["converged"] for x in st0 + st1)
    assert [x["ace_warm"] for x in st1] == [False, True, True]
    assert not any(x["ace_warm"] for x in st0)
    assert np.isnan(st1[1]["total_energy"]) and np.isfinite(st1[0]["total_energy"])
    assert np.linalg.norm(p1 - p0) <= bar * np.linalg.norm(p0)
    assert np.abs(s1 - s0).max() <= bar
    print("ACE builds per step cold", [x["outer"] for x in st0], "warm", [x["outer"] for x in st1],
          "inner cold", [x["inner"] for x in st0], "warm", [x["inner"] for x in st1])


def test_warm_start_needs_the_previous_output(ctx):
    """A perturbed input, another system and a trimmed context all build their own first operator."""
    w = synth.small_cell(78, 12, 8.0, 6, kT=0.05, ecut=6.0)
    phi = torch.from_numpy(w.phi.copy()).cuda()
    sigma = torch.from_numpy(w.sigma.copy()).cuda()
    vloc = torch.from_numpy(w.vloc).cuda()
    kw = dict(cell=w.cell, kernel=w.kernel, precision="fp64", dt=0.5, ecut=6.0, tol=1e-10)
    ctx.set_option("ptim_ace_warm", 1)
    ctx.trim()
    try:
        assert not ctx.ptim_step(phi, sigma, vloc, **kw)["ace_warm"]
        assert ctx.ptim_step(phi, sigma, vloc, **kw)["ace_warm"]
        phi[0, 0, 0, 0] += 1e-12  # any change of the state
        assert not ctx.ptim_step(phi, sigma, vloc, **kw)["ace_warm"]
        assert ctx.ptim_step(phi, sigma, vloc, **kw)["ace_warm"]
        ctx.trim()
        assert not ctx.ptim_step(phi, sigma, vloc, **kw)["ace_warm"]
        w2 = synth.small_cell(79, 12, 8.0, 6, kT=0.05, ecut=6.0)
        assert not ctx.ptim_step(torch.from_numpy(w2.phi).cuda(), torch.from_numpy(w2.sigma.copy()).cuda(),
                                 torch.from_numpy(w2.vloc).cuda(), **kw)["ace_warm"]
    finally:
        ctx.set_option("ptim_ace_warm", 1)


def test_warm_start_sees_a_one_ulp_change_fp32(ctx):
    """The state fingerprint hashes bit patterns: one unit in the last place of one element of Phi
    (complex64) or of sigma (complex128) is a different input."""
    w = synth.small_cell(77, 12, 8.0, 6, kT=0.05, ecut=6.0)
    phi = torch.from_numpy(w.phi.astype(np.complex64)).cuda()
    sigma = torch.from_numpy(w.sigma.copy()).cuda()
    vloc = torch.from_numpy(w.vloc).cuda()
    kw = dict(cell=w.cell, kernel=w.kernel, precision="fp32", dt=0.5, ecut=6.0, tol=1e-5)
    ctx.set_option("ptim_ace_warm", 1)
    ctx.trim()
    try:
        assert not ctx.ptim_step(phi, sigma, vloc, **kw)["ace_warm"]
        assert ctx.ptim_step(phi, sigma, vloc, **kw)["ace_warm"]
        re = torch.view_as_real(phi)
        re[3, 1, 2, 0, 1] = torch.nextafter(re[3, 1, 2, 0, 1], torch.tensor(np.inf, device="cuda"))
        assert not ctx.ptim_step(phi, sigma, vloc, **kw)["ace_warm"]
        assert ctx.ptim_step(phi, sigma, vloc, **kw)["ace_warm"]
        sr = torch.view_as_real(sigma)
        sr[2, 4, 0] = torch.nextafter(sr[2, 4, 0], torch.tensor(-np.inf, device="cuda", dtype=torch.float64))
        assert not ctx.ptim_step(phi, sigma, vloc, **kw)["ace_warm"]
        assert ctx.ptim_step(phi, sigma, vloc, **kw)["ace_warm"]
    finally:
        ctx.set_option("ptim_ace_warm", 1)
