"""The PT-IM step in the plane-wave basis of the Ecut sphere (context option ptim_pw): the orbital
blocks of the step held as unitary-FFT coefficients at the plane waves |G|^2/2 <= Ecut.  Inner
products are those of the grid, so the step lands on the state of the grid form to its tolerance;
an input with weight outside the sphere, or a grid without compile-time FFT kernels, runs on the
grid."""
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


def step(ctx, w, pw, precision, tol, phi=None, **extra):
    ctype = np.complex128 if precision == "fp64" else np.complex64
    phi = torch.from_numpy(np.ascontiguousarray((w.phi if phi is None else phi).astype(ctype))).cuda()
    sigma = torch.from_numpy(w.sigma.copy()).cuda()
    ctx.set_option("ptim_pw", pw)
    try:
        st = ctx.ptim_step(phi, sigma, torch.from_numpy(w.vloc).cuda(), cell=w.cell, kernel=w.kernel,
                           precision=precision, dt=0.5, ecut=10.0, tol=tol, **extra)
    finally:
        ctx.set_option("ptim_pw", 1)  # the library's default
    return phi.cpu().numpy().astype(np.complex128), sigma.cpu().numpy(), st


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-11, 1e-9), ("fp32", 1e-6, 2e-5)])
@pytest.mark.parametrize("n,N", [(16, 12), (24, 20)])
def test_plane_wave_step_matches_the_grid_step(ctx, precision, tol, bar, n, N):
    w = synth.small_cell(40 + n, n, 10.0, N, kT=0.05, ecut=10.0)
    phi0, sig0, st0 = step(ctx, w, 0, precision, tol)
    phi1, sig1, st1 = step(ctx, w, 1, precision, tol)
    npw = synth.sphere_indices(w.cell, 10.0).size
    assert st0["plane_waves"] == 0 and st1["plane_waves"] == npw
    assert st0["converged"] and st1["converged"]
    ep, es = rel(phi1, phi0), rel(sig1, sig0)
    print(precision, n, "plane waves", npw, "of", n ** 3, "phi %.2e sigma %.2e" % (ep, es),
          "inner", st0["inner"], st1["inner"])
    assert ep < bar and es < bar
    # the output lies in the sphere: its coefficients outside it vanish to rounding
    c = np.fft.fftn(phi1.reshape((N,) + w.cell.n), axes=(1, 2, 3)).reshape(N, -1)
    inside = np.zeros(c.shape[1], bool)
    inside[synth.sphere_indices(w.cell, 10.0)] = True
    frac = (np.abs(c[:, ~inside]) ** 2).sum() / (np.abs(c) ** 2).sum()
    assert frac < (1e-26 if precision == "fp64" else 1e-12)


def test_weight_outside_the_sphere_runs_on_the_grid(ctx):
    w = synth.small_cell(52, 16, 10.0, 8, kT=0.05, ecut=10.0)
    rng = np.random.default_rng(3)
    noisy = w.phi + 1e-3 * (rng.standard_normal(w.phi.shape) + 1j * rng.standard_normal(w.phi.shape))
    q, _ = np.linalg.qr(noisy.reshape(8, -1).T)  # orthonormal again, but not band-limited
    phi = np.ascontiguousarray((q.T * np.sqrt(1.0 / w.cell.dV)).reshape(w.phi.shape))
    _, _, st = step(ctx, w, 1, "fp64", 1e-10, phi=phi)
    assert st["plane_waves"] == 0 and st["converged"]


def test_default_step_uses_the_plane_wave_basis(ctx):
    w = synth.small_cell(53, 16, 10.0, 8, kT=0.05, ecut=10.0)
    _, _, st = step(ctx, w, 1, "fp64", 1e-10)
    assert st["plane_waves"] > 0
