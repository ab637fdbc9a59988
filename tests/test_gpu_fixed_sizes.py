"""GPU parity of the compile-time-size FFT kernels (cubic grids with sides 16 .. 64) for the
exchange and for H psi, against the FP64 oracle, in both precision forms."""
import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIDES = [16, 20, 30, 32, 36, 40, 48, 54, 60, 64]


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
@pytest.mark.parametrize("n", SIDES)
def test_exchange_cubic_side(ctx, n, precision):
    rng = np.random.default_rng(500 + n)
    cell = synth.cubic(n, 0.32 * n)
    phi = synth.random_orbitals(rng, cell, 4, ecut=4.0)
    occ = np.array([1.0, 0.6, 0.0, 0.3])
    g = O.grid_of(cell)
    ref = O.apply_exchange(phi, occ, phi, O.exchange_kernel(g, 1, synth.SCREENED_MU))
    dt = np.complex128 if precision == "fp64" else np.complex64
    out = ctx.apply_exchange(dev(phi.astype(dt)), dev(occ), cell=cell, kernel={"type": 1, "mu": synth.SCREENED_MU},
                             precision=precision)
    assert rel(out.cpu().numpy().astype(np.complex128), ref) <= (1e-11 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", SIDES)
def test_apply_H_cubic_side(ctx, n, precision):
    rng = np.random.default_rng(600 + n)
    cell = synth.cubic(n, 0.32 * n)
    psi = synth.random_orbitals(rng, cell, 3, ecut=5.0)
    v = synth.gaussian_wells(cell, np.array([[1.0, 2.0, 3.0], [0.5 * cell.L[0], 0.4 * cell.L[1], 0.3 * cell.L[2]]]))
    g = O.grid_of(cell)
    dt = np.complex128 if precision == "fp64" else np.complex64
    # an ACE operator with a known action: from W = -psi (orthonormal psi), M = -I, xi = -psi and
    # V_ACE psi = -xi <xi|psi> = -psi
    ace = ctx.build_ace_from(dev(-psi.astype(dt)), dev(psi.astype(dt)), cell=cell, precision=precision)
    out = ctx.apply_H(dev(psi.astype(dt)), dev(v), ace, 0.25, 5.0, cell=cell, precision=precision)
    ref = O.apply_H(psi, v, g, 5.0, 0.25, -psi)
    assert rel(out.cpu().numpy().astype(np.complex128), ref) <= (1e-11 if precision == "fp64" else 1e-5)
    ace.close()


@pytest.mark.parametrize("ft", [128, 512])
@pytest.mark.parametrize("n", SIDES + [24])
def test_exchange_cubic_side_fp32_cta_sizes(ctx, n, ft):
    """The FP32 compile-time exchange kernels with 128 or 512 threads per CTA (the batched form's
    autotuner chooses among 128, 256 and 512 per grid) against the oracle, in several pair batches.
    64^3 runs the compile-time kernels (engine 1) instead of the TMA pipeline here."""
    rng = np.random.default_rng(700 + n + ft)
    cell = synth.cubic(n, 0.32 * n)
    phi = synth.random_orbitals(rng, cell, 5, ecut=4.0)
    occ = np.array([1.0, 0.6, 0.0, 0.3, 0.9])
    g = O.grid_of(cell)
    ref = O.apply_exchange(phi, occ, phi, O.exchange_kernel(g, 1, synth.SCREENED_MU))
    ctx.set_option("fft_threads", ft)
    ctx.set_option("exchange64_engine", 1)
    ctx.set_option("scratch_bytes", 4 * g.ng * 8)  # 2 x 2 pair tiles: several batches
    try:
        out = ctx.apply_exchange(dev(phi.astype(np.complex64)), dev(occ), cell=cell,
                                 kernel={"type": 1, "mu": synth.SCREENED_MU}, precision="fp32")
    finally:
        ctx.set_option("fft_threads", 256)
        ctx.set_option("exchange64_engine", 0)
        ctx.set_option("scratch_bytes", 512 << 20)
    assert rel(out.cpu().numpy().astype(np.complex128), ref) <= 1e-5
