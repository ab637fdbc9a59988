"""Algorithm 2 on the GPU (pt_apply_exchange_mixed): the undiagonalised mixed-state exchange
(Sec. II-B Eq. mixed_vx; Sec. III-B, the triple loop with N^3 pair FFTs) against the FP64 oracle's
triple sum, and against the library's diagonalised form of the same operator (Sec. IV-A1:
sigma = Q D Q^*, phit = Phi Q, Eq. vxdiag) on the same inputs — the identity behind the paper's
"Diag" step, checked on the device.  FP64 to 1e-11, FP32 to 1e-5 (relative Frobenius)."""
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


def hermitian(rng, N, scale=0.05):
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    return np.diag(np.linspace(1.0, 0.1, N)) + scale * (A + A.conj().T)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
@pytest.mark.parametrize("shape,M", [((12, 10, 8), None), ((16, 16, 16), 3), ((15, 12, 10), 4)])
def test_mixed_exchange_matches_oracle_triple_sum(ctx, precision, tol, shape, M):
    rng = np.random.default_rng(sum(shape) + (M or 0))
    cell = synth.Cell(shape, (8.0, 7.0, 6.0))
    N = 5
    phi = synth.random_orbitals(rng, cell, N, ecut=5.0)
    tgt = None if M is None else synth.random_orbitals(rng, cell, M, ecut=5.0)
    sigma = hermitian(rng, N)
    g = O.grid_of(cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    ref = O.apply_exchange_mixed(phi, sigma, phi if tgt is None else tgt, K)
    dt = np.complex128 if precision == "fp64" else np.complex64
    out, n = ctx.apply_exchange_mixed(dev(phi.astype(dt)), dev(sigma), None if tgt is None else dev(tgt.astype(dt)),
                                      cell=cell, kernel={"type": 1, "mu": synth.SCREENED_MU}, precision=precision)
    assert n == N * N * (N if M is None else M)
    assert rel(out.cpu().numpy().astype(np.complex128), ref) <= tol


def test_mixed_exchange_non_hermitian_sigma_used_as_given(ctx):
    """The triple sum takes sigma as given (no symmetrisation): a non-Hermitian sigma still matches the
    oracle's triple sum (which the diagonalised form could not reproduce)."""
    rng = np.random.default_rng(9)
    cell = synth.cubic(12, 7.0)
    N = 4
    phi = synth.random_orbitals(rng, cell, N, ecut=5.0)
    sigma = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    g = O.grid_of(cell)
    ref = O.apply_exchange_mixed(phi, sigma, phi, O.exchange_kernel(g, 1, synth.SCREENED_MU))
    out, _ = ctx.apply_exchange_mixed(dev(phi), dev(sigma), cell=cell, kernel={"type": 1, "mu": synth.SCREENED_MU})
    assert rel(out.cpu().numpy(), ref) <= 1e-11


def test_mixed_exchange_config1_cell_fp64(ctx):
    """The plain-FP64 exchange cell (24^3, L = 10, N = 16) with a Hermitian sigma: 4096 pair FFTs."""
    w = synth.exchange_small()
    rng = np.random.default_rng(1000)
    sigma = hermitian(rng, w.N, 0.02)
    g = O.grid_of(w.cell)
    ref = O.apply_exchange_mixed(w.phi, sigma, w.phi, O.exchange_kernel(g, 1, synth.SCREENED_MU))
    out, n = ctx.apply_exchange_mixed(dev(w.phi), dev(sigma), cell=w.cell, kernel=w.kernel, precision="fp64")
    assert n == 16 ** 3
    assert rel(out.cpu().numpy(), ref) <= 1e-11


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-6)])
def test_triple_loop_equals_diagonalised_form_on_the_device(ctx, precision, tol):
    """Algorithm 2's triple loop and the diagonalised double loop (eigensolve, rotation, symmetric pair
    FFTs, rotation back), both on the GPU, on a 32^3 cell with N = 12: the same V_x[P] Phi."""
    rng = np.random.default_rng(32)
    cell = synth.cubic(32, 10.25)
    N = 12
    phi = synth.random_orbitals(rng, cell, N, ecut=8.0)
    sigma = hermitian(rng, N, 0.03)
    dt = np.complex128 if precision == "fp64" else np.complex64
    kern = {"type": 1, "mu": synth.SCREENED_MU}
    p = dev(phi.astype(dt))
    mixed, _ = ctx.apply_exchange_mixed(p, dev(sigma), cell=cell, kernel=kern, precision=precision)
    Q, d = ctx.diag_occupations(dev(sigma))
    phit = ctx.rotate(p, Q, cell=cell, precision=precision)
    wt = ctx.apply_exchange(phit, d, cell=cell, kernel=kern, precision=precision)
    diag = ctx.rotate(wt, Q.conj().T.contiguous(), cell=cell, precision=precision)
    a = mixed.cpu().numpy().astype(np.complex128)
    b = diag.cpu().numpy().astype(np.complex128)
    assert rel(a, b) <= tol
