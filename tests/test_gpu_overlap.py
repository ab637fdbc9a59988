"""GPU parity of the two grid contractions: the overlap C = dV A^* B (ACE's M = <phi|W>,
PT-IM's S = <phi|phi>) and the rotation out_j = sum_k B[k][j] A_k (phit = Phi Q, xi = W L^-*).

The FP32 forms are compared with the FP64 oracle evaluated on the same FP32-rounded inputs, so
the bound measures the contraction alone: |C_gpu - C_ref| <= tol * dV sum_r |a_i(r)| |b_j(r)|
element by element (the scale a product-sum's rounding error is proportional to), with
tol 1e-6 for compensated FP32 on CUDA cores, 1e-5 for the 3-product TF32 tensor-core form,
2e-3 for a single TF32 product (10 explicit mantissa bits: unit roundoff 2^-11 per product) and
4e-3 for a single BF16 product (7 explicit mantissa bits: unit roundoff u = 2^-9, and a product of
two rounded factors is off by at most (2u + u^2) |a| |b| = 3.91e-3 |a| |b|; the FP32 sums in TMEM
and the compensated readout add about 1e-5 of that scale).
"""
import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "fp32_tc": 1e-5, "tf32": 2e-3, "bf16": 4e-3}


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


def fields(rng, cell, n, offset=True):
    """n complex64 fields on the grid; with `offset` each carries a random constant so that the
    inner products are not dominated by cancellation."""
    nx, ny, nz = cell.n
    a = rng.standard_normal((n, nz, ny, nx)) + 1j * rng.standard_normal((n, nz, ny, nx))
    if offset:
        a += (rng.standard_normal(n) + 1j * rng.standard_normal(n))[:, None, None, None]
    return a.astype(np.complex64)


def run(ctx, mode, A, B, cell, wide=1):
    """Overlap on the GPU in one of the forms: fp64, fp32 (CUDA cores), fp32_tc, tf32; `wide`
    selects the 64 x 128 tensor-core tiles (1, used when N2 > 64) or the 64 x 64 ones (0)."""
    prec = {"fp32_tc": "fp32"}.get(mode, mode)
    dt = np.complex128 if prec == "fp64" else np.complex64
    a = dev(A.astype(dt))
    b = a if B is A else dev(B.astype(dt))
    ctx.set_option("tc_gram", 1 if mode == "fp32_tc" else 0)
    ctx.set_option("tc_gram_wide", wide)
    try:
        return ctx.overlap(a, b, cell=cell, precision=prec).cpu().numpy()
    finally:
        ctx.set_option("tc_gram", 0)
        ctx.set_option("tc_gram_wide", 1)


def check(got, A, B, dV, tol):
    A64, B64 = A.astype(np.complex128), B.astype(np.complex128)
    ref = O.overlap(A64, B64, dV)
    scale = dV * (np.abs(A64).reshape(len(A64), -1) @ np.abs(B64).reshape(len(B64), -1).T)
    err = np.abs(got - ref)
    assert np.all(err <= tol * scale), float((err / scale).max())
    return float((err / scale).max())


@pytest.mark.parametrize("wide", [1, 0])
@pytest.mark.parametrize("mode", ["fp64", "fp32", "fp32_tc", "tf32", "bf16"])
def test_overlap_general_ragged(ctx, mode, wide):
    """N1 = 70, N2 = 130 (ragged 64-wide tiles; 64 x 128 tensor-core tiles with an absent second
    half in the last one), 24^3 grid."""
    rng = np.random.default_rng(301)
    cell = synth.cubic(24, 10.0)
    A, B = fields(rng, cell, 70), fields(rng, cell, 130)
    got = run(ctx, mode, A, B, cell, wide)
    if mode == "fp64":
        ref = O.overlap(A.astype(np.complex128), B.astype(np.complex128), O.grid_of(cell).dV)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    else:
        check(got, A, B, O.grid_of(cell).dV, TOL[mode])


@pytest.mark.parametrize("wide", [1, 0])
@pytest.mark.parametrize("mode", ["fp32", "fp32_tc", "tf32", "bf16"])
def test_overlap_hermitian_ragged_K_tail(ctx, mode, wide):
    """S = <A|A> with N = 97 (mirrored tiles) on a 9 x 10 x 12 grid: 2 Ng = 2160 floats is not a
    multiple of the 32-float stage, so the last stage is partly zero-filled."""
    rng = np.random.default_rng(302)
    cell = synth.Cell((9, 10, 12), (5.0, 5.5, 6.0))
    A = fields(rng, cell, 97)
    got = run(ctx, mode, A, A, cell, wide)
    check(got, A, A, O.grid_of(cell).dV, TOL[mode])
    # tiles below the diagonal are mirrors of the ones above: exact conjugates across tiles
    t = np.arange(97) // 64
    off = t[:, None] != t[None, :]
    assert np.abs(got - got.conj().T)[off].max() == 0.0


@pytest.mark.parametrize("mode", ["fp32", "fp32_tc"])
def test_overlap_orthonormal_orbitals(ctx, mode):
    """Orthonormal band-limited orbitals: S = I to FP32 rounding of the inputs."""
    rng = np.random.default_rng(303)
    cell = synth.cubic(24, 10.0)
    phi = synth.random_orbitals(rng, cell, 40).astype(np.complex64)
    got = run(ctx, mode, phi, phi, cell)
    check(got, phi, phi, O.grid_of(cell).dV, TOL[mode])
    assert np.abs(got - np.eye(40)).max() <= 1e-5


@pytest.mark.parametrize("wide", [1, 0])
def test_overlap_64cubed_N320_tensor_cores_sampled(ctx, wide):
    """Full size of the PT-IM overlap (64^3 grid, N = 320): the tensor-core form (64 x 128 or
    64 x 64 tiles) on sampled entries against the FP64 oracle's definition, and against the
    CUDA-core form everywhere."""
    rng = np.random.default_rng(304)
    cell = synth.cubic(64, 20.5)
    A = fields(rng, cell, 320)
    a = dev(A)
    ctx.set_option("tc_gram", 1)
    ctx.set_option("tc_gram_wide", wide)
    try:
        tc = ctx.overlap(a, a, cell=cell, precision="fp32").cpu().numpy()
    finally:
        ctx.set_option("tc_gram", 0)
        ctx.set_option("tc_gram_wide", 1)
    simt = ctx.overlap(a, a, cell=cell, precision="fp32").cpu().numpy()
    dV = O.grid_of(cell).dV
    Af = A.reshape(320, -1).astype(np.complex128)
    absn = np.abs(Af)
    idx = rng.integers(0, 320, size=(64, 2))
    for i, j in idx:
        ref = dV * np.vdot(Af[i], Af[j])
        scale = dV * float(absn[i] @ absn[j])
        assert abs(tc[i, j] - ref) <= TOL["fp32_tc"] * scale
        assert abs(simt[i, j] - ref) <= TOL["fp32"] * scale
    diag = dV * (absn ** 2).sum(axis=1)
    assert np.abs(tc - simt).max() <= 2 * TOL["fp32_tc"] * diag.max()


def run_rotate(ctx, mode, A, B, cell):
    prec = {"fp32_tc": "fp32"}.get(mode, mode)
    dt = np.complex128 if prec == "fp64" else np.complex64
    ctx.set_option("tc_gram", 1 if mode == "fp32_tc" else 0)
    try:
        return ctx.rotate(dev(A.astype(dt)), dev(B), cell=cell, precision=prec).cpu().numpy()
    finally:
        ctx.set_option("tc_gram", 0)


def check_rotate(got, A, B, tol):
    A64 = A.astype(np.complex128)
    ref = O.rotate(A64, B)
    scale = (np.abs(B).T @ np.abs(A64).reshape(len(A64), -1)).reshape(ref.shape)
    err = np.abs(got - ref)
    assert np.all(err <= tol * scale), float((err / scale).max())


ROT_TOL = {"fp32": 1e-5, "fp32_tc": 1e-5, "tf32": 2e-3, "bf16": 4e-3}


@pytest.mark.parametrize("mode", ["fp64", "fp32", "fp32_tc", "tf32", "bf16"])
@pytest.mark.parametrize("shape", [(24, 24, 24), (9, 10, 12)])
def test_rotate_ragged(ctx, mode, shape):
    """N1 = 70 (partial last K stage of 16 orbitals), N2 = 130 (partial last 64-orbital tile);
    9 x 10 x 12 = 1080 points leaves a partial 128-point tile."""
    rng = np.random.default_rng(311)
    cell = synth.Cell(shape, (6.0, 6.5, 7.0))
    A = fields(rng, cell, 70)
    B = rng.standard_normal((70, 130)) + 1j * rng.standard_normal((70, 130))
    got = run_rotate(ctx, mode, A, B, cell)
    if mode == "fp64":
        ref = O.rotate(A.astype(np.complex128), B)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    else:
        check_rotate(got, A, B, ROT_TOL[mode])


def test_rotate_64cubed_N320_tensor_cores_sampled(ctx):
    """Full size of the PT-IM rotations (64^3 grid, N = 320, a unitary B as for phit = Phi Q)."""
    rng = np.random.default_rng(312)
    cell = synth.cubic(64, 20.5)
    A = fields(rng, cell, 320)
    Q, _ = np.linalg.qr(rng.standard_normal((320, 320)) + 1j * rng.standard_normal((320, 320)))
    got = run_rotate(ctx, "fp32_tc", A, Q, cell).reshape(320, -1)
    simt = run_rotate(ctx, "fp32", A, Q, cell).reshape(320, -1)
    Af = A.reshape(320, -1).astype(np.complex128)
    for _ in range(64):
        j, r = int(rng.integers(0, 320)), int(rng.integers(0, Af.shape[1]))
        ref = np.sum(Q[:, j] * Af[:, r])
        scale = float(np.sum(np.abs(Q[:, j]) * np.abs(Af[:, r])))
        assert abs(got[j, r] - ref) <= ROT_TOL["fp32_tc"] * scale
        assert abs(simt[j, r] - ref) <= ROT_TOL["fp32"] * scale


def test_bf16_64cubed_N320_sampled(ctx):
    """The BF16 form at the full size of the ACE contractions (64^3 grid, N = 320): the overlap and
    the rotation on sampled entries against the FP64 definitions, within the single-BF16-product
    bound."""
    rng = np.random.default_rng(320)
    cell = synth.cubic(64, 20.5)
    A = fields(rng, cell, 320)
    a = dev(A)
    S = ctx.overlap(a, a, cell=cell, precision="bf16").cpu().numpy()
    Q, _ = np.linalg.qr(rng.standard_normal((320, 320)) + 1j * rng.standard_normal((320, 320)))
    R = ctx.rotate(a, dev(Q), cell=cell, precision="bf16").cpu().numpy().reshape(320, -1)
    dV = O.grid_of(cell).dV
    Af = A.reshape(320, -1).astype(np.complex128)
    absn = np.abs(Af)
    for _ in range(64):
        i, j = (int(v) for v in rng.integers(0, 320, size=2))
        ref = dV * np.vdot(Af[i], Af[j])
        assert abs(S[i, j] - ref) <= TOL["bf16"] * dV * float(absn[i] @ absn[j])
        r = int(rng.integers(0, Af.shape[1]))
        ref = np.sum(Q[:, j] * Af[:, r])
        assert abs(R[j, r] - ref) <= ROT_TOL["bf16"] * float(np.sum(np.abs(Q[:, j]) * absn[:, r]))
    # tiles below the diagonal are exact conjugate mirrors of the ones above
    t = np.arange(320) // 64
    off = t[:, None] != t[None, :]
    assert np.abs(S - S.conj().T)[off].max() == 0.0
