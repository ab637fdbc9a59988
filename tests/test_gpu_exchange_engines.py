"""The alternative 64^3 FP32 exchange engines.  The persistent engine (exchange64_engine = 2: one cooperative
launch per application, pair fields in an L2-sized ring) against the FP64 oracle and against the
launch-pipelined engine: symmetric and general targets, ragged tiles, exact-zero occupations,
ring slots reused many times within a call (small tiles, the smallest ring the schedule admits),
every stage lag, and the benchmark cell's sampled targets (Sec. IV-A1, Eq. vxdiag).  The fused
engine (exchange64_engine = 3: the pipelined TMA kernel whose accumulate role runs the inverse plane
transforms itself) against the oracle over tile sizes and on the benchmark cell.
"""
import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def run(ctx, src, occ, tgt, cell, engine, tile=4, ring=24, lag=2):
    opts = {"exchange64_engine": engine, "exchange64p_tile": tile, "exchange64p_ring": ring,
            "exchange64p_lag": lag}
    for k, v in opts.items():
        ctx.set_option(k, v)
    try:
        out = ctx.apply_exchange(dev(src.astype(np.complex64)), dev(occ),
                                 None if tgt is None else dev(tgt.astype(np.complex64)), cell=cell,
                                 kernel={"type": 1, "mu": synth.SCREENED_MU}, precision="fp32")
        torch.cuda.synchronize()
    finally:
        for k, v in (("exchange64_engine", 0), ("exchange64p_tile", 4), ("exchange64p_ring", 24),
                     ("exchange64p_lag", 2)):
            ctx.set_option(k, v)
    return out.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("sym,N,M,tile,lag", [(True, 7, None, 2, 1), (True, 9, None, 3, 2), (False, 7, 5, 3, 1),
                                              (False, 5, 9, 2, 3)])
def test_persistent_engine_matches_oracle(ctx, sym, N, M, tile, lag):
    rng = np.random.default_rng(700 + 10 * N + tile)
    cell = synth.cubic(64, 20.5)
    src = synth.random_orbitals(rng, cell, N)
    tgt = None if sym else synth.random_orbitals(rng, cell, M)
    occ = np.linspace(1.0, 0.05, N)
    occ[1] = 0.0  # exactly zero: pairs skipped on the device
    g = O.grid_of(cell)
    ref = O.apply_exchange(src, occ, src if sym else tgt, O.exchange_kernel(g, 1, synth.SCREENED_MU))
    got = run(ctx, src, occ, tgt, cell, 2, tile=tile, ring=1, lag=lag)  # ring raised to its minimum
    assert rel(got, ref) <= FP32_TOL


@pytest.mark.parametrize("tile,ring,lag", [(4, 24, 2), (2, 1, 1), (6, 64, 3), (8, 80, 2)])
def test_persistent_engine_matches_pipelined_engine(ctx, tile, ring, lag):
    """N = 40 symmetric (820 pair FFTs): many reuses of every ring slot, against the launch-pipelined
    engine (itself pinned to the oracle): the same sums in another order."""
    rng = np.random.default_rng(41)
    cell = synth.cubic(64, 20.5)
    N = 40
    src = synth.random_orbitals(rng, cell, N)
    occ = synth.fermi_dirac_occupations(N, 0.02)
    occ[5] = 0.0
    a = run(ctx, src, occ, None, cell, 0)
    b = run(ctx, src, occ, None, cell, 2, tile=tile, ring=ring, lag=lag)
    assert rel(b, a) <= 2e-6


def test_persistent_engine_benchmark_cell_sampled_targets(ctx):
    """64^3, N = 320 (the benchmark's V_x application) against the oracle on sampled targets."""
    w = synth.ptim_cell128()
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    got = run(ctx, w.phi, w.occ, None, w.cell, 2)
    for j in (0, 97, 319):
        ref = O.apply_exchange(w.phi, w.occ, w.phi[j:j + 1], K)[0]
        assert rel(got[j], ref) <= FP32_TOL, j


@pytest.mark.parametrize("sym", [True, False])
@pytest.mark.parametrize("tile", [2, 6, 16])
def test_fused_cd_engine_matches_oracle(ctx, sym, tile):
    """Engine 3: the launch-pipelined TMA kernel with C's inverse plane transforms fused into the
    accumulate (three scratch slots).  Several batches of 2x2, 6x6 or 16x16 pair tiles, ragged at the
    edge, an exact-zero occupation, separate targets."""
    rng = np.random.default_rng(900 + 10 * tile + sym)
    cell = synth.cubic(64, 20.5)
    n = {2: 7, 6: 13, 16: 21}[tile]
    src = synth.random_orbitals(rng, cell, n)
    tgt = None if sym else synth.random_orbitals(rng, cell, {2: 3, 6: 8, 16: 18}[tile])
    occ = np.linspace(1.0, 0.05, n)
    occ[2] = 0.0
    g = O.grid_of(cell)
    ref = O.apply_exchange(src, occ, src if sym else tgt, O.exchange_kernel(g, 1, synth.SCREENED_MU))
    ctx.set_option("exchange64_scratch_bytes", tile * tile * g.ng * 8)
    try:
        got = run(ctx, src, occ, tgt, cell, 3)
    finally:
        ctx.set_option("exchange64_scratch_bytes", 512 << 20)
    assert rel(got, ref) <= FP32_TOL


def test_fused_cd_engine_benchmark_cell(ctx):
    """64^3, N = 320 with the fused engine: sampled targets against the oracle, the whole result against
    the four-role engine."""
    w = synth.ptim_cell128()
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    got = run(ctx, w.phi, w.occ, None, w.cell, 3)
    for j in (1, 200, 318):
        ref = O.apply_exchange(w.phi, w.occ, w.phi[j:j + 1], K)[0]
        assert rel(got[j], ref) <= FP32_TOL, j
    four = run(ctx, w.phi, w.occ, None, w.cell, 0)
    assert rel(got, four) <= 2e-6
