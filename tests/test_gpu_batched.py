"""GPU tests of the batched exchange (heterogeneous items, autotuned pair tiles, CUDA graph replay)."""
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


def make_items(precision):
    """Four systems: two symmetric (24^3 N=12, 64^3 N=9 on the specialised path), one with
    separate targets on an orthorhombic grid, one 30^3 with an exact-zero occupation."""
    dt = np.complex128 if precision == "fp64" else np.complex64
    rng = np.random.default_rng(401)
    specs = [
        (synth.cubic(24, 10.0), 12, None, 0.106),
        (synth.Cell((20, 24, 30), (7.5, 9.0, 11.0)), 7, 5, 0.2),
        (synth.cubic(64, 20.5), 9, None, 0.106),
        (synth.cubic(30, 12.0), 10, None, 0.106),
    ]
    items, host = [], []
    for cell, N, M, mu in specs:
        src = synth.random_orbitals(rng, cell, N, ecut=5.0)
        tgt = None if M is None else synth.random_orbitals(rng, cell, M, ecut=5.0)
        occ = np.linspace(1.0, 0.05, N)
        if N == 10:
            occ[3] = 0.0
        kern = {"type": 1, "mu": mu}
        items.append({"src": dev(src.astype(dt)), "occ": dev(occ), "cell": cell, "kernel": kern,
                      "tgt": None if tgt is None else dev(tgt.astype(dt))})
        host.append((cell, src.astype(dt).astype(np.complex128), occ,
                     None if tgt is None else tgt.astype(dt).astype(np.complex128), mu))
    return items, host


def oracle_out(h):
    cell, src, occ, tgt, mu = h
    g = O.grid_of(cell)
    return O.apply_exchange(src, occ, src if tgt is None else tgt, O.exchange_kernel(g, 1, mu))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_matches_oracle_and_single_calls(ctx, precision):
    items, host = make_items(precision)
    outs, pairs, _ = ctx.apply_exchange_batched(items, precision=precision)
    tol = 1e-11 if precision == "fp64" else 1e-5
    assert pairs == 12 * 13 // 2 + 7 * 5 + 9 * 10 // 2 + 10 * 11 // 2
    for it, h, out in zip(items, host, outs):
        ref = oracle_out(h)
        assert rel(out.cpu().numpy().astype(np.complex128), ref) <= tol
        single = ctx.apply_exchange(it["src"], it["occ"], it["tgt"], cell=it["cell"], kernel=it["kernel"],
                                    precision=precision)
        assert rel(out.cpu().numpy(), single.cpu().numpy()) <= (1e-13 if precision == "fp64" else 1e-6)


def test_batched_graph_replay_reads_new_inputs(ctx):
    """Second and third calls replay the captured graph on the same buffers.  Halving every
    source orbital (exact in binary floating point) scales each output by exactly 1/8."""
    items, _ = make_items("fp32")
    outs0, _, nodes0 = ctx.apply_exchange_batched(items, precision="fp32")
    first = [o.clone() for o in outs0]
    for it, o in zip(items, outs0):
        it["out"] = o
    outs1, _, nodes1 = ctx.apply_exchange_batched(items, precision="fp32")
    assert nodes0 > 0 and nodes1 == nodes0  # eager pass recorded the graph; this call replayed it
    for a, b in zip(first, outs1):
        assert torch.equal(a, b)
    for it in items:
        it["src"].mul_(0.5)
        if it["tgt"] is not None:
            it["tgt"].mul_(0.5)
    outs2, _, nodes2 = ctx.apply_exchange_batched(items, precision="fp32")
    assert nodes2 == nodes0
    for it, a, b in zip(items, first, outs2):
        # separate targets: W = V_x[src] tgt scales by 1/4 * 1/2; symmetric: by 1/8 as well
        assert torch.equal(b, a * 0.125)


def test_batched_eager_equals_graph(ctx):
    items, _ = make_items("fp32")
    ctx.set_option("graphs", 0)
    try:
        eager, _, nodes = ctx.apply_exchange_batched(items, precision="fp32")
        assert nodes == 0
    finally:
        ctx.set_option("graphs", 1)
    eager = [o.clone() for o in eager]
    for it in items:
        it["out"] = None
    g1, _, _ = ctx.apply_exchange_batched(items, precision="fp32")
    for it, o in zip(items, g1):
        it["out"] = o
    g2, _, nodes2 = ctx.apply_exchange_batched(items, precision="fp32")
    assert nodes2 > 0
    for a, b in zip(eager, g2):
        assert torch.equal(a, b)


def test_batched_rejects_bad_item(ctx):
    from paper_2501_03061_gb300 import api
    items, _ = make_items("fp32")
    items[1]["cell"] = synth.Cell((7, 24, 30), (7.5, 9.0, 11.0))  # 7 is not 2,3,5-smooth
    with pytest.raises(api.PtimError, match="item 1"):
        ctx.apply_exchange_batched(items, precision="fp32")


@pytest.mark.parametrize("graphs", [0, 1])
def test_batched_concurrent_branches_equal_one_stream(ctx, graphs):
    """Items dealt to four concurrent streams (each with its own scratch) give bit-identical outputs
    to the same items run in order on one stream: every item's arithmetic is independent of when it
    runs.  Eager and replayed from a captured graph with parallel branches."""
    items, _ = make_items("fp32")
    ctx.set_option("graphs", graphs)
    try:
        ctx.set_option("batch_streams", 1)
        one, _, _ = ctx.apply_exchange_batched(items, precision="fp32")
        one = [o.clone() for o in one]
        ctx.set_option("batch_streams", 4)
        for it in items:
            it["out"] = None
        four, _, _ = ctx.apply_exchange_batched(items, precision="fp32")
        if graphs:
            for it, o in zip(items, four):
                it["out"] = o
            four, _, nodes = ctx.apply_exchange_batched(items, precision="fp32")  # replay
            assert nodes > 0
        torch.cuda.synchronize()
    finally:
        ctx.set_option("graphs", 1)
        ctx.set_option("batch_streams", 4)
    for a, b in zip(one, four):
        assert torch.equal(a, b)
