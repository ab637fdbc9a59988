"""The bounded device waits end in PT_TIMEOUT, not a hang: a kernel waits on an mbarrier that
nothing completes (through the deadline-bounded wait every TMA and tensor-core pipeline uses),
gives up at its deadline, records the expiry and returns; the host reads PT_TIMEOUT and the
context keeps working.  No fault, trap or endless loop is involved."""
import time

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


def test_wait_that_nothing_completes_returns_timeout(ctx):
    t0 = time.perf_counter()
    assert ctx.selftest_wait(arrive=False, timeout_s=0.05) == "PT_TIMEOUT"
    assert time.perf_counter() - t0 < 30.0
    assert "deadline" in ctx.lib.pt_last_error(ctx.h).decode()
    # the control: the same wait on a barrier that completes
    assert ctx.selftest_wait(arrive=True, timeout_s=0.05) == "PT_OK"


def test_context_still_computes_after_a_timeout(ctx):
    assert ctx.selftest_wait(arrive=False, timeout_s=0.02) == "PT_TIMEOUT"
    w = synth.small_cell(7, 12, 8.0, 6, kT=0.02, ecut=8.0)
    g = O.grid_of(w.cell)
    ref = O.apply_exchange(w.phi, w.occ, w.phi, O.exchange_kernel(g, 1, synth.SCREENED_MU))
    out = ctx.apply_exchange(torch.from_numpy(w.phi).cuda(), torch.from_numpy(w.occ).cuda(), cell=w.cell,
                             kernel=w.kernel, precision="fp64")
    assert np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-11


def test_selftest_argument_checks(ctx):
    from paper_2501_03061_gb300 import _lib as L
    for arrive, t in ((2, 0.05), (0, 0.0), (0, 2.5), (1, -1.0)):
        assert ctx.lib.pt_selftest_wait(ctx.h, arrive, t, None) == L.PT_INVALID_ARG
