"""Serving loop: each request's result is the same alone and in the mix (requests overlapping on
the device through separate contexts and streams), and admission respects the HBM budget."""
import numpy as np
import pytest

from paper_2501_03061_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _requests():
    from paper_2501_03061_gb300.serve import Request
    reqs = []
    for k, (n, N) in enumerate([(16, 8), (20, 12), (24, 10), (16, 6)]):
        w = synth.small_cell(500 + k, n, 0.32 * n * 2, N, kT=0.05, ecut=8.0)
        if k == 3:
            reqs.append(Request(phi=w.phi, sigma=None, occ=w.occ, vloc=None, cell=w.cell, kernel=w.kernel,
                                kind="exchange", precision="fp32"))
        else:
            reqs.append(Request(phi=w.phi, sigma=w.sigma, occ=None, vloc=w.vloc, cell=w.cell, kernel=w.kernel,
                                kind="ptim", precision="fp32", params={"ecut": 8.0, "tol": 1e-6}))
    return reqs


def _results(server, reqs):
    futs = [server.submit(r) for r in reqs]
    return [f.result(timeout=300) for f in futs]


def test_results_alone_equal_results_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300.serve import Server
    alone = []
    srv = Server(slots=1)
    try:
        for r in _requests():
            alone.append(_results(srv, [r])[0])
    finally:
        srv.close()
    srv = Server(slots=4)
    try:
        mixed = _results(srv, _requests())
        assert max(r.t_start for r in mixed) < min(r.t_end for r in mixed)  # they overlapped
    finally:
        srv.close()
    for a, b in zip(alone, mixed):
        assert a.error is None and b.error is None, (a.error, b.error)
        for key in ("phi", "sigma", "vx"):
            if key in a.result:
                x, y = a.result[key], b.result[key]
                assert np.linalg.norm(x - y) <= 1e-6 * np.linalg.norm(x), key


def test_admission_rejects_oversize_and_queues_within_budget():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300.serve import Server
    reqs = _requests()[:3]
    need = max(Server.footprint(None, r) for r in reqs)  # pure arithmetic, no server state used
    srv = Server(slots=3, hbm_budget=int(need * 1.2))  # room for one request at a time
    try:
        done = _results(srv, reqs)
        assert all(r.error is None for r in done)
        spans = sorted((r.t_start, r.t_end) for r in done)
        for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
            assert s1 >= e0 - 1e-3  # serialized by the budget
        big = _requests()[0]
        big.phi = np.zeros((4000,) + big.phi.shape[1:], dtype=np.complex128)
        rej = srv.submit(big).result(timeout=10)
        assert rej.error == "larger than the HBM budget"
    finally:
        srv.close()


def test_session_steps_equal_chained_requests():
    """A session (state resident on the device) serving two requests of two steps each gives the
    state that four chained ordinary requests give, the state copied through the host in between."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300.serve import Request, Server
    w = synth.small_cell(531, 16, 8.0, 8, kT=0.05, ecut=8.0)
    # each worker's context warm-starts its sigma eigensolve from its own last basis, so two routes
    # agree to the order of the tolerance they converge to, not to rounding
    params = {"ecut": 8.0, "tol": 1e-11}
    srv = Server(slots=2)
    try:
        phi, sig = w.phi, w.sigma
        for _ in range(4):
            r = _results(srv, [Request(phi=phi, sigma=sig, occ=None, vloc=w.vloc, cell=w.cell, kernel=w.kernel,
                                       kind="ptim", precision="fp64", params=params)])[0]
            assert r.error is None, r.error
            phi, sig = r.result["phi"], r.result["sigma"]
        sid = srv.open_session(w.phi, w.sigma, w.vloc, w.cell, w.kernel, "fp64")
        futs = [srv.submit(Request(phi=None, sigma=None, occ=None, vloc=None, cell=None, kernel={}, session=sid,
                                   steps=2, params=params)) for _ in range(2)]
        res = [f.result(timeout=300) for f in futs]
        assert all(r.error is None for r in res), [r.error for r in res]
        assert res[0].t_end <= res[1].t_start  # one request of a session at a time, in order
        st = srv.close_session(sid)
    finally:
        srv.close()
    assert st["steps_done"] == 4
    assert np.linalg.norm(st["phi"] - phi) <= 1e-9 * np.linalg.norm(phi)
    assert np.abs(st["sigma"] - sig).max() <= 1e-9
