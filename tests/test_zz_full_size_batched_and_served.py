"""The batched and served forms at the benchmark's full sizes, in the launch configuration bench.py
times, against the FP64 oracle where the oracle can follow.

Batched form (64 instances, N ~ U{16..256}, grids 24^3..64^3, FP32; concurrent branches, captured
graph, autotuned pair tiles and engines): sampled targets of three items — the largest 64^3 item, a
non-64 item and the smallest grid — against the oracle's exchange for those targets, on the eager
pass and on a graph replay (Sec. IV-A1, Eq. vxdiag).

Serving form: one served PT-IM step request of the serving stream's kind (a 48^3 cell, N = 200, FP32,
tol 1e-6, in a server with other requests in flight) satisfies the step's fixed-point equation for
sampled orbitals, evaluated by the oracle (Sec. II-A, Eqs. lisan and x=tx), with its trace invariants.
"""
import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth
from test_zz_full_size_step import fixed_point_defect

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_config4_batch_sampled_targets_against_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300 import api
    specs = synth.batched_instances()
    templates = {n: synth.small_cell(3000 + n, n, 0.32 * n, 256, kT=0.02, natoms=8)
                 for n in sorted({s["n"] for s in specs})}
    host, items = [], []
    for sp in specs:
        w = templates[sp["n"]]
        N = sp["N"]
        src = np.ascontiguousarray(w.phi[:N].astype(np.complex64))
        occ = synth.fermi_dirac_occupations(N, 0.02)
        host.append((w, src, occ))
        items.append({"src": torch.from_numpy(src).cuda(), "occ": torch.from_numpy(occ).cuda(), "cell": w.cell,
                      "kernel": w.kernel})
    sizes = [sp["n"] for sp in specs]
    big = max(range(len(specs)), key=lambda k: (sizes[k], specs[k]["N"]))
    small = min(range(len(specs)), key=lambda k: (sizes[k], specs[k]["N"]))
    mid = next(k for k in range(len(specs)) if sizes[k] not in (64, sizes[small]))
    ctx = api.Context(0)
    try:
        outs, pairs, _ = ctx.apply_exchange_batched(items, precision="fp32")  # tunes, runs eagerly, captures
        eager = [outs[k].cpu().numpy().astype(np.complex128) for k in (big, mid, small)]
        for it, o in zip(items, outs):
            it["out"] = o
        _, _, nodes = ctx.apply_exchange_batched(items, precision="fp32")  # graph replay
        assert nodes > 0
        replay = [outs[k].cpu().numpy().astype(np.complex128) for k in (big, mid, small)]
    finally:
        ctx.close()
    assert pairs == sum(sp["N"] * (sp["N"] + 1) // 2 for sp in specs)
    for slot, k in enumerate((big, mid, small)):
        w, src, occ = host[k]
        g = O.grid_of(w.cell)
        K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
        s128 = src.astype(np.complex128)
        N = src.shape[0]
        for j in (0, N // 2, N - 1):
            ref = O.apply_exchange(s128, occ, s128[j:j + 1], K)[0]
            assert rel(eager[slot][j], ref) <= 1e-5, (k, j)
            assert rel(replay[slot][j], ref) <= 1e-5, (k, j)


def test_served_request_satisfies_its_fixed_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300.serve import Request, Server
    n, N = 48, 200
    w = synth.small_cell(2000 + n, n, 0.32 * n, 320, kT=0.02, natoms=8)
    phi = np.ascontiguousarray(w.phi[:N])
    f = synth.fermi_dirac_occupations(N, 0.02)
    sig = np.diag(f).astype(np.complex128)
    srv = Server(slots=3)
    try:
        others = [Request(phi=np.ascontiguousarray(w.phi[:64]), sigma=np.diag(f[:64]).astype(np.complex128),
                          occ=None, vloc=w.vloc, cell=w.cell, kernel=w.kernel, params={"tol": 1e-6})
                  for _ in range(2)]
        futs = [srv.submit(r) for r in others]
        fut = srv.submit(Request(phi=phi, sigma=sig, occ=None, vloc=w.vloc, cell=w.cell, kernel=w.kernel,
                                 params={"tol": 1e-6}))
        r = fut.result(timeout=600)
        for x in futs:
            x.result(timeout=600)
    finally:
        srv.close()
    assert r.error is None, r.error
    assert r.result["stats"]["converged"]
    phi1 = r.result["phi"].astype(np.complex128)
    sig1 = r.result["sigma"]
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    phi_n = phi.astype(np.complex64).astype(np.complex128)  # the request's orbitals as the FP32 form holds them
    defect = fixed_point_defect(phi_n, sig, phi1, sig1, w.vloc, g, K, 0.5, 10.0, 0.25, (0, N // 2, N - 1))
    assert defect <= 1e-5, defect
    assert abs(np.trace(sig1) - np.trace(sig)) <= 1e-5 * abs(np.trace(sig))
