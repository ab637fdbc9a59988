"""The allocation-free exchange entry point against the regular one.

pt_apply_exchange_noalloc serves callers that cannot allocate device memory while it runs (a
host application whose pool allocator owns all device memory, or a loop that cannot take the
device synchronisation of cudaMalloc).  It keeps its scratch in static device arrays, so it must
give the same V_x tgt as pt_apply_exchange — on every call, including a second call that finds
the previous call's data still in those arrays — and it must not allocate: after warm-up calls
(which also let lazy module loading bring in the kernels), further calls leave the device's free
memory and torch's allocated bytes unchanged.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2501_03061_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(lib, src, occ, tgt, out, cell, kernel, precision):
    from paper_2501_03061_gb300 import _lib as L
    from paper_2501_03061_gb300.api import _grid, _kernel

    g, k = _grid(cell), _kernel(kernel)
    st = lib.pt_apply_exchange_noalloc(C.c_void_p(src.data_ptr()), C.c_void_p(occ.data_ptr()), src.shape[0],
                                       None if tgt is None else C.c_void_p(tgt.data_ptr()),
                                       (src if tgt is None else tgt).shape[0], C.c_void_p(out.data_ptr()),
                                       C.byref(g), C.byref(k), L.PRECISIONS[precision],
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == L.PT_OK, L.STATUS_NAMES.get(st, st)
    return out


CASES = [
    # (grid, L, N, M (None = symmetric), precision, tolerance)
    (24, 10.0, 16, None, "fp64", 1e-12),
    (24, 10.0, 9, 5, "fp32", 1e-6),
    (64, 20.5, 6, None, "fp32", 1e-6),   # several batches of the 32 MiB scratch
    (30, 9.6, 7, 4, "fp64", 1e-12),
    ((24, 30, 20), (7.5, 9.4, 6.3), 6, None, "fp32", 1e-6),  # non-cubic: table key and twiddle layout
]


def _cell(n, L):
    return synth.cubic(n, L) if isinstance(n, int) else synth.Cell(n, L)


@pytest.mark.parametrize("n,L,N,M,precision,tol", CASES)
def test_noalloc_matches_regular_exchange_twice(n, L, N, M, precision, tol):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300 import _lib, api

    lib = _lib.load()
    ctx = api.Context(0)
    try:
        rng = np.random.default_rng((n if isinstance(n, int) else sum(n)) * 100 + N)
        cell = _cell(n, L)
        dt = np.complex128 if precision == "fp64" else np.complex64
        kernel = {"type": 1, "mu": synth.SCREENED_MU}
        for call in range(2):  # the second call reuses the static arrays the first one filled
            src = torch.from_numpy(synth.random_orbitals(rng, cell, N, ecut=6.0).astype(dt)).cuda()
            tgt = None if M is None else torch.from_numpy(synth.random_orbitals(rng, cell, M, ecut=6.0).astype(dt)).cuda()
            occ = torch.from_numpy(np.concatenate([[0.0], rng.uniform(0.05, 1.0, N - 1)])).cuda()
            ref = ctx.apply_exchange(src, occ, tgt, cell=cell, kernel=kernel, precision=precision)
            out = torch.full_like(ref, float("nan"))
            _noalloc(lib, src, occ, tgt, out, cell, kernel, precision)
            torch.cuda.synchronize()
            err = float(torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref))
            assert err <= tol, (call, err)
    finally:
        ctx.close()


def test_noalloc_rejects_oversize_requests():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300 import _lib

    lib = _lib.load()
    cell = synth.cubic(8, 5.0)
    src = torch.zeros((1025, 8, 8, 8), dtype=torch.complex64, device="cuda")
    occ = torch.ones(1025, dtype=torch.float64, device="cuda")
    out = torch.empty_like(src)
    from paper_2501_03061_gb300.api import _grid, _kernel
    st = lib.pt_apply_exchange_noalloc(C.c_void_p(src.data_ptr()), C.c_void_p(occ.data_ptr()), 1025, None, 1025,
                                       C.c_void_p(out.data_ptr()), C.byref(_grid(cell)), C.byref(_kernel(None)), 1,
                                       None)
    assert st == _lib.PT_INVALID_ARG


def test_noalloc_calls_allocate_nothing():
    """Two warm-up calls (a 64^3 symmetric FP32 request and a 24x30x20 FP64 request with separate
    targets), then the same two requests with other data: the device's free memory and torch's
    allocated bytes are the same before and after the second pair of calls."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300 import _lib

    lib = _lib.load()
    rng = np.random.default_rng(77)
    kernel = {"type": 1, "mu": synth.SCREENED_MU}
    reqs = []
    for cell, N, M, precision in ((synth.cubic(64, 20.5), 5, None, "fp32"),
                                  (synth.Cell((24, 30, 20), (7.5, 9.4, 6.3)), 4, 3, "fp64")):
        dt = np.complex128 if precision == "fp64" else np.complex64
        for _ in range(2):
            src = torch.from_numpy(synth.random_orbitals(rng, cell, N, ecut=5.0).astype(dt)).cuda()
            tgt = None if M is None else torch.from_numpy(synth.random_orbitals(rng, cell, M, ecut=5.0).astype(dt)).cuda()
            occ = torch.from_numpy(rng.uniform(0.1, 1.0, N)).cuda()
            out = torch.empty_like(src if tgt is None else tgt)
            reqs.append((src, occ, tgt, out, cell, precision))
    for r in reqs[0::2]:  # warm-up: one call of each kind
        _noalloc(lib, r[0], r[1], r[2], r[3], r[4], kernel, r[5])
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for r in reqs[1::2]:
        _noalloc(lib, r[0], r[1], r[2], r[3], r[4], kernel, r[5])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    for r in reqs:
        assert bool(torch.isfinite(torch.view_as_real(r[3])).all())
