"""The C ABI's error behaviour as include/ptim.h states it: invalid arguments come back as
PT_INVALID_ARG with a message in pt_last_error, before any kernel runs, and the context stays
usable afterwards.  Calls go straight through ctypes with raw pointers so the library's own checks
(not the Python binding's) are what is tested."""
import ctypes as C

import pytest

from paper_2501_03061_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300 import _lib as L
    from paper_2501_03061_gb300 import api
    ctx = api.Context(0)
    yield ctx, L, api
    ctx.close()


def p(t):
    return C.c_void_p(t.data_ptr())


def grid(cell):
    from paper_2501_03061_gb300 import api
    return api._grid(cell)


def kern():
    from paper_2501_03061_gb300 import api
    return api._kernel({"type": 1, "mu": 0.106})


def stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def expect_invalid(ctx, L, st, fragment):
    assert st == L.PT_INVALID_ARG, L.STATUS_NAMES.get(st, st)
    msg = ctx.lib.pt_last_error(ctx.h).decode()
    assert fragment in msg, msg


def test_exchange_argument_checks(env):
    ctx, L, api = env
    cell = synth.cubic(8, 5.0)
    g, k = grid(cell), kern()
    phi = torch.zeros((3, 8, 8, 8), dtype=torch.complex128, device="cuda")
    occ = torch.ones(3, dtype=torch.float64, device="cuda")
    out = torch.empty_like(phi)
    lib, h = ctx.lib, ctx.h
    fp64 = L.PRECISIONS["fp64"]
    # N <= 0
    st = lib.pt_apply_exchange(h, p(phi), p(occ), 0, None, 0, p(out), C.byref(g), C.byref(k), fp64, stream())
    assert st == L.PT_INVALID_ARG
    # out aliasing the sources
    st = lib.pt_apply_exchange(h, p(phi), p(occ), 3, None, 3, p(phi), C.byref(g), C.byref(k), fp64, stream())
    assert st == L.PT_INVALID_ARG
    # a source block that does not start on a 16-byte boundary (one complex64 element in)
    f32 = torch.zeros(3 * 512 + 1, dtype=torch.complex64, device="cuda")
    st = lib.pt_apply_exchange(h, C.c_void_p(f32.data_ptr() + 8), p(occ), 3, None, 3, p(out), C.byref(g), C.byref(k),
                               L.PRECISIONS["fp32"], stream())
    expect_invalid(ctx, L, st, "align")
    # an unknown precision
    st = lib.pt_apply_exchange(h, p(phi), p(occ), 3, None, 3, p(out), C.byref(g), C.byref(k), 7, stream())
    expect_invalid(ctx, L, st, "precision")
    # a grid side that is not 2,3,5-smooth
    bad = grid(synth.cubic(14, 5.0))
    st = lib.pt_apply_exchange(h, p(phi), p(occ), 3, None, 3, p(out), C.byref(bad), C.byref(k), fp64, stream())
    assert st == L.PT_INVALID_ARG
    # the context still works
    res = ctx.apply_exchange(phi, occ, cell=cell)
    assert float(res.abs().max()) == 0.0


def test_contraction_and_h_argument_checks(env):
    ctx, L, api = env
    cell = synth.cubic(8, 5.0)
    g = grid(cell)
    lib, h = ctx.lib, ctx.h
    a = torch.zeros((4, 8, 8, 8), dtype=torch.complex64, device="cuda")
    Cm = torch.zeros((4, 4), dtype=torch.complex128, device="cuda")
    fp32 = L.PRECISIONS["fp32"]
    assert lib.pt_overlap(h, p(a), 0, p(a), 4, C.byref(g), fp32, p(Cm), stream()) == L.PT_INVALID_ARG
    # rotation output overlapping its input
    assert lib.pt_rotate(h, p(a), 4, p(Cm), 4, C.byref(g), fp32, p(a), stream()) == L.PT_INVALID_ARG
    v = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
    # H with out == psi, and with a NULL potential
    st = lib.pt_apply_H(h, p(a), 4, p(a), p(v), None, 0.25, 10.0, None, C.byref(g), fp32, stream())
    assert st == L.PT_INVALID_ARG
    out = torch.empty_like(a)
    st = lib.pt_apply_H(h, p(a), 4, p(out), None, None, 0.25, 10.0, None, C.byref(g), fp32, stream())
    assert st == L.PT_INVALID_ARG


def test_step_and_local_potential_argument_checks(env):
    ctx, L, api = env
    cell = synth.cubic(8, 5.0)
    g, k = grid(cell), kern()
    lib, h = ctx.lib, ctx.h
    phi = torch.zeros((2, 8, 8, 8), dtype=torch.complex128, device="cuda")
    sig = torch.eye(2, dtype=torch.complex128, device="cuda")
    v = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
    stats = L.pt_ptim_stats()
    fp64 = L.PRECISIONS["fp64"]

    def params(**kw):
        d = dict(dt=0.5, alpha=0.25, ecut=10.0, tol=1e-6, max_outer=5, max_inner=5, anderson_depth=5,
                 anderson_beta=1.0, use_ace=1, spin=2.0, hxc=0)
        d.update(kw)
        prm = L.pt_ptim_params(d["dt"], d["alpha"], d["ecut"], d["tol"], d["max_outer"], d["max_inner"],
                               d["anderson_depth"], d["anderson_beta"], d["use_ace"], d["spin"], d["hxc"])
        return prm

    for bad in (dict(dt=0.0), dict(tol=-1.0), dict(anderson_depth=21), dict(max_inner=0), dict(hxc=2),
                dict(hxc=1, spin=0.0)):
        prm = params(**bad)
        st = lib.pt_ptim_step(h, p(phi), p(sig), 2, p(v), C.byref(g), C.byref(k), C.byref(prm), fp64,
                              C.byref(stats), stream())
        expect_invalid(ctx, L, st, "PT-IM parameters")
    # density: N = 0, non-positive spin
    rho = torch.empty((8, 8, 8), dtype=torch.float64, device="cuda")
    assert lib.pt_density(h, p(phi), p(sig), 0, C.byref(g), fp64, 2.0, p(rho), stream()) == L.PT_INVALID_ARG
    assert lib.pt_density(h, p(phi), p(sig), 2, C.byref(g), fp64, 0.0, p(rho), stream()) == L.PT_INVALID_ARG
    # current: NULL output
    assert lib.pt_current(h, p(phi), p(sig), 2, C.byref(g), fp64, None, 2.0, None, stream()) == L.PT_INVALID_ARG


def test_options_are_checked(env):
    ctx, L, api = env
    lib, h = ctx.lib, ctx.h
    for key, val in ((b"no_such_option", 1.0), (b"scratch_bytes", 0.0), (b"exchange64_scratch_bytes", 0.0),
                     (b"tc_period", 0.0), (b"tc_period", 65.0), (b"ptim_inner_kappa", -0.5)):
        assert lib.pt_set_option(h, key, val) == L.PT_INVALID_ARG, key
    assert lib.pt_set_option(h, b"tc_period", 2.0) == L.PT_OK
