"""The Python binding rejects buffers that do not match the call before the C library sees a
pointer (no GPU needed).  The library addresses its arguments by pointer and size, so a tensor
that is shorter than the cell and orbital count imply would be read or written past its end;
the binding compares every tensor's element count with what the call addresses and raises
PtimError(PT_INVALID_ARG) instead.  These tests drive a Context whose library handle refuses to
be called, on CPU tensors, so any check that let a bad buffer through fails loudly here."""
import pytest

torch = pytest.importorskip("torch")

from paper_2501_03061_gb300 import _lib as L  # noqa: E402
from paper_2501_03061_gb300 import api, synth  # noqa: E402


class NoLibrary:
    def __getattr__(self, name):
        raise AssertionError(f"the library was called ({name}) with a buffer the binding should have rejected")


@pytest.fixture
def ctx():
    c = object.__new__(api.Context)  # the binding's checks only: no device, no pt_ctx
    c.lib = NoLibrary()
    c.device = torch.device("cpu")
    c.h = None
    return c


CELL = synth.cubic(8, 5.0)
OTHER = synth.Cell((8, 8, 6), (5.0, 5.0, 4.0))


def block(N, cell=CELL, dtype=torch.complex128):
    nx, ny, nz = cell.n
    return torch.zeros((N, nz, ny, nx), dtype=dtype)


def invalid(fn, fragment):
    with pytest.raises(api.PtimError) as ei:
        fn()
    assert ei.value.status == L.PT_INVALID_ARG
    assert fragment in str(ei.value), str(ei.value)


def test_exchange_checks(ctx):
    phi, occ = block(3), torch.ones(3, dtype=torch.float64)
    invalid(lambda: ctx.apply_exchange(phi, occ, cell=OTHER), "src holds")
    invalid(lambda: ctx.apply_exchange(phi, occ, block(2, OTHER), cell=CELL), "tgt holds")
    invalid(lambda: ctx.apply_exchange(phi, torch.ones(2, dtype=torch.float64), cell=CELL), "occ holds 2")
    invalid(lambda: ctx.apply_exchange(phi, occ, out=block(2), cell=CELL), "out holds")
    invalid(lambda: ctx.apply_exchange(phi, occ, block(2), out=block(3), cell=CELL), "out holds")
    with pytest.raises(ValueError):
        ctx.apply_exchange(phi, occ, out=block(3, dtype=torch.complex64), cell=CELL)


def test_batched_checks_name_the_item(ctx):
    good = {"src": block(3), "occ": torch.ones(3, dtype=torch.float64), "cell": CELL}
    bad = {"src": block(3), "occ": torch.ones(3, dtype=torch.float64), "cell": OTHER}
    invalid(lambda: ctx.apply_exchange_batched([good, bad], precision="fp64"), "item 1: src holds")
    short = dict(good, out=block(1))
    invalid(lambda: ctx.apply_exchange_batched([short], precision="fp64"), "item 0: out holds")
    few = dict(good, occ=torch.ones(1, dtype=torch.float64))
    invalid(lambda: ctx.apply_exchange_batched([good, good, few], precision="fp64"), "item 2: occ holds 1")


def test_ace_checks(ctx):
    phi = block(4)
    invalid(lambda: ctx.build_ace(phi, torch.ones(4, dtype=torch.float64), cell=OTHER), "phi holds")
    invalid(lambda: ctx.build_ace(phi, torch.ones(3, dtype=torch.float64), cell=CELL), "occ holds 3")
    invalid(lambda: ctx.build_ace_from(block(3), phi, cell=CELL), "W holds")
    ace = object.__new__(api.Ace)
    ace.ctx, ace.handle, ace.N, ace.cell, ace.precision = ctx, None, 4, CELL, "fp64"
    invalid(lambda: ctx.apply_ace(ace, block(2, OTHER)), "psi holds")
    invalid(lambda: ctx.apply_ace(ace, block(2), out=block(1)), "out holds")


def test_contraction_checks(ctx):
    a, b = block(4), block(5)
    invalid(lambda: ctx.overlap(a, b, cell=OTHER), "A holds")
    invalid(lambda: ctx.overlap(a, block(5, OTHER), cell=CELL), "B holds")
    invalid(lambda: ctx.overlap(a, b, cell=CELL, out=torch.zeros((4, 4), dtype=torch.complex128)), "out holds 16")
    B = torch.zeros((4, 6), dtype=torch.complex128)
    invalid(lambda: ctx.rotate(a, B, cell=OTHER), "A holds")
    invalid(lambda: ctx.rotate(a, B, cell=CELL, out=block(5)), "out holds")
    with pytest.raises(ValueError):
        ctx.rotate(a, torch.zeros((3, 6), dtype=torch.complex128), cell=CELL)


def test_hamiltonian_and_observable_checks(ctx):
    psi, v = block(3), torch.zeros((8, 8, 8), dtype=torch.float64)
    invalid(lambda: ctx.apply_H(psi, v, cell=OTHER), "psi holds")
    invalid(lambda: ctx.apply_H(psi, torch.zeros((8, 8, 6), dtype=torch.float64), cell=CELL), "vloc holds")
    invalid(lambda: ctx.apply_H(psi, v, cell=CELL, out=block(2)), "out holds")
    sig = torch.eye(3, dtype=torch.complex128)
    invalid(lambda: ctx.density(psi, torch.eye(2, dtype=torch.complex128), cell=CELL), "sigma holds 4")
    invalid(lambda: ctx.density(psi, sig, cell=CELL, out=torch.zeros(10, dtype=torch.float64)), "out holds 10")
    invalid(lambda: ctx.current(psi, torch.eye(4, dtype=torch.complex128), cell=CELL), "sigma holds 16")
    invalid(lambda: ctx.current(block(3, OTHER), sig, cell=CELL), "phi holds")
    invalid(lambda: ctx.hxc_potential(torch.zeros(100, dtype=torch.float64), cell=CELL), "rho holds 100")
    invalid(lambda: ctx.hxc_potential(v, torch.zeros(5, dtype=torch.float64), cell=CELL), "vloc holds 5")
    invalid(lambda: ctx.hxc_potential(v, cell=CELL, out=torch.zeros(7, dtype=torch.float64)), "out holds 7")
    invalid(lambda: ctx.diag_occupations(torch.zeros((3, 4), dtype=torch.complex128)), "square")


def test_step_checks(ctx):
    phi, v = block(3), torch.zeros((8, 8, 8), dtype=torch.float64)
    sig = torch.eye(3, dtype=torch.complex128)
    invalid(lambda: ctx.ptim_step(phi, sig, v, cell=OTHER), "phi holds")
    invalid(lambda: ctx.ptim_step(phi, torch.eye(2, dtype=torch.complex128), v, cell=CELL), "sigma holds 4")
    invalid(lambda: ctx.ptim_step(phi, sig, torch.zeros(9, dtype=torch.float64), cell=CELL), "vloc holds 9")


def test_matching_buffers_reach_the_library(ctx):
    """Control: buffers that match the call pass every check and reach the (refusing) library."""
    phi, v = block(3), torch.zeros((8, 8, 8), dtype=torch.float64)
    sig = torch.eye(3, dtype=torch.complex128)
    for call in (lambda: ctx.apply_exchange(phi, torch.ones(3, dtype=torch.float64), cell=CELL),
                 lambda: ctx.overlap(phi, cell=CELL),
                 lambda: ctx.apply_H(phi, v, cell=CELL),
                 lambda: ctx.density(phi, sig, cell=CELL),
                 lambda: ctx.hxc_potential(v, v, cell=CELL),
                 lambda: ctx.ptim_step(phi, sig, v, cell=CELL)):
        with pytest.raises(AssertionError, match="the library was called"):
            call()
