"""pt_ptim_stats.total_energy is E(t_n) of the step's input state: spin Tr[P (-Lap/2 + V_loc)]
with the field's vector potential in the kinetic term, plus E_x, plus E_H + E_xc when the step
rebuilds V_Hxc.  Compared with the FP64 oracle's total energy on the same state, for the first
step and for the second (whose input is the GPU's own output of the first)."""
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


def case():
    w = synth.small_cell(23, 12, 8.0, 6, kT=0.05, ecut=6.0)
    sig = np.diag(w.occ).astype(np.complex128)
    sig[0, 1] = sig[1, 0] = 0.03
    sig[2, 4] = 0.02j
    sig[4, 2] = -0.02j
    return w, sig


@pytest.mark.parametrize("precision,use_ace,hxc,A,tc_gram,tol", [
    ("fp64", True, False, None, 0, 1e-10),
    ("fp64", False, False, None, 0, 1e-10),
    ("fp64", True, True, None, 0, 1e-10),
    ("fp64", True, False, (0.3, -0.2, 0.1), 0, 1e-10),
    ("fp32", True, True, (0.3, -0.2, 0.1), 1, 1e-5),
])
def test_step_reports_the_input_states_total_energy(ctx, precision, use_ace, hxc, A, tc_gram, tol):
    w, sig = case()
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    dt = np.complex128 if precision == "fp64" else np.complex64
    phi0 = w.phi.astype(dt)
    phi = torch.from_numpy(phi0).cuda()
    sigma = torch.from_numpy(sig).cuda()
    vloc = torch.from_numpy(w.vloc).cuda()
    Av = None if A is None else np.array(A)
    # the input state's energy does not depend on how far the step converges
    kw = dict(cell=w.cell, kernel=w.kernel, precision=precision, dt=0.5, ecut=6.0,
              tol=1e-10 if precision == "fp64" else 2e-6, use_ace=use_ace, hxc=hxc, A=A, allow_unconverged=True)
    ctx.set_option("tc_gram", tc_gram)
    # the second step chains on the first one's output: without the warm-started ACE operator, so that
    # its first iteration's exchange is exact on its input and the energy is reported
    ctx.set_option("ptim_ace_warm", 0)
    try:
        s1 = ctx.ptim_step(phi, sigma, vloc, **kw)
        phi1 = phi.cpu().numpy().astype(np.complex128)
        sig1 = sigma.cpu().numpy()
        s2 = ctx.ptim_step(phi, sigma, vloc, **kw)
    finally:
        ctx.set_option("tc_gram", 0)
        ctx.set_option("ptim_ace_warm", 1)
    e0 = O.total_energy(phi0.astype(np.complex128), sig, w.vloc, g, K, 6.0, hxc=hxc, A=Av)
    e1 = O.total_energy(phi1, sig1, w.vloc, g, K, 6.0, hxc=hxc, A=Av)
    assert abs(s1["total_energy"] - e0) <= tol * abs(e0), (s1["total_energy"], e0)
    assert abs(s2["total_energy"] - e1) <= tol * abs(e1), (s2["total_energy"], e1)
