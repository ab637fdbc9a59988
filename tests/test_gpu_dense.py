"""GPU FP64 dense kernels exercised through the C ABI: ACE Cholesky at sizes spanning several panels."""
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


@pytest.mark.parametrize("N", [31, 32, 33, 70, 97, 160, 200])
def test_ace_from_w_multi_panel_cholesky(ctx, N):
    """build_ace_from runs the blocked Cholesky (32-wide panels) and the bottom-up blocked
    triangular inverse; the resulting xi must match the oracle's construction for N across panel
    boundaries and merge levels (N = 200: blocks of 32 merged into 64, 128 and a partial 72)."""
    rng = np.random.default_rng(N)
    cell = synth.cubic(12, 9.0)
    phi = synth.random_orbitals(rng, cell, N, ecut=20.0)
    occ = rng.uniform(0.05, 1.0, N)
    g = O.grid_of(cell)
    W = O.apply_exchange(phi, occ, phi, O.exchange_kernel(g, 1, 0.106))
    xi_ref = O.build_ace(phi, W, g.dV)
    ace = ctx.build_ace_from(torch.from_numpy(W).cuda(), torch.from_numpy(phi).cuda(), cell=cell, precision="fp64")
    xi = ace.xi().cpu().numpy()
    assert np.linalg.norm(xi - xi_ref) / np.linalg.norm(xi_ref) < 1e-11
    ace.close()
