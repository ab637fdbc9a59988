"""The benchmark's library comparison (cuFFT exchange through torch.fft) computes the same V_x
as the oracle; checked on the CPU at small sizes so that the timed comparison on the GPU compares
like with like."""
import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("N,batch", [(5, 2), (7, 64), (6, 1)])
def test_library_exchange_matches_oracle(N, batch):
    import bench
    cell = synth.Cell((8, 10, 12), (6.0, 7.0, 8.0))
    rng = np.random.default_rng(70 + N)
    phi = synth.random_orbitals(rng, cell, N, ecut=5.0)
    occ = np.linspace(1.0, 0.1, N)
    occ[2] = 0.0
    g = O.grid_of(cell)
    ref = O.apply_exchange(phi, occ, phi, O.exchange_kernel(g, 1, 0.3))
    K = bench.screened_kernel_table(cell, 0.3, torch.float64, "cpu")
    assert np.abs(K.numpy() - O.exchange_kernel(g, 1, 0.3)).max() <= 1e-12 * np.abs(K.numpy()).max()
    got = bench.library_exchange(torch.from_numpy(phi), torch.from_numpy(occ), K, batch=batch).numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-12
