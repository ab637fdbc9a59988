"""The exchange energy at the benchmark's full size (64^3 grid, N = 320, 128 sites) against the
FP64 oracle: the FP32 form within 1e-6 Ha/atom and the plain FP64 form within 1e-11 relative.

E_x = spin (alpha/2) sum_i d_i <phi_i|V_x phi_i> (Sec. II-B; Sec. IV-A1, Eq. vxdiag with
sigma = diag(d)).  The GPU value contracts the library's V_x Phi (pt_apply_exchange, the
benchmark's launch configuration) with Phi in FP64 on the host; the oracle value takes the
one-forward-FFT-per-pair route (exchange_energy_pairs, pinned against the exchange route and the
plane-wave closed form on the CPU) on the same inputs — the orbitals rounded to complex64 for the
FP32 comparison — with the 51,360 pairs split over the host's cores in spawned worker processes.
"""
import multiprocessing as mp
import os
import tempfile

import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPIN, ALPHA = 2.0, 0.25

_W = {}


def _init(path, occ_path, n, L, mu):
    _W["phi"] = np.load(path, mmap_mode="r")
    _W["d"] = np.load(occ_path)
    g = O.grid_of(synth.cubic(n, L))
    _W["K"] = O.exchange_kernel(g, 1, mu)
    _W["dV"] = g.dV


def _rows(rows):
    return O.exchange_energy_pairs(_W["phi"], _W["d"], _W["K"], _W["dV"], rows=rows)


def oracle_energy(phi128, occ, n, L):
    """spin alpha/2 * sum_ij pairs, the rows i dealt out so that every worker gets a similar share."""
    N = phi128.shape[0]
    nproc = max(1, min(32, os.cpu_count() or 1))
    order = sorted(range(N), key=lambda i: -(N - i))  # longest rows first
    chunks = [order[k::4 * nproc] for k in range(4 * nproc)]
    with tempfile.TemporaryDirectory() as td:
        path, opath = os.path.join(td, "phi.npy"), os.path.join(td, "occ.npy")
        np.save(path, phi128)
        np.save(opath, occ)
        with mp.get_context("spawn").Pool(nproc, initializer=_init,
                                          initargs=(path, opath, n, L, synth.SCREENED_MU)) as pool:
            parts = pool.map(_rows, [c for c in chunks if c])
    return SPIN * 0.5 * ALPHA * float(np.sum(parts))


def gpu_energy(ctx, phi_np, occ, w, precision):
    phi = torch.from_numpy(phi_np).cuda()
    W = ctx.apply_exchange(phi, torch.from_numpy(occ).cuda(), cell=w.cell, kernel=w.kernel, precision=precision)
    Wh = W.cpu().numpy().astype(np.complex128)
    del W, phi
    dV = w.cell.volume / w.cell.ng
    N = phi_np.shape[0]
    p = phi_np.reshape(N, -1).astype(np.complex128)
    diag = dV * np.einsum("ir,ir->i", p.conj(), Wh.reshape(N, -1)).real
    return SPIN * 0.5 * ALPHA * float(np.sum(occ * diag))


@pytest.fixture(scope="module")
def cell128():
    return synth.ptim_cell128()


def test_exchange_energy_fp32_at_64cubed_N320(cell128):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300 import api
    w = cell128
    phi32 = w.phi.astype(np.complex64)
    ctx = api.Context(0)
    try:
        e_gpu = gpu_energy(ctx, phi32, w.occ, w, "fp32")
    finally:
        ctx.close()
    e_ref = oracle_energy(phi32.astype(np.complex128), w.occ, 64, w.cell.L[0])
    err = abs(e_gpu - e_ref) / w.natoms
    print(f"E_x FP32 GPU {e_gpu:.12f} Ha, oracle {e_ref:.12f} Ha, |dE|/atom {err:.3e} Ha")
    assert e_ref < 0
    assert err <= 1e-6, err


def test_exchange_energy_fp64_at_64cubed_N320(cell128):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300 import api
    w = cell128
    ctx = api.Context(0)
    try:
        e_gpu = gpu_energy(ctx, w.phi, w.occ, w, "fp64")
    finally:
        ctx.close()
    e_ref = oracle_energy(w.phi, w.occ, 64, w.cell.L[0])
    rel = abs(e_gpu - e_ref) / abs(e_ref)
    print(f"E_x FP64 GPU {e_gpu:.15f} Ha, oracle {e_ref:.15f} Ha, relative {rel:.3e}")
    assert rel <= 1e-11, rel
