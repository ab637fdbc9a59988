"""The seeded input generators follow their stated recipe (no GPU): orthonormal band-limited
orbitals, Fermi-Dirac occupations with the stated electron count, the diamond-like site sets,
periodic Gaussian wells, and reproducibility from the seed."""
import math

import numpy as np
import pytest

from paper_2501_03061_gb300 import synth


def test_random_orbitals_orthonormal_and_band_limited():
    cell = synth.Cell((12, 10, 9), (7.0, 6.0, 5.5))
    rng = np.random.default_rng(3)
    phi = synth.random_orbitals(rng, cell, 20, ecut=6.0)
    dV = cell.volume / cell.ng
    P = phi.reshape(20, -1)
    S = dV * P.conj() @ P.T
    assert np.abs(S - np.eye(20)).max() < 1e-13
    spec = np.fft.fftn(phi, axes=(1, 2, 3)).reshape(20, -1)
    outside = np.ones(cell.ng, bool)
    outside[synth.sphere_indices(cell, 6.0)] = False
    assert np.abs(spec[:, outside]).max() < 1e-10 * np.abs(spec).max()


def test_random_orbitals_reproducible_and_reject_too_many():
    cell = synth.cubic(8, 5.0)
    a = synth.random_orbitals(np.random.default_rng(9), cell, 4, ecut=4.0)
    b = synth.random_orbitals(np.random.default_rng(9), cell, 4, ecut=4.0)
    assert np.array_equal(a, b)
    n = synth.sphere_indices(cell, 4.0).size
    with pytest.raises(ValueError):
        synth.random_orbitals(np.random.default_rng(9), cell, n + 1, ecut=4.0)


@pytest.mark.parametrize("N,kT", [(16, 0.01), (320, 0.02), (64, 0.05)])
def test_fermi_dirac_occupations(N, kT):
    f = synth.fermi_dirac_occupations(N, kT)
    assert abs(f.sum() - 0.8 * N) < 1e-9
    assert np.all(np.diff(f) <= 0) and np.all((f > 0) & (f <= 1))
    # Fermi-Dirac form on the ladder: log(1/f - 1) is linear in the level with slope spacing/kT
    # (away from f ~ 1, where 1/f - 1 loses digits to cancellation)
    x = np.log(1.0 / f[(f > 1e-6) & (f < 1 - 1e-6)] - 1.0)
    if x.size > 2:
        assert np.allclose(np.diff(x), (0.5 / N) / kT, rtol=1e-6)


def test_site_sets():
    d = synth.diamond_sites(1, 1.0)
    assert d.shape == (8, 3)
    # nearest-neighbour distance of diamond: sqrt(3)/4 of the lattice constant
    dist = np.linalg.norm(d[:, None] - d[None], axis=-1) + np.eye(8) * 10
    assert abs(dist.min() - math.sqrt(3) / 4) < 1e-12
    rng = np.random.default_rng(1)
    s128 = synth.silicon_like_sites(rng, 128, 20.5, jitter=0.0)
    assert s128.shape == (128, 3)
    # all distinct sites inside the cell
    assert np.all((s128 >= 0) & (s128 < 20.5))
    assert len({tuple(np.round(p, 9)) for p in s128}) == 128


def test_gaussian_wells_periodic_and_normalised():
    cell = synth.cubic(32, 16.0)
    centre = np.array([[8.0, 8.0, 8.0]])
    v = synth.gaussian_wells(cell, centre, depth=1.0, width=1.0)
    assert v.min() == pytest.approx(-1.0, abs=1e-12)  # grid point at the centre
    # integral of a 3-D Gaussian: -(2 pi w^2)^(3/2)
    dV = cell.volume / cell.ng
    assert v.sum() * dV == pytest.approx(-(2 * math.pi) ** 1.5, rel=1e-9)
    # a well centred on the cell boundary is the same field shifted by half the cell
    v2 = synth.gaussian_wells(cell, np.array([[0.0, 0.0, 0.0]]), depth=1.0, width=1.0)
    assert np.allclose(np.roll(v2, (16, 16, 16), axis=(0, 1, 2)), v, atol=1e-12)


def test_named_workloads_shapes():
    w = synth.exchange_small()
    assert w.phi.shape == (16, 24, 24, 24) and w.occ.shape == (16,)
    specs = synth.batched_instances()
    assert len(specs) == 64 and all(16 <= s["N"] <= 256 for s in specs)
    reqs = synth.serving_stream(count=50)
    t = [r["t"] if isinstance(r, dict) else r.t for r in reqs]
    assert all(b >= a for a, b in zip(t, t[1:]))
