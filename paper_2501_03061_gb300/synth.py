"""Seeded synthetic inputs for the PT-IM hybrid-functional hot path.

This module is shared by the tests, the FP64 oracle's callers and the benchmark.
It holds no arithmetic of the method itself (no exchange kernel, no Hamiltonian,
no propagation): it only draws the inputs the method is applied to.

The workloads mirror the paper's silicon cells (Sec. VI "physical system": cubic
Si cells, N = 2.5 N_atom orbitals, Ecut = 10 Ha, fractional Fermi-Dirac
occupations at finite temperature).  Real pseudopotentials are not available,
so a sum of seeded Gaussian wells stands in for the local potential.

Layouts (shared with the C ABI):
  * orbitals: complex array of shape (N, nz, ny, nx), C order, i.e. orbital j,
    point (x, y, z) sits at flat index j*Ng + (z*ny + y)*nx + x;
  * occupation matrix sigma: complex (N, N), sigma[i, j] = sigma_ij;
  * local potential: real (nz, ny, nx).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# 2·3·5-smooth grid sizes the batched and serving workloads draw from.
BATCH_GRID_SIZES = (24, 30, 32, 36, 40, 48, 54, 60, 64)
SERVE_GRID_SIZES = (32, 36, 40, 48, 54, 60, 64)


@dataclasses.dataclass
class Cell:
    """A cubic or orthorhombic periodic cell sampled on an nx×ny×nz grid."""

    n: tuple  # (nx, ny, nz)
    L: tuple  # (Lx, Ly, Lz) in bohr

    @property
    def ng(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def volume(self) -> float:
        return self.L[0] * self.L[1] * self.L[2]

    @property
    def dV(self) -> float:
        return self.volume / self.ng


def cubic(n: int, L: float) -> Cell:
    return Cell((n, n, n), (L, L, L))


def integer_frequencies(n: int) -> np.ndarray:
    """Grid frequencies m wrapped to [-n/2, n/2) (numpy FFT ordering)."""
    return np.fft.fftfreq(n, 1.0 / n).round().astype(np.int64)


def _g2_axes(cell: Cell):
    gx = 2 * np.pi * integer_frequencies(cell.n[0]) / cell.L[0]
    gy = 2 * np.pi * integer_frequencies(cell.n[1]) / cell.L[1]
    gz = 2 * np.pi * integer_frequencies(cell.n[2]) / cell.L[2]
    return gx, gy, gz


def sphere_indices(cell: Cell, ecut: float) -> np.ndarray:
    """Flat (z, y, x) indices of the plane waves with |G|^2/2 <= ecut."""
    gx, gy, gz = _g2_axes(cell)
    g2 = gz[:, None, None] ** 2 + gy[None, :, None] ** 2 + gx[None, None, :] ** 2
    return np.flatnonzero((0.5 * g2).ravel() <= ecut)


def random_orbitals(rng: np.random.Generator, cell: Cell, N: int, ecut: float = 10.0,
                    dtype=np.complex128) -> np.ndarray:
    """N orbitals with N(0,1)+iN(0,1) plane-wave coefficients inside the Ecut sphere,
    orthonormalised under <a|b> = dV sum_r conj(a) b by a Householder QR.

    Because sum_r e^{-iG.r} e^{iG'.r} = Ng delta_GG', orthonormalising the
    coefficient vectors with weight Omega is the same as orthonormalising the
    real-space orbitals with weight dV; the QR is done on the (smaller)
    coefficient matrix and the result is then placed on the grid.
    """
    idx = sphere_indices(cell, ecut)
    if idx.size < N:
        raise ValueError(f"Ecut sphere holds {idx.size} plane waves < N={N}")
    coef = rng.standard_normal((idx.size, N)) + 1j * rng.standard_normal((idx.size, N))
    q, r = np.linalg.qr(coef * math.sqrt(cell.volume))
    q = q * np.sign(np.real(np.diag(r)))[None, :]  # unique QR: positive diagonal
    coef = q / math.sqrt(cell.volume)
    nx, ny, nz = cell.n
    spec = np.zeros((N, cell.ng), dtype=np.complex128)
    spec[:, idx] = coef.T
    # phi(r) = sum_G c(G) e^{iG.r} = Ng * ifftn(c)
    phi = np.fft.ifftn(spec.reshape(N, nz, ny, nx), axes=(1, 2, 3)) * cell.ng
    return np.ascontiguousarray(phi.astype(dtype))


def plane_wave_orbitals(cell: Cell, freqs) -> np.ndarray:
    """phi_j(r) = exp(i G_j . r)/sqrt(Omega) for integer frequency triples (mx, my, mz)."""
    nx, ny, nz = cell.n
    x = np.arange(nx) / nx
    y = np.arange(ny) / ny
    z = np.arange(nz) / nz
    out = np.empty((len(freqs), nz, ny, nx), dtype=np.complex128)
    for j, (mx, my, mz) in enumerate(freqs):
        ph = (2j * np.pi) * (mz * z[:, None, None] + my * y[None, :, None] + mx * x[None, None, :])
        out[j] = np.exp(ph) / math.sqrt(cell.volume)
    return out


def fermi_dirac_occupations(N: int, kT: float, n_occ: float | None = None,
                            spacing: float | None = None) -> np.ndarray:
    """Occupations f_i = 1/(1+exp((eps_i - mu)/kT)) on an equally spaced level ladder.

    eps_i = (i + 1/2 - n_occ) * spacing, spacing = 0.5 Ha / N, n_occ = 0.8 N by
    default; mu is found by bisection so that sum_i f_i = n_occ to 1e-14.
    """
    if n_occ is None:
        n_occ = 0.8 * N
    if spacing is None:
        spacing = 0.5 / N
    eps = (np.arange(N) + 0.5 - n_occ) * spacing

    def occ(mu):
        x = np.clip((eps - mu) / kT, -700, 700)
        return 1.0 / (1.0 + np.exp(x))

    lo, hi = eps[0] - 50 * kT - 1.0, eps[-1] + 50 * kT + 1.0
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if occ(mid).sum() > n_occ:
            hi = mid
        else:
            lo = mid
        if hi - lo < 1e-16:
            break
    f = occ(0.5 * (lo + hi))
    return f


def diamond_sites(cells: int, a: float) -> np.ndarray:
    """Cartesian sites of a cells^3 supercell of the 8-atom cubic diamond cell (lattice a)."""
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    basis = np.concatenate([fcc, fcc + 0.25])
    out = []
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                out.append((basis + np.array([i, j, k])) * a)
    return np.concatenate(out)


def silicon_like_sites(rng: np.random.Generator, natoms: int, L: float, jitter: float = 0.1) -> np.ndarray:
    """natoms jittered sites in a cubic cell of side L.

    8 atoms: the cubic diamond cell.  64: its 2x2x2 supercell.  128: the 64
    diamond sites of the 2x2x2 supercell plus the same set shifted by half the
    small cell's body diagonal.  Each site gets N(0, jitter) bohr noise.
    """
    if natoms == 8:
        base = diamond_sites(1, L)
    elif natoms == 64:
        base = diamond_sites(2, L / 2)
    elif natoms == 128:
        d = diamond_sites(2, L / 2)
        base = np.concatenate([d, d + 0.5 * (L / 2)])
    else:
        raise ValueError("natoms must be 8, 64 or 128")
    sites = base + rng.normal(0.0, jitter, size=base.shape)
    return np.mod(sites, L)


def gaussian_wells(cell: Cell, sites: np.ndarray, depth: float = 1.0, width: float = 1.0) -> np.ndarray:
    """V(r) = -sum_a depth * exp(-|r - R_a|^2 / (2 width^2)) with periodic images."""
    nx, ny, nz = cell.n
    Lx, Ly, Lz = cell.L
    x = np.arange(nx) * Lx / nx
    y = np.arange(ny) * Ly / ny
    z = np.arange(nz) * Lz / nz
    v = np.zeros((nz, ny, nx))
    for R in sites:
        def axis(c, Rc, Lc):
            d = c - Rc
            d = d - Lc * np.round(d / Lc)  # minimum image
            acc = np.zeros_like(c)
            for img in (-1, 0, 1):  # two more images keep the tails exact for width << L
                acc += np.exp(-((d + img * Lc) ** 2) / (2 * width ** 2))
            return acc
        ex = axis(x, R[0], Lx)
        ey = axis(y, R[1], Ly)
        ez = axis(z, R[2], Lz)
        v -= depth * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    return v


# ----------------------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------------------

SCREENED_MU = 0.106  # bohr^-1, the screening length of the erfc-screened (HSE-like) kernel


@dataclasses.dataclass
class Workload:
    name: str
    cell: Cell
    phi: np.ndarray          # (N, nz, ny, nx) complex128, orthonormal
    occ: np.ndarray          # (N,) Fermi-Dirac occupations
    sigma: np.ndarray        # (N, N) complex128 = diag(occ)
    vloc: np.ndarray | None  # (nz, ny, nx) float64
    natoms: int
    kernel: dict             # {"type": 1, "mu": 0.106}
    params: dict             # dt, alpha, ecut, ...

    @property
    def N(self) -> int:
        return self.phi.shape[0]


def exchange_small(seed: int = 1000, n: int = 24, L: float = 10.0, N: int = 16, kT: float = 0.01) -> Workload:
    """Exchange + ACE workload: L = 10 bohr, 24^3 grid, N = 16 orbitals, kT = 0.01 Ha."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cell = cubic(n, L)
    phi = random_orbitals(rng, cell, N)
    f = fermi_dirac_occupations(N, kT)
    sites = silicon_like_sites(rng, 8, L)
    vloc = gaussian_wells(cell, sites)
    return Workload(f"exchange_{n}^3_N{N}", cell, phi, f, np.diag(f).astype(np.complex128), vloc, 8,
                    {"type": 1, "mu": SCREENED_MU}, {"dt": 0.5, "alpha": 0.25, "ecut": 10.0})


def ptim_cell128(seed: int = 1001, n: int = 64, L: float = 20.5, N: int = 320, kT: float = 0.02) -> Workload:
    """PT-IM step workload on a 128-site silicon-like cell: L = 20.5 bohr, 64^3, N = 320, kT = 0.02 Ha."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cell = cubic(n, L)
    phi = random_orbitals(rng, cell, N)
    f = fermi_dirac_occupations(N, kT)
    sites = silicon_like_sites(rng, 128, L)
    vloc = gaussian_wells(cell, sites)
    return Workload(f"ptim_{n}^3_N{N}_128site", cell, phi, f, np.diag(f).astype(np.complex128), vloc, 128,
                    {"type": 1, "mu": SCREENED_MU}, {"dt": 0.5, "alpha": 0.25, "ecut": 10.0})


def small_cell(seed: int, n: int, L: float, N: int, kT: float = 0.01, natoms: int = 8,
               ecut: float = 10.0) -> Workload:
    """A reduced cell for tests (any 2·3·5-smooth n, any N below the sphere size)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cell = cubic(n, L)
    phi = random_orbitals(rng, cell, N, ecut)
    f = fermi_dirac_occupations(N, kT)
    sites = silicon_like_sites(rng, natoms, L)
    vloc = gaussian_wells(cell, sites)
    return Workload(f"cell_{n}^3_N{N}", cell, phi, f, np.diag(f).astype(np.complex128), vloc, natoms,
                    {"type": 1, "mu": SCREENED_MU}, {"dt": 0.5, "alpha": 0.25, "ecut": ecut})


def batched_instances(seed: int = 1003, count: int = 64, nmin: int = 16, nmax: int = 256):
    """Specs of the batched form: N ~ U{16..256}, n drawn from BATCH_GRID_SIZES, L = 0.32 n bohr."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for k in range(count):
        n = int(rng.choice(BATCH_GRID_SIZES))
        N = int(rng.integers(nmin, nmax + 1))
        specs.append({"n": n, "L": 0.32 * n, "N": N, "seed": int(rng.integers(1 << 31))})
    return specs


def serving_stream(seed: int = 1005, count: int = 2000, rate: float = 200.0, nmin: int = 32, nmax: int = 320):
    """Poisson arrivals (exponential gaps at `rate` per second) of PT-IM step requests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(rng.choice(SERVE_GRID_SIZES))
        N = int(rng.integers(nmin, nmax + 1))
        reqs.append({"t": t, "n": n, "L": 0.32 * n, "N": N, "seed": int(rng.integers(1 << 31))})
    return reqs
