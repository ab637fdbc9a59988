"""The stored fixtures under tests/golden/ (written by tests/golden/make_golden.py from the FP64
oracle) against the oracle recomputed through a different route where it has one:

* exchange: the fixtures hold the triple sum of the mixed-state exchange (Sec. II-B); here the
  diagonalised form (Sec. IV-A1: sigma = Q D Q^*, rotated orbitals, one double loop) recomputes it;
* ACE: the fixtures hold the Cholesky factor of -<Phi|W>; here it is read back from the
  compressed operator itself (<xi|Phi> = -L^*) with W from the diagonalised exchange;
* density: rho = 2 sum_i d_i |phit_i|^2 from the eigenpairs of sigma instead of the double sum;
* PT-IM step: the fixtures hold the PT-IM-ACE fixed point; here the step runs with the exchange
  applied exactly in every inner iteration (same fixed point, different iteration);
* field: the stored current against the field derivative of the total energy, and the stored step
  with a vector potential against the exact-exchange iteration.

A failing fixture means the oracle's arithmetic changed; the generating script is rerun only with
a commit that names the passage of the paper justifying the change.
"""
import os

import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SAMPLE_POINTS = [(0, 0, 0), (1, 2, 3), (5, 0, 11), (6, 6, 6), (11, 7, 2), (3, 10, 8), (9, 4, 1), (7, 11, 10)]


def load(name):
    """Parse a fixture: '# ' header lines, then blocks '@ name rows cols real|complex' + rows."""
    out, header = {}, []
    with open(os.path.join(GOLDEN, name)) as f:
        lines = f.read().splitlines()
    k = 0
    while k < len(lines):
        line = lines[k]
        if line.startswith("#"):
            header.append(line)
            k += 1
            continue
        tag, key, rows, cols, kind = line.split()
        assert tag == "@"
        rows, cols = int(rows), int(cols)
        vals = np.array([[float(x) for x in lines[k + 1 + r].split()] for r in range(rows)])
        if kind == "complex":
            vals = vals[:, 0::2] + 1j * vals[:, 1::2]
        assert vals.shape == (rows, cols)
        out[key] = vals[0, 0] if (rows, cols) == (1, 1) and kind == "real" else vals
        k += 1 + rows
    return out, header


def samples(field):
    return np.stack([field[(Ellipsis,) + p] for p in SAMPLE_POINTS], axis=-1)


def mixed_sigma(occ):
    s = np.diag(occ).astype(np.complex128)
    s[0, 1] = s[1, 0] = 0.03
    s[2, 4] = 0.02j
    s[4, 2] = -0.02j
    s[1, 5] = 0.01 - 0.01j
    s[5, 1] = 0.01 + 0.01j
    return s


def close(got, want, rtol):
    got, want = np.atleast_2d(got), np.atleast_2d(want)
    assert got.shape == want.shape
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= rtol, f"relative error {err:.3e} > {rtol:.0e}"


@pytest.fixture(scope="module")
def exchange_input():
    w = synth.small_cell(7, 12, 8.0, 6, kT=0.02, ecut=8.0)
    return w, mixed_sigma(w.occ), O.grid_of(w.cell)


def test_every_fixture_is_cited():
    names = sorted(n for n in os.listdir(GOLDEN) if n.endswith(".txt"))
    assert names == ["ace_12cubed_N6.txt", "exchange_12cubed_N6.txt", "field_12cubed_N6.txt", "hxc_12cubed_N6.txt",
                     "ptim_step_12cubed_N6.txt"]
    for n in names:
        data, header = load(n)
        assert data and any("Sec." in h for h in header), n


@pytest.mark.parametrize("name,ktype", [("screened", 1), ("coulomb", 0)])
def test_exchange_fixture_by_diagonalised_form(exchange_input, name, ktype):
    w, sig, g = exchange_input
    ref, _ = load("exchange_12cubed_N6.txt")
    K = O.exchange_kernel(g, ktype, synth.SCREENED_MU)
    vx = O.apply_exchange_sigma(w.phi, sig, w.phi, K)
    close(O.overlap(w.phi, vx, g.dV), ref[f"vx_matrix_{name}"], 1e-12)
    close(samples(vx), ref[f"vx_samples_{name}"], 1e-12)
    assert O.exchange_energy(w.phi, sig, K, g.dV) == pytest.approx(ref[f"ex_{name}"], rel=1e-12)
    # the stored matrix is Hermitian negative definite (V_x of a positive definite sigma)
    M = ref[f"vx_matrix_{name}"]
    assert np.abs(M - M.conj().T).max() <= 1e-14 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.conj().T)).max() < 0


def test_ace_fixture_from_the_compressed_operator(exchange_input):
    w, sig, g = exchange_input
    ref, _ = load("ace_12cubed_N6.txt")
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    W = O.apply_exchange_sigma(w.phi, sig, w.phi, K)
    xi = O.build_ace(w.phi, W, g.dV)
    L = -O.overlap(xi, w.phi, g.dV).conj().T  # <xi|Phi> = L^{-1} <W|Phi> = L^{-1} M = -L^*
    assert np.abs(np.triu(L, 1)).max() <= 1e-12 * np.abs(L).max()
    close(L, ref["cholesky_L"], 1e-11)
    close(O.overlap(xi, xi, g.dV), ref["xi_gram"], 1e-11)
    close(samples(xi), ref["xi_samples"], 1e-11)
    # the stored factor has a real positive diagonal
    d = np.diag(ref["cholesky_L"])
    assert np.all(d.real > 0) and np.abs(d.imag).max() == 0


def test_hxc_fixture_from_the_diagonal_density(exchange_input):
    w, sig, g = exchange_input
    ref, _ = load("hxc_12cubed_N6.txt")
    Q, d = O.diagonalize_occupations(sig)
    phit = O.rotate(w.phi, Q)
    rho = 2.0 * np.einsum("i,irst->rst", d, np.abs(phit) ** 2)
    assert g.dV * rho.sum() == pytest.approx(ref["electrons"], rel=1e-13)
    assert ref["electrons"] == pytest.approx(2.0 * np.trace(sig).real, rel=1e-13)
    eh, exc = O.hxc_energy(rho, g)
    assert eh == pytest.approx(ref["e_hartree"], rel=1e-12)
    assert exc == pytest.approx(ref["e_xc"], rel=1e-12)
    close(samples(rho), ref["rho_samples"], 1e-12)
    close(samples(O.hxc_potential(rho, g)), ref["vhxc_samples"], 1e-12)


@pytest.mark.parametrize("suffix,hxc", [("", False), ("_hxc", True)])
def test_ptim_fixture_by_exact_exchange_iteration(suffix, hxc):
    w = synth.small_cell(23, 12, 8.0, 6, kT=0.05, ecut=6.0)
    sig = mixed_sigma(w.occ)
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    ref, _ = load("ptim_step_12cubed_N6.txt")
    phi1, sig1, st = O.ptim_step(w.phi, sig, w.vloc, g, K, O.PtimParams(tol=1e-12, ecut=6.0, hxc=hxc, use_ace=False))
    assert st.converged
    close(sig1, ref["sigma1" + suffix], 1e-9)
    close(O.overlap(w.phi, phi1, g.dV), ref["proj" + suffix], 1e-9)
    assert O.total_energy(w.phi, sig, w.vloc, g, K, 6.0, hxc=hxc) == pytest.approx(ref["energy0" + suffix], rel=1e-12)
    assert O.total_energy(phi1, sig1, w.vloc, g, K, 6.0, hxc=hxc) == pytest.approx(ref["energy1" + suffix], rel=1e-9)
    # stored invariants of the implicit midpoint step: sigma stays Hermitian with its trace; both
    # orbital blocks are orthonormal, so the overlap between them has singular values <= 1
    s1 = ref["sigma1" + suffix]
    assert np.abs(s1 - s1.conj().T).max() <= 1e-12
    assert np.trace(s1).real == pytest.approx(np.trace(sig).real, rel=1e-11)
    sv = np.linalg.svd(ref["proj" + suffix], compute_uv=False)
    assert sv.max() <= 1 + 1e-12 and sv.min() > 0.5


def test_field_fixture_by_energy_derivative_and_exact_exchange_iteration():
    """The stored current against Omega J_a = dE/dA_a by central differences of the total energy, and
    the stored field step against the step with the exchange applied exactly in every iteration."""
    w = synth.small_cell(23, 12, 8.0, 6, kT=0.05, ecut=6.0)
    sig = mixed_sigma(w.occ)
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    A = np.array([0.3, -0.2, 0.1])
    ref, header = load("field_12cubed_N6.txt")
    assert any("0.3, -0.2, 0.1" in h for h in header)
    h = 1e-4
    dE = []
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        dE.append((O.total_energy(w.phi, sig, w.vloc, g, K, 6.0, A=A + e)
                   - O.total_energy(w.phi, sig, w.vloc, g, K, 6.0, A=A - e)) / (2 * h) / g.volume)
    close(np.array(dE), ref["current0"], 1e-6)
    phi1, sig1, st = O.ptim_step(w.phi, sig, w.vloc, g, K,
                                 O.PtimParams(tol=1e-12, ecut=6.0, A=tuple(A), use_ace=False))
    assert st.converged
    close(sig1, ref["sigma1"], 1e-9)
    close(O.overlap(w.phi, phi1, g.dV), ref["proj"], 1e-9)
    close(O.current(phi1, sig1, g, A), ref["current1"], 1e-8)
    assert O.total_energy(w.phi, sig, w.vloc, g, K, 6.0, A=A) == pytest.approx(ref["energy0"], rel=1e-12)
    assert O.total_energy(phi1, sig1, w.vloc, g, K, 6.0, A=A) == pytest.approx(ref["energy1"], rel=1e-9)
