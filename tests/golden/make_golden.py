"""Write the stored expected values under tests/golden/ from the FP64 oracle.

Only `oracle/` computes here; `paper_2501_03061_gb300.synth` supplies the seeded
inputs (it holds none of the method's arithmetic).  The paper prints no worked
example small enough to store (its results are timings and spectra of 384- to
3072-atom silicon cells), so these fixtures freeze the oracle's answers on small
seeded cells, each value computed by a stated route.  tests/test_golden.py
recomputes them, where possible through a different route of the oracle (the
diagonalised exchange of Sec. IV-A1 against the triple sum of the mixed-state
exchange written here), so that a later change of the oracle's arithmetic shows
up as a failing fixture.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import ptim_oracle as O  # noqa: E402
from paper_2501_03061_gb300 import synth  # noqa: E402

# grid points (z, y, x) at which fields are sampled
SAMPLE_POINTS = [(0, 0, 0), (1, 2, 3), (5, 0, 11), (6, 6, 6), (11, 7, 2), (3, 10, 8), (9, 4, 1), (7, 11, 10)]


def mixed_sigma(occ):
    """A Hermitian positive definite occupation matrix with off-diagonal coherences:
    diag(occ) plus a few small Hermitian couplings (smallest eigenvalue 0.046 for the exchange
    input, 0.26 for the step's)."""
    s = np.diag(occ).astype(np.complex128)
    s[0, 1] = s[1, 0] = 0.03
    s[2, 4] = 0.02j
    s[4, 2] = -0.02j
    s[1, 5] = 0.01 - 0.01j
    s[5, 1] = 0.01 + 0.01j
    return s


def exchange_case():
    w = synth.small_cell(7, 12, 8.0, 6, kT=0.02, ecut=8.0)
    return w, mixed_sigma(w.occ)


def ptim_case():
    w = synth.small_cell(23, 12, 8.0, 6, kT=0.05, ecut=6.0)
    return w, mixed_sigma(w.occ)


class Writer:
    def __init__(self, path, header):
        self.f = open(path, "w")
        for line in header.strip().splitlines():
            self.f.write("# " + line.strip() + "\n")

    def scalar(self, name, v):
        self.f.write(f"@ {name} 1 1 real\n{float(v)!r}\n")

    def array(self, name, a):
        a = np.atleast_2d(np.asarray(a))
        cplx = np.iscomplexobj(a)
        self.f.write(f"@ {name} {a.shape[0]} {a.shape[1]} {'complex' if cplx else 'real'}\n")
        for row in a:
            if cplx:
                self.f.write(" ".join(f"{float(z.real)!r} {float(z.imag)!r}" for z in row) + "\n")
            else:
                self.f.write(" ".join(f"{float(x)!r}" for x in row) + "\n")

    def close(self):
        self.f.close()


def samples(field):
    """field (..., nz, ny, nx) sampled at SAMPLE_POINTS -> (..., len(SAMPLE_POINTS))."""
    return np.stack([field[(Ellipsis,) + p] for p in SAMPLE_POINTS], axis=-1)


def write_exchange(path):
    w, sig = exchange_case()
    g = O.grid_of(w.cell)
    hdr = f"""
    Mixed-state Fock exchange (Sec. II-B, the mixed-state V_x equation) on a seeded 12^3 cell.
    Input: synth.small_cell(seed 7, n 12, L 8.0 bohr, N 6, kT 0.02 Ha, ecut 8.0 Ha) with the occupation
    matrix diag(f) + Hermitian couplings (tests/golden/make_golden.py: mixed_sigma).
    Route: the triple sum over (i, k) of sigma_ik phi_i IFFT[K FFT[conj(phi_k) phi_j]], FP64.
    vx_matrix_<k>[i, j] = <phi_i|V_x[P] phi_j>; ex_<k> = spin (alpha/2) Tr[P V_x[P]] with spin 2,
    alpha 0.25; vx_samples_<k>[j, s] = (V_x[P] phi_j)(r_s) at the grid points {SAMPLE_POINTS}.
    Kernels: screened = 4 pi/G^2 (1 - exp(-G^2/(4 mu^2))), mu = {synth.SCREENED_MU}; coulomb = 4 pi/G^2
    (both with the G = 0 limit of the oracle's kernel).
    """
    out = Writer(path, hdr)
    for name, ktype in (("screened", 1), ("coulomb", 0)):
        K = O.exchange_kernel(g, ktype, synth.SCREENED_MU)
        vx = O.apply_exchange_mixed(w.phi, sig, w.phi, K)
        M = O.overlap(w.phi, vx, g.dV)
        ex = 2.0 * 0.5 * 0.25 * float(np.real(np.sum(sig * M.T)))
        out.array(f"vx_matrix_{name}", M)
        out.scalar(f"ex_{name}", ex)
        out.array(f"vx_samples_{name}", samples(vx))
    out.close()


def write_ace(path):
    w, sig = exchange_case()
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    vx = O.apply_exchange_mixed(w.phi, sig, w.phi, K)
    M = O.overlap(w.phi, vx, g.dV)
    M = 0.5 * (M + M.conj().T)
    L = np.linalg.cholesky(-M)
    xi = O.build_ace(w.phi, vx, g.dV)
    hdr = """
    Adaptively compressed exchange (Sec. IV-A2) built from W = V_x[P] Phi of the exchange fixture's input
    (screened kernel).  M = <Phi|W> (Hermitian part), -M = L L^* (lower Cholesky, positive diagonal),
    xi = W L^{-*}.  cholesky_L is L; xi_gram[k, l] = <xi_k|xi_l>; xi_samples[k, s] = xi_k(r_s) at the
    exchange fixture's sample points.
    """
    out = Writer(path, hdr)
    out.array("cholesky_L", L)
    out.array("xi_gram", O.overlap(xi, xi, g.dV))
    out.array("xi_samples", samples(xi))
    out.close()


def write_hxc(path):
    w, sig = exchange_case()
    g = O.grid_of(w.cell)
    rho = 2.0 * O.density(w.phi, sig).real
    eh, exc = O.hxc_energy(rho, g)
    v = O.hxc_potential(rho, g)
    hdr = """
    Density and Hartree + LDA potential (Sec. III-C item 1; the V_Hxc term of Eq. 1) of the exchange
    fixture's input.  rho = 2 sum_ij phi_i sigma_ij conj(phi_j); Hartree with V_H(G = 0) = 0;
    LDA = Slater exchange + Perdew-Zunger 1981 correlation.  electrons = dV sum rho;
    rho_samples / vhxc_samples at the exchange fixture's sample points.
    """
    out = Writer(path, hdr)
    out.scalar("electrons", g.dV * rho.sum())
    out.scalar("e_hartree", eh)
    out.scalar("e_xc", exc)
    out.array("rho_samples", samples(rho))
    out.array("vhxc_samples", samples(v))
    out.close()


def write_ptim(path):
    w, sig = ptim_case()
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    hdr = """
    One PT-IM-ACE step (Sec. II-A, the midpoint and fixed-point equations; the double loop of Sec. IV-A2)
    on a seeded 12^3 cell: synth.small_cell(seed 23, n 12, L 8.0 bohr, N 6, kT 0.05 Ha, ecut 6.0 Ha) with
    the occupation matrix of mixed_sigma, dt 0.5 au, alpha 0.25, tol 1e-12; without V_Hxc (frozen local
    potential) and with V_Hxc[rho_{n+1/2}] (suffix _hxc).  sigma1 = sigma_{n+1}; proj[i, j] = <phi_n,i|phi_{n+1},j>
    (the step's rotation of the orbital block); energy0 / energy1 = the total energy before and after.
    """
    out = Writer(path, hdr)
    for suffix, hxc in (("", False), ("_hxc", True)):
        p = O.PtimParams(tol=1e-12, ecut=6.0, hxc=hxc)
        phi1, sig1, st = O.ptim_step(w.phi, sig, w.vloc, g, K, p)
        if not st.converged:
            raise RuntimeError("oracle PT-IM step did not converge")
        e0 = O.total_energy(w.phi, sig, w.vloc, g, K, 6.0, hxc=hxc)
        e1 = O.total_energy(phi1, sig1, w.vloc, g, K, 6.0, hxc=hxc)
        out.array("sigma1" + suffix, sig1)
        out.array("proj" + suffix, O.overlap(w.phi, phi1, g.dV))
        out.scalar("energy0" + suffix, e0)
        out.scalar("energy1" + suffix, e1)
    out.close()


FIELD_A = (0.3, -0.2, 0.1)  # bohr^-1, a uniform vector potential


def write_field(path):
    w, sig = ptim_case()
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    A = np.array(FIELD_A)
    hdr = f"""
    Velocity-gauge field (Eq. 1's V_ext(t) as a uniform vector potential A = {FIELD_A} bohr^-1) on the
    step fixture's input: current = (spin/Omega) Re Tr[P (-i grad + A)] with spin 2 (current0 before the
    step, current1 after), and one PT-IM-ACE step with A at the midpoint time (Sec. II-A), dt 0.5 au,
    tol 1e-12: sigma1, proj[i, j] = <phi_n,i|phi_{{n+1}},j>, energy0 / energy1 with A in the kinetic term.
    """
    out = Writer(path, hdr)
    out.array("current0", O.current(w.phi, sig, g, A))
    phi1, sig1, st = O.ptim_step(w.phi, sig, w.vloc, g, K, O.PtimParams(tol=1e-12, ecut=6.0, A=FIELD_A))
    if not st.converged:
        raise RuntimeError("oracle PT-IM step did not converge")
    out.array("current1", O.current(phi1, sig1, g, A))
    out.array("sigma1", sig1)
    out.array("proj", O.overlap(w.phi, phi1, g.dV))
    out.scalar("energy0", O.total_energy(w.phi, sig, w.vloc, g, K, 6.0, A=A))
    out.scalar("energy1", O.total_energy(phi1, sig1, w.vloc, g, K, 6.0, A=A))
    out.close()


def main():
    write_field(os.path.join(HERE, "field_12cubed_N6.txt"))
    write_exchange(os.path.join(HERE, "exchange_12cubed_N6.txt"))
    write_ace(os.path.join(HERE, "ace_12cubed_N6.txt"))
    write_hxc(os.path.join(HERE, "hxc_12cubed_N6.txt"))
    write_ptim(os.path.join(HERE, "ptim_step_12cubed_N6.txt"))


if __name__ == "__main__":
    main()
