"""Planted mistakes in the FP64 oracle are caught by its pins.

Each case edits the source of one oracle function on the CPU (for the duration of the test only:
the edited copy is compiled and patched into the oracle module, the file is never touched) with one
plausible mistake (a dropped term or factor, a wrong sign, index or constant, a transposed or
unconjugated operand) and runs the pins that should notice it.  The case passes when at least one
of those pins fails.  Mistakes that leave the converged answer unchanged (the Anderson history,
the Loewdin compensation of sigma at a fixed point where S = I) are not mistakes of the result and
are not planted.
"""
import __future__
import functools
import inspect
import textwrap

import numpy as np
import pytest

import test_oracle_field_pins as F
import test_oracle_hxc_pins as H
import test_oracle_pins as P
from oracle import ptim_oracle as O


def plant(monkeypatch, name, old, new, count=1):
    """Replace `old` by `new` in the source of O.<name> and patch the edited function in."""
    src = textwrap.dedent(inspect.getsource(getattr(O, name)))
    assert src.count(old) == count, f"{name}: {old!r} occurs {src.count(old)} times, expected {count}"
    ns = dict(vars(O))
    code = compile(src.replace(old, new), O.__file__, "exec",
                   flags=__future__.annotations.compiler_flag, dont_inherit=True)
    exec(code, ns)
    monkeypatch.setattr(O, name, ns[name])


def caught(pin):
    """True when the pin fails: an assertion, or a factorisation the mistake makes impossible
    (any other exception means the planted edit itself is broken and is raised)."""
    try:
        pin()
    except (AssertionError, np.linalg.LinAlgError):
        return True
    return False


conv = functools.partial(P.test_pair_potential_matches_direct_convolution, shape=(6, 8, 10))
pw = P.test_exchange_of_plane_waves_closed_form
triple = functools.partial(P.test_diagonalised_exchange_equals_triple_sum, 4)

# (id, oracle function, text, replacement, occurrences, pins)
CASES = [
    # pair potential and kernel
    ("pair density conjugates the target", "pair_potential", "np.conj(phi_i) * phi_j", "phi_i * np.conj(phi_j)", 1,
     [functools.partial(conv, 1)]),
    ("pair potential without the kernel", "pair_potential", "K * np.fft.fftn(rho)", "np.fft.fftn(rho)", 1,
     [functools.partial(conv, 0)]),
    ("screening exponent G^2/(2 mu^2)", "exchange_kernel", "(4 * mu * mu)", "(2 * mu * mu)", 1,
     [functools.partial(pw, 1)]),
    ("screened kernel loses its G = 0 term", "exchange_kernel", "np.pi / (mu * mu) if g0", "0.0 if g0", 1,
     [functools.partial(pw, 1), P.test_kernel_small_g_limit_and_coulomb_zero]),
    ("Coulomb kernel without 4 pi", "exchange_kernel", "K[nz] = 4 * np.pi / g2[nz]\n", "K[nz] = 1.0 / g2[nz]\n", 1,
     [functools.partial(pw, 0)]),
    ("|G|^2 takes Lz for the x axis", "g_squared", "_wrapped(g.nx) / g.Lx", "_wrapped(g.nx) / g.Lz", 1,
     [functools.partial(conv, 1), functools.partial(pw, 1)]),
    # exchange sums
    ("exchange without its minus sign", "apply_exchange", "out[j] = -acc", "out[j] = acc", 1,
     [P.test_exchange_is_hermitian_negative_semidefinite]),
    ("exchange weighted by the target's occupation", "apply_exchange", "occ[i] * src[i]", "occ[j] * src[i]", 1,
     [functools.partial(pw, 1)]),
    ("exchange multiplies the pair potential by the target", "apply_exchange", "occ[i] * src[i] *",
     "occ[i] * tgt[j] *", 1, [functools.partial(pw, 1)]),
    ("mixed-state exchange with sigma transposed", "apply_exchange_mixed", "acc += sigma[i, k] * phi[i] * v",
     "acc += sigma[k, i] * phi[i] * v", 1, [triple, P.test_mixed_exchange_of_plane_waves_closed_form]),
    ("eigenvectors of sigma conjugated", "diagonalize_occupations", "return Q, d", "return Q.conj(), d", 1,
     [triple]),
    ("rotation by Q instead of Q^T", "rotate", "(Q.T @ P)", "(Q @ P)", 1,
     [triple, P.test_ace_reproduces_exchange_on_its_orbitals]),
    ("inner product without the conjugate", "overlap", "A.conj() @ B.T", "A @ B.T", 1,
     [P.test_exchange_is_hermitian_negative_semidefinite, P.test_ace_reproduces_exchange_on_its_orbitals]),
    ("inner product without the volume element", "overlap", "dV * (A.conj() @ B.T)", "(A.conj() @ B.T)", 1,
     [P.test_ptim_quadratic_invariants, P.test_ptim_free_electron_cayley_closed_form]),
    ("exchange energy without the 1/2", "exchange_energy", "spin * 0.5 * alpha", "spin * alpha", 1,
     [functools.partial(pw, 1)]),
    ("pair energy counts off-diagonal pairs once", "exchange_energy_pairs", "1.0 if i == j else 2.0", "1.0", 1,
     [functools.partial(P.test_exchange_energy_by_pairs_plane_waves_closed_form, 1)]),
    ("pair energy weights one occupation twice", "exchange_energy_pairs", "d[i] * d[j]", "d[i] * d[i]", 1,
     [P.test_exchange_energy_by_pairs_matches_the_exchange_route]),
    ("pair energy without the 1/Ng of Parseval", "exchange_energy_pairs", "-dV / ng * s", "-dV * s", 1,
     [functools.partial(P.test_exchange_energy_by_pairs_plane_waves_closed_form, 0)]),
    # ACE
    ("ACE factor without the conjugate of L^-1", "build_ace", "(Linv.conj() @ Wm)", "(Linv @ Wm)", 1,
     [P.test_ace_reproduces_exchange_on_its_orbitals]),
    ("ACE Cholesky of the transposed M", "build_ace", "np.linalg.cholesky(-M)", "np.linalg.cholesky(-M.T)", 1,
     [P.test_ace_reproduces_exchange_on_its_orbitals]),
    ("ACE applied with a plus sign", "apply_ace", "return -rotate(xi, C)", "return rotate(xi, C)", 1,
     [P.test_ace_reproduces_exchange_on_its_orbitals]),
    # Hamiltonian
    ("kinetic energy |G|^2 without the 1/2", "kinetic_factor", "return 0.5 * g_squared(g)",
     "return g_squared(g)", 1, [P.test_ptim_free_electron_cayley_closed_form, P.test_ptim_eigenstates_are_stationary]),
    ("velocity gauge with |G - A|^2", "kinetic_factor", "(G[a] + A[a]) ** 2", "(G[a] - A[a]) ** 2", 1,
     [F.test_plane_waves_are_eigenfunctions_with_field]),
    ("local potential with the wrong sign", "apply_kinetic_local", "kin + vloc[None] * phi",
     "kin - vloc[None] * phi", 1, [P.test_ptim_eigenstates_are_stationary]),
    ("plane-wave sphere |G|^2 <= Ecut", "sphere_mask", "(0.5 * g_squared(g) <= ecut)", "(g_squared(g) <= ecut)", 1,
     [P.test_ptim_eigenstates_are_stationary]),
    ("exchange term of H with the wrong sign", "apply_H", "+ alpha * vx_phi", "- alpha * vx_phi", 1,
     [P.test_ptim_energy_drift_is_second_order]),
    # PT-IM step
    ("sigma commutator reversed", "ptim_step", "A @ sig_h - sig_h @ A", "sig_h @ A - A @ sig_h", 1,
     [P.test_ptim_free_electron_cayley_closed_form]),
    ("orbital update without the projector I - Pt", "ptim_step", "(Hphi - rotate(phi_h, SinvA))", "(Hphi)", 1,
     [P.test_ptim_free_electron_cayley_closed_form]),
    ("orbital midpoint taken at the new time", "ptim_step", "0.5 * (phi + phi_n)", "phi", 2,
     [P.test_ptim_quadratic_invariants, P.test_ptim_matches_rk4_and_is_second_order]),
    ("orbital update with +i dt", "ptim_step", "T_phi = phi_n - 1j * p.dt", "T_phi = phi_n + 1j * p.dt", 1,
     [P.test_ptim_matches_rk4_and_is_second_order]),
    ("ACE built from W not rotated back by Q^*", "ptim_step",
     "W = rotate(apply_exchange(phit, d, phit, K), Q.conj().T)", "W = apply_exchange(phit, d, phit, K)", 1,
     [P.test_ptim_ace_and_exact_share_the_fixed_point]),
    ("V_Hxc of the density without the spin factor", "ptim_step", "hxc_potential(p.spin * density(",
     "hxc_potential(density(", 1, [H.test_ptim_hxc_matches_rk4_and_is_second_order]),
    # V_Hxc and observables
    ("Hartree without 4 pi", "hartree_potential", "4 * np.pi * rg[nz] / g2[nz]", "rg[nz] / g2[nz]", 1,
     [H.test_hartree_of_cosine_densities_closed_form]),
    ("Hartree over |G| instead of |G|^2", "hartree_potential", "/ g2[nz]", "/ np.sqrt(g2[nz])", 1,
     [H.test_hartree_of_cosine_densities_closed_form]),
    ("Slater exchange constant (r/pi)^(1/3)", "lda_xc", "np.cbrt(3.0 * r / np.pi)", "np.cbrt(r / np.pi)", 1,
     [H.test_slater_exchange_of_the_uniform_gas]),
    ("exchange potential equal to the energy density", "lda_xc", "vx = 4.0 / 3.0 * ex", "vx = ex", 1,
     [functools.partial(H.test_vxc_is_the_derivative_of_rho_eps, 2.5)]),
    ("PZ high-density-branch potential coefficient 6/7", "lda_xc", "7.0 / 6.0 * PZ_BETA1", "6.0 / 7.0 * PZ_BETA1", 1,
     [functools.partial(H.test_vxc_is_the_derivative_of_rho_eps, 2.5)]),
    ("PZ low-density-branch potential sign", "lda_xc", "(2.0 * PZ_D - PZ_C) / 3.0", "(2.0 * PZ_D + PZ_C) / 3.0", 1,
     [functools.partial(H.test_vxc_is_the_derivative_of_rho_eps, 0.4)]),
    ("density with sigma transposed", "density", "P, sigma, P.conj()", "P, sigma.T, P.conj()", 1,
     [H.test_density_integrates_to_trace_and_matches_diagonal_form]),
    ("current with -A", "current", "(G[a] + A[a])[None]", "(G[a] - A[a])[None]", 1,
     [F.test_current_of_plane_waves]),
    ("current without the spin factor", "current", "spin / g.volume", "1.0 / g.volume", 1,
     [F.test_current_of_plane_waves]),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(monkeypatch, case):
    _, name, old, new, count, pins = case
    plant(monkeypatch, name, old, new, count)
    assert any(caught(pin) for pin in pins), f"no pin caught: {case[0]}"


@pytest.mark.parametrize("const,value", [("PZ_D", 0.0116), ("PZ_BETA1", 1.529), ("PZ_A", 0.0131)])
def test_planted_constant_typo_is_caught(monkeypatch, const, value):
    """A mistyped Perdew-Zunger constant breaks the join of the two branches at rs = 1 or the
    Gell-Mann-Brueckner high-density coefficient."""
    monkeypatch.setattr(O, const, value)
    assert caught(H.test_pz_high_density_limit_and_branch_continuity)


def test_unplanted_oracle_passes_the_same_pins():
    """Control: the pins used above pass on the oracle as it stands (a pin that always failed
    would catch every mistake)."""
    pins = {id(p): p for c in CASES for p in c[5]}
    pins[id(H.test_pz_high_density_limit_and_branch_continuity)] = H.test_pz_high_density_limit_and_branch_continuity
    for pin in pins.values():
        pin()
