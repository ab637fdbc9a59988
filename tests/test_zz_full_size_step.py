"""One PT-IM step at the benchmark's full size (64^3 grid, N = 320, FP32 form with tensor-core
contractions, tol 1e-6), checked where the oracle cannot run the whole step: through properties
that hold at any size and through the step's own fixed-point equation evaluated by the oracle for
sampled orbitals.

Fixed-point check (Sec. II-A, the midpoint and fixed-point equations): with Phi_h, sigma_h the
midpoints of the step's input and output, the converged output must satisfy, orbital by orbital,
    Phi_{n+1, j} = Phi_{n, j} - i dt [ (H Phi_h)_j - Phi_h S^{-1} <Phi_h|(H Phi_h)_j> ],
where H = P_sph[-Lap/2 + V_loc + alpha V_x[Phi_h sigma_h Phi_h^*]] and S = <Phi_h|Phi_h>.  Only
column j of H Phi_h is needed (N pair FFTs of the exchange for one target), and the Gram S and the
sigma_h eigenbasis are single contractions, so the check costs seconds on the host at full size.
The same check is first run on an oracle step (CPU, small cell), where it must hold to the step's
tolerance and must fail for a step taken with another time step.
"""
import numpy as np
import pytest

from oracle import ptim_oracle as O
from paper_2501_03061_gb300 import synth


def fixed_point_defect(phi_n, sig_n, phi1, sig1, vloc, g, K, dt, ecut, alpha, js):
    """max over sampled j of ||Phi_{n+1,j} - T_Phi(x)_j|| / ||Phi_{n+1,j}|| (FP64, oracle routines)."""
    phi_h = 0.5 * (phi_n + phi1)
    sig_h = 0.5 * (sig_n + sig1)
    S = O.overlap(phi_h, phi_h, g.dV)
    Q, d = O.diagonalize_occupations(sig_h)
    phit = O.rotate(phi_h, Q)
    worst = 0.0
    for j in js:
        tgt = phi_h[j:j + 1]
        vx = O.apply_exchange(phit, d, tgt, K)
        hphi = O.apply_H(tgt, vloc, g, ecut, alpha, vx)
        a = O.overlap(phi_h, hphi, g.dV)[:, 0]
        r = hphi[0] - O.rotate(phi_h, np.linalg.solve(S, a)[:, None])[0]
        t = phi_n[j] - 1j * dt * r
        worst = max(worst, float(np.linalg.norm(phi1[j] - t) / np.linalg.norm(phi1[j])))
    return worst


def test_fixed_point_check_on_an_oracle_step():
    """The check itself, on a step the oracle takes (12^3, N = 6, a complex sigma): it holds to the
    step's tolerance, and a step taken with half the time step fails it by orders of magnitude."""
    w = synth.small_cell(23, 12, 8.0, 6, kT=0.05, ecut=6.0)
    sig = np.diag(w.occ).astype(np.complex128)
    sig[0, 1] = sig[1, 0] = 0.03
    sig[2, 4] = 0.02j
    sig[4, 2] = -0.02j
    g = O.grid_of(w.cell)
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    phi1, sig1, st = O.ptim_step(w.phi, sig, w.vloc, g, K, O.PtimParams(tol=1e-12, ecut=6.0))
    assert st.converged
    ok = fixed_point_defect(w.phi, sig, phi1, sig1, w.vloc, g, K, 0.5, 6.0, 0.25, range(6))
    assert ok <= 1e-9, ok
    phi2, sig2, _ = O.ptim_step(w.phi, sig, w.vloc, g, K, O.PtimParams(tol=1e-12, ecut=6.0, dt=0.25))
    bad = fixed_point_defect(w.phi, sig, phi2, sig2, w.vloc, g, K, 0.5, 6.0, 0.25, range(6))
    assert bad > 1e3 * max(ok, 1e-12), (ok, bad)


@pytest.mark.gpu
def test_full_size_fp32_step_satisfies_its_fixed_point_and_invariants():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03061_gb300 import api
    w = synth.ptim_cell128()  # 64^3, N = 320, 128 sites, kT = 0.02 Ha
    g = O.grid_of(w.cell)
    N = w.phi.shape[0]
    phi_n = w.phi.astype(np.complex64)
    sig_n = w.sigma.copy()
    ctx = api.Context(0)
    try:
        ctx.set_option("tc_gram", 1)
        phi = torch.from_numpy(phi_n).cuda()
        sigma = torch.from_numpy(sig_n).cuda()
        st = ctx.ptim_step(phi, sigma, torch.from_numpy(w.vloc).cuda(), cell=w.cell, kernel=w.kernel,
                           precision="fp32", dt=0.5, alpha=0.25, ecut=10.0, tol=1e-6, max_outer=20,
                           max_inner=100, anderson_depth=20)
        phi1 = phi.cpu().numpy().astype(np.complex128)
        sig1 = sigma.cpu().numpy()
    finally:
        ctx.close()
    assert st["converged"]
    del phi, sigma
    # invariants of the implicit midpoint step (quadratic invariants, exact at the fixed point):
    # sigma Hermitian with its trace and tr sigma^2; an orthonormal orbital block.  Bounds: the
    # step stops at a relative residual of tol = 1e-6 on x = (Phi, sigma), which bounds the drift
    # of the traces to a few tol; the orbitals are stored in FP32 (unit roundoff 6e-8), whose
    # rounding after the final orthonormalisation leaves max |Phi^*Phi - I| near 1e-6.
    tr_drift = abs(np.trace(sig1) - np.trace(sig_n)) / abs(np.trace(sig_n))
    tr2_drift = abs(np.trace(sig1 @ sig1) - np.trace(sig_n @ sig_n)) / abs(np.trace(sig_n @ sig_n))
    G = O.overlap(phi1, phi1, g.dV)
    orth = float(np.abs(G - np.eye(N)).max())
    # the orbital equation of the fixed point for sampled orbitals, through the oracle
    K = O.exchange_kernel(g, 1, synth.SCREENED_MU)
    defect = fixed_point_defect(phi_n.astype(np.complex128), sig_n, phi1, sig1, w.vloc, g, K, 0.5, 10.0, 0.25,
                                (0, 177, 319))
    print(f"full-size FP32 step: outer {st['outer']} inner {st['inner']} residual {st['residual']:.3e}; "
          f"tr sigma drift {tr_drift:.3e}, tr sigma^2 drift {tr2_drift:.3e}, max|Phi*Phi - I| {orth:.3e}, "
          f"fixed-point defect {defect:.3e}")
    assert np.abs(sig1 - sig1.conj().T).max() <= 1e-12
    assert tr_drift <= 1e-5, tr_drift
    assert tr2_drift <= 1e-5, tr2_drift
    assert orth <= 1e-5, orth
    # the step moved the state (a no-op would pass the invariants)
    assert np.abs(sig1 - sig_n).max() > 1e-4
    # the defect of the fixed-point equation: the inner residual (tol), the ACE operator's distance
    # from the exact V_x at the final midpoint (the anchor moved less than tol) and the final
    # orthonormalisation (~1e-6) each enter at the 1e-6 level, FP32 rounding of the orbitals at 1e-7
    assert defect <= 1e-5, defect
