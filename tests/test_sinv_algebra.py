"""The algebra behind the step's routes to S^{-1} A (no GPU): the Neumann series and the product form
in E = S - I meet their stated error bounds, and an FP32 factor of S refined twice with FP64
residuals reaches FP64 accuracy for the overlaps the step meets (kappa(S) ~ 7: eigenvalues of the
midpoint overlap between 1/(1 + (e dt/2)^2) and 1).  These are the bounds the library uses to pick
a route (a series when its bound reaches 1e-17; the refinement's last correction checked against
1e-10)."""
import numpy as np
import pytest


def hermitian_with_spectrum(rng, N, lo, hi):
    q, _ = np.linalg.qr(rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    lam = np.linspace(lo, hi, N)
    return (q * lam) @ q.conj().T


@pytest.mark.parametrize("e_target", [1e-3, 3e-2, 0.2])
def test_series_forms_meet_their_bounds(e_target):
    rng = np.random.default_rng(11)
    N = 40
    E = hermitian_with_spectrum(rng, N, -1.0, 1.0)
    E *= e_target / np.linalg.norm(E)  # ||E||_F = e
    S = np.eye(N) + E
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    exact = np.linalg.solve(S, A)
    e = np.linalg.norm(E)
    for K in range(1, 12):  # Horner: Y <- A - E Y, K times
        Y = A.copy()
        for _ in range(K):
            Y = A - E @ Y
        bound = e ** (K + 1) / (1 - e)
        assert np.linalg.norm(Y - exact) <= (bound + 1e-14) * np.linalg.norm(A) / (1 - e)
    for J in range(0, 5):  # product: (I - E)(I + E^2)...(I + E^{2^J}) A
        Y = A - E @ A
        P = E.copy()
        for _ in range(J):
            P = P @ P
            Y = Y + P @ Y
        bound = e ** (2 ** (J + 1)) / (1 - e)
        assert np.linalg.norm(Y - exact) <= (bound + 1e-14) * np.linalg.norm(A) / (1 - e)


def test_fp32_factor_refined_twice_reaches_fp64():
    rng = np.random.default_rng(12)
    N = 96
    S = hermitian_with_spectrum(rng, N, 1.0 / (1.0 + 2.5 ** 2), 1.0)  # kappa ~ 7
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    exact = np.linalg.solve(S, A)
    L32 = np.linalg.cholesky(S.astype(np.complex64))
    Li32 = np.linalg.inv(L32).astype(np.complex64)
    Si32 = (Li32.conj().T @ Li32).astype(np.complex64)  # S32^{-1}
    X = (Si32 @ A.astype(np.complex64)).astype(np.complex128)
    errs = [np.linalg.norm(X - exact) / np.linalg.norm(exact)]
    for _ in range(2):
        R = A - S @ X  # FP64 residual
        C = (Si32 @ R.astype(np.complex64)).astype(np.complex128)
        X = X + C
        errs.append(np.linalg.norm(X - exact) / np.linalg.norm(exact))
    assert errs[0] < 1e-5
    assert errs[1] < 1e-10
    assert errs[2] < 1e-14
    assert np.linalg.norm(C) <= 1e-10 * np.linalg.norm(X)  # the library's acceptance test passes
