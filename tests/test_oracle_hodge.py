"""Pins of the oracle's Hodge-Laplacian solver (Sec. 5.3): the mixed
system's inertia, MINRES against the direct solve and against the
brute-force Krylov least-squares minimum, the Chebyshev residual polynomial
in closed form."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.hodge import HodgeMixed, chebyshev, minres, ritz_interval
from paper_2211_14284_gb300 import inputs


def test_chebyshev_residual_is_the_chebyshev_polynomial():
    """On a diagonal operator with B = I, 4 Chebyshev steps on [a, b] leave
    the residual r_4 = T_4((b + a - 2 lam) / (b - a)) / T_4((b + a) / (b - a)) r
    eigenvalue by eigenvalue (the defining minimax property)."""
    lam = np.linspace(0.3, 2.0, 40)
    r = np.random.default_rng(0).standard_normal(40)
    a, b = 0.25, 2.2
    x = chebyshev(np.diag(lam), np.eye(40), r, a, b, its=4)
    T4 = np.polynomial.chebyshev.Chebyshev([0, 0, 0, 0, 1])
    want = T4((b + a - 2 * lam) / (b - a)) / T4((b + a) / (b - a)) * r
    assert np.abs((r - lam * x) - want).max() <= 1e-13 * np.abs(r).max()


def test_ritz_interval_brackets_the_spectrum():
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    lam = np.linspace(1.0, 30.0, 60)
    A = (Q * lam) @ Q.T
    a, b = ritz_interval(A, np.eye(60), 60, seed=2, steps=30)
    assert a <= lam.min() and b >= lam.max()
    assert a >= 0.85 * lam.min() and b <= 1.15 * lam.max()


def test_minres_minimises_the_residual_over_the_krylov_space():
    """MINRES with P = I: after m steps the residual is the least-squares
    minimum of ||b - A x|| over x in K_m(A, b) (brute force, indefinite A)."""
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    lam = np.concatenate([-np.linspace(1, 3, 10), np.linspace(0.5, 4, 20)])
    A = (Q * lam) @ Q.T
    b = rng.standard_normal(30)
    for m in (3, 6, 9):
        x, info = minres(A, b, np.eye(30), rtol=0.0, maxit=m)
        K = np.stack([np.linalg.matrix_power(A, j) @ b for j in range(m)], 1)
        c, *_ = np.linalg.lstsq(A @ K, b, rcond=None)
        best = np.linalg.norm(b - A @ K @ c)
        assert np.linalg.norm(b - A @ x) == pytest.approx(best, rel=1e-8)
        # the recursively updated norm is the true one (P = I)
        assert info["history_natural"][-1] * np.linalg.norm(b) == pytest.approx(best, rel=1e-8)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_hodge_system_inertia(k):
    """-M on V^{k-1} and the positive Schur complement: the mixed system has
    exactly n_sigma negative and n_u positive eigenvalues (nonsingular: the
    cube has no harmonic forms in these degrees)."""
    n, p = 2, 2
    H = HodgeMixed(k, n, p, inputs.vertices(n, perturb=0.1, seed=4))
    ev = np.linalg.eigvalsh(H.K.toarray())
    tol = 1e-10 * np.abs(ev).max()
    assert np.sum(ev < -tol) == H.n0 and np.sum(ev > tol) == H.nk


@pytest.mark.slow
@pytest.mark.parametrize("k", [1, 2, 3])
def test_hodge_minres_reaches_the_direct_solution(k):
    n, p = 2, 3
    H = HodgeMixed(k, n, p, inputs.vertices(n, perturb=0.1, seed=5))
    F = inputs.normal_rhs(H.nk, 6)
    x, info = H.solve(F, rtol=1e-11, maxit=200)
    assert info["converged"]
    xd = spla.spsolve(H.K.tocsc(), np.concatenate([np.zeros(H.n0), F]))
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    # robust counts, as in tab. hodge-iter (6-23)
    _, i8 = H.solve(F, rtol=1e-8)
    assert i8["iterations"] <= 30, i8["iterations"]
