"""Pins of the oracle's (flexible) preconditioned CG.

Flexible CG takes beta = z_new . (r_new - r_old) / (r_old . z_old)
(Polak-Ribiere); for a fixed symmetric positive definite preconditioner
z_new . r_old vanishes in exact arithmetic, so its iterates are those of
plain PCG (beta = r_new . z_new / r_old . z_old)."""
import numpy as np
import scipy.sparse as sp

from oracle.krylov import pcg


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    return M @ M.T / n + np.diag(rng.uniform(0.01, 1.0, n))


def test_flexible_equals_plain_for_fixed_preconditioner():
    n = 60
    A = _spd(n, 1)
    B = np.linalg.inv(np.diag(np.diag(A)) + 0.3 * _spd(n, 2))  # SPD, fixed
    b = np.random.default_rng(3).standard_normal(n)
    x1, i1 = pcg(A, b, B, rtol=1e-10, maxit=200)
    x2, i2 = pcg(A, b, B, rtol=1e-10, maxit=200, flexible=True)
    assert i1["converged"] and i2["converged"]
    assert i1["iterations"] == i2["iterations"]
    # identical in exact arithmetic; in floating point the two recurrences
    # drift apart only as the residual falls (rounding grows relative to it)
    h1, h2 = np.array(i1["history_l2"]), np.array(i2["history_l2"])
    early = h1 > 1e-6
    assert early.sum() > 10
    assert np.abs(h1[early] - h2[early]).max() <= 1e-9 * h1[early].min()
    assert np.allclose(x1, x2, rtol=1e-8, atol=1e-9 * np.abs(x1).max())


def test_unpreconditioned_cg_reaches_direct_solution():
    n = 40
    A = sp.csr_matrix(_spd(n, 4))
    b = np.random.default_rng(5).standard_normal(n)
    x, info = pcg(A, b, None, rtol=1e-13, maxit=2000)
    assert info["converged"]
    assert np.allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-9, atol=1e-12)
    # the recursive residual history ends at or below the tolerance
    assert info["history_l2"][-1] <= 1e-13
