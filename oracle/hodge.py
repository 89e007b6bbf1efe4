"""Mixed formulation of the Hodge Laplacians with the Riesz-map block
preconditioner (Sec. 5.3): find (sigma, u) in V^{k-1} x V^k with

    -(tau, sigma) + (d tau, u)       = 0      for all tau in V^{k-1},
     (v, d sigma) + (d v, d u)        = F(v)   for all v in V^k,

Gamma_D empty; MINRES preconditioned by blockdiag(R_{k-1}^-1, R_k^-1), each
Riesz map (alpha = beta = 1) inverted approximately by 4 Chebyshev
iterations preconditioned by its SC relaxation with the p = 1 coarse
correction (SC-PAFW for V^0, SC-PH for V^1 and V^2, point-Jacobi for the L2
block of k = 3); stopping on the natural norm.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings where the paper is silent:
* Chebyshev interval: the extreme Ritz values theta_min, theta_max of 20
  preconditioned Lanczos (CG) steps on a seeded N(0,1) right-hand side,
  widened to [0.9 theta_min, 1.1 theta_max] (Ritz values lie inside the
  spectrum; the widening keeps the polynomial preconditioner positive
  definite);
* the Chebyshev iteration is the classical three-term recurrence for the
  preconditioned operator started from zero (Saad, Iterative methods for
  sparse linear systems, Alg. 12.1), 4 applications of the inner
  preconditioner and 3 of the Riesz operator per block solve;
* MINRES is the preconditioned minimum residual method of Paige and
  Saunders in the Lanczos form (Elman, Silvester and Wathen, Finite
  elements and fast iterative solvers, Alg. 2.4); the natural norm is the
  preconditioned residual norm sqrt(r^T P r) that it updates.

Pins (tests/test_oracle_hodge.py): the system's inertia (n_sigma negative,
n_u positive eigenvalues); MINRES reaches the direct solution; its residual
is the least-squares minimum over the Krylov space (brute force); the
Chebyshev residual is the scaled Chebyshev polynomial at every eigenvalue.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .auxiliary import assemble_aux
from .discretization import Problem
from .krylov import pcg
from .relaxation import SCPAFW, SCPH, discrete_derivative


def chebyshev(A, B, r, a, b, its=4):
    """its steps of the preconditioned Chebyshev iteration for A x = r from
    x = 0, B the inner preconditioner, [a, b] the interval of the spectrum
    of B A.  Returns x (a fixed polynomial in B A times B r)."""
    Aop = A if callable(A) else (lambda v: A @ v)
    Bop = B if callable(B) else (lambda v: B @ v)
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = np.zeros_like(r)
    res = r.copy()
    d = Bop(res) / theta
    for k in range(its):
        x = x + d
        if k == its - 1:
            break
        res = res - Aop(d)
        z = Bop(res)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * z
        rho = rho_new
    return x


def ritz_interval(A, B, n, seed=0, steps=20):
    """[0.9 theta_min, 1.1 theta_max] from the CG tridiagonal of `steps`
    preconditioned CG iterations on a seeded N(0,1) right-hand side."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(n)
    Aop = A if callable(A) else (lambda v: A @ v)
    Bop = B if callable(B) else (lambda v: B @ v)
    x = np.zeros(n)
    r = b.copy()
    z = Bop(r)
    p = z.copy()
    rz = r @ z
    alphas, betas = [], []
    for _ in range(steps):
        q = Aop(p)
        a = rz / (p @ q)
        r = r - a * q
        z = Bop(r)
        rz_new = r @ z
        bt = rz_new / rz
        alphas.append(a)
        betas.append(bt)
        rz = rz_new
        p = z + bt * p
        if rz <= 1e-30 * (b @ b):
            break
    m = len(alphas)
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < m:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    ev = np.linalg.eigvalsh(T)
    return 0.9 * ev[0], 1.1 * ev[-1]


def minres(A, b, P, rtol=1e-8, maxit=500):
    """Preconditioned MINRES (P symmetric positive definite) from x = 0.
    Stops when the natural norm sqrt(r^T P r) has fallen by 1/rtol.
    Returns x and {iterations, history_natural, converged}."""
    Aop = A if callable(A) else (lambda v: A @ v)
    Pop = P if callable(P) else (lambda v: P @ v)
    n = len(b)
    x = np.zeros(n)
    v_old = np.zeros(n)
    v = b.copy()
    z = Pop(v)
    gamma = np.sqrt(v @ z)
    gamma_old = 1.0
    eta = gamma
    eta0 = gamma
    s_old = s = 0.0
    c_old = c = 1.0
    w_old = np.zeros(n)
    w = np.zeros(n)
    hist = [1.0]
    it = 0
    converged = eta0 == 0.0
    while not converged and it < maxit:
        z = z / gamma
        Az = Aop(z)
        delta = z @ Az
        v_new = Az - (delta / gamma) * v - (gamma / gamma_old) * v_old
        z_new = Pop(v_new)
        gamma_new = np.sqrt(max(v_new @ z_new, 0.0))
        a0 = c * delta - c_old * s * gamma
        a1 = np.sqrt(a0 * a0 + gamma_new * gamma_new)
        a2 = s * delta + c_old * c * gamma
        a3 = s_old * gamma
        c_new, s_new = a0 / a1, gamma_new / a1
        w_new = (z - a3 * w_old - a2 * w) / a1
        x = x + c_new * eta * w_new
        eta = -s_new * eta
        it += 1
        hist.append(abs(eta) / eta0)
        converged = abs(eta) <= rtol * eta0
        v_old, v = v, v_new
        z = z_new
        gamma_old, gamma = gamma, gamma_new
        w_old, w = w, w_new
        c_old, c = c, c_new
        s_old, s = s, s_new
    return x, {"iterations": it, "history_natural": hist, "converged": converged}


class HodgeMixed:
    """The block system of the k-th Hodge Laplacian (k = 1, 2, 3) on a
    structured mesh with Gamma_D empty, and its block preconditioner."""

    def __init__(self, k, n, p, X, cheb_its=4, seed=0):
        assert k in (1, 2, 3)
        self.k, self.p = k, p
        one = 1.0
        # V^{k-1}: the mass (-(tau, sigma)) and the Riesz map (alpha = beta = 1)
        self.p0 = Problem(k - 1, n, p, X, 0.0, one, bc="none")
        self.M0 = self.p0.A_free()
        r0 = Problem(k - 1, n, p, X, one, one, bc="none")
        self.R0 = r0.A_free()
        # V^k: the mass, the derivative term (d v, d u) and the Riesz map
        pk = Problem(k, n, p, X, 0.0, one, bc="none")
        self.Mk = pk.A_free()
        self.Kk = (Problem(k, n, p, X, one, 0.0, bc="none").A_free() if k < 3
                   else sp.csr_matrix(self.Mk.shape))
        rk = Problem(k, n, p, X, one, one, bc="none") if k < 3 else pk
        self.Rk = rk.A_free()
        D = discrete_derivative(k - 1, self.p0.lat, pk.lat)
        self.D = D[pk.free][:, self.p0.free].tocsr()
        self.n0, self.nk = self.M0.shape[0], self.Mk.shape[0]
        MkD = (self.Mk @ self.D).tocsr()
        self.K = sp.bmat([[-self.M0, MkD.T], [MkD, self.Kk]]).tocsr()
        # inner preconditioners of the two Riesz maps
        self.B0 = self._relaxation(r0)
        if k < 3:
            self.Bk = self._relaxation(rk)
        else:
            dk = self.Rk.diagonal()
            self.Bk = lambda v: v / dk
        self.cheb_its = cheb_its
        self.int0 = ritz_interval(self.R0, self.B0, self.n0, seed)
        self.intk = ritz_interval(self.Rk, self.Bk, self.nk, seed + 1)

    @staticmethod
    def _relaxation(pr):
        P = assemble_aux(pr)[pr.free][:, pr.free]
        if pr.k == 0:
            return SCPAFW(pr, P, factor="icc").apply
        return SCPH(pr, P).apply

    def precondition(self, r):
        r0, rk = r[:self.n0], r[self.n0:]
        z0 = chebyshev(self.R0, self.B0, r0, *self.int0, its=self.cheb_its)
        zk = chebyshev(self.Rk, self.Bk, rk, *self.intk, its=self.cheb_its)
        return np.concatenate([z0, zk])

    def solve(self, F, rtol=1e-8, maxit=500):
        """MINRES for K (sigma, u) = (0, F)."""
        b = np.concatenate([np.zeros(self.n0), F])
        return minres(self.K, b, self.precondition, rtol=rtol, maxit=maxit)
