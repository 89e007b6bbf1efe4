"""1D FDM bases on the reference interval [-1, 1] (Sec. 2.2 and 2.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Pins (tests/test_oracle_basis.py): GLL nodes and weights against textbook
values; B-hat identity on the interior and zero interior-interface block
(Sec. 2.2, unisolvence); A-hat interior block diagonal (Eq. eigs); r-hat
L2-orthonormal (Sec. 2.3); D-hat sparsity and the identity s_j' = sum_i D_ij
r_i at random points; lambda_1 decreasing to pi^2/4 (Rayleigh-Ritz).

Readings where the paper is silent:
* the interior eigenvector sign: each interior function s_j is scaled so
  that s_j'(-1) > 0;
* eigenvalues ascending (LAPACK order);
* the GLL mass and stiffness matrices are integrated exactly ((p+1)-point
  Gauss), not lumped.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg
from numpy.polynomial import legendre as npleg


def gll_nodes(p: int) -> np.ndarray:
    """The p+1 Gauss-Lobatto-Legendre points: -1, 1 and the roots of P_p'."""
    if p < 1:
        raise ValueError("p >= 1")
    if p == 1:
        return np.array([-1.0, 1.0])
    inner = np.sort(npleg.Legendre.basis(p).deriv().roots().real)
    return np.concatenate([[-1.0], inner, [1.0]])


def gll_rule(q: int):
    """q-point GLL quadrature: nodes and weights 2 / (q (q-1) P_{q-1}(x)^2)."""
    x = gll_nodes(q - 1)
    P = npleg.Legendre.basis(q - 1)(x)
    w = 2.0 / (q * (q - 1) * P * P)
    return x, w


def gauss_rule(m: int):
    """m-point Gauss-Legendre rule (exact for degree 2m-1)."""
    return npleg.leggauss(m)


def lagrange(nodes: np.ndarray, x: np.ndarray):
    """Values and derivatives of the Lagrange polynomials on `nodes` at x.

    Returns (L, dL) with L[k, j] = l_j(x_k), dL[k, j] = l_j'(x_k), using the
    product formula and its derivative written out term by term.
    """
    nodes = np.asarray(nodes, float)
    x = np.atleast_1d(np.asarray(x, float))
    n = len(nodes)
    L = np.ones((len(x), n))
    dL = np.zeros((len(x), n))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
        for m in range(n):
            if m == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[m]))
            for l in range(n):
                if l == j or l == m:
                    continue
                term *= (x - nodes[l]) / (nodes[j] - nodes[l])
            dL[:, j] += term
    return L, dL


class FDM1D:
    """FDM element for P_p and the derived basis of DP_{p-1} (Sec. 2.2-2.3).

    Attributes
    ----------
    p      degree
    xi     GLL nodes (p+1)
    Bgll   (l_i, l_j) exact             Agll  (l_i', l_j') exact
    S      tabulation S[i, j] = s_j(xi_i), columns 0..p
    lam    lam[0] = |I| = 2, lam[j] = (s_j', s_j') for j in 1..p-1
    Bhat   (s_i, s_j)                   Ahat  (s_i', s_j')
    D      D[i, j] = (r_i, s_j'), shape p x (p+1), by Gauss quadrature
    """

    def __init__(self, p: int):
        if p < 1:
            raise ValueError("p >= 1")
        self.p = p
        self.xi = gll_nodes(p)
        xg, wg = gauss_rule(p + 1)
        L, dL = lagrange(self.xi, xg)
        self.Bgll = L.T @ np.diag(wg) @ L
        self.Agll = dL.T @ np.diag(wg) @ dL
        I = list(range(1, p))
        G = [0, p]
        S = np.zeros((p + 1, p + 1))
        S[0, 0] = 1.0
        S[p, p] = 1.0
        lam_int = np.zeros(0)
        if p >= 2:
            # Eq. eigs: S_II^T A_II S_II = Lambda, S_II^T B_II S_II = I.
            lam_int, V = scipy.linalg.eigh(self.Agll[np.ix_(I, I)],
                                           self.Bgll[np.ix_(I, I)])
            # sign reading: s_j'(-1) > 0
            _, dL_left = lagrange(self.xi, np.array([-1.0]))
            slope = dL_left[0, I] @ V
            if np.any(np.abs(slope) < 1e-8 * np.abs(slope).max()):
                raise RuntimeError("sign rule undefined: s_j'(-1) ~ 0")
            V = V * np.sign(slope)[None, :]
            S[np.ix_(I, I)] = V
            # duality (Eq. unisolvence): S_IG = -S_II S_II^T B_IG
            S[np.ix_(I, G)] = -V @ V.T @ self.Bgll[np.ix_(I, G)]
        self.S = S
        self.lam = np.concatenate([[2.0], lam_int])
        self.Bhat = S.T @ self.Bgll @ S
        self.Ahat = S.T @ self.Agll @ S
        # D_ij = (r_i, s_j') by (p+1)-point Gauss (exact, degree 2p-2)
        r = self.r(xg)
        ds = self.ds(xg)
        self.D = r.T @ np.diag(wg) @ ds

    # -- evaluation at arbitrary points ------------------------------------
    def s(self, x):
        """s_j(x_k), shape (len(x), p+1)."""
        L, _ = lagrange(self.xi, x)
        return L @ self.S

    def ds(self, x):
        """s_j'(x_k), shape (len(x), p+1)."""
        _, dL = lagrange(self.xi, x)
        return dL @ self.S

    def r(self, x):
        """r_j(x_k), shape (len(x), p): r_0 = lam_0^{-1/2}, r_j = lam_j^{-1/2} s_j'."""
        x = np.atleast_1d(np.asarray(x, float))
        out = np.empty((len(x), self.p))
        out[:, 0] = 1.0 / np.sqrt(self.lam[0])
        if self.p >= 2:
            ds = self.ds(x)
            for j in range(1, self.p):
                out[:, j] = ds[:, j] / np.sqrt(self.lam[j])
        return out

    def injection_from_p1(self):
        """Coefficients of the p=1 basis in this basis (coarse space, Sec. 4.3).

        Returns (Js, Jr): Js[:, c] are the FDM-P_p coefficients of the linear
        hat c in {0: (1-x)/2, 1: (1+x)/2}, obtained by applying the dual
        functionals of Eq. fdmdualbasis; Jr[:, 0] are the DP_{p-1}
        coefficients of the p=1 L2 function r_0 = 2^{-1/2}.
        """
        p = self.p
        xg, wg = gauss_rule(p + 2)
        hats = np.stack([(1 - xg) / 2, (1 + xg) / 2], axis=1)
        s = self.s(xg)
        Js = np.zeros((p + 1, 2))
        Js[0, 0] = 1.0       # v(-1)
        Js[p, 1] = 1.0       # v(1)
        for i in range(1, p):
            Js[i, :] = (s[:, i] * wg) @ hats
        r = self.r(xg)
        coarse_r0 = np.full(len(xg), 1.0 / np.sqrt(2.0))
        Jr = (r * wg[:, None]).T @ coarse_r0[:, None]
        return Js, Jr
