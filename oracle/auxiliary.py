"""Sparse auxiliary operator P (Sec. 3.2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

P_K = G^T diag(Mbar^k_beta) G + Dbar^T diag(Mbar^{k+1}_alpha) Dbar,
Dbar = G D-hat (Eq. sum-factorization_approx), where G is the basis change
to the broken space whose interface functions are orthogonalised
(Eq. mass_in_broken_basis).

Reading where the paper is silent: the interface pair (s_0, s_p) is replaced
by the orthonormal rotation sbar_0 = (s_0 + s_p)/sqrt 2,
sbar_p = (s_0 - s_p)/sqrt 2, which diagonalises the symmetric 2x2 block
B-hat_GG = [[a, b], [b, a]].  Any scaling of the broken functions gives the
same P; only the rotation matters.

Pins: P = A on Cartesian cells with constant coefficients (the broken mass
matrix is then diagonal); P symmetric positive definite; the interior block
P_II has the Cartesian sparsity (1 nonzero per row for k=0, blocks <= 3x3 for
k=1,2; Remark after Eq. schur).  The spectral equivalence of P and A on
distorted cells has no value in the paper: parity unpinned there.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.linalg

from .discretization import (SPACE_TYPES, ReferenceElement, dhat_3d,
                             form_weight, trilinear)


def broken_transform_1d(p: int) -> np.ndarray:
    """G with ubar = G u for the P_p basis (identity on the interior)."""
    G = np.eye(p + 1)
    h = 1.0 / np.sqrt(2.0)
    G[0, 0], G[0, p], G[p, 0], G[p, p] = h, h, h, -h
    return G


def broken_transform(kk: int, p: int) -> np.ndarray:
    """Block-diagonal G for V^kk(K-hat): one Kronecker block per component."""
    G1 = broken_transform_1d(p)
    blocks = []
    for t in SPACE_TYPES[kk]:
        T = [G1 if t[d] == "s" else np.eye(p) for d in range(3)]
        blocks.append(np.kron(T[2], np.kron(T[1], T[0])))
    return scipy.linalg.block_diag(*blocks)


def broken_tabulation(ref: ReferenceElement, kk: int):
    """The broken functions tabulated at the quadrature points, Phi G^{-1}."""
    G = broken_transform(kk, ref.p)
    nq, c, nd = ref.values.shape
    return (ref.values.reshape(nq * c, nd) @ np.linalg.inv(G)).reshape(nq, c, nd)


def broken_mass_diagonal(Phib, W):
    """diag of the weighted mass matrix in the broken basis:
    d_K = sum_q Phib_K(q)^T W(q) Phib_K(q).

    W: (nq, c, c) weight including the quadrature weight and coefficient."""
    return np.einsum("qak,qab,qbk->k", Phib, W, Phib)


class AuxElement:
    """Builds P_K for form degree k on a given quadrature."""

    def __init__(self, k: int, p: int, x1d, w1d):
        self.k, self.p = k, p
        self.ref_k = ReferenceElement(k, p, x1d, w1d)
        self.ref_k1 = ReferenceElement(k + 1, p, x1d, w1d)
        self.Gk = broken_transform(k, p)
        self.Gk1 = broken_transform(k + 1, p)
        self.D = dhat_3d(k, self.ref_k.e)
        self.Dbar = self.Gk1 @ self.D
        self.Phib_k = broken_tabulation(self.ref_k, k)
        self.Phib_k1 = broken_tabulation(self.ref_k1, k + 1)

    def matrix(self, V8, mass_coef: float, stiff_coef: float):
        _, J = trilinear(V8, self.ref_k.xi)
        w = self.ref_k.w[:, None, None]
        db = broken_mass_diagonal(self.Phib_k, mass_coef * form_weight(self.k, J) * w)
        da = broken_mass_diagonal(self.Phib_k1, stiff_coef * form_weight(self.k + 1, J) * w)
        return (self.Gk.T @ np.diag(db) @ self.Gk
                + self.Dbar.T @ np.diag(da) @ self.Dbar)


def assemble_aux(problem, mass_coef=None, stiff_coef=None):
    """Global P over the full lattice for a discretization.Problem.

    mass_coef / stiff_coef default to the problem's beta / alpha; the
    Hiptmair potential operator uses mass 0 and stiffness beta on V^0."""
    from .basis import gll_rule
    from .discretization import quadrature_points
    k, p = problem.k, problem.p
    x1d, w1d = gll_rule(quadrature_points(p))
    el = AuxElement(k, p, x1d, w1d)
    mc = problem.beta if mass_coef is None else mass_coef
    sc = problem.alpha if stiff_coef is None else stiff_coef
    rows, cols, vals = [], [], []
    for e, c in problem.lat.cells():
        dofs = problem.lat.cell_dofs(e)
        PK = el.matrix(problem.mesh.cell_vertices(e), mc[c], sc[c])
        rows.append(np.repeat(dofs, len(dofs)))
        cols.append(np.tile(dofs, len(dofs)))
        vals.append(PK.ravel())
    N = problem.lat.size
    return sp.coo_matrix((np.concatenate(vals),
                          (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N)).tocsr()
