"""Tensor-product de Rham spaces on structured hexahedral meshes, element
matrices by full-tensor quadrature, and global assembly.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages: the spaces Q_p, NCE_p, NCF_p, DQ_{p-1} and their bases (Sec.
2.4, Eqs. hgrad-basis, hcurl-basis, hdiv-basis, ltwo-basis); the weak form
a^k(v,u) = (v, beta u) + (d v, alpha d u) (Eq. common_weak_formulation); the
pullbacks F^k (Sec. 3.1); the cell matrices [A_K]_ij = a^k(F(psi_i), F(psi_j)).
The quadrature is the GLL rule with ceil(3(p+1)/2) points per direction
(Sec. 5, the rule of the paper's generated residual code).

Pins (tests/test_oracle_discretization.py): the complete-sequence identities
(Eqs. gradbasis, curlbasis, divbasis) at random points; the Cartesian cell
matrix equals the Kronecker closed form built from B-hat, A-hat; the interior
block of the Cartesian stiffness has 1 (k=0) or <= 3 (k=1,2) nonzeros per
row; curl grad = 0 and div curl = 0 on distorted cells; L2 convergence of
order p+1 for the sin-product solution.

Layout (shared convention with the CUDA path, stated independently there):
* component m of form degree k has type t_d in {'s', 'r'} per direction d;
  its lattice has N_d = n_d p + 1 (s) or n_d p (r) points, lattice index
  g_d = e_d p + i_d for local index i_d in cell e_d;
* a component's entries are stored g1 fastest, components concatenated;
* Dirichlet DOFs (Gamma_D = boundary of the unit cube) are the entries with
  an s-type index g_d in {0, n_d p};
* cell-local DOFs are ordered component-major, then i3, i2, i1 (i1 fastest).
"""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .basis import FDM1D, gauss_rule, gll_rule

# component types per form degree (Sec. 2.4)
SPACE_TYPES = {
    0: [("s", "s", "s")],
    1: [("r", "s", "s"), ("s", "r", "s"), ("s", "s", "r")],
    2: [("s", "r", "r"), ("r", "s", "r"), ("r", "r", "s")],
    3: [("r", "r", "r")],
}

# d^k in reference coordinates: for each target component of V^{k+1}, the
# terms (source component of V^k, direction differentiated, sign).
DERIVATIVE_TERMS = {
    0: [[(0, 0, +1)], [(0, 1, +1)], [(0, 2, +1)]],                  # grad
    1: [[(2, 1, +1), (1, 2, -1)],                                    # curl
        [(0, 2, +1), (2, 0, -1)],
        [(1, 0, +1), (0, 1, -1)]],
    2: [[(0, 0, +1), (1, 1, +1), (2, 2, +1)]],                       # div
}


def quadrature_points(p: int) -> int:
    """ceil(3(p+1)/2) GLL points per direction."""
    return (3 * (p + 1) + 1) // 2


def kron3(T3, T2, T1):
    """Matrix of the tensor product, rows (q3,q2,q1) and cols (i3,i2,i1)."""
    return np.kron(T3, np.kron(T2, T1))


class Lattice:
    """Global DOF lattice of V^k_{h,p} on an n1 x n2 x n3 mesh.

    bc = "dirichlet": Gamma_D is the whole boundary of the cube (entries with
    an s-type index on the boundary are not DOFs); bc = "none": Gamma_D is
    empty and every lattice entry is a DOF (Eq. common_weak_formulation with
    natural boundary conditions everywhere)."""

    def __init__(self, k: int, n, p: int, bc: str = "dirichlet"):
        if bc not in ("dirichlet", "none"):
            raise ValueError(bc)
        self.k, self.p, self.bc = k, p, bc
        self.n = (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)
        self.types = SPACE_TYPES[k]
        self.ncomp = len(self.types)
        self.dims = []
        self.loc_dims = []
        for t in self.types:
            self.dims.append(tuple(self.n[d] * p + (1 if t[d] == "s" else 0)
                                   for d in range(3)))
            self.loc_dims.append(tuple(p + 1 if t[d] == "s" else p
                                       for d in range(3)))
        self.sizes = [d[0] * d[1] * d[2] for d in self.dims]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(int)
        self.size = int(self.offsets[-1])
        self.loc_sizes = [d[0] * d[1] * d[2] for d in self.loc_dims]
        self.loc_offsets = np.concatenate([[0], np.cumsum(self.loc_sizes)]).astype(int)
        self.nloc = int(self.loc_offsets[-1])

    def index(self, m, g1, g2, g3):
        N1, N2, _ = self.dims[m]
        return self.offsets[m] + g1 + N1 * (g2 + N2 * g3)

    def coords(self):
        """(comp, g1, g2, g3) of every lattice entry, as integer arrays."""
        comp, G = [], [[], [], []]
        for m in range(self.ncomp):
            N1, N2, N3 = self.dims[m]
            g3, g2, g1 = np.meshgrid(np.arange(N3), np.arange(N2),
                                     np.arange(N1), indexing="ij")
            comp.append(np.full(g1.size, m))
            G[0].append(g1.ravel())
            G[1].append(g2.ravel())
            G[2].append(g3.ravel())
        return (np.concatenate(comp), np.concatenate(G[0]),
                np.concatenate(G[1]), np.concatenate(G[2]))

    def dirichlet_mask(self):
        mask = np.zeros(self.size, bool)
        if self.bc == "none":
            return mask
        comp, g1, g2, g3 = self.coords()
        G = (g1, g2, g3)
        for m in range(self.ncomp):
            sel = comp == m
            for d in range(3):
                if self.types[m][d] == "s":
                    edge = (G[d] == 0) | (G[d] == self.n[d] * self.p)
                    mask |= sel & edge
        return mask

    def free(self):
        return np.flatnonzero(~self.dirichlet_mask())

    def cell_dofs(self, e):
        """Global indices of the local DOFs of cell e = (e1, e2, e3)."""
        out = []
        p = self.p
        for m in range(self.ncomp):
            l1, l2, l3 = self.loc_dims[m]
            i3, i2, i1 = np.meshgrid(np.arange(l3), np.arange(l2),
                                     np.arange(l1), indexing="ij")
            out.append(self.index(m, e[0] * p + i1.ravel(), e[1] * p + i2.ravel(),
                                  e[2] * p + i3.ravel()))
        return np.concatenate(out)

    def cells(self):
        n1, n2, n3 = self.n
        for e3 in range(n3):
            for e2 in range(n2):
                for e1 in range(n1):
                    yield (e1, e2, e3), e1 + n1 * (e2 + n2 * e3)


class Mesh:
    """Structured hex mesh with trilinear cells (vertex layout of inputs.py)."""

    def __init__(self, n, X):
        self.n = (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)
        n1, n2, n3 = self.n
        self.X = np.asarray(X, float).reshape((n3 + 1) * (n2 + 1) * (n1 + 1), 3)

    def cell_vertices(self, e):
        """8 x 3 corner coordinates, corner c = c1 + 2 c2 + 4 c3."""
        n1, n2, _ = self.n
        out = np.empty((8, 3))
        for c3 in range(2):
            for c2 in range(2):
                for c1 in range(2):
                    a = (e[0] + c1) + (n1 + 1) * ((e[1] + c2) + (n2 + 1) * (e[2] + c3))
                    out[c1 + 2 * c2 + 4 * c3] = self.X[a]
        return out


def trilinear(V, xi):
    """x(xi) and J(xi) = dx/dxi of the trilinear map with corners V (8x3).

    xi: (nq, 3).  Returns x (nq, 3), J (nq, 3, 3) with J[q, a, d] = dx_a/dxi_d.
    """
    xi = np.asarray(xi, float)
    N = [np.stack([(1 - xi[:, d]) / 2, (1 + xi[:, d]) / 2], 1) for d in range(3)]
    dN = np.array([-0.5, 0.5])
    x = np.zeros((len(xi), 3))
    J = np.zeros((len(xi), 3, 3))
    for c3 in range(2):
        for c2 in range(2):
            for c1 in range(2):
                v = V[c1 + 2 * c2 + 4 * c3]
                w = N[0][:, c1] * N[1][:, c2] * N[2][:, c3]
                x += w[:, None] * v[None, :]
                d1 = dN[c1] * N[1][:, c2] * N[2][:, c3]
                d2 = N[0][:, c1] * dN[c2] * N[2][:, c3]
                d3 = N[0][:, c1] * N[1][:, c2] * dN[c3]
                J[:, :, 0] += d1[:, None] * v[None, :]
                J[:, :, 1] += d2[:, None] * v[None, :]
                J[:, :, 2] += d3[:, None] * v[None, :]
    return x, J


def form_weight(kk: int, J):
    """Pullback weight of the L2 product of kk-forms in reference values
    (Sec. 3.1): 0: |det J|; 1: |det J| J^-1 J^-T; 2: J^T J / |det J|;
    3: 1/|det J|.  Returns (nq, c, c) with c = 1 or 3."""
    det = np.linalg.det(J)
    if np.any(det <= 0):
        raise ValueError("inverted cell")
    if kk == 0:
        return det[:, None, None]
    if kk == 3:
        return (1.0 / det)[:, None, None]
    if kk == 1:
        Ji = np.linalg.inv(J)
        return det[:, None, None] * np.einsum("qab,qcb->qac", Ji, Ji)
    if kk == 2:
        return np.einsum("qba,qbc->qac", J, J) / det[:, None, None]
    raise ValueError(kk)


class ReferenceElement:
    """Tabulations of V^k(K-hat) and of d^k V^k(K-hat) at quadrature points."""

    def __init__(self, k: int, p: int, x1d, w1d):
        self.k, self.p = k, p
        self.e = FDM1D(p)
        self.x1d, self.w1d = np.asarray(x1d), np.asarray(w1d)
        q = len(x1d)
        self.nq = q ** 3
        g3, g2, g1 = np.meshgrid(self.x1d, self.x1d, self.x1d, indexing="ij")
        self.xi = np.stack([g1.ravel(), g2.ravel(), g3.ravel()], 1)
        self.w = kron3(self.w1d[:, None], self.w1d[:, None], self.w1d[:, None]).ravel()
        self.tab = {"s": self.e.s(self.x1d), "r": self.e.r(self.x1d)}
        self.dtab = self.e.ds(self.x1d)
        self.values = self._values(k)
        self.dvalues = self._dvalues(k) if k < 3 else None

    def _comp_table(self, types, deriv_dir=None):
        T = []
        for d in range(3):
            if d == deriv_dir:
                assert types[d] == "s"
                T.append(self.dtab)
            else:
                T.append(self.tab[types[d]])
        return kron3(T[2], T[1], T[0])

    def _values(self, kk):
        types = SPACE_TYPES[kk]
        c = 3 if len(types) == 3 else 1
        blocks = []
        for m, t in enumerate(types):
            V = self._comp_table(t)
            B = np.zeros((self.nq, c, V.shape[1]))
            B[:, m if c == 3 else 0, :] = V
            blocks.append(B)
        return np.concatenate(blocks, axis=2)

    def _dvalues(self, k):
        """Reference exterior derivative of every basis function of V^k,
        computed from the tabulated derivatives s_j' (not from D-hat)."""
        src = SPACE_TYPES[k]
        tgt_terms = DERIVATIVE_TERMS[k]
        c = len(tgt_terms) if len(tgt_terms) == 3 else 1
        blocks = []
        for m, t in enumerate(src):
            B = np.zeros((self.nq, c, int(np.prod([self.p + 1 if x == "s" else self.p
                                                   for x in t]))))
            for tc, terms in enumerate(tgt_terms):
                for (sm, d, sgn) in terms:
                    if sm == m:
                        B[:, tc, :] += sgn * self._comp_table(t, deriv_dir=d)
            blocks.append(B)
        return np.concatenate(blocks, axis=2)


def element_matrix(ref: ReferenceElement, V8, alpha: float, beta: float):
    """A_K = sum_q w_q [ Phi^T (beta W^k) Phi + dPhi^T (alpha W^{k+1}) dPhi ]
    (Eq. common_weak_formulation in reference values, Sec. 3.1-3.2)."""
    k = ref.k
    _, J = trilinear(V8, ref.xi)
    Wb = beta * form_weight(k, J) * ref.w[:, None, None]
    Phi = ref.values
    nq, c, nd = Phi.shape
    WPhi = np.einsum("qab,qbj->qaj", Wb, Phi)
    A = Phi.reshape(nq * c, nd).T @ WPhi.reshape(nq * c, nd)
    if k < 3:
        Wa = alpha * form_weight(k + 1, J) * ref.w[:, None, None]
        dPhi = ref.dvalues
        c2 = dPhi.shape[1]
        WdPhi = np.einsum("qab,qbj->qaj", Wa, dPhi)
        A += dPhi.reshape(nq * c2, nd).T @ WdPhi.reshape(nq * c2, nd)
    return A


class Problem:
    """a^k on a structured mesh with per-cell alpha, beta (Eq.
    common_weak_formulation), Gamma_D = boundary of the cube (bc =
    "dirichlet") or empty (bc = "none")."""

    def __init__(self, k, n, p, X, alpha, beta, bc="dirichlet"):
        self.k, self.p, self.bc = k, p, bc
        self.mesh = Mesh(n, X)
        self.n = self.mesh.n
        self.lat = Lattice(k, self.n, p, bc)
        ncell = self.n[0] * self.n[1] * self.n[2]
        self.alpha = np.broadcast_to(np.asarray(alpha, float), (ncell,)).copy()
        self.beta = np.broadcast_to(np.asarray(beta, float), (ncell,)).copy()
        q = quadrature_points(p)
        self.ref = ReferenceElement(k, p, *gll_rule(q))
        self.free = self.lat.free()
        self._A = None

    def element(self, e, c):
        return element_matrix(self.ref, self.mesh.cell_vertices(e),
                              self.alpha[c], self.beta[c])

    def assemble(self):
        """Global A over the full lattice (Dirichlet rows/cols included)."""
        if self._A is None:
            rows, cols, vals = [], [], []
            for e, c in self.lat.cells():
                dofs = self.lat.cell_dofs(e)
                AK = self.element(e, c)
                rows.append(np.repeat(dofs, len(dofs)))
                cols.append(np.tile(dofs, len(dofs)))
                vals.append(AK.ravel())
            N = self.lat.size
            self._A = sp.coo_matrix((np.concatenate(vals),
                                     (np.concatenate(rows), np.concatenate(cols))),
                                    shape=(N, N)).tocsr()
        return self._A

    def A_free(self):
        A = self.assemble()
        return A[self.free][:, self.free].tocsr()

    def apply(self, x):
        """y = R_f^T A_ff R_f x on the full lattice (Dirichlet entries of x
        ignored, of y zero)."""
        A = self.assemble()
        xf = np.zeros(self.lat.size)
        xf[self.free] = x[self.free]
        y = np.zeros(self.lat.size)
        y[self.free] = (A @ xf)[self.free]
        return y

    def apply_rows(self, x, rows):
        """(A x)_i for selected lattice rows i, one by one from the cells
        that touch each row (no global assembly)."""
        xf = np.zeros(self.lat.size)
        xf[self.free] = x[self.free]
        dmask = self.lat.dirichlet_mask()
        out = np.zeros(len(rows))
        want = {int(r): i for i, r in enumerate(rows)}
        n1, n2, n3 = self.n
        p = self.p
        comp, g1, g2, g3 = self.lat.coords()
        cells_of = {}
        for r in want:
            cs = []
            G = (g1[r], g2[r], g3[r])
            t = self.lat.types[comp[r]]
            ranges = []
            for d in range(3):
                if t[d] == "s" and G[d] % p == 0:
                    e = G[d] // p
                    ranges.append([x for x in (e - 1, e) if 0 <= x < self.n[d]])
                else:
                    ranges.append([G[d] // p])
            for a in ranges[0]:
                for b in ranges[1]:
                    for c in ranges[2]:
                        cs.append((a, b, c))
            for cc in cs:
                cells_of.setdefault(cc, []).append(r)
        ref = self.ref
        for e, rs in cells_of.items():
            c = e[0] + n1 * (e[1] + n2 * e[2])
            dofs = self.lat.cell_dofs(e)
            _, J = trilinear(self.mesh.cell_vertices(e), ref.xi)
            xK = xf[dofs]
            u = np.einsum("qaj,j->qa", ref.values, xK)
            v = np.einsum("qab,qb->qa", self.beta[c] * form_weight(self.k, J)
                          * ref.w[:, None, None], u)
            if self.k < 3:
                du = np.einsum("qaj,j->qa", ref.dvalues, xK)
                dv = np.einsum("qab,qb->qa", self.alpha[c] * form_weight(self.k + 1, J)
                               * ref.w[:, None, None], du)
            loc = {int(g): i for i, g in enumerate(dofs)}
            for r in rs:
                i = loc[r]
                val = np.sum(ref.values[:, :, i] * v)
                if self.k < 3:
                    val += np.sum(ref.dvalues[:, :, i] * dv)
                out[want[r]] += val
        out[dmask[np.asarray(rows)]] = 0.0
        return out

    # -- manufactured solution (H(grad) only) ------------------------------
    def load_vector_hgrad(self, f, extra=3):
        """b_i = (f, psi_i) with a (p+extra)-point Gauss rule per direction."""
        assert self.k == 0
        xg, wg = gauss_rule(self.p + extra)
        ref = ReferenceElement(0, self.p, xg, wg)
        b = np.zeros(self.lat.size)
        for e, c in self.lat.cells():
            x, J = trilinear(self.mesh.cell_vertices(e), ref.xi)
            det = np.linalg.det(J)
            fw = f(x) * det * ref.w
            b[self.lat.cell_dofs(e)] += ref.values[:, 0, :].T @ fw
        b[~np.isin(np.arange(self.lat.size), self.free)] = 0.0
        return b

    def l2_error_hgrad(self, u_coef, u_exact, extra=4):
        assert self.k == 0
        xg, wg = gauss_rule(self.p + extra)
        ref = ReferenceElement(0, self.p, xg, wg)
        err = 0.0
        for e, c in self.lat.cells():
            x, J = trilinear(self.mesh.cell_vertices(e), ref.xi)
            det = np.linalg.det(J)
            uh = ref.values[:, 0, :] @ u_coef[self.lat.cell_dofs(e)]
            err += np.sum(ref.w * det * (uh - u_exact(x)) ** 2)
        return math.sqrt(err)


def dhat_3d(k: int, e: FDM1D):
    """Reference exterior derivative d^k in FDM coefficients, V^k -> V^{k+1},
    as Kronecker products of the 1D D-hat (Sec. 2.3-2.4, fig. fdmbasis(c))."""
    p = e.p
    src = SPACE_TYPES[k]
    tgt = SPACE_TYPES[k + 1]
    I = {"s": np.eye(p + 1), "r": np.eye(p)}
    ncol = [int(np.prod([p + 1 if x == "s" else p for x in t])) for t in src]
    nrow = [int(np.prod([p + 1 if x == "s" else p for x in t])) for t in tgt]
    coff = np.concatenate([[0], np.cumsum(ncol)])
    roff = np.concatenate([[0], np.cumsum(nrow)])
    M = np.zeros((roff[-1], coff[-1]))
    for tc, terms in enumerate(DERIVATIVE_TERMS[k]):
        for (sm, d, sgn) in terms:
            T = [e.D if dd == d else I[src[sm][dd]] for dd in range(3)]
            M[roff[tc]:roff[tc + 1], coff[sm]:coff[sm + 1]] += sgn * kron3(T[2], T[1], T[0])
    return M
