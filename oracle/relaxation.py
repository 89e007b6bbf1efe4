"""Subspace-correction relaxation: stars, patches, static condensation,
Cholesky / ICC(0) patch factors, the p=1 coarse space, additive and hybrid
compositions (Sec. 4).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Passages: stars and V_h|star (Sec. 4.1, fig. stars); PAFW and PH
decompositions (Eqs. pafw, ph) and their algebraic forms (Eqs. asm-afw,
asm-hiptmair); static condensation (Eqs. LDU, schur) and the SC forms
(Eqs. sc-pafw, sc-ph, sc-asm-afw, sc-asm-hiptmair); ICC on the
static-condensation pattern and edge-star Cholesky (Sec. 4.5); hybrid
multigrid/Schwarz V(1,1) (Sec. 5).

Readings where the paper is silent or ambiguous:
* stars are taken over ALL vertices / edges / faces (Eq. pafw sums over
  E^0), boundary entities included; Dirichlet DOFs are never in a patch;
* a DOF belongs to the star of an entity when, in every direction, its
  support lies in the cells around the entity and it vanishes on the star's
  boundary (the support rule of Sec. 4.1);
* patch ordering is nested dissection by entity: cell interiors, then faces,
  then edges, then vertices, lexicographic in the global index within each
  group; this fixes the ICC(0) factor;
* the patch matrix is taken on its sparsity pattern: entries with
  |S_ij| <= 1e-12 sqrt(|S_ii S_jj|) are numerically zero couplings and are
  not part of it; ICC(0) keeps exactly the remaining entries and exact
  Cholesky factors the matrix restricted to them; a non-positive pivot is a
  breakdown;
* the coarse correction R_0^T A_0^{-1} R_0 acts on the full space; R_0^T is
  the injection of V_{h,1} into V_{h,p} (dual functionals of Eq.
  fdmdualbasis applied to the p=1 basis) and A_0 is a^k rediscretised at p=1
  with its own ceil(3*2/2)=3-point GLL rule;
* in the SC forms the interior solve uses the auxiliary operator's P_II and
  the harmonic extension uses its P_GI (the preconditioner is built from P);
* the H(curl) Hiptmair potential operator is B = D^T P^1 D, which equals the
  H(grad) auxiliary operator with mass 0 and stiffness beta; D-tilde is the
  discrete gradient restricted to interface rows and columns;
* hybrid V(1,1): pre-smooth omega*M^{-1}, exact coarse correction,
  post-smooth omega*M^{-1}, with M^{-1} the additive fine-level relaxation.

Pins: a dense patch Cholesky solve equals numpy.linalg.solve; ICC(0) with
the full pattern equals Cholesky; the SC identity A^{-1} = R_I^T A_II^{-1}
R_I + R_G^T S^{-1} R_G and R_G A R_I^T = 0 (Eq. schur); Galerkin
R_0 A R_0^T = A_0 on Cartesian cells; hybrid V(1,1) with p = 1 converges in
one CG iteration (tab. hgrad-iter, l = 0 entries "1/1").
"""

from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .basis import FDM1D
from .discretization import Lattice, Problem

ICC_DROP = 1e-12


# ---------------------------------------------------------------------------
# stars and patches
# ---------------------------------------------------------------------------
class DofGeometry:
    """Per lattice entry: lattice coordinates and which directions are
    'vertex-type' (an s-type index on a mesh plane)."""

    def __init__(self, lat: Lattice):
        self.lat = lat
        comp, g1, g2, g3 = lat.coords()
        self.comp = comp
        self.G = np.stack([g1, g2, g3], 1)
        p = lat.p
        stype = np.array([[t[d] == "s" for d in range(3)] for t in lat.types])
        self.vtx = stype[comp] & (self.G % p == 0)
        self.cell = self.G // p              # owning cell for non-vertex type
        self.plane = self.G // p             # mesh plane for vertex type
        self.dim = 3 - self.vtx.sum(1)       # dimension of the entity the DOF lives on

    def star(self, corner, span, candidates):
        """DOFs (among `candidates`, lattice indices) supported in the star of
        the entity with lower corner `corner` spanning directions `span`."""
        c = candidates
        ok = np.ones(len(c), bool)
        for d in range(3):
            a = corner[d]
            vt = self.vtx[c, d]
            if d in span:
                ok &= (~vt) & (self.cell[c, d] == a)
            else:
                ok &= (vt & (self.plane[c, d] == a)) | \
                      ((~vt) & ((self.cell[c, d] == a - 1) | (self.cell[c, d] == a)))
        sel = c[ok]
        order = np.lexsort((sel, -self.dim[sel]))
        return sel[order]


def entities(n, span):
    """Lower corners of all entities spanning `span` on an n1 x n2 x n3 mesh."""
    rng = [range(n[d]) if d in span else range(n[d] + 1) for d in range(3)]
    out = []
    for a3 in rng[2]:
        for a2 in rng[1]:
            for a1 in rng[0]:
                out.append((a1, a2, a3))
    return out


def patch_lists(lat: Lattice, span, candidates):
    """Patches (lattice indices, nested-dissection order) of every entity."""
    geo = DofGeometry(lat)
    pats = []
    for a in entities(lat.n, span):
        s = geo.star(a, span, candidates)
        if len(s):
            pats.append(s)
    return pats


# ---------------------------------------------------------------------------
# patch factorizations
# ---------------------------------------------------------------------------
def icc0(Adense: np.ndarray, drop: float = ICC_DROP) -> np.ndarray:
    """Incomplete Cholesky with zero fill-in on the pattern of Adense
    (right-looking elimination restricted to the pattern)."""
    A = np.array(Adense, float, copy=True)
    n = A.shape[0]
    d = np.sqrt(np.abs(np.diag(A)))
    mask = np.abs(A) > drop * np.outer(d, d)
    np.fill_diagonal(mask, True)
    A[~mask] = 0.0
    for k in range(n):
        if A[k, k] <= 0.0:
            raise np.linalg.LinAlgError(f"ICC(0) breakdown at pivot {k}")
        A[k, k] = np.sqrt(A[k, k])
        col = k + 1 + np.flatnonzero(mask[k + 1:, k])
        A[col, k] /= A[k, k]
        if len(col):
            upd = np.outer(A[col, k], A[col, k]) * mask[np.ix_(col, col)]
            A[np.ix_(col, col)] -= upd
    return np.tril(A)


def pattern_matrix(Adense: np.ndarray, drop: float = ICC_DROP) -> np.ndarray:
    """The patch matrix on its sparsity pattern: entries with
    |A_ij| <= drop sqrt(|A_ii A_jj|) (numerically zero couplings) removed."""
    d = np.sqrt(np.abs(np.diag(Adense)))
    A = np.array(Adense, float, copy=True)
    A[np.abs(A) <= drop * np.outer(d, d)] = 0.0
    np.fill_diagonal(A, np.diag(Adense))
    return A


def cholesky(Adense: np.ndarray) -> np.ndarray:
    """Exact Cholesky factor of the patch matrix on its sparsity pattern."""
    return np.linalg.cholesky(pattern_matrix(Adense))


class PatchSolver:
    """sum_j R_j^T (L_j L_j^T)^{-1} R_j over patches of a matrix (free DOF
    numbering)."""

    def __init__(self, M: sp.csr_matrix, patches, factor: str):
        self.patches = patches
        self.L = []
        M = M.tocsr()
        for idx in patches:
            Aj = M[idx][:, idx].toarray()
            self.L.append(icc0(Aj) if factor == "icc" else cholesky(Aj))

    def apply(self, r):
        z = np.zeros_like(r)
        for idx, L in zip(self.patches, self.L):
            y = scipy.linalg.solve_triangular(L, r[idx], lower=True)
            z[idx] += scipy.linalg.solve_triangular(L.T, y, lower=False)
        return z


# ---------------------------------------------------------------------------
# coarse space
# ---------------------------------------------------------------------------
def prolongation(lat_f: Lattice, lat_c: Lattice) -> sp.csr_matrix:
    """Injection V_{h,1} -> V_{h,p} on the full lattices (fine x coarse)."""
    e = FDM1D(lat_f.p)
    Js, Jr = e.injection_from_p1()
    J = {"s": Js, "r": Jr}
    blocks = []
    for t in lat_f.types:
        blocks.append(np.kron(J[t[2]], np.kron(J[t[1]], J[t[0]])))
    Jloc = scipy.linalg.block_diag(*blocks)
    entries = {}
    for cell, _ in lat_f.cells():
        fd = lat_f.cell_dofs(cell)
        cd = lat_c.cell_dofs(cell)
        for i in range(len(fd)):
            for j in range(len(cd)):
                v = Jloc[i, j]
                if v != 0.0:
                    entries[(int(fd[i]), int(cd[j]))] = v
    r = np.array([k[0] for k in entries], int)
    c = np.array([k[1] for k in entries], int)
    v = np.array(list(entries.values()))
    return sp.coo_matrix((v, (r, c)), shape=(lat_f.size, lat_c.size)).tocsr()


def refinement(lat_f: Lattice, lat_c: Lattice) -> sp.csr_matrix:
    """Lowest-order (p=1) refinement from the mesh n/2 (lat_c) to n (lat_f),
    on the full lattices: along an s-type direction the coarse hat is 1 at
    its own vertex and 1/2 at the two fine vertices beside it; along an
    r-type direction a coarse cell's constant is carried by its two fine
    halves with weight 1/2 each (the reference-value scaling of the 1- and
    2-form pullbacks when the cell length halves)."""
    rows, cols, vals = [], [], []
    comp, g1, g2, g3 = lat_f.coords()
    G = np.stack([g1, g2, g3], 1)
    for idx in range(lat_f.size):
        m = comp[idx]
        opts = []
        for d in range(3):
            g = G[idx, d]
            if lat_f.types[m][d] == "s":
                opts.append([(g // 2, 1.0)] if g % 2 == 0 else [((g - 1) // 2, 0.5), ((g + 1) // 2, 0.5)])
            else:
                opts.append([(g // 2, 0.5)])
        for (a, wa) in opts[0]:
            for (b, wb) in opts[1]:
                for (c, wc) in opts[2]:
                    rows.append(idx)
                    cols.append(lat_c.index(m, a, b, c))
                    vals.append(wa * wb * wc)
    return sp.coo_matrix((vals, (rows, cols)), shape=(lat_f.size, lat_c.size)).tocsr()


class Coarse:
    """R_0^T A_0^{-1} R_0 with A_0 the p=1 rediscretisation (Eq. asm-afw).

    mode "exact": A_0^{-1} by a dense Cholesky solve.  mode "gmg": A_0^{-1}
    replaced by one symmetric V(2,2) cycle of geometric multigrid (the
    paper's p-coarse multigrid, Sec. 5.1): Galerkin levels P^T A P with the
    lowest-order refinement while every n_d is even and >= 4 and the level
    has more than 512 DOFs; a dense solve on the coarsest level (the h-coarse
    Cholesky of the solver diagram).  Smoother: damped point Jacobi with
    weight 1 / ||D^-1 A||_inf for k = 0; for k = 1, 2 smoother = "default":
    additive vertex stars (weight 1/8), "hiptmair": the paper's
    Hiptmair-Jacobi relaxation (damped Jacobi on A, then damped Jacobi on
    the potential operator G^T A G through the discrete gradient or curl G),
    "jacobi": damped Jacobi on A alone (no potential correction; for
    comparison)."""

    def __init__(self, problem: Problem, mode: str = "exact", smoother: str = "default"):
        X = problem.mesh.X
        self.mode = mode
        self.smoother = smoother if problem.k >= 1 else "default"
        self.cp = Problem(problem.k, problem.n, 1, X, problem.alpha, problem.beta, problem.bc)
        P0 = prolongation(problem.lat, self.cp.lat)
        self.R0T = P0[problem.free][:, self.cp.free].tocsr()
        A0 = self.cp.A_free().tocsr()
        self.A0 = A0.toarray()
        if mode == "exact":
            self.A0_chol = scipy.linalg.cho_factor(self.A0, lower=True)
            return
        self.levels = []
        A, lat, free, n = A0, self.cp.lat, self.cp.free, list(problem.n)
        while all(v % 2 == 0 and v >= 4 for v in n) and A.shape[0] > 512:
            nh = [v // 2 for v in n]
            lat_h = Lattice(problem.k, tuple(nh), 1, problem.bc)
            free_h = lat_h.free()
            P = refinement(lat, lat_h)[free][:, free_h].tocsr()
            D = A.diagonal()
            omega = 1.0 / np.max(np.asarray(abs(A).sum(1)).ravel() / D)
            star = None
            if problem.k >= 1 and self.smoother == "hiptmair":
                star = self._hiptmair_level(problem.k, A, lat, free, tuple(n))
            elif problem.k >= 1 and self.smoother != "jacobi":
                pos = free_position(free, lat.size)
                star = PatchSolver(A, [pos[s] for s in patch_lists(lat, (), free)], "chol")
            self.levels.append((A, P, omega / D, star))
            A = (P.T @ A @ P).tocsr()
            lat, free, n = lat_h, free_h, nh
        self.A_last = A.toarray()

    @staticmethod
    def _hiptmair_level(k, A, lat, free, n):
        """Hiptmair-Jacobi data of one level (the paper's p-coarse relaxation,
        Sec. 5.1 and its solver diagram): the discrete gradient (k = 1) or curl
        (k = 2) G from the level's V^{k-1}_{h,1} into its V^k_{h,1}, the
        potential operator B = G^T A G and the damped Jacobi weights of A and
        of B (omega = 1 / ||D^-1 M||_inf each)."""
        lat0 = Lattice(k - 1, n, 1, lat.bc)
        free0 = lat0.free()
        G = discrete_derivative(k - 1, lat0, lat)[free][:, free0].tocsr()
        B = (G.T @ A @ G).tocsr()
        Db = B.diagonal()
        wb = 1.0 / np.max(np.asarray(abs(B).sum(1)).ravel() / Db) / Db
        return ("hiptmair", G, wb)

    def _hiptmair_sweep(self, A, w, G, wb, b, x, space_first):
        """One multiplicative Hiptmair-Jacobi sweep: damped Jacobi on A, then
        damped Jacobi on the potential, x += G W_B G^T (b - A x) (reversed
        for the post-smoother, so that the cycle stays symmetric)."""
        def space(x):
            return x + w * (b - A @ x)

        def potential(x):
            return x + G @ (wb * (G.T @ (b - A @ x)))
        return potential(space(x)) if space_first else space(potential(x))

    def _vcycle(self, l, b):
        if l == len(self.levels):
            return np.linalg.solve(self.A_last, b)
        A, P, w, star = self.levels[l]
        if isinstance(star, tuple):
            _, G, wb = star
            x = np.zeros_like(b)
            for _ in range(2):
                x = self._hiptmair_sweep(A, w, G, wb, b, x, True)
            x = x + P @ self._vcycle(l + 1, P.T @ (b - A @ x))
            for _ in range(2):
                x = self._hiptmair_sweep(A, w, G, wb, b, x, False)
            return x
        if star is not None:
            # H(curl)/H(div): additive vertex-star smoother (Arnold-Falk-Winther),
            # weight 1/8 (at most 8 stars overlap a DOF)
            om = 0.125
            x = om * star.apply(b)
            x = x + om * star.apply(b - A @ x)
            x = x + P @ self._vcycle(l + 1, P.T @ (b - A @ x))
            x = x + om * star.apply(b - A @ x)
            return x + om * star.apply(b - A @ x)
        x = w * b
        x = x + w * (b - A @ x)
        x = x + P @ self._vcycle(l + 1, P.T @ (b - A @ x))
        x = x + w * (b - A @ x)
        return x + w * (b - A @ x)

    def apply(self, r):
        c = self.R0T.T @ r
        if self.mode == "exact":
            return self.R0T @ scipy.linalg.cho_solve(self.A0_chol, c)
        return self.R0T @ self._vcycle(0, c)


# ---------------------------------------------------------------------------
# static condensation
# ---------------------------------------------------------------------------
def interior_mask(lat: Lattice, free):
    """Free DOFs interior to a cell: no s-type index on a mesh plane."""
    geo = DofGeometry(lat)
    return ~geo.vtx[free].any(1)


class Condensed:
    """Block split of a free-DOF matrix P into interior I and interface G,
    with S = P_GG - P_GI P_II^{-1} P_IG (Eqs. LDU, schur)."""

    def __init__(self, P: sp.csr_matrix, lat: Lattice, free):
        self.free = free
        imask = interior_mask(lat, free)
        self.I = np.flatnonzero(imask)
        self.G = np.flatnonzero(~imask)
        P = P.tocsc()
        self.PII = P[self.I][:, self.I].tocsc()
        self.PIG = P[self.I][:, self.G].tocsc()
        self.PGI = P[self.G][:, self.I].tocsr()
        PGG = P[self.G][:, self.G].tocsr()
        # P_II is block diagonal (blocks of at most d x d, Remark after Eq.
        # schur): factor it block by block on its connected components
        # (couplings below 1e-13 sqrt(|P_ii P_jj|) are quadrature round-off),
        # P_II = L L^T.  Then P_II^{-1} = L^{-T} L^{-1} and
        # S = P_GG - W^T W with W = L^{-1} P_IG: the quantities of Eq. schur,
        # formed so that they stay symmetric positive definite in floating
        # point when P_II is ill conditioned (beta << alpha: its interior
        # gradients or curls are nearly singular), where an explicit inverse
        # in P_GI P_II^{-1} P_IG loses both properties.
        PIId = self.PII.tocsr()
        dg = np.sqrt(np.abs(PIId.diagonal()))
        C = PIId.tocoo()
        keep = np.abs(C.data) > 1e-13 * dg[C.row] * dg[C.col]
        graph = sp.csr_matrix((np.ones(keep.sum()), (C.row[keep], C.col[keep])),
                              shape=PIId.shape)
        ncomp, lab = sp.csgraph.connected_components(graph, directed=False)
        rows, cols, vals, lvals = [], [], [], []
        for c in range(ncomp):
            ix = np.flatnonzero(lab == c)
            L = np.linalg.cholesky(PIId[ix][:, ix].toarray())
            Li = scipy.linalg.solve_triangular(L, np.eye(len(ix)), lower=True)
            Bi = Li.T @ Li
            rows.append(np.repeat(ix, len(ix)))
            cols.append(np.tile(ix, len(ix)))
            vals.append((0.5 * (Bi + Bi.T)).ravel())   # symmetric to the last bit
            lvals.append(Li.ravel())
        nI = len(self.I)
        r_, c_ = np.concatenate(rows), np.concatenate(cols)
        self.PII_inv = sp.csr_matrix((np.concatenate(vals), (r_, c_)), shape=(nI, nI))
        Linv = sp.csr_matrix((np.concatenate(lvals), (r_, c_)), shape=(nI, nI))
        W = (Linv @ self.PIG).tocsr()
        self.S = (PGG - (W.T @ W)).tocsr()
        # the harmonic extension E = P_GI P_II^{-1} as one matrix, used with
        # its exact transpose in condense and expand: the condensed
        # preconditioner [[P_II^-1 + E^T M E, -E^T M], [-M E, M]] is then
        # symmetric in floating point too (applying P_II^{-1} and P_IG in
        # sequence leaves an asymmetry amplified by cond(P_II), 1e11 at
        # beta / alpha = 1e-8, which CG does not survive)
        self.E = (self.PGI @ self.PII_inv).tocsr()
        self.Et = self.E.T.tocsr()

    def condense(self, r):
        """(y_I, R_G r) with y_I = P_II^{-1} r_I and R_G r = r_G - E r_I."""
        yI = self.PII_inv @ r[self.I]
        return yI, r[self.G] - self.E @ r[self.I]

    def expand(self, yI, zG):
        """z = R_I^T y_I + R_G^T z_G, written as [y_I - E^T z_G; z_G]."""
        z = np.zeros(len(self.free))
        z[self.I] = yI - self.Et @ zG
        z[self.G] = zG
        return z


# ---------------------------------------------------------------------------
# preconditioners (free-DOF numbering)
# ---------------------------------------------------------------------------
def free_position(free, size):
    pos = -np.ones(size, int)
    pos[free] = np.arange(len(free))
    return pos


class PAFW:
    """Non-condensed PAFW, Eq. asm-afw: sum over vertex stars of A_v^{-1}
    (exact Cholesky or ICC(0) of R_v M R_v^T), optionally plus the coarse
    correction."""

    def __init__(self, problem: Problem, M=None, factor="chol", coarse=True):
        self.problem = problem
        free = problem.free
        M = problem.A_free() if M is None else M
        pos = free_position(free, problem.lat.size)
        pats = patch_lists(problem.lat, (), free)
        self.patches = PatchSolver(M, [pos[s] for s in pats], factor)
        self.coarse = (Coarse(problem, coarse if isinstance(coarse, str) else "exact")
                       if coarse else None)

    def smooth(self, r):
        return self.patches.apply(r)

    def apply(self, r):
        z = self.smooth(r)
        if self.coarse is not None:
            z += self.coarse.apply(r)
        return z


class SCPAFW:
    """SC-PAFW (Eqs. sc-pafw, sc-asm-afw) on the auxiliary operator P:
    interior solve + harmonic extension of sum_v S_v^{-1}, plus coarse."""

    def __init__(self, problem: Problem, P_free, factor="icc", coarse=True):
        self.problem = problem
        free = problem.free
        self.sc = Condensed(P_free, problem.lat, free)
        pos = free_position(free[self.sc.G], problem.lat.size)
        pats = patch_lists(problem.lat, (), free[self.sc.G])
        self.patches = PatchSolver(self.sc.S, [pos[s] for s in pats], factor)
        self.coarse = (Coarse(problem, coarse if isinstance(coarse, str) else "exact")
                       if coarse else None)

    def smooth(self, r):
        yI, rG = self.sc.condense(r)
        return self.sc.expand(yI, self.patches.apply(rG))

    def apply(self, r):
        z = self.smooth(r)
        if self.coarse is not None:
            z += self.coarse.apply(r)
        return z


def discrete_derivative(kk: int, lat_a: Lattice, lat_b: Lattice) -> sp.csr_matrix:
    """d^kk: V^kk lattice -> V^{kk+1} lattice (full lattices), cellwise
    D-hat_3d (the gradient for kk = 0, the curl for kk = 1)."""
    from .discretization import dhat_3d
    Dl = dhat_3d(kk, FDM1D(lat_a.p))
    entries = {}
    for cell, _ in lat_a.cells():
        da = lat_a.cell_dofs(cell)
        db = lat_b.cell_dofs(cell)
        nz = np.nonzero(Dl)
        for i, j in zip(*nz):
            entries[(int(db[i]), int(da[j]))] = Dl[i, j]
    r = np.array([k[0] for k in entries], int)
    c = np.array([k[1] for k in entries], int)
    v = np.array(list(entries.values()))
    return sp.coo_matrix((v, (r, c)), shape=(lat_b.size, lat_a.size)).tocsr()


def discrete_gradient(lat0: Lattice, lat1: Lattice) -> sp.csr_matrix:
    """D: V^0 lattice -> V^1 lattice (full lattices), cellwise D-hat_3d."""
    return discrete_derivative(0, lat0, lat1)


# eps of the H(div) potential operator B_eps = (curl phi, beta curl psi) +
# eps (phi, beta psi): the Remark after Eq. ph adds "a small multiple of the
# mass matrix" to the singular curl-curl patch matrices without giving it
HDIV_POTENTIAL_EPS = 1e-2


class SCPH:
    """SC-PH (Eqs. sc-ph, sc-asm-hiptmair) for H(curl) and H(div): stars of
    the k-dimensional entities on S (exact Cholesky; edge stars for H(curl),
    face stars for H(div), where the face-star blocks of S are diagonal and
    the relaxation is point-Jacobi on S, Sec. 4.5), plus the potential term
    D-tilde (sum_j B-tilde_j^{-1}) D-tilde^T on the stars of the
    (k-1)-dimensional entities (vertex stars of V^0 for H(curl), edge stars of
    V^1 for H(div)) with B = (d phi, beta d psi) (Sec. 4.3) -- for H(div) plus
    eps (phi, beta psi), the Remark on its singular potential problem --
    built as the auxiliary operator of V^{k-1} with mass coefficient 0 (H(curl))
    or eps beta (H(div)) and derivative coefficient beta; interior solve,
    harmonic extension and coarse correction as in SC-PAFW."""

    def __init__(self, problem: Problem, P_free, edge_factor="chol",
                 vertex_factor="icc", coarse=True, eps=HDIV_POTENTIAL_EPS):
        from .auxiliary import assemble_aux
        k = problem.k
        assert k in (1, 2)
        self.problem = problem
        lat1 = problem.lat
        free1 = problem.free
        self.sc = Condensed(P_free, lat1, free1)
        G1 = free1[self.sc.G]
        pos1 = free_position(G1, lat1.size)
        self.edge = []
        for m in range(3):
            span = (m,) if k == 1 else tuple(d for d in range(3) if d != m)
            pats = patch_lists(lat1, span, G1)
            self.edge.append(PatchSolver(self.sc.S, [pos1[s] for s in pats],
                                         edge_factor))
        # potential space V^{k-1}
        p0 = Problem(k - 1, problem.n, problem.p, problem.mesh.X,
                     problem.alpha, problem.beta, problem.bc)
        mass = np.zeros_like(problem.beta) if k == 1 else eps * problem.beta
        B = assemble_aux(p0, mass_coef=mass, stiff_coef=problem.beta)
        self.B = B
        free0 = p0.free
        self.sc0 = Condensed(B[free0][:, free0].tocsr(), p0.lat, free0)
        G0 = free0[self.sc0.G]
        pos0 = free_position(G0, p0.lat.size)
        spans0 = [()] if k == 1 else [(m,) for m in range(3)]
        self.potential = [PatchSolver(self.sc0.S, [pos0[s] for s in patch_lists(p0.lat, sp0, G0)],
                                      vertex_factor) for sp0 in spans0]
        self.vertex = self.potential[0] if k == 1 else None
        D = discrete_derivative(k - 1, p0.lat, lat1)
        self.Dt = D[G1][:, G0].tocsr()
        self.coarse = (Coarse(problem, coarse if isinstance(coarse, str) else "exact")
                       if coarse else None)

    def interface(self, rG):
        z = np.zeros_like(rG)
        for ps in self.edge:
            z += ps.apply(rG)
        u = self.Dt.T @ rG
        v = np.zeros_like(u)
        for ps in self.potential:
            v += ps.apply(u)
        z += self.Dt @ v
        return z

    def smooth(self, r):
        yI, rG = self.sc.condense(r)
        return self.sc.expand(yI, self.interface(rG))

    def apply(self, r):
        z = self.smooth(r)
        if self.coarse is not None:
            z += self.coarse.apply(r)
        return z


class Hybrid:
    """Hybrid multigrid/Schwarz V(1,1) (Sec. 5): smoother omega*M^{-1}
    (additive fine-level relaxation), exact coarse solve in between."""

    def __init__(self, A, relax, coarse: Coarse, omega: float):
        self.A, self.relax, self.coarse, self.omega = A, relax, coarse, omega

    def apply(self, r):
        z = self.omega * self.relax.smooth(r)
        z = z + self.coarse.apply(r - self.A @ z)
        return z + self.omega * self.relax.smooth(r - self.A @ z)
