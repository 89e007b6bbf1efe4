"""Pins of the oracle's spaces, element matrices and assembly (Sec. 2.4, 3.1)."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.basis import FDM1D, gll_rule
from oracle.discretization import (Lattice, Problem, ReferenceElement,
                                   dhat_3d, element_matrix, kron3,
                                   quadrature_points)
from oracle.relaxation import discrete_gradient, prolongation
from paper_2211_14284_gb300 import inputs


def _random_points(m=11, seed=0):
    x = np.random.default_rng(seed).uniform(-1, 1, m)
    return x, np.full(m, 1.0)


@pytest.mark.parametrize("k", [0, 1, 2])
@pytest.mark.parametrize("p", [1, 2, 4])
def test_dhat_commutes_with_tabulation(k, p):
    """Reference values of d^k psi (tabulated derivatives) equal the V^{k+1}
    tabulation of D-hat coefficients: the sum-factorisation of Eq.
    sum-factorization rests on this."""
    x, w = _random_points()
    rk = ReferenceElement(k, p, x, w)
    rk1 = ReferenceElement(k + 1, p, x, w)
    D = dhat_3d(k, rk.e)
    lhs = rk.dvalues
    rhs = np.einsum("qaj,jk->qak", rk1.values, D)
    assert np.abs(lhs - rhs).max() < 1e-10


@pytest.mark.parametrize("p", [3, 5])
def test_complete_sequence_interior(p):
    """Eqs. gradbasis, curlbasis, divbasis for interior indices."""
    x, w = _random_points(7)
    e = FDM1D(p)
    r0 = ReferenceElement(0, p, x, w)
    r1 = ReferenceElement(1, p, x, w)
    r2 = ReferenceElement(2, p, x, w)
    r3 = ReferenceElement(3, p, x, w)
    L1 = Lattice(1, 1, p)
    L2 = Lattice(2, 1, p)
    sq = np.sqrt(e.lam)

    def idx(lat, m, i, j, l):
        n1, n2, _ = lat.loc_dims[m]
        return lat.loc_offsets[m] + i + n1 * (j + n2 * l)

    for (i, j, l) in [(1, 1, 1), (1, 2, p - 1), (p - 1, 1, 2)]:
        psi = i + (p + 1) * (j + (p + 1) * l)
        g = r0.dvalues[:, :, psi]
        want = (sq[i] * r1.values[:, :, idx(L1, 0, i, j, l)]
                + sq[j] * r1.values[:, :, idx(L1, 1, i, j, l)]
                + sq[l] * r1.values[:, :, idx(L1, 2, i, j, l)])
        assert np.abs(g - want).max() < 1e-10
        # curl (f e1) = (0, d3 f, -d2 f), so curl Psi^(1) =
        # lam_l^{1/2} Phi^(2) - lam_j^{1/2} Phi^(3).  Eq. curlbasis prints the
        # opposite global sign; the standard curl is taken here.
        c = r1.dvalues[:, :, idx(L1, 0, i, j, l)]
        want = (sq[l] * r2.values[:, :, idx(L2, 1, i, j, l)]
                - sq[j] * r2.values[:, :, idx(L2, 2, i, j, l)])
        assert np.abs(c - want).max() < 1e-10
        # div Phi^(2) = lam_j^{1/2} phi
        dv = r2.dvalues[:, :, idx(L2, 1, i, j, l)]
        phi = r3.values[:, :, i + p * (j + p * l)]
        assert np.abs(dv - sq[j] * phi).max() < 1e-10


def _box(h, origin=(0.1, 0.2, 0.3)):
    V = np.zeros((8, 3))
    for c3 in range(2):
        for c2 in range(2):
            for c1 in range(2):
                V[c1 + 2 * c2 + 4 * c3] = np.array(origin) + np.array([c1, c2, c3]) * h
    return V


@pytest.mark.parametrize("p", [1, 3, 5])
def test_cartesian_hgrad_kronecker(p):
    """On a box cell A^0_K = beta detJ B(x)B(x)B + alpha detJ sum_d (2/h_d)^2
    (A-hat in d, B-hat elsewhere) (Sec. 2.2: Kronecker products of the 1D
    mass and stiffness)."""
    h = np.array([0.5, 0.25, 1 / 3])
    alpha, beta = 2.0, 3.0
    ref = ReferenceElement(0, p, *gll_rule(quadrature_points(p)))
    A = element_matrix(ref, _box(h), alpha, beta)
    e = FDM1D(p)
    B, Ah = e.Bhat, e.Ahat
    det = np.prod(h / 2)
    K = beta * det * kron3(B, B, B)
    K += alpha * det * (2 / h[0]) ** 2 * kron3(B, B, Ah)
    K += alpha * det * (2 / h[1]) ** 2 * kron3(B, Ah, B)
    K += alpha * det * (2 / h[2]) ** 2 * kron3(Ah, B, B)
    assert np.abs(A - K).max() < 1e-12 * np.abs(K).max()


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("p", [1, 3, 4])
def test_cartesian_hcurl_hdiv_kronecker(k, p):
    """On a box cell the k-form mass is diagonal across components with
    1D factors B-hat (s-type) and I (r-type, orthonormal), and the
    derivative term is D-hat^T M^{k+1} D-hat (Eq. sum-factorization)."""
    h = np.array([0.5, 0.25, 1 / 3])
    alpha, beta = 2.0, 3.0
    ref = ReferenceElement(k, p, *gll_rule(quadrature_points(p)))
    A = element_matrix(ref, _box(h), alpha, beta)
    e = FDM1D(p)
    det = np.prod(h / 2)

    def mass(kk, coef):
        from oracle.discretization import SPACE_TYPES
        import scipy.linalg
        blocks = []
        types = SPACE_TYPES[kk]
        for m, t in enumerate(types):
            T = [e.Bhat if t[d] == "s" else np.eye(p) for d in range(3)]
            if kk == 1:
                s = det * (2 / h[m]) ** 2
            elif kk == 2:
                s = (h[m] / 2) ** 2 / det
            else:
                s = 1 / det
            blocks.append(coef * s * kron3(T[2], T[1], T[0]))
        return scipy.linalg.block_diag(*blocks)

    D = dhat_3d(k, e)
    K = mass(k, beta) + D.T @ mass(k + 1, alpha) @ D
    assert np.abs(A - K).max() < 1e-12 * np.abs(K).max()


@pytest.mark.parametrize("k,bound", [(0, 1), (1, 3), (2, 3)])
def test_interior_block_sparsity(k, bound):
    """Cartesian interior block: 1 nonzero per row (k=0) or <= d = 3 per row
    (k=1,2), end of Sec. 2.4."""
    p = 4
    ref = ReferenceElement(k, p, *gll_rule(quadrature_points(p)))
    A = element_matrix(ref, _box(np.array([0.3, 0.5, 0.7])), 1.3, 0.7)
    lat = Lattice(k, 1, p)
    interior = []
    for m, t in enumerate(lat.types):
        l1, l2, l3 = lat.loc_dims[m]
        for i3 in range(l3):
            for i2 in range(l2):
                for i1 in range(l1):
                    ii = (i1, i2, i3)
                    if all(t[d] == "r" or 0 < ii[d] < p for d in range(3)):
                        interior.append(lat.loc_offsets[m] + i1 + l1 * (i2 + l2 * i3))
    AII = A[np.ix_(interior, interior)]
    nnz = (np.abs(AII) > 1e-12 * np.abs(A).max()).sum(1)
    assert nnz.max() <= bound


def test_curl_grad_and_div_curl_vanish_distorted():
    """With beta = 0 on a distorted cell, A^1 D-hat_grad = 0 and
    A^2 D-hat_curl = 0: the pullbacks commute with d (Eq. commutativity)."""
    p = 3
    V = _box(np.array([1.0, 1.0, 1.0]))
    V += np.random.default_rng(3).uniform(-0.15, 0.15, V.shape)
    e = FDM1D(p)
    for k in (1, 2):
        ref = ReferenceElement(k, p, *gll_rule(quadrature_points(p)))
        A = element_matrix(ref, V, 1.0, 0.0)
        D = dhat_3d(k - 1, e)
        assert np.abs(A @ D).max() < 1e-11 * np.abs(A).max()


def test_linear_function_in_kernel_of_stiffness():
    """beta = 0, distorted mesh: a globally linear u = c.x lies in Q_1 and
    (grad psi_i, grad u) = 0 for every free psi_i (divergence theorem)."""
    n, p = 3, 3
    X = inputs.vertices(n, perturb=0.2, seed=11)
    pr = Problem(0, n, p, X, 1.0, 0.0)
    A = pr.assemble()
    lat1 = Lattice(0, n, 1)
    c = np.array([0.3, -1.2, 0.7])
    u1 = X @ c      # Q1 vertex values = nodal coefficients at p = 1
    u = prolongation(pr.lat, lat1) @ u1
    r = (A @ u)[pr.free]
    assert np.abs(r).max() < 1e-12 * np.abs(A).max()


def test_global_discrete_gradient_kernel():
    """A^1 D = M^1_beta D on a distorted mesh when alpha-terms vanish:
    with beta = 0 the global H(curl) operator annihilates discrete gradients."""
    n, p = 2, 3
    X = inputs.vertices(n, perturb=0.1, seed=5)
    p1 = Problem(1, n, p, X, 1.0, 0.0)
    D = discrete_gradient(Lattice(0, n, p), p1.lat)
    A = p1.assemble()
    AD = A @ D
    assert abs(AD).max() < 1e-11 * abs(A).max()


def _solve_sin(n, p, perturb):
    X = inputs.vertices(n, perturb=perturb, seed=7)
    pr = Problem(0, n, p, X, 1.0, 1.0)
    u = lambda x: np.prod(np.sin(np.pi * x), axis=1)
    f = lambda x: (1 + 3 * np.pi ** 2) * u(x)
    b = pr.load_vector_hgrad(f)
    x = np.zeros(pr.lat.size)
    x[pr.free] = spla.spsolve(pr.A_free().tocsc(), b[pr.free])
    return pr.l2_error_hgrad(x, u)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("perturb", [0.0, 0.1])
def test_l2_convergence_order(p, perturb):
    """||u - u_h||_L2 = O(h^{p+1}) for the sin-product solution."""
    errs = [_solve_sin(n, p, perturb) for n in (2, 4, 8)]
    rate = np.log2(errs[-2] / errs[-1])
    assert rate > p + 1 - 0.35, (errs, rate)


# -- natural boundary conditions (Gamma_D empty) ------------------------------
@pytest.mark.parametrize("bc", ["none", "dirichlet"])
def test_kernel_dimensions_follow_the_sequence(bc):
    """With beta = 0 the kernel of a^k is d^{k-1} V^{k-1}, whose dimension the
    exactness of the discrete de Rham sequence on the cube fixes (Sec. 2.4):
    H(grad): the constants (Gamma_D empty) or nothing (Dirichlet); H(curl):
    dim V^0 - dim ker grad; H(div): dim V^1 - dim ker curl.  Counting them
    checks which boundary entries are DOFs under each condition."""
    from oracle.discretization import Problem
    n, p = 2, 2
    X = inputs.vertices(n, perturb=0.1, seed=3)
    dims = {}
    for k in (0, 1, 2):
        pr = Problem(k, n, p, X, 1.0, 0.0, bc=bc)
        A = pr.A_free().toarray()
        ev = np.linalg.eigvalsh(A)
        dims[k] = (len(pr.free), int(np.sum(ev < 1e-10 * ev.max())))
    ker0 = 1 if bc == "none" else 0
    assert dims[0][1] == ker0
    assert dims[1][1] == dims[0][0] - ker0
    assert dims[2][1] == dims[1][0] - dims[1][1]
    if bc == "none":
        # every lattice entry is a DOF
        assert dims[0][0] == (n * p + 1) ** 3


@pytest.mark.parametrize("k", [0, 1, 2])
def test_natural_bc_operator_is_definite(k):
    """Gamma_D empty with beta > 0: A is symmetric positive definite."""
    from oracle.discretization import Problem
    n, p = 2, 2
    X = inputs.vertices(n, perturb=0.1, seed=4)
    be = inputs.loguniform_coefficient(n, 1e-3, 1.0, seed=5)
    pr = Problem(k, n, p, X, 1.0, be, bc="none")
    A = pr.A_free().toarray()
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


def test_neumann_manufactured_convergence():
    """Gamma_D empty, H(grad): u = cos(pi x) cos(pi y) cos(pi z) has zero
    normal derivative on the cube, so it solves u - div grad u = (1 + 3 pi^2) u
    with natural boundary conditions; the L2 error falls at order p + 1
    (boundary entries solved for, not fixed)."""
    import scipy.sparse.linalg as spla
    from oracle.discretization import Problem
    u = lambda x: np.prod(np.cos(np.pi * x), axis=1)
    for p in (1, 2):
        errs = []
        for n in (2, 4):
            pr = Problem(0, n, p, inputs.vertices(n), 1.0, 1.0, bc="none")
            b = pr.load_vector_hgrad(lambda x: (1 + 3 * np.pi ** 2) * u(x))
            xh = spla.spsolve(pr.A_free().tocsc(), b)
            errs.append(pr.l2_error_hgrad(xh, u))
        order = np.log2(errs[0] / errs[1])
        assert order > p + 1 - 0.35, (p, errs, order)
