"""Pins of the oracle's 1D FDM basis against textbook values and the
properties the paper fixes (Sec. 2.2-2.3)."""

import numpy as np
import pytest

from oracle.basis import FDM1D, gauss_rule, gll_nodes, gll_rule, lagrange


def test_gll_nodes_textbook():
    # Gauss-Lobatto nodes: p=2 {0}, p=3 {+-1/sqrt5}, p=4 {0, +-sqrt(3/7)}
    assert np.allclose(gll_nodes(2), [-1, 0, 1], atol=1e-15)
    assert np.allclose(gll_nodes(3), [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1], atol=1e-15)
    assert np.allclose(gll_nodes(4), [-1, -np.sqrt(3 / 7), 0, np.sqrt(3 / 7), 1], atol=1e-15)


def test_gll_weights_textbook():
    _, w3 = gll_rule(3)
    assert np.allclose(w3, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    _, w4 = gll_rule(4)
    assert np.allclose(w4, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    # exact for degree 2q-3
    for q in range(3, 12):
        x, w = gll_rule(q)
        for deg in range(0, 2 * q - 2):
            exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
            assert abs(np.sum(w * x ** deg) - exact) < 1e-13


def test_lagrange_p1_closed_form():
    L, dL = lagrange(np.array([-1.0, 1.0]), np.array([-0.3, 0.7]))
    assert np.allclose(L, [[0.65, 0.35], [0.15, 0.85]])
    assert np.allclose(dL, [[-0.5, 0.5], [-0.5, 0.5]])
    e = FDM1D(1)
    assert np.allclose(e.Bgll, [[2 / 3, 1 / 3], [1 / 3, 2 / 3]], atol=1e-15)
    assert np.allclose(e.Agll, [[0.5, -0.5], [-0.5, 0.5]], atol=1e-15)


@pytest.mark.parametrize("p", [2, 3, 4, 7, 10, 12])
def test_bhat_structure(p):
    """B-hat: identity on the interior, zero interior-interface block, the
    only off-diagonal entry at (0, p) (Sec. 2.2, after Eq. unisolvence)."""
    B = FDM1D(p).Bhat
    I = np.arange(1, p)
    assert np.allclose(B[np.ix_(I, I)], np.eye(p - 1), atol=1e-12)
    assert np.abs(B[np.ix_(I, [0, p])]).max() < 1e-12
    assert abs(B[0, p]) > 1e-5 and abs(B[0, p] - B[p, 0]) < 1e-14


@pytest.mark.parametrize("p", [2, 3, 4, 7, 10, 12])
def test_ahat_interior_diagonal(p):
    """A-hat_II = Lambda (Eq. eigs); A-hat is an arrowhead."""
    e = FDM1D(p)
    I = np.arange(1, p)
    AII = e.Ahat[np.ix_(I, I)]
    assert np.abs(AII - np.diag(e.lam[1:])).max() < 1e-12 * e.lam[-1]
    assert np.all(np.diff(e.lam[1:]) > 0)


@pytest.mark.parametrize("p", [2, 3, 5, 8])
def test_duality_and_traces(p):
    """Eq. unisolvence evaluated with an independent Gauss rule on the
    tabulated functions: s_i(+-1) = 0 for interior i, s_0(-1)=1, s_0(1)=0,
    (s_i, s_0) = (s_i, s_p) = 0, (s_i, s_j) = delta_ij."""
    e = FDM1D(p)
    ends = e.s(np.array([-1.0, 1.0]))
    assert np.allclose(ends[:, 1:p], 0.0, atol=1e-13)
    assert np.allclose(ends[:, [0, p]], np.eye(2), atol=1e-13)
    xg, wg = gauss_rule(2 * p + 4)
    s = e.s(xg)
    Mf = s.T @ (wg[:, None] * s)
    I = np.arange(1, p)
    assert np.allclose(Mf[np.ix_(I, I)], np.eye(p - 1), atol=1e-12)
    assert np.abs(Mf[np.ix_(I, [0, p])]).max() < 1e-12
    # sign reading: s_j'(-1) > 0
    assert np.all(e.ds(np.array([-1.0]))[0, 1:p] > 0)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 7, 8, 11])
def test_reflection_parity(p):
    """Under x -> -x the interface pair swaps, s_p(x) = s_0(-x); the interior
    s_j (the j-th eigenfunction of the interior eigenproblem, Eq. eigs) is
    even for odd j and odd for even j; r_i is even for even i (r_0 constant,
    r_j proportional to s_j').  The reflection split of the interpolations
    at the mirrored GLL points rests on this structure (Sec. 2.2-2.3)."""
    e = FDM1D(p)
    x = np.random.default_rng(1).uniform(-1, 1, 23)
    s, sm = e.s(x), e.s(-x)
    assert np.allclose(sm[:, p], s[:, 0], atol=1e-12)
    assert np.allclose(sm[:, 0], s[:, p], atol=1e-12)
    for j in range(1, p):
        sign = 1.0 if j % 2 == 1 else -1.0
        assert np.allclose(sm[:, j], sign * s[:, j], atol=1e-11 * np.abs(s[:, j]).max())
    r, rm = e.r(x), e.r(-x)
    for i in range(p):
        sign = 1.0 if i % 2 == 0 else -1.0
        assert np.allclose(rm[:, i], sign * r[:, i], atol=1e-11 * np.abs(r[:, i]).max())


@pytest.mark.parametrize("p", [1, 2, 4, 7, 11])
def test_r_orthonormal(p):
    """r-hat is L2-orthonormal, (r_0, r_j) = 0 (Sec. 2.3)."""
    e = FDM1D(p)
    xg, wg = gauss_rule(2 * p + 4)
    r = e.r(xg)
    assert np.allclose(r.T @ (wg[:, None] * r), np.eye(p), atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 4, 7, 11])
def test_dhat_sparsity_and_derivative(p):
    """D-hat_ij = (r_i, s_j'): interior columns hold lam_j^{1/2} on row j
    only; row 0 is (-2^{-1/2}, 0, ..., 0, 2^{-1/2}) (fig. fdmbasis(c));
    s_j' = sum_i D_ij r_i pointwise."""
    e = FDM1D(p)
    D = e.D
    for j in range(1, p):
        col = D[:, j].copy()
        assert abs(col[j] - np.sqrt(e.lam[j])) < 1e-12 * np.sqrt(e.lam[j])
        col[j] = 0.0
        assert np.abs(col).max() < 1e-12
    h = 1 / np.sqrt(2)
    assert np.allclose(D[0], np.r_[-h, np.zeros(p - 1), h], atol=1e-13)
    x = np.random.default_rng(0).uniform(-1, 1, 17)
    assert np.allclose(e.ds(x), e.r(x) @ D, atol=1e-11)


def test_lambda1_rayleigh_ritz():
    """lam_j(p) are Rayleigh-Ritz upper bounds of the Dirichlet eigenvalues
    (j pi / 2)^2 of -u'' on [-1, 1], non-increasing in p, -> pi^2/4."""
    prev = np.inf
    for p in range(2, 16):
        lam = FDM1D(p).lam[1:]
        exact = (np.arange(1, p) * np.pi / 2) ** 2
        assert np.all(lam >= exact * (1 - 1e-12))
        assert lam[0] <= prev + 1e-12
        prev = lam[0]
    assert abs(prev - np.pi ** 2 / 4) < 1e-10


@pytest.mark.parametrize("p", [1, 2, 3, 6])
def test_injection_reproduces_p1(p):
    """The p=1 hats and r_0 are reproduced exactly by their FDM-P_p
    coefficients (the coarse injection V_{h,1} in V_{h,p})."""
    e = FDM1D(p)
    Js, Jr = e.injection_from_p1()
    x = np.linspace(-1, 1, 13)
    hats = np.stack([(1 - x) / 2, (1 + x) / 2], 1)
    assert np.allclose(e.s(x) @ Js, hats, atol=1e-13)
    assert np.allclose(e.r(x) @ Jr, 1 / np.sqrt(2), atol=1e-13)
