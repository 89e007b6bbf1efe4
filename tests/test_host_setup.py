"""CPU checks of the CUDA path's host FP64 setup (librm_host.so) against the
oracle: 1D basis, auxiliary operator, Schur complement, patch lists and
factors, coarse operator.  No GPU needed; the oracle only supplies expected
values."""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.auxiliary import assemble_aux
from oracle.basis import FDM1D
from oracle.discretization import Lattice, Problem
from oracle.relaxation import (Coarse, Condensed, cholesky, discrete_gradient,
                               icc0, patch_lists)
from paper_2211_14284_gb300 import inputs
from paper_2211_14284_gb300.rm import HostProbe


@pytest.fixture(scope="module")
def probe():
    return HostProbe()


@pytest.mark.parametrize("p", [1, 2, 3, 4, 7, 10, 12])
def test_basis_matches_oracle(probe, p):
    h = probe.basis(p)
    e = FDM1D(p)
    assert np.abs(h["S"] - e.S).max() < 1e-12
    assert np.abs(h["lam"] - e.lam).max() < 1e-11 * e.lam.max()
    assert np.abs(h["Bhat"] - e.Bhat).max() < 1e-12
    assert np.abs(h["Ahat"] - e.Ahat).max() < 1e-11 * np.abs(e.Ahat).max()
    assert np.abs(h["D"] - e.D).max() < 1e-11 * np.abs(e.D).max()
    Js, _ = e.injection_from_p1()
    assert np.abs(h["Js"] - Js).max() < 1e-12


def _csr_dense(ptr, col, val, n):
    return sp.csr_matrix((val, col, ptr), shape=(n, n)).toarray()


def _case(k, n, p, perturb, seed=3, coef=False):
    X = inputs.vertices(n, perturb=perturb, seed=seed)
    if coef:
        al = inputs.loguniform_coefficient(n, 0.1, 10, seed=seed + 1)
        be = inputs.loguniform_coefficient(n, 0.1, 10, seed=seed + 2)
    else:
        al = inputs.constant_coefficient(n, 1.0)
        be = inputs.constant_coefficient(n, 1.0)
    return X, al, be, Problem(k, n, p, X, al, be)


@pytest.mark.parametrize("k,p,perturb,coef", [(0, 3, 0.15, True), (1, 2, 0.15, False),
                                              (2, 2, 0.1, True), (0, 4, 0.0, False)])
def test_aux_and_schur_match_oracle(probe, k, p, perturb, coef):
    n = 2
    X, al, be, pr = _case(k, n, p, perturb, coef=coef)
    probe.build(k, n, p, X, al, be, mode=1, factor=0, coarse=False)
    nf = len(pr.free)
    P = _csr_dense(*probe.csr(0), nf)
    Po = assemble_aux(pr)[pr.free][:, pr.free]
    scale = abs(Po).max()
    assert np.abs(P - Po.toarray()).max() < 1e-12 * scale
    sc = Condensed(Po, pr.lat, pr.free)
    S = _csr_dense(*probe.csr(1), nf)
    assert np.abs(S[np.ix_(sc.G, sc.G)] - sc.S.toarray()).max() < 1e-11 * scale
    assert np.abs(S[np.ix_(sc.I, sc.I)]).max() == 0.0


def _compare_family(fam, pats_lat, Mfree_fn, factor, free, rel=1e-12):
    """fam: C++ family; pats_lat: oracle patch lists (lattice ids);
    Mfree_fn(idx_lat) -> dense patch matrix from the oracle; rel: the
    agreement of the two patch matrices relative to their largest entry,
    which the inverse amplifies by the condition number."""
    assert fam["npatch"] == len(pats_lat)
    rp, col = fam["rowptr"], fam["col"]
    ns = fam["nslots"]
    if fam["inverse"] is not None:
        # exact factorisation stored as block inverses: compare with the
        # inverse of the oracle's (pattern) patch matrix
        assert factor == "chol"
        for pi, want in enumerate(pats_lat):
            sm = fam["slotmap"][pi]
            valid = np.flatnonzero(sm >= 0)
            assert np.array_equal(sm[valid], want)
            Minv = HostProbe.patch_inverse(fam, pi)
            Lo = cholesky(Mfree_fn(want))
            Ao = Lo @ Lo.T
            Ao_inv = np.linalg.inv(Ao)
            # setup round-off (~1e-13 relative) amplified by cond(A_v)
            tol = max(1e-10, rel * np.linalg.cond(Ao))
            assert np.abs(Minv[np.ix_(valid, valid)] - Ao_inv).max() < tol * np.abs(Ao_inv).max()
            inval = np.flatnonzero(sm < 0)
            if len(inval):
                assert np.allclose(Minv[np.ix_(inval, inval)], np.eye(len(inval)))
                assert np.abs(Minv[np.ix_(valid, inval)]).max(initial=0.0) == 0.0
        return
    for pi, want in enumerate(pats_lat):
        sm = fam["slotmap"][pi]
        valid = np.flatnonzero(sm >= 0)
        assert np.array_equal(sm[valid], want)
        Ld = np.zeros((ns, ns))
        for i in range(ns):
            Ld[i, col[rp[i]:rp[i + 1]]] = fam["val"][pi, rp[i]:rp[i + 1]]
        Lv = Ld[np.ix_(valid, valid)]
        A = Mfree_fn(want)
        Lo = icc0(A) if factor == "icc" else cholesky(A)
        tol = max(1e-10, rel * np.linalg.cond(Lo) ** 2)
        assert np.abs(Lv - Lo).max() < tol * np.abs(Lo).max()
        inval = np.flatnonzero(sm < 0)
        if len(inval):
            assert np.allclose(Ld[np.ix_(inval, inval)], np.eye(len(inval)))


def _free_pos(free, size):
    pos = -np.ones(size, int)
    pos[free] = np.arange(len(free))
    return pos


@pytest.mark.parametrize("k,p,factor", [(0, 2, "icc"), (0, 3, "chol"), (1, 3, "chol"),
                                        (2, 2, "icc")])
def test_sc_pafw_patches_match_oracle(probe, k, p, factor):
    n = 3
    X, al, be, pr = _case(k, n, p, 0.1, coef=True)
    probe.build(k, n, p, X, al, be, mode=1, factor=int(factor == "icc"), coarse=False)
    fams = probe.families()
    Po = assemble_aux(pr)[pr.free][:, pr.free]
    sc = Condensed(Po, pr.lat, pr.free)
    G = pr.free[sc.G]
    pats = patch_lists(pr.lat, (), G)
    posG = _free_pos(G, pr.lat.size)
    S = sc.S.tocsr()
    _compare_family(fams[0], pats, lambda idx: S[posG[idx]][:, posG[idx]].toarray(),
                    factor, pr.free)


def test_pafw_cholesky_patches_match_oracle(probe):
    n, p = 3, 3
    X, al, be, pr = _case(0, n, p, 0.0)
    probe.build(0, n, p, X, al, be, mode=0, factor=0, coarse=False)
    fams = probe.families()
    A = pr.A_free().tocsr()
    pats = patch_lists(pr.lat, (), pr.free)
    pos = _free_pos(pr.free, pr.lat.size)
    _compare_family(fams[0], pats, lambda idx: A[pos[idx]][:, pos[idx]].toarray(),
                    "chol", pr.free)


def test_sc_ph_matches_oracle(probe):
    n, p = 2, 3
    X, al, be, pr = _case(1, n, p, 0.1)
    probe.build(1, n, p, X, al, be, mode=2, factor=1, coarse=False)
    fams = probe.families()
    Po = assemble_aux(pr)[pr.free][:, pr.free]
    sc = Condensed(Po, pr.lat, pr.free)
    G1 = pr.free[sc.G]
    pos1 = _free_pos(G1, pr.lat.size)
    S = sc.S.tocsr()
    for m in range(3):
        pats = patch_lists(pr.lat, (m,), G1)
        _compare_family(fams[m], pats, lambda idx: S[pos1[idx]][:, pos1[idx]].toarray(),
                        "chol", pr.free)
    p0 = Problem(0, n, p, X, al, be)
    B = assemble_aux(p0, mass_coef=np.zeros_like(be), stiff_coef=be)
    sc0 = Condensed(B[p0.free][:, p0.free].tocsr(), p0.lat, p0.free)
    S0 = _csr_dense(*probe.csr(5), len(p0.free))
    assert np.abs(S0[np.ix_(sc0.G, sc0.G)] - sc0.S.toarray()).max() < 1e-11 * abs(B).max()
    G0 = p0.free[sc0.G]
    pos0 = _free_pos(G0, p0.lat.size)
    S0o = sc0.S.tocsr()
    _compare_family(fams[3], patch_lists(p0.lat, (), G0),
                    lambda idx: S0o[pos0[idx]][:, pos0[idx]].toarray(), "icc", p0.free)
    ptr, col, val = probe.csr(6)
    Dh = sp.csr_matrix((val, col, ptr), shape=(pr.lat.size, p0.lat.size))
    Do = discrete_gradient(p0.lat, pr.lat)[G1][:, G0]
    assert abs(Dh[G1][:, G0] - Do).max() < 1e-12 * abs(Do).max()


def test_sc_ph_hdiv_matches_oracle(probe):
    """SC-PH for H(div): face-star families of S, the eps-shifted NCE
    potential's Schur complement, its edge-star ICC(0) factors and the
    discrete curl on the interfaces."""
    from oracle.relaxation import HDIV_POTENTIAL_EPS, discrete_derivative
    n, p = 2, 3
    X, al, be, pr = _case(2, n, p, 0.1, coef=True)
    probe.build(2, n, p, X, al, be, mode=2, factor=1, coarse=False)
    fams = probe.families()
    Po = assemble_aux(pr)[pr.free][:, pr.free]
    sc = Condensed(Po, pr.lat, pr.free)
    G2 = pr.free[sc.G]
    pos2 = _free_pos(G2, pr.lat.size)
    S = sc.S.tocsr()
    # S agrees to 1e-11 of its largest entry (test_aux_and_schur_match_oracle);
    # a face block is diagonal, so its inverse carries that times cond
    for m in range(3):
        span = tuple(d for d in range(3) if d != m)
        _compare_family(fams[m], patch_lists(pr.lat, span, G2),
                        lambda idx: S[pos2[idx]][:, pos2[idx]].toarray(), "chol", pr.free, rel=1e-11)
    p1 = Problem(1, n, p, X, al, be)
    B = assemble_aux(p1, mass_coef=HDIV_POTENTIAL_EPS * be, stiff_coef=be)
    sc1 = Condensed(B[p1.free][:, p1.free].tocsr(), p1.lat, p1.free)
    S1 = _csr_dense(*probe.csr(5), len(p1.free))
    assert np.abs(S1[np.ix_(sc1.G, sc1.G)] - sc1.S.toarray()).max() < 1e-11 * abs(B).max()
    G1 = p1.free[sc1.G]
    pos1 = _free_pos(G1, p1.lat.size)
    S1o = sc1.S.tocsr()
    # the eps-shifted curl-curl patches are ill conditioned (cond ~ 1/eps
    # and more): their ICC(0) factors carry the Schur agreement times cond
    for m in range(3):
        _compare_family(fams[3 + m], patch_lists(p1.lat, (m,), G1),
                        lambda idx: S1o[pos1[idx]][:, pos1[idx]].toarray(), "icc", p1.free, rel=1e-11)
    ptr, col, val = probe.csr(6)
    Ch = sp.csr_matrix((val, col, ptr), shape=(pr.lat.size, p1.lat.size))
    Co = discrete_derivative(1, p1.lat, pr.lat)[G2][:, G1]
    assert abs(Ch[G2][:, G1] - Co).max() < 1e-12 * abs(Co).max()


@pytest.mark.parametrize("k,perturb", [(0, 0.0), (0, 0.15), (1, 0.1), (2, 0.1)])
def test_coarse_matches_oracle(probe, k, perturb):
    n, p = 3, 3
    X, al, be, pr = _case(k, n, p, perturb, coef=True)
    probe.build(k, n, p, X, al, be, mode=1, factor=0, coarse=True)
    Ainv = probe.coarse_inverse()
    c = Coarse(pr)
    want = np.linalg.inv(c.A0)
    assert np.abs(Ainv - want).max() < 1e-10 * np.abs(want).max()
    ptr, col, val = probe.csr(4)
    R0 = sp.csr_matrix((val, col, ptr), shape=(len(c.cp.free), pr.lat.size))
    assert abs(R0[:, pr.free] - c.R0T.T).max() < 1e-12


@pytest.mark.parametrize("k,mode", [(0, 1), (1, 2), (2, 1)])
def test_natural_boundary_setup_matches_oracle(probe, k, mode):
    """Gamma_D empty: every lattice entry is a DOF; the auxiliary operator,
    its Schur complement, the patch lists and factors (boundary-vertex stars
    now hold the boundary entries) and the coarse space match the oracle's
    natural-boundary problem."""
    n, p = 2, 2
    X = inputs.vertices(n, perturb=0.1, seed=13)
    al = inputs.loguniform_coefficient(n, 0.1, 10, seed=14)
    be = inputs.loguniform_coefficient(n, 0.1, 10, seed=15)
    pr = Problem(k, n, p, X, al, be, bc="none")
    assert len(pr.free) == pr.lat.size
    probe.build(k, n, p, X, al, be, mode=mode | 16, factor=0, coarse=True)
    nf = pr.lat.size
    Po = assemble_aux(pr)
    P = _csr_dense(*probe.csr(0), nf)
    assert np.abs(P - Po.toarray()).max() < 1e-12 * abs(Po).max()
    sc = Condensed(Po.tocsr(), pr.lat, pr.free)
    S = sc.S.tocsr()
    G = pr.free[sc.G]
    pos = _free_pos(G, pr.lat.size)
    fams = probe.families()
    spans = [()] if mode == 1 else [(0,), (1,), (2,)]
    for f, span in enumerate(spans):
        _compare_family(fams[f], patch_lists(pr.lat, span, G),
                        lambda idx: S[pos[idx]][:, pos[idx]].toarray(), "chol", pr.free)
    c = Coarse(pr)
    want = np.linalg.inv(c.A0)
    assert c.A0.shape[0] == c.cp.lat.size
    assert np.abs(probe.coarse_inverse() - want).max() < 1e-10 * np.abs(want).max()


def test_icc_breakdown_agrees(probe):
    """ICC(0) of NCE_2 vertex-star Schur complements has a non-positive pivot
    (the paper notes that ICC(0) may fail); both sides report it."""
    X, al, be, pr = _case(1, 2, 2, 0.0)
    with pytest.raises(RuntimeError, match="breakdown"):
        probe.build(1, 2, 2, X, al, be, mode=1, factor=1, coarse=False)
    from oracle.relaxation import SCPAFW
    P = assemble_aux(pr)[pr.free][:, pr.free]
    with pytest.raises(np.linalg.LinAlgError):
        SCPAFW(pr, P, factor="icc", coarse=False)


def test_inverted_cell_is_an_error(probe):
    """A cell whose trilinear map folds over (negative Jacobian) is reported
    as an error by the multithreaded assembly, not a process abort."""
    n = 2
    X = inputs.vertices(n, seed=1).reshape(n + 1, n + 1, n + 1, 3).copy()
    X[1, 1, 1] += 1.2 / n  # the interior vertex beyond its neighbours
    al = inputs.constant_coefficient(n)
    with pytest.raises(RuntimeError, match="inverted or degenerate cell"):
        probe.build(0, n, 2, X.reshape(-1, 3), al, al, mode=0, factor=0, coarse=False)


_DIGEST = r"""
import hashlib, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2211_14284_gb300 import inputs
from paper_2211_14284_gb300.rm import HostProbe
n = 3
X = inputs.vertices(n, perturb=0.12, seed=8)
al = inputs.loguniform_coefficient(n, 0.1, 10, seed=9)
be = inputs.loguniform_coefficient(n, 0.1, 10, seed=10)
h = hashlib.sha256()
for k, mode in ((0, 1), (1, 2)):
    hp = HostProbe()
    hp.build(k, n, 4, X, al, be, mode, 1)
    for which in (0, 1, 2, 3, 4):
        for a in hp.csr(which):
            h.update(np.ascontiguousarray(a).tobytes())
    for f in hp.families():
        for key in sorted(f):
            v = f[key]
            if isinstance(v, dict):
                for kk in sorted(v):
                    h.update(np.ascontiguousarray(v[kk]).tobytes())
            elif v is not None:
                h.update(np.ascontiguousarray(v).tobytes())
print(h.hexdigest())
"""


def test_setup_is_independent_of_the_thread_count():
    """The multithreaded setup (assembly, condensation, patch factors, coarse
    operator) gives bit-identical matrices for any number of threads: summed
    duplicates are merged in a canonical order."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    digests = []
    for threads in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        out = subprocess.run([sys.executable, "-c", _DIGEST, root], env=env, capture_output=True,
                             text=True, timeout=300, check=True)
        digests.append(out.stdout.strip())
    assert digests[0] == digests[1] and len(digests[0]) == 64
