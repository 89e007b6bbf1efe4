"""GPU parity of the mixed Hodge-Laplacian solver (Sec. 5.3, rm_hodge_*)
against the oracle (oracle/hodge.py): the block operator elementwise, the
Chebyshev block preconditioner (with the GPU's own Chebyshev intervals fed
to the oracle), MINRES against the direct solve and the oracle's iteration
count."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.hodge import HodgeMixed, ritz_interval
from paper_2211_14284_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.asarray(a, float), dtype=torch.float64, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _pair(k, n, p, perturb, seed):
    from paper_2211_14284_gb300.rm import HodgeSolver
    X = inputs.vertices(n, perturb=perturb, seed=seed)
    s = HodgeSolver(k, n, p, vertices=X, factor=1, rtol=1e-8, max_it=300)
    H = HodgeMixed(k, n, p, X)
    assert (s.n_sigma, s.n_u) == (H.n0, H.nk)
    # the oracle runs with the GPU's Chebyshev intervals
    i0, i1 = s.intervals()
    H.int0, H.intk = i0, i1
    return s, H


@pytest.mark.parametrize("k,perturb", [(1, 0.1), (2, 0.1), (3, 0.1), (2, 0.0)])
def test_hodge_apply_and_precondition_parity(k, perturb):
    s, H = _pair(k, 2, 3, perturb, 80 + k)
    x = inputs.normal_rhs(s.size, 81)
    y = torch.zeros(s.size, dtype=torch.float64, device="cuda")
    s.apply(_dev(x), y)
    want = H.K @ x
    assert np.abs(_host(y) - want).max() <= 1e-12 * np.abs(want).max()
    z = torch.zeros_like(y)
    s.precondition(_dev(x), z)
    want = H.precondition(x)
    # each block: 4 Chebyshev steps through the SC relaxation (tolerance of
    # the relaxation parity, times the few steps)
    assert np.abs(_host(z) - want).max() <= 1e-9 * np.abs(want).max()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_hodge_intervals_bracket_the_spectrum(k):
    """The GPU's Chebyshev intervals (Ritz values of 20 preconditioned CG
    steps, widened by 10%) agree with the oracle's own estimate from another
    random vector to 15%."""
    s, H = _pair(k, 2, 3, 0.1, 90 + k)
    for (a, b), (R, B, n) in zip(s.intervals(), ((H.R0, H.B0, H.n0), (H.Rk, H.Bk, H.nk))):
        ao, bo = ritz_interval(R, B, n, seed=3)
        assert abs(a - ao) <= 0.15 * ao and abs(b - bo) <= 0.15 * bo, (a, b, ao, bo)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_hodge_minres_parity(k):
    """MINRES to 1e-11: the solution within 1e-8 of the direct solve; to
    1e-8: the oracle's MINRES count (+-1) and the paper's range (tab.
    hodge-iter: 6-23)."""
    from paper_2211_14284_gb300.rm import HodgeSolver
    X = inputs.vertices(2, perturb=0.1, seed=95)
    s11 = HodgeSolver(k, 2, 3, vertices=X, factor=1, rtol=1e-11, max_it=300)
    H = HodgeMixed(k, 2, 3, X)
    H.int0, H.intk = s11.intervals()
    F = inputs.normal_rhs(H.nk, 96)
    b = np.concatenate([np.zeros(H.n0), F])
    x = torch.zeros(s11.size, dtype=torch.float64, device="cuda")
    info = s11.solve(_dev(b), x)
    assert info["status"] == "RM_OK"
    xd = spla.spsolve(H.K.tocsc(), b)
    assert np.linalg.norm(_host(x) - xd) <= 1e-8 * np.linalg.norm(xd)
    s8 = HodgeSolver(k, 2, 3, vertices=X, factor=1, rtol=1e-8, max_it=300)
    i8 = s8.solve(_dev(b), torch.zeros_like(x))
    H.int0, H.intk = s8.intervals()
    _, io = H.solve(F, rtol=1e-8)
    assert abs(i8["iterations"] - io["iterations"]) <= 1, (i8, io["iterations"])
    assert i8["iterations"] <= 30


@pytest.mark.slow
@pytest.mark.parametrize("k", [1, 2, 3])
def test_hodge_iterations_robust_in_p_and_h(k):
    """Counts flat in h and p, as in tab. hodge-iter (Cartesian meshes)."""
    from paper_2211_14284_gb300.rm import HodgeSolver
    its = {}
    for n, p in ((4, 3), (8, 3), (4, 6)):
        s = HodgeSolver(k, n, p, factor=1, rtol=1e-8, max_it=300)
        b = np.concatenate([np.zeros(s.n_sigma), inputs.normal_rhs(s.n_u, 97)])
        info = s.solve(_dev(b), torch.zeros(s.size, dtype=torch.float64, device="cuda"))
        assert info["status"] == "RM_OK"
        its[(n, p)] = info["iterations"]
        s.close()
    assert max(its.values()) - min(its.values()) <= 4 and max(its.values()) <= 30, its
