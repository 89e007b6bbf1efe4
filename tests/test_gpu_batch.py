"""Batched solves (rm_batch_*): uneven H(curl) problems solved together in
lock step (one graph-captured iteration) must give each problem's own
solution: the same iterates as the single-problem solver up to summation
order, and the oracle's direct solution."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.discretization import Problem
from paper_2211_14284_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OPTS = dict(static_condensation=1, decomposition=1, factor=1, rtol=1e-11, max_it=400,
            check_every=4)


def _problems():
    spec = [(2, 2, 0.3), (3, 3, 2.0), (2, 4, 7.5), ((3, 2, 2), 3, 0.15), (4, 2, 1.0)]
    out = []
    for i, (n, p, beta) in enumerate(spec):
        nn = (n, n, n) if isinstance(n, int) else n
        ncell = nn[0] * nn[1] * nn[2]
        out.append({"space": 1, "n": n, "p": p, "alpha": np.ones(ncell),
                    "beta": np.full(ncell, beta), "rhs_seed": 300 + i})
    return out


def test_batch_matches_single_and_direct():
    from paper_2211_14284_gb300.rm import BatchSolver, Solver
    probs = _problems()
    B = BatchSolver(probs, **OPTS)
    bs, xs = [], []
    for pr, size in zip(probs, B.sizes):
        bs.append(torch.tensor(inputs.normal_rhs(size, pr["rhs_seed"]), device="cuda"))
        xs.append(torch.zeros(size, dtype=torch.float64, device="cuda"))
    infos = B.solve(bs, xs)
    # iteration counts at 1e-8 (near 1e-11 the count depends on rounding order)
    B8 = BatchSolver(probs, **dict(OPTS, rtol=1e-8))
    x8 = [torch.zeros_like(x) for x in xs]
    infos8 = B8.solve(bs, x8)
    for pr, b, x, info, info8 in zip(probs, bs, xs, infos, infos8):
        assert info["status"] == "RM_OK" and info["rel_res_l2"] <= 1e-11
        s = Solver(1, pr["n"], pr["p"], alpha=pr["alpha"], beta=pr["beta"], **OPTS)
        x1 = torch.zeros_like(x)
        s.solve(b, x1)
        # check_every = 1: the single solver then stops at the exact iteration
        # (the batch records it on the device whatever check_every is)
        s8 = Solver(1, pr["n"], pr["p"], alpha=pr["alpha"], beta=pr["beta"],
                    **dict(OPTS, rtol=1e-8, check_every=1))
        i8 = s8.solve(b, torch.zeros_like(x))
        assert abs(i8["iterations"] - info8["iterations"]) <= 1
        xb, xa = x.cpu().numpy(), x1.cpu().numpy()
        assert np.linalg.norm(xb - xa) <= 1e-9 * np.linalg.norm(xa)
        opr = Problem(1, pr["n"], pr["p"], inputs.vertices(pr["n"]), pr["alpha"], pr["beta"])
        if opr.lat.size < 20000:
            xd = spla.spsolve(opr.A_free().tocsc(), b.cpu().numpy()[opr.free])
            assert np.linalg.norm(xb[opr.free] - xd) <= 1e-9 * np.linalg.norm(xd)


def test_batch_mixed_precision():
    from paper_2211_14284_gb300.rm import BatchSolver
    probs = _problems()
    B = BatchSolver(probs, **dict(OPTS, precision=1, flexible=1, rtol=1e-8))
    bs = [torch.tensor(inputs.normal_rhs(sz, 9 + i), device="cuda") for i, sz in enumerate(B.sizes)]
    xs = [torch.zeros_like(b) for b in bs]
    infos = B.solve(bs, xs)
    assert all(i["status"] == "RM_OK" and i["rel_res_l2"] <= 1e-8 for i in infos)


def test_batch_rejects_distorted_meshes():
    from paper_2211_14284_gb300.rm import BatchSolver, RmError
    X = inputs.vertices(2, perturb=0.1, seed=1)
    with pytest.raises(RmError, match="Cartesian"):
        BatchSolver([{"space": 1, "n": 2, "p": 2, "vertices": X}], **OPTS)


def test_batch_rejects_deterministic():
    """The deterministic relaxation is for single-problem handles."""
    from paper_2211_14284_gb300.rm import BatchSolver, RmError
    with pytest.raises(RmError, match="deterministic"):
        BatchSolver([{"space": 1, "n": 2, "p": 2}], **dict(OPTS, deterministic=1))


def test_batch_nan_problem_stops_alone():
    """A problem whose right-hand side holds a NaN is flagged RM_ERR_NAN on
    the device and frozen at once; the other problems still converge and the
    lock step does not run on to max_it."""
    from paper_2211_14284_gb300.rm import BatchSolver
    probs = _problems()[:3]
    B = BatchSolver(probs, **dict(OPTS, rtol=1e-8, max_it=300))
    bs = [torch.tensor(inputs.normal_rhs(sz, 60 + i), device="cuda") for i, sz in enumerate(B.sizes)]
    from oracle.discretization import Lattice
    free1 = Lattice(1, probs[1]["n"], probs[1]["p"]).free()
    bs[1][int(free1[len(free1) // 2])] = float("nan")        # a free entry of problem 1
    xs = [torch.zeros_like(b) for b in bs]
    infos = B.solve(bs, xs, check=False)
    assert infos[1]["status"] == "RM_ERR_NAN"
    assert infos[0]["status"] == "RM_OK" and infos[2]["status"] == "RM_OK"
    assert max(i["iterations"] for i in infos) < 100


@pytest.mark.parametrize("arith", [0, 1], ids=["fp64", "df64"])
def test_batch_high_degree_matches_single(arith):
    """Degrees up to 12 (the top of the uneven batch's range) on small
    meshes: every problem's batched solution equals the single solver's."""
    from paper_2211_14284_gb300.rm import BatchSolver, Solver
    spec = [(2, 12, 0.5), (2, 10, 3.0), (3, 9, 1.0)]
    probs = []
    for i, (n, p, beta) in enumerate(spec):
        probs.append({"space": 1, "n": n, "p": p, "alpha": np.ones(n ** 3),
                      "beta": np.full(n ** 3, beta), "rhs_seed": 70 + i})
    opts = dict(OPTS, rtol=1e-10, arith=arith)
    B = BatchSolver(probs, **opts)
    bs = [torch.tensor(inputs.normal_rhs(sz, pr["rhs_seed"]), device="cuda")
          for pr, sz in zip(probs, B.sizes)]
    xs = [torch.zeros_like(b) for b in bs]
    infos = B.solve(bs, xs)
    for pr, b, x, info in zip(probs, bs, xs, infos):
        assert info["status"] == "RM_OK"
        s = Solver(1, pr["n"], pr["p"], alpha=pr["alpha"], beta=pr["beta"], **opts)
        x1 = torch.zeros_like(x)
        assert s.solve(b, x1)["status"] == "RM_OK"
        xa = x1.cpu().numpy()
        assert np.linalg.norm(x.cpu().numpy() - xa) <= 1e-8 * np.linalg.norm(xa)
