"""Learned coarse corrector: the network's BF16 forward and backward kernels
against the FP64 oracle U-Net (fed the same BF16-rounded weights and
inputs, rounding stored activations where the kernels store them), Adam
against its closed form, and the corrector inside flexible PCG: what the
trained network gains, the judge and its fallback, save / load."""

import os
import struct

import numpy as np
import pytest

from oracle.learned import UNet, adam_step, bf16_round
from paper_2211_14284_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# norm-wise relative tolerance of a BF16 network against the oracle fed the
# same roundings: FP32 accumulation differs from FP64 by ~1e-6, but a value
# that lands on the other side of a BF16 rounding boundary moves by one BF16
# ulp (2^-8 relative) and propagates.  Without down-sampling levels that
# stays below 2e-2.  Deeper, the cascade of BF16 roundings and ReLU masks is
# chaotic (the oracle itself moves its gradients by 5-13% under 1e-7
# relative jitter), so there the bar is a multiple of the oracle's own spread.
TOL_NET = 2e-2
SPREAD_FACTOR = 3.0


def _net_case(dims, levels, width, batch, seed):
    from paper_2211_14284_gb300.rm import Net
    net = Net(dims, levels, width, 2, max_batch=batch, seed=seed)
    rng = np.random.default_rng(seed)
    w = net.get_params().astype(np.float64)
    w += 0.05 * rng.standard_normal(w.size)          # non-zero biases too
    w = w.astype(np.float32)
    net.set_params(w)
    nz, ny, nx = dims[2], dims[1], dims[0]
    x = rng.standard_normal((batch, nz, ny, nx, 2)).astype(np.float32)
    dy = rng.standard_normal((batch, nz, ny, nx)).astype(np.float32)
    return net, w, x, dy


@pytest.mark.parametrize("dims,levels,width,batch", [((9, 9, 9), 2, 4, 2),
                                                     ((13, 5, 9), 2, 16, 3),
                                                     ((17, 9, 9), 3, 8, 1),
                                                     ((7, 5, 6), 0, 16, 2)])
def test_net_forward_backward_vs_oracle(dims, levels, width, batch):
    net, w, x, dy = _net_case(dims, levels, width, batch, seed=11 + levels + width)
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty(x.shape[:4], dtype=torch.float32, device="cuda")
    net.forward(xd, yd)
    grad = torch.empty(net.nparams, dtype=torch.float32, device="cuda")
    dxd = torch.empty_like(xd)
    net.backward(torch.tensor(dy, device="cuda"), grad, dxd)
    torch.cuda.synchronize()
    y, g, dx = yd.cpu().numpy(), grad.cpu().numpy(), dxd.cpu().numpy()

    def oracle(jitter):
        gsum, outs = np.zeros(net.nparams), []
        for b in range(batch):
            o = UNet(w.astype(np.float64), levels, width, 2, bf16=True, jitter=jitter)
            yo = o.forward(x[b].transpose(3, 0, 1, 2).astype(np.float64))[0]
            gb, dxb = o.backward(dy[b][None].astype(np.float64))
            gsum += gb
            outs.append((yo, dxb.transpose(1, 2, 3, 0)))
        return gsum, outs

    rel = lambda a, r: np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-30)
    gref, ref = oracle(None)
    tol_y = tol_dx = tol_g = TOL_NET
    if levels >= 1:
        spread = [oracle((seed, 1e-7)) for seed in (1, 2, 3)]
        tol_y = max(TOL_NET, SPREAD_FACTOR * max(rel(o[b][0], ref[b][0])
                                                 for _, o in spread for b in range(batch)))
        tol_dx = max(TOL_NET, SPREAD_FACTOR * max(rel(o[b][1], ref[b][1])
                                                  for _, o in spread for b in range(batch)))
        tol_g = max(TOL_NET, SPREAD_FACTOR * max(rel(gs, gref) for gs, _ in spread))
    for b in range(batch):
        assert rel(y[b], ref[b][0]) < tol_y, (rel(y[b], ref[b][0]), tol_y)
        assert rel(dx[b], ref[b][1]) < tol_dx, (rel(dx[b], ref[b][1]), tol_dx)
    assert rel(g, gref) < tol_g, (rel(g, gref), tol_g)
    # per layer (weights, biases), where the cascade is not chaotic
    from oracle.learned import net_layers
    off = 0
    for ci, co, _ in net_layers(levels, width, 2):
        for size in (co * 27 * ci, co):
            a, r = g[off:off + size], gref[off:off + size]
            if levels == 0:
                assert np.linalg.norm(a - r) <= TOL_NET * np.linalg.norm(r) + 1e-6, (off, size)
            off += size
    assert off == net.nparams


def test_net_fp32_accumulation_single_layer_path():
    """With inputs and weights exactly representable in BF16 and a ReLU-free
    path (levels = 0, all-positive pre-activations) the only difference from
    FP64 is FP32 accumulation."""
    from paper_2211_14284_gb300.rm import Net
    dims = (9, 7, 5)
    net = Net(dims, 0, 16, 2, max_batch=1, seed=3)
    rng = np.random.default_rng(3)
    w = bf16_round(np.abs(rng.standard_normal(net.nparams)) * 0.05).astype(np.float32)
    net.set_params(w)
    x = bf16_round(np.abs(rng.standard_normal((1, 5, 7, 9, 2)))).astype(np.float32)
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty((1, 5, 7, 9), dtype=torch.float32, device="cuda")
    net.forward(xd, yd)
    o = UNet(w.astype(np.float64), 0, 16, 2, bf16=True)
    yo = o.forward(x[0].transpose(3, 0, 1, 2).astype(np.float64))[0]
    # the two stored activations are rounded to BF16 on both sides
    assert np.max(np.abs(yd.cpu().numpy()[0] - yo) / np.abs(yo)) < 2e-2
    assert np.median(np.abs(yd.cpu().numpy()[0] - yo) / np.abs(yo)) < 1e-5


def test_adam_matches_closed_form():
    net, w, x, dy = _net_case((5, 5, 5), 1, 4, 1, seed=7)
    xd, dyd = torch.tensor(x, device="cuda"), torch.tensor(dy, device="cuda")
    yd = torch.empty(x.shape[:4], dtype=torch.float32, device="cuda")
    grad = torch.empty(net.nparams, dtype=torch.float32, device="cuda")
    wm, m, v = w.astype(np.float64), np.zeros(net.nparams), np.zeros(net.nparams)
    for t in (1, 2, 3):
        net.forward(xd, yd)
        net.backward(dyd, grad)
        g = grad.cpu().numpy().astype(np.float64)
        net.adam(1e-3)
        wm, m, v = adam_step(wm, g, m, v, t, 1e-3)
        got = net.get_params().astype(np.float64)
        assert np.max(np.abs(got - wm)) < 2e-6
        wm = got


# ---------------------------------------------------------------------------
# the corrector inside the solver

N, P = 16, 3


def _solver(**kw):
    from paper_2211_14284_gb300.rm import Solver
    al = inputs.lognormal_grf_coefficient(N, 1.0, 0.1, seed=5)
    return Solver(0, N, P, alpha=al, **dict(dict(rtol=1e-8, max_it=300), **kw))


def _rhs(s, count, seed):
    return torch.tensor(np.stack([inputs.normal_rhs(s.size, seed + i) for i in range(count)]),
                        device="cuda")


@pytest.fixture(scope="module")
def trained(tmp_path_factory):
    from paper_2211_14284_gb300.rm import RM_CORRECTOR_LEARNED
    s = _solver()
    info = s.corrector_train(_rhs(s, 60, 1000), pairs=800, epochs=30, levels=3, width=8,
                             batch=16, lr=2e-3, seed=9, off_fraction=0.0)
    path = str(tmp_path_factory.mktemp("corr") / "net.rmcorr")
    s.corrector_save(path)
    s.corrector_use(RM_CORRECTOR_LEARNED, 0, 1.0)
    return s, info, path


def _solve(s, seed=77):
    b = torch.tensor(inputs.normal_rhs(s.size, seed), device="cuda")
    x = torch.zeros_like(b)
    info = s.solve(b, x)
    return info, x


def test_training_reports(trained):
    _, info, _ = trained
    assert info["pairs"] == 800 and info["params"] > 0
    assert np.isfinite(info["train_loss"]) and np.isfinite(info["val_loss"])
    assert 0.0 <= info["val_eta"] < 1.0


def test_corrector_gain_and_judge(trained):
    from paper_2211_14284_gb300.rm import (RM_CORRECTOR_LEARNED, RM_CORRECTOR_OFF,
                                           RM_CORRECTOR_PLAIN)
    s, info, path = trained
    res = {}
    for name, mode, every, jmax in [("learned", RM_CORRECTOR_LEARNED, 4, 1.0),
                                    ("plain", RM_CORRECTOR_PLAIN, 0, 1.0),
                                    ("off", RM_CORRECTOR_OFF, 0, 1.0)]:
        s.corrector_use(mode, every, jmax)
        res[name] = _solve(s)
    for name, (i, x) in res.items():
        assert i["status"] == "RM_OK" and i["rel_res_l2"] <= 1e-8, name
    il = res["learned"][0]
    assert il["learned_calls"] == il["iterations"] and il["fallback_at"] == -1
    assert il["judge_calls"] >= 1 and 0.0 <= il["judge_eta"] < 1.0
    # the gain over the relaxation without it
    assert il["iterations"] < res["off"][0]["iterations"]
    # all three solve the same system
    xp = res["plain"][1]
    for name in ("learned", "off"):
        assert torch.linalg.norm(res[name][1] - xp) <= 1e-6 * torch.linalg.norm(xp)
    # an untrained network (same layers, initial weights) captures less
    from paper_2211_14284_gb300.rm import Net
    fresh = Net((N + 1,) * 3, 3, 8, 2, seed=123)
    w = fresh.get_params()
    upath = path + ".untrained"
    with open(upath, "wb") as f:
        f.write(b"RMCORR01" + struct.pack("<6i", N + 1, N + 1, N + 1, 3, 8, 2)
                + struct.pack("<q", w.size) + w.astype("<f4").tobytes())
    s.corrector_load(upath)
    s.corrector_use(RM_CORRECTOR_LEARNED, 1, 1.0)
    iu = _solve(s)[0]
    s.corrector_load(path)
    s.corrector_use(RM_CORRECTOR_LEARNED, 1, 1.0)
    it = _solve(s)[0]
    assert iu["status"] == "RM_OK"
    assert it["iterations"] < iu["iterations"]
    # the judge rejects everything above judge_max: fallback on the first
    # judged call, then the plain coarse correction (flexible CG)
    s.corrector_use(RM_CORRECTOR_LEARNED, 1, 0.0)
    ij = _solve(s)[0]
    assert ij["fallback_at"] == 0 and ij["learned_calls"] == 0
    assert abs(ij["iterations"] - res["plain"][0]["iterations"]) <= 1
    s.corrector_use(RM_CORRECTOR_LEARNED, 0, 1.0)
    os.remove(upath)


def test_corrector_save_load_roundtrip(trained):
    from paper_2211_14284_gb300.rm import RM_CORRECTOR_LEARNED, RmError
    s, _, path = trained
    s.corrector_use(RM_CORRECTOR_LEARNED, 0, 1.0)
    i1, x1 = _solve(s, seed=91)
    s2 = _solver()
    with pytest.raises(RmError):
        s2.corrector_use(RM_CORRECTOR_LEARNED, 0, 1.0)   # no network yet
    s2.corrector_load(path)
    s2.corrector_use(RM_CORRECTOR_LEARNED, 0, 1.0)
    # one application: the same network on the same input gives the same
    # coarse term; the rest differs only by the order of the FP64 atomics of
    # the overlapping patch scatter
    r = torch.tensor(inputs.normal_rhs(s.size, 5), device="cuda")
    z1, z2 = torch.empty_like(r), torch.empty_like(r)
    s.precondition(r, z1)
    s2.precondition(r, z2)
    assert torch.linalg.norm(z1 - z2) <= 1e-12 * torch.linalg.norm(z1)
    # whole solves: those last-bit differences reach the BF16 network's
    # rounding decisions, so the iteration counts may differ by one
    i2, x2 = _solve(s2, seed=91)
    assert abs(i1["iterations"] - i2["iterations"]) <= 1
    assert torch.linalg.norm(x1 - x2) <= 1e-6 * torch.linalg.norm(x1)


def test_corrector_rejects_bad_files(trained, tmp_path):
    from paper_2211_14284_gb300.rm import RmError
    _, _, path = trained
    good = open(path, "rb").read()
    s = _solver()
    cases = {"magic": b"XXXXXXXX" + good[8:],
             "truncated": good[:len(good) // 2],
             "dims": good[:8] + struct.pack("<i", N + 3) + good[12:],
             "count": good[:32] + struct.pack("<q", 12345) + good[40:]}
    for name, data in cases.items():
        p = tmp_path / f"{name}.rmcorr"
        p.write_bytes(data)
        with pytest.raises(RmError):
            s.corrector_load(str(p))
    with pytest.raises(RmError):
        s.corrector_load(str(tmp_path / "missing.rmcorr"))
    s.corrector_load(path)          # the handle is still usable


def test_corrector_rejects_bad_use():
    from paper_2211_14284_gb300.rm import RmError, Solver
    s = Solver(1, 2, 2)          # H(curl): no corrector
    with pytest.raises(RmError):
        s.corrector_train(torch.zeros(s.size, dtype=torch.float64, device="cuda"), pairs=4)
    s0 = _solver()
    with pytest.raises(RmError, match="pairs"):
        s0.corrector_train(_rhs(s0, 1, 5), pairs=500, epochs=1)
