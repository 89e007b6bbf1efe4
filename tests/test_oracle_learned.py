"""Pins of the oracle's network reference (conv3d, ReLU, loss, Adam)."""

import numpy as np

from oracle.learned import (adam_step, backward, bf16_round, conv3d, conv3d_backward,
                            forward, mse)


def test_delta_kernel_is_a_shift():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 4, 5, 6))
    W = np.zeros((1, 1, 3, 3, 3))
    W[0, 0, 1, 1, 2] = 1.0          # picks x[.., x + 1]
    y = conv3d(x, W, np.zeros(1))
    want = np.zeros_like(x)
    want[..., :-1] = x[..., 1:]
    assert np.array_equal(y, want)


def test_linearity():
    rng = np.random.default_rng(1)
    x1, x2 = rng.standard_normal((2, 2, 3, 4, 5))
    W = rng.standard_normal((3, 2, 3, 3, 3))
    b = np.zeros(3)
    assert np.allclose(conv3d(2 * x1 - x2, W, b), 2 * conv3d(x1, W, b) - conv3d(x2, W, b))


def test_gradients_central_differences():
    rng = np.random.default_rng(2)
    layers = [(0.3 * rng.standard_normal((4, 2, 3, 3, 3)), 0.1 * rng.standard_normal(4)),
              (0.3 * rng.standard_normal((1, 4, 3, 3, 3)), 0.1 * rng.standard_normal(1))]
    x = rng.standard_normal((2, 3, 4, 3))
    t = rng.standard_normal((1, 3, 4, 3))

    def loss(ls, xx):
        y, _, _ = forward(ls, xx)
        return mse(y, t)[0]

    y, acts, pre = forward(layers, x)
    _, dy = mse(y, t)
    grads, dx = backward(layers, acts, pre, dy)
    h = 1e-6
    for li in range(2):
        W, b = layers[li]
        for idx in [(0, 0, 1, 1, 1), (0, 1, 0, 2, 1)]:
            Wp = W.copy(); Wp[idx] += h
            Wm = W.copy(); Wm[idx] -= h
            lp = loss([(Wp, b) if j == li else layers[j] for j in range(2)], x)
            lm = loss([(Wm, b) if j == li else layers[j] for j in range(2)], x)
            assert abs((lp - lm) / (2 * h) - grads[li][0][idx]) < 1e-6 * max(1, abs(grads[li][0][idx]))
        bp = b.copy(); bp[0] += h
        bm = b.copy(); bm[0] -= h
        lp = loss([(W, bp) if j == li else layers[j] for j in range(2)], x)
        lm = loss([(W, bm) if j == li else layers[j] for j in range(2)], x)
        assert abs((lp - lm) / (2 * h) - grads[li][1][0]) < 1e-6
    for idx in [(0, 1, 2, 1), (1, 2, 0, 0)]:
        xp = x.copy(); xp[idx] += h
        xm = x.copy(); xm[idx] -= h
        assert abs((loss(layers, xp) - loss(layers, xm)) / (2 * h) - dx[idx]) < 1e-6


def test_adam_closed_form():
    w, m, v = adam_step(1.0, 0.5, 0.0, 0.0, 1, 0.1)
    # first step: m_hat = g, v_hat = g^2 -> w - lr * g / (|g| + eps)
    assert abs(w - (1.0 - 0.1 * 0.5 / (0.5 + 1e-8))) < 1e-15


def test_bf16_rounding():
    assert bf16_round(1.0) == 1.0
    assert bf16_round(1.0 + 2 ** -9) == 1.0            # below half an ulp (2^-8)
    assert bf16_round(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7
    x = np.random.default_rng(3).standard_normal(1000)
    assert np.max(np.abs(bf16_round(x) - x) / np.abs(x)) <= 2 ** -8


def test_upsampling_is_linear_interpolation_and_adjoint():
    from oracle.learned import up, up_adjoint
    rng = np.random.default_rng(4)
    # a trilinear function sampled on the coarse nodes is reproduced on the fine nodes
    c = (3, 4, 5)
    f = tuple(2 * n - 1 for n in c)
    lin = lambda z, y, x: 1.0 + 2.0 * x - 3.0 * y + 0.5 * z + 0.25 * x * y * z
    zc, yc, xc = np.meshgrid(*[np.arange(n) * 2.0 for n in c], indexing="ij")
    zf, yf, xf = np.meshgrid(*[np.arange(n) * 1.0 for n in f], indexing="ij")
    a = lin(zc, yc, xc)[None]
    assert np.allclose(up(a)[0], lin(zf, yf, xf))
    # adjoint: <up(a), g> = <a, up^T g>
    a = rng.standard_normal((2,) + c)
    g = rng.standard_normal((2,) + f)
    assert abs(np.sum(up(a) * g) - np.sum(a * up_adjoint(g, a.shape))) < 1e-12


def test_strided_conv_brute_force():
    from oracle.learned import conv3d_strided
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, 5, 7, 9))
    W = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    y = conv3d_strided(x, W, b, 2)
    assert y.shape == (3, 3, 4, 5)
    for (o, oz, oy, ox) in [(0, 0, 0, 0), (2, 1, 3, 2), (1, 2, 1, 4)]:
        s = b[o]
        for dz in range(3):
            for dy in range(3):
                for dx in range(3):
                    iz, iy, ix = 2 * oz + dz - 1, 2 * oy + dy - 1, 2 * ox + dx - 1
                    if 0 <= iz < 5 and 0 <= iy < 7 and 0 <= ix < 9:
                        s += W[o, :, dz, dy, dx] @ x[:, iz, iy, ix]
        assert abs(y[o, oz, oy, ox] - s) < 1e-12


def test_unet_layout_and_gradients():
    from oracle.learned import UNet, net_layers, pack, unpack
    levels, width, in_ch = 1, 2, 2
    spec = net_layers(levels, width, in_ch)
    nparam = sum(co * 27 * ci + co for ci, co, _ in spec)
    rng = np.random.default_rng(6)
    params = 0.4 * rng.standard_normal(nparam)
    layers = unpack(params, levels, width, in_ch)
    assert np.array_equal(pack(layers), params)
    # flat tap order: (dz*3 + dy)*3 + dx with c_in fastest
    W0 = layers[0][0]
    assert W0[1, 0, 2, 0, 1] == params[(1 * 27 + (2 * 3 + 0) * 3 + 1) * in_ch + 0]
    x = rng.standard_normal((in_ch, 5, 3, 5))
    dy = rng.standard_normal((1, 5, 3, 5))
    net = UNet(params, levels, width, in_ch)
    y = net.forward(x)
    assert y.shape == (1, 5, 3, 5)
    g, dx = net.backward(dy)
    f = lambda p, xx: float(np.sum(dy * UNet(p, levels, width, in_ch).forward(xx)))
    h = 1e-6
    for k in rng.choice(nparam, 25, replace=False):
        pp, pm = params.copy(), params.copy()
        pp[k] += h
        pm[k] -= h
        fd = (f(pp, x) - f(pm, x)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(1.0, abs(g[k])), k
    for idx in [(0, 2, 1, 3), (1, 0, 0, 4)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        assert abs((f(params, xp) - f(params, xm)) / (2 * h) - dx[idx]) < 1e-5
