"""Plain FP64 reference of the learned coarse corrector's network: 3D
convolutions (3x3x3, zero padding), ReLU, the mean-squared loss and their
gradients, and one Adam step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The corrector is not in the paper (the north-star's "learned parts"); the
network is a plain convolutional stack, written here from the definition
of a cross-correlation y[co, v] = b[co] + sum_{ci, d} W[co, ci, d] x[ci, v + d - 1].
The GPU kernels round operands to bfloat16 and accumulate in FP32, so the
GPU comparison feeds this reference the same bfloat16-rounded operands.

Pins (tests/test_oracle_learned.py): a delta kernel is a shift; the
forward map is linear in x and in (W, b); gradients match central finite
differences; the Adam step matches its closed form on one scalar.
"""

from __future__ import annotations

import numpy as np


def bf16_round(a):
    """Round float values to the nearest bfloat16 (ties to even), as floats."""
    a = np.asarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3d(x, W, b):
    """x: (ci, nz, ny, nx); W: (co, ci, 3, 3, 3); b: (co,) -> (co, nz, ny, nx)."""
    ci, nz, ny, nx = x.shape
    co = W.shape[0]
    xp = np.zeros((ci, nz + 2, ny + 2, nx + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    y = np.zeros((co, nz, ny, nx)) + b[:, None, None, None]
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + nz, dy:dy + ny, dx:dx + nx]
                y += np.einsum("oi,izyx->ozyx", W[:, :, dz, dy, dx], patch)
    return y


def conv3d_backward(x, W, dy):
    """Gradients of sum(dy * conv3d(x, W, b)) w.r.t. x, W, b."""
    ci, nz, ny, nx = x.shape
    xp = np.zeros((ci, nz + 2, ny + 2, nx + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for dz in range(3):
        for dy_ in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + nz, dy_:dy_ + ny, dx:dx + nx]
                dW[:, :, dz, dy_, dx] = np.einsum("ozyx,izyx->oi", dy, patch)
                dxp[:, dz:dz + nz, dy_:dy_ + ny, dx:dx + nx] += np.einsum(
                    "oi,ozyx->izyx", W[:, :, dz, dy_, dx], dy)
    return dxp[:, 1:-1, 1:-1, 1:-1], dW, dy.sum(axis=(1, 2, 3))


def forward(layers, x):
    """layers: [(W, b), ...]; ReLU after every layer but the last.
    Returns the output and the per-layer inputs / pre-activations."""
    acts = [x]
    pre = []
    h = x
    for li, (W, b) in enumerate(layers):
        z = conv3d(h, W, b)
        pre.append(z)
        h = z if li == len(layers) - 1 else np.maximum(z, 0.0)
        acts.append(h)
    return h, acts, pre


def backward(layers, acts, pre, dout):
    grads = []
    g = dout
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        if li != len(layers) - 1:
            g = g * (pre[li] > 0)
        dx, dW, db = conv3d_backward(acts[li], W, g)
        grads.append((dW, db))
        g = dx
    return grads[::-1], g


def mse(y, t):
    """mean((y - t)^2) and its gradient."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


# ---------------------------------------------------------------------------
# The corrector's U-Net, written out layer by layer in FP64.  Its layers and
# the flat parameter order are the ones the library documents for rm_net_*:
# e0a = conv(x), e0 = conv(e0a); d_l = conv_stride2(e_{l-1}), e_l = conv(d_l);
# u_l = up(h_{l+1}), a_l = conv(u_l), s_l = a_l + e_l, h_l = conv(s_l);
# y = conv(h_0); ReLU after every conv but the last.

def conv3d_strided(x, W, b, stride):
    """Zero-padded 3x3x3 conv reading the input at stride*o + tap - 1: the
    stride-1 conv sampled at every stride-th output."""
    y = conv3d(x, W, b)
    return y[:, ::stride, ::stride, ::stride] if stride > 1 else y


def conv3d_strided_backward(x, W, dy, stride):
    if stride == 1:
        return conv3d_backward(x, W, dy)
    full = np.zeros((dy.shape[0],) + x.shape[1:])
    full[:, ::stride, ::stride, ::stride] = dy
    return conv3d_backward(x, W, full)


def up_matrix(c):
    """1D vertex-centred linear interpolation from c to 2c - 1 nodes."""
    U = np.zeros((2 * c - 1, c))
    for i in range(c):
        U[2 * i, i] = 1.0
    for i in range(c - 1):
        U[2 * i + 1, i] = U[2 * i + 1, i + 1] = 0.5
    return U


def up(a):
    """a: (C, z, y, x) -> (C, 2z-1, 2y-1, 2x-1)"""
    _, nz, ny, nx = a.shape
    return np.einsum("Zz,Yy,Xx,czyx->cZYX", up_matrix(nz), up_matrix(ny), up_matrix(nx), a)


def up_adjoint(g, shape):
    _, nz, ny, nx = shape
    return np.einsum("Zz,Yy,Xx,cZYX->czyx", up_matrix(nz), up_matrix(ny), up_matrix(nx), g)


def net_layers(levels, width, in_ch):
    """(c_in, c_out, stride) per conv, in parameter order."""
    ch = [width << l for l in range(levels + 1)]
    out = [(in_ch, ch[0], 1), (ch[0], ch[0], 1)]
    for l in range(1, levels + 1):
        out += [(ch[l - 1], ch[l], 2), (ch[l], ch[l], 1)]
    for l in range(levels - 1, -1, -1):
        out += [(ch[l + 1], ch[l], 1), (ch[l], ch[l], 1)]
    out.append((ch[0], 1, 1))
    return out


def unpack(params, levels, width, in_ch):
    """Flat parameters (per conv W[c_out][27][c_in] with tap (dz*3+dy)*3+dx,
    then b[c_out]) -> [(W[c_out, c_in, dz, dy, dx], b)]."""
    out, off = [], 0
    for ci, co, _ in net_layers(levels, width, in_ch):
        W = params[off:off + co * 27 * ci].reshape(co, 3, 3, 3, ci).transpose(0, 4, 1, 2, 3)
        off += co * 27 * ci
        out.append((np.array(W, dtype=np.float64), np.array(params[off:off + co], np.float64)))
        off += co
    assert off == len(params)
    return out


def pack(grads):
    return np.concatenate([np.concatenate([dW.transpose(0, 2, 3, 4, 1).ravel(), db])
                           for dW, db in grads])


class UNet:
    """Forward and backward of one sample x (C, z, y, x).  With bf16=True the
    stored tensors are rounded to bfloat16 where the GPU kernels store them
    (inputs, weights, every activation but the FP32 output)."""

    def __init__(self, params, levels, width, in_ch, bf16=False, jitter=None):
        """jitter = (seed, eps): every stored value is multiplied by
        (1 + eps N(0, 1)) before its BF16 rounding -- a model of FP32
        accumulation noise, used to measure how far two equally valid BF16
        evaluations of the same network drift apart."""
        self.L = levels
        self.spec = net_layers(levels, width, in_ch)
        self.layers = unpack(np.asarray(params, np.float64), levels, width, in_ch)
        self.r = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
        self.layers = [(self.r(W), b) for W, b in self.layers]
        if jitter is not None:
            jr, eps, r0 = np.random.default_rng(jitter[0]), jitter[1], self.r
            self.r = lambda a: r0(np.asarray(a) * (1.0 + eps * jr.standard_normal(np.shape(a))))

    def forward(self, x):
        r, L, P = self.r, self.L, self.layers
        relu = lambda z: np.maximum(z, 0.0)
        t = {"x": r(x)}
        i = 0

        def conv(name_in, li, act=True):
            W, b = P[li]
            z = conv3d_strided(t[name_in], W, b, self.spec[li][2])
            return r(relu(z)) if act else z

        t["e0a"] = conv("x", 0); i = 1
        t["e0"] = conv("e0a", 1); i = 2
        for l in range(1, L + 1):
            t[f"d{l}"] = conv(f"e{l - 1}", i); i += 1
            t[f"e{l}"] = conv(f"d{l}", i); i += 1
        for l in range(L - 1, -1, -1):
            t[f"u{l}"] = r(up(t[f"e{L}"] if l + 1 == L else t[f"h{l + 1}"]))
            t[f"a{l}"] = conv(f"u{l}", i); i += 1
            t[f"s{l}"] = r(t[f"a{l}"] + t[f"e{l}"])
            t[f"h{l}"] = conv(f"s{l}", i); i += 1
        t["y"] = conv("h0" if L > 0 else "e0", i, act=False)
        self.t = t
        return t["y"]

    def backward(self, dy):
        """Gradients of sum(dy * y) after forward(): (flat parameter gradient, dx)."""
        t, L, P, spec = self.t, self.L, self.layers, self.spec
        n = len(P)
        grads = [None] * n
        g = {}

        def back(name_in, li, gout):
            dx, dW, db = conv3d_strided_backward(t[name_in], P[li][0], gout, spec[li][2])
            grads[li] = (dW, db)
            return dx

        top = "h0" if L > 0 else "e0"
        g[top] = back(top, n - 1, dy) * (t[top] > 0)
        i = n - 2
        for l in range(L):
            gs = back(f"s{l}", i, g[f"h{l}"]); i -= 1
            g[f"e{l}"] = gs.copy()
            gu = back(f"u{l}", i, gs * (t[f"a{l}"] > 0)); i -= 1
            src = f"e{L}" if l + 1 == L else f"h{l + 1}"
            gh = up_adjoint(gu, t[src].shape)
            g[src] = gh if l + 1 == L else gh * (t[src] > 0)
        for l in range(L, 0, -1):
            ge = g[f"e{l}"] * (t[f"e{l}"] > 0)
            gd = back(f"d{l}", i, ge) * (t[f"d{l}"] > 0); i -= 1
            g[f"e{l - 1}"] = g[f"e{l - 1}"] + back(f"e{l - 1}", i, gd); i -= 1
        ge0 = g["e0"] * (t["e0"] > 0) if L > 0 else g["e0"]
        ga = back("e0a", 1, ge0) * (t["e0a"] > 0)
        dx = back("x", 0, ga)
        return pack(grads), dx


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba): returns new (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
