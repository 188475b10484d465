"""FP64 reference of the channel-data denoiser (test infrastructure only).

A 4-level 2D convolutional U-Net over the analytic channel data of one
transmit, seen as an image of n_el rows (elements) by n_s columns (samples)
with 2 channels (rf, quad).  Encoder levels: two 3x3 convolutions with ReLU,
then 2x2 average pooling; bottleneck: two 3x3 convolutions; decoder levels:
nearest-neighbour 2x upsampling, concatenation with the encoder features of the
same level, two 3x3 convolutions with ReLU; a 1x1 head adds its 2 outputs to
the input (residual).  Widths C, 2C, 4C, 8C with C = 32 give about 2M
parameters.  Loss: mean squared error against the high-ray channel data;
optimiser: Adam (Kingma & Ba, 2015).

Tensors are NHWC numpy arrays; convolution weights use the layout
[tap = 3 ky + kx][c_out][c_in], zero padding keeps the spatial size.  Plain
loops over the 9 taps with tensordot; the backward pass is written out by hand.
Never imported by the CUDA package.
"""
from __future__ import annotations

import numpy as np

LAYERS = ("e1a", "e1b", "e2a", "e2b", "e3a", "e3b", "e4a", "e4b", "d3a", "d3b", "d2a", "d2b", "d1a", "d1b")


def layer_shapes(c=32, c_in=2):
    """(c_in, c_out) of every 3x3 convolution, then the 1x1 head."""
    w = [c, 2 * c, 4 * c, 8 * c]
    return {"e1a": (c_in, w[0]), "e1b": (w[0], w[0]), "e2a": (w[0], w[1]), "e2b": (w[1], w[1]),
            "e3a": (w[1], w[2]), "e3b": (w[2], w[2]), "e4a": (w[2], w[3]), "e4b": (w[3], w[3]),
            "d3a": (w[3] + w[2], w[2]), "d3b": (w[2], w[2]), "d2a": (w[2] + w[1], w[1]), "d2b": (w[1], w[1]),
            "d1a": (w[1] + w[0], w[0]), "d1b": (w[0], w[0]), "head": (w[0], c_in)}


def init_params(rng, c=32, c_in=2):
    """He-normal weights, zero biases (float64)."""
    p = {}
    for name, (ci, co) in layer_shapes(c, c_in).items():
        taps = 1 if name == "head" else 9
        p[name + ".w"] = rng.standard_normal((taps, co, ci)) * np.sqrt(2.0 / (taps * ci))
        p[name + ".b"] = np.zeros(co)
    return p


# ------------------------------------------------------------------ operators

def _shift(x, dy, dx):
    """x[n, y + dy, x + dx, c] with zero padding."""
    N, H, W, C = x.shape
    out = np.zeros_like(x)
    ys, yd = (slice(dy, H), slice(0, H - dy)) if dy >= 0 else (slice(0, H + dy), slice(-dy, H))
    xs, xd = (slice(dx, W), slice(0, W - dx)) if dx >= 0 else (slice(0, W + dx), slice(-dx, W))
    out[:, yd, xd, :] = x[:, ys, xs, :]
    return out


def conv3x3(x, w, b):
    """y[p, co] = b[co] + sum_{tap, ci} w[tap, co, ci] x[p + offset(tap), ci]."""
    y = np.zeros(x.shape[:3] + (w.shape[1],))
    for tap in range(9):
        ky, kx = divmod(tap, 3)
        y += np.tensordot(_shift(x, ky - 1, kx - 1), w[tap], axes=([3], [1]))
    return y + b


def conv3x3_dgrad(dy, w):
    """dL/dx of conv3x3 given dL/dy."""
    dx = np.zeros(dy.shape[:3] + (w.shape[2],))
    for tap in range(9):
        ky, kx = divmod(tap, 3)
        dx += _shift(np.tensordot(dy, w[tap], axes=([3], [0])), 1 - ky, 1 - kx)
    return dx


def conv3x3_wgrad(x, dy):
    """dL/dw [9, co, ci] and dL/db [co] of conv3x3."""
    dw = np.zeros((9, dy.shape[3], x.shape[3]))
    for tap in range(9):
        ky, kx = divmod(tap, 3)
        dw[tap] = np.tensordot(dy, _shift(x, ky - 1, kx - 1), axes=([0, 1, 2], [0, 1, 2]))
    return dw, dy.sum(axis=(0, 1, 2))


def conv1x1(x, w, b):
    return np.tensordot(x, w[0], axes=([3], [1])) + b


def pool2(x):
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool2_bwd(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_bwd(g):
    N, H, W, C = g.shape
    return g.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def relu(x):
    return np.maximum(x, 0.0)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# ------------------------------------------------------------------ network

def forward(p, x, q=None):
    """x [N, H, W, 2] -> (output [N, H, W, 2], cache).  With q (a rounding
    function, e.g. bf16) the stored tensors are rounded where a BF16 network
    stores them: input, convolution weights, every convolution output after
    ReLU and every pooled tensor; accumulation stays exact."""
    r = q if q is not None else (lambda v: v)
    x = r(x)
    c = {"x": x}

    def block(name_a, name_b, inp):
        a = r(relu(conv3x3(inp, r(p[name_a + ".w"]), p[name_a + ".b"])))
        bb = r(relu(conv3x3(a, r(p[name_b + ".w"]), p[name_b + ".b"])))
        c[name_a + ".in"], c[name_a + ".out"], c[name_b + ".out"] = inp, a, bb
        return bb

    e1 = block("e1a", "e1b", x)
    e2 = block("e2a", "e2b", r(pool2(e1)))
    e3 = block("e3a", "e3b", r(pool2(e2)))
    e4 = block("e4a", "e4b", r(pool2(e3)))
    d3 = block("d3a", "d3b", np.concatenate([up2(e4), e3], axis=3))
    d2 = block("d2a", "d2b", np.concatenate([up2(d3), e2], axis=3))
    d1 = block("d1a", "d1b", np.concatenate([up2(d2), e1], axis=3))
    c["d1"] = d1
    y = x + conv1x1(d1, p["head.w"], p["head.b"])
    return y, c


def backward(p, c, g_out):
    """Gradients of every parameter given dL/d(output)."""
    g = {}
    g["head.w"] = np.tensordot(g_out, c["d1"], axes=([0, 1, 2], [0, 1, 2]))[None]
    g["head.b"] = g_out.sum(axis=(0, 1, 2))
    d = np.tensordot(g_out, p["head.w"][0], axes=([3], [0]))

    def block_bwd(name_a, name_b, d_out):
        d_pre_b = d_out * (c[name_b + ".out"] > 0)
        g[name_b + ".w"], g[name_b + ".b"] = conv3x3_wgrad(c[name_a + ".out"], d_pre_b)
        d_a = conv3x3_dgrad(d_pre_b, p[name_b + ".w"])
        d_pre_a = d_a * (c[name_a + ".out"] > 0)
        g[name_a + ".w"], g[name_a + ".b"] = conv3x3_wgrad(c[name_a + ".in"], d_pre_a)
        return conv3x3_dgrad(d_pre_a, p[name_a + ".w"])

    def split(d_in, c_low):
        return up2_bwd(d_in[..., :c_low]), d_in[..., c_low:]

    c1 = c["e1b.out"].shape[3]
    c2 = c["e2b.out"].shape[3]
    c3 = c["e3b.out"].shape[3]
    d_d2, d_e1 = split(block_bwd("d1a", "d1b", d), c["d2b.out"].shape[3])
    d_d3, d_e2 = split(block_bwd("d2a", "d2b", d_d2), c["d3b.out"].shape[3])
    d_e4, d_e3 = split(block_bwd("d3a", "d3b", d_d3), c["e4b.out"].shape[3])
    d_e3 = d_e3 + pool2_bwd(block_bwd("e4a", "e4b", d_e4))
    d_e2 = d_e2 + pool2_bwd(block_bwd("e3a", "e3b", d_e3))
    d_e1 = d_e1 + pool2_bwd(block_bwd("e2a", "e2b", d_e2))
    block_bwd("e1a", "e1b", d_e1)
    del c1, c2, c3
    return g


def mse(y, t):
    """Mean squared error and its gradient."""
    diff = y - t
    return float(np.mean(diff * diff)), 2.0 * diff / diff.size


def adam_step(p, g, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments), in place; state holds m, v and the step."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m." + k, np.zeros_like(p[k]))
        v = state.setdefault("v." + k, np.zeros_like(p[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] * g[k]
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p
