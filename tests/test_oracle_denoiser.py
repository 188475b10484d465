"""Pins for the FP64 denoiser reference: convolution against torch's conv2d
(a library primitive), its data/weight gradients and the whole U-Net gradient
against finite differences, pooling identities, and one Adam step by hand."""
import numpy as np
import pytest

from oracle import denoiser as D


def test_conv3x3_matches_torch_conv2d():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 7, 11, 5))
    w = rng.standard_normal((9, 6, 5))
    b = rng.standard_normal(6)
    y = D.conv3x3(x, w, b)
    wt = torch.from_numpy(w.reshape(3, 3, 6, 5).transpose(2, 3, 0, 1).copy())
    ref = torch.nn.functional.conv2d(torch.from_numpy(x.transpose(0, 3, 1, 2).copy()), wt, torch.from_numpy(b),
                                     padding=1).numpy().transpose(0, 2, 3, 1)
    assert np.allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_conv_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 5, 6, 3))
    w = rng.standard_normal((9, 4, 3))
    b = rng.standard_normal(4)
    gy = rng.standard_normal((1, 5, 6, 4))
    f = lambda xx, ww, bb: float(np.sum(gy * D.conv3x3(xx, ww, bb)))   # linear in each argument
    dx = D.conv3x3_dgrad(gy, w)
    dw, db = D.conv3x3_wgrad(x, gy)
    h = 1.0
    for idx in [(0, 0, 0, 0), (0, 2, 3, 1), (0, 4, 5, 2)]:
        e = np.zeros_like(x)
        e[idx] = h
        assert dx[idx] == pytest.approx((f(x + e, w, b) - f(x - e, w, b)) / (2 * h), rel=1e-10)
    for idx in [(0, 0, 0), (4, 3, 2), (8, 1, 1)]:
        e = np.zeros_like(w)
        e[idx] = h
        assert dw[idx] == pytest.approx((f(x, w + e, b) - f(x, w - e, b)) / (2 * h), rel=1e-10)
    e = np.zeros_like(b)
    e[2] = h
    assert db[2] == pytest.approx((f(x, w, b + e) - f(x, w, b - e)) / (2 * h), rel=1e-10)


def test_pool_and_upsample_identities():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 4, 6, 3))
    assert np.allclose(D.pool2(D.up2(x)), x)
    g = rng.standard_normal((2, 2, 3, 3))
    # adjoint pairs: <pool2(x), g> = <x, pool2_bwd(g)>, <up2(y), h> = <y, up2_bwd(h)>
    assert np.sum(D.pool2(x) * g) == pytest.approx(np.sum(x * D.pool2_bwd(g)))
    h = rng.standard_normal((2, 4, 6, 3))
    assert np.sum(D.up2(g) * h) == pytest.approx(np.sum(g * D.up2_bwd(h)))


def test_unet_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = D.init_params(rng, c=4)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    x = rng.standard_normal((2, 8, 16, 2))
    t = rng.standard_normal((2, 8, 16, 2))
    y, cache = D.forward(p, x)
    assert y.shape == x.shape
    loss, g_out = D.mse(y, t)
    g = D.backward(p, cache, g_out)
    assert set(g) == set(p)
    h = 1e-6
    for k in ("e1a.w", "e2b.w", "e4a.w", "e4b.b", "d3a.w", "d2b.b", "d1a.w", "d1b.w", "head.w", "head.b"):
        for _ in range(2):
            idx = tuple(rng.integers(0, s) for s in p[k].shape)
            pp = {kk: vv.copy() for kk, vv in p.items()}
            pm = {kk: vv.copy() for kk, vv in p.items()}
            pp[k][idx] += h
            pm[k][idx] -= h
            fd = (D.mse(D.forward(pp, x)[0], t)[0] - D.mse(D.forward(pm, x)[0], t)[0]) / (2 * h)
            assert g[k][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (k, idx)


def test_default_width_has_about_two_million_parameters():
    p = D.init_params(np.random.default_rng(0), c=32)
    n = sum(v.size for v in p.values())
    assert 1.9e6 < n < 2.0e6


def test_adam_step_by_hand():
    p = {"w": np.array([1.0, -2.0])}
    g = {"w": np.array([0.5, 0.1])}
    st = {}
    D.adam_step(p, g, st, lr=0.01)
    # first step: m_hat = g, v_hat = g^2 -> update lr * sign(g) (up to eps)
    assert np.allclose(p["w"], [1.0 - 0.01, -2.0 - 0.01], atol=1e-9)


def test_receptive_field_of_the_unet():
    """An output column depends only on the inputs within 46 columns of it, for a crop aligned to
    the pooling grid: the oracle on a crop reproduces the full frame's outputs exactly from the
    46th column inside each inner crop edge on, and not nearer (the full-size GPU parity test
    compares crops with a 96-column margin on the strength of this)."""
    rng = np.random.default_rng(1)
    P = D.init_params(rng)
    for k in P:
        if k.endswith(".b"):
            P[k] = rng.standard_normal(P[k].shape) * 0.05
    P["head.w"] = rng.standard_normal(P["head.w"].shape) * 0.3
    x = rng.standard_normal((1, 32, 512, 2))
    y, _ = D.forward(P, x, q=D.bf16)
    x0, cw = 128, 256
    yc, _ = D.forward(P, x[:, :, x0:x0 + cw], q=D.bf16)
    same = np.all(yc == y[:, :, x0:x0 + cw], axis=(0, 1, 3))
    exact = np.nonzero(same)[0]
    assert exact[0] == 46 and exact[-1] == cw - 1 - 46
    assert same[46:cw - 46].all()
