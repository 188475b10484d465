"""The BF16 U-Net denoiser through the C ABI against the FP64 reference
(oracle/denoiser.py) with the same BF16 rounding of stored tensors: forward
output, full parameter gradient, one Adam update, and that training lowers the
loss.

Tolerances: both sides round the same 17 stored tensors (input, 14 conv
outputs, 3 pooled tensors) to BF16 (unit roundoff u = 2^-9), but their sums
are accumulated in different orders (FP32 on the tensor cores, FP64 here), so
an element near a rounding boundary can round one ulp (2u) apart and the flip
spreads through later layers; the output then differs by about u sqrt(17)
~ 8e-3 relative in the learned part.  A wrong tap, edge, bias or channel
offset gives errors 10-100x larger.  Gradients also store every data
gradient in BF16 (28 more roundings) and sum small bias gradients over few
pixels, hence the looser bounds there."""
import numpy as np
import pytest

from oracle import denoiser as D
from _parity import rel_l2

pytestmark = pytest.mark.gpu

H, W, B = 16, 64, 2


@pytest.fixture(scope="module")
def net():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05828_gb300 as ur
    dn = ur.Denoiser(0, max_batch=B, n_el=H, n_s=W, width=32, seed=3)
    rng = np.random.default_rng(4)
    p = dn.params()
    lay = ur.nn_layout(32)
    for name, (wo, ws, bo, co) in lay.items():   # non-zero biases exercise the bias paths
        p[bo:bo + co] = rng.standard_normal(co).astype(np.float32) * 0.05
    wo, ws, bo, co = lay["head"]                 # a head large enough that the residual matters
    p[wo:wo + 64] = rng.standard_normal(64).astype(np.float32) * 0.3
    dn.set_params(p)
    dn.set_scale(2.0)
    return torch, ur, dn, lay


def to_oracle(p, lay):
    out = {}
    for name, (wo, ws, bo, co) in lay.items():
        w = p[wo:wo + int(np.prod(ws))].reshape(ws).astype(np.float64)
        if name == "e1a":
            w = w[:, :, :2]
        out[name + ".w"] = w
        out[name + ".b"] = p[bo:bo + co].astype(np.float64)
    return out


def inputs(torch, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, H, W, 2)).astype(np.float32) * 2.0
    t = (x * 0.5 + rng.standard_normal((B, H, W, 2)) * 0.3).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return x, t, dev(x[..., 0]), dev(x[..., 1]), dev(t[..., 0]), dev(t[..., 1])


def test_forward_matches_oracle(net):
    torch, ur, dn, lay = net
    x, t, rf, q, trf, tq = inputs(torch, 0)
    orf, oq = dn.forward(rf, q)
    torch.cuda.synchronize()
    P = to_oracle(dn.params(), lay)
    y, _ = D.forward(P, x.astype(np.float64) / 2.0, q=D.bf16)
    gpu = np.stack([orf.cpu().numpy(), oq.cpu().numpy()], -1) / 2.0
    xb = D.bf16(x.astype(np.float64) / 2.0)
    e_all, e_res = rel_l2(gpu, y), rel_l2(gpu - xb, y - xb)
    print(f"forward rel_l2: output {e_all:.2e}, learned part {e_res:.2e}")
    assert e_all <= 5e-3
    assert e_res <= 2e-2          # the learned part alone


def test_forward_matches_unrounded_network(net):
    """The same forward against the FP64 network with no BF16 rounding at all.  Each of the 17
    stored activations and 14 convolution weight tensors carries a relative rounding error of at
    most u = 2^-9 (RMS u / sqrt(3) for round-to-nearest), independent between tensors, so with
    layer gains near one the learned part moves by about sqrt(31) u / sqrt(3) ~ 6e-3; the bar
    allows about 3x that.  A GPU error that the shared rounding points happened to mirror would
    show here."""
    torch, ur, dn, lay = net
    x, t, rf, q, trf, tq = inputs(torch, 0)
    orf, oq = dn.forward(rf, q)
    torch.cuda.synchronize()
    P = to_oracle(dn.params(), lay)
    y, _ = D.forward(P, x.astype(np.float64) / 2.0)
    gpu = np.stack([orf.cpu().numpy(), oq.cpu().numpy()], -1) / 2.0
    x64 = x.astype(np.float64) / 2.0
    e_all, e_res = rel_l2(gpu, y), rel_l2(gpu - x64, y - x64)
    print(f"forward vs unrounded rel_l2: output {e_all:.2e}, learned part {e_res:.2e}")
    assert e_all <= 1e-2
    assert e_res <= 2e-2


def test_gradient_matches_oracle(net):
    torch, ur, dn, lay = net
    x, t, rf, q, trf, tq = inputs(torch, 1)
    loss, g = dn.train_step(rf, q, trf, tq, 0.0, grad=True)
    g = g.cpu().numpy()
    P = to_oracle(dn.params(), lay)
    y, cache = D.forward(P, x.astype(np.float64) / 2.0, q=D.bf16)
    ol, og = D.mse(y, t.astype(np.float64) / 2.0)
    assert loss == pytest.approx(ol, rel=1e-2)
    G = D.backward(P, cache, og)
    worst = 0.0
    for name, (wo, ws, bo, co) in lay.items():
        gw = g[wo:wo + int(np.prod(ws))].reshape(ws)
        if name == "e1a":
            assert np.all(gw[:, :, 2:] == 0.0)      # padded input channels stay untouched
            gw = gw[:, :, :2]
        gb = g[bo:bo + co]
        for kind, a, b in (("w", gw, G[name + ".w"]), ("b", gb, G[name + ".b"])):
            e = rel_l2(a.astype(np.float64), b)
            worst = max(worst, e)
            print(f"{name}.{kind}: rel_l2 {e:.2e}")
            assert e <= (5e-2 if kind == "w" else 1e-1), (name, kind, e)
    assert worst > 0.0


def test_adam_update_matches_oracle(net):
    torch, ur, dn, lay = net
    x, t, rf, q, trf, tq = inputs(torch, 5)
    p0 = dn.params()
    lr = 1e-3
    _, g = dn.train_step(rf, q, trf, tq, lr, grad=True)
    p1 = dn.params()
    P = {"all": p0.astype(np.float64)}
    D.adam_step(P, {"all": g.cpu().numpy().astype(np.float64)}, {}, lr)
    assert np.max(np.abs(p1 - P["all"])) <= 1e-3 * lr + 1e-7
    dn.set_params(p0)


def test_training_lowers_the_loss(net):
    torch, ur, dn, lay = net
    x, t, rf, q, trf, tq = inputs(torch, 2)
    p0 = dn.params()
    first = dn.train_step(rf, q, trf, tq, 2e-3)
    for _ in range(60):
        last = dn.train_step(rf, q, trf, tq, 2e-3)
    assert last < 0.2 * first
    dn.set_params(p0)


def test_forward_matches_oracle_across_tiles():
    """8 x 320 frames: several convolution tiles per image row (128-pixel tiles of the
    per-tap kernel, 126-output tiles of the fused-kx kernel) and a ragged last tile."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05828_gb300 as ur
    h, w = 8, 320
    dn = ur.Denoiser(0, max_batch=1, n_el=h, n_s=w, width=32, seed=7)
    lay = ur.nn_layout(32)
    rng = np.random.default_rng(8)
    p = dn.params()
    for name, (wo, ws, bo, co) in lay.items():
        p[bo:bo + co] = rng.standard_normal(co).astype(np.float32) * 0.05
    wo, ws, bo, co = lay["head"]
    p[wo:wo + 64] = rng.standard_normal(64).astype(np.float32) * 0.3
    dn.set_params(p)
    x = rng.standard_normal((1, h, w, 2)).astype(np.float32)
    rf = torch.from_numpy(np.ascontiguousarray(x[..., 0])).cuda()
    q = torch.from_numpy(np.ascontiguousarray(x[..., 1])).cuda()
    orf, oq = dn.forward(rf, q)
    torch.cuda.synchronize()
    y, _ = D.forward(to_oracle(dn.params(), lay), x.astype(np.float64), q=D.bf16)
    gpu = np.stack([orf.cpu().numpy(), oq.cpu().numpy()], -1)
    xb = D.bf16(x.astype(np.float64))
    e_res = rel_l2(gpu - xb, y - xb)
    # per-column error profile: a wrong tile seam shows up as a spike at x = 126, 252 or 128, 256
    col = np.sqrt(np.sum((gpu - y) ** 2, axis=(0, 1, 3)) / (np.sum((y - xb) ** 2, axis=(0, 1, 3)) + 1e-30))
    print(f"wide forward: learned part {e_res:.2e}, worst column {col.max():.2e} at x = {col.argmax()}")
    assert e_res <= 2e-2
    assert col.max() <= 0.1
    dn.close()


def test_forward_full_size_sampled_columns():
    """The forward pass at the benchmarked frame size [128 x 3200] (batch 1, the launch
    configuration of the benchmark's convolutions) against the oracle on crops.  An output pixel
    depends only on the inputs in its receptive field: on the oracle itself, a crop's outputs
    equal the full frame's from 46 columns inside each crop edge that is not an image edge (four
    levels of two 3x3 convolutions with 2x pooling and nearest upsampling).  So a crop of 384
    columns aligned to the pooling grid (a multiple of 8) gives the full frame's exact outputs on
    all but 96 columns at each inner edge.  Three crops: the left image edge, the middle, the
    right image edge."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05828_gb300 as ur
    h, w, cw, margin = 128, 3200, 384, 96
    dn = ur.Denoiser(0, max_batch=1, n_el=h, n_s=w, width=32, seed=13)
    lay = ur.nn_layout(32)
    rng = np.random.default_rng(14)
    p = dn.params()
    for name, (wo, ws, bo, co) in lay.items():
        p[bo:bo + co] = rng.standard_normal(co).astype(np.float32) * 0.05
    wo, ws, bo, co = lay["head"]
    p[wo:wo + 64] = rng.standard_normal(64).astype(np.float32) * 0.3
    dn.set_params(p)
    x = rng.standard_normal((1, h, w, 2)).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    orf, oq = dn.forward(dev(x[..., 0]), dev(x[..., 1]))
    torch.cuda.synchronize()
    gpu = np.stack([orf.cpu().numpy(), oq.cpu().numpy()], -1)
    P = to_oracle(dn.params(), lay)
    for x0 in (0, 1408, w - cw):
        assert x0 % 8 == 0
        y, _ = D.forward(P, x[:, :, x0:x0 + cw].astype(np.float64), q=D.bf16)
        lo = 0 if x0 == 0 else margin
        hi = cw if x0 + cw == w else cw - margin
        g, o = gpu[:, :, x0 + lo:x0 + hi], y[:, :, lo:hi]
        xb = D.bf16(x[:, :, x0 + lo:x0 + hi].astype(np.float64))
        e_all, e_res = rel_l2(g, o), rel_l2(g - xb, o - xb)
        print(f"full size, columns {x0 + lo}..{x0 + hi - 1}: output {e_all:.2e}, learned part {e_res:.2e}")
        assert e_all <= 5e-3
        assert e_res <= 2e-2
    dn.close()


@pytest.mark.parametrize("w", [320, 256, 1088])
def test_gradient_matches_oracle_across_tiles(w):
    """Parameter gradients on an 8 x w frame: several K steps per image row, so the x-shifted
    boxes of the fused-kx weight gradient cross block seams and the image edges (w = 320: 64-pixel
    steps at every level; w = 256: 128-pixel steps at the two upper levels, whose widths are
    multiples of 128; w = 1088: 128-pixel steps with a ragged last block at the top level)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05828_gb300 as ur
    h = 8
    dn = ur.Denoiser(0, max_batch=1, n_el=h, n_s=w, width=32, seed=11)
    lay = ur.nn_layout(32)
    rng = np.random.default_rng(12)
    p = dn.params()
    for name, (wo, ws, bo, co) in lay.items():
        p[bo:bo + co] = rng.standard_normal(co).astype(np.float32) * 0.05
    wo, ws, bo, co = lay["head"]
    p[wo:wo + 64] = rng.standard_normal(64).astype(np.float32) * 0.3
    dn.set_params(p)
    x = rng.standard_normal((1, h, w, 2)).astype(np.float32)
    t = (0.5 * x + 0.3 * rng.standard_normal((1, h, w, 2))).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    _, g = dn.train_step(dev(x[..., 0]), dev(x[..., 1]), dev(t[..., 0]), dev(t[..., 1]), 0.0, grad=True)
    g = g.cpu().numpy()
    P = to_oracle(dn.params(), lay)
    y, cache = D.forward(P, x.astype(np.float64), q=D.bf16)
    _, og = D.mse(y, t.astype(np.float64))
    G = D.backward(P, cache, og)
    for name in ("e1b", "e2a", "e2b", "d2a", "d2b", "d1a", "d1b", "e3b", "d3a"):
        wo, ws, bo, co = lay[name]
        e = rel_l2(g[wo:wo + int(np.prod(ws))].reshape(ws).astype(np.float64), G[name + ".w"])
        print(f"wide ({w}) {name}.w: rel_l2 {e:.2e}")
        assert e <= 5e-2, (name, e)
    dn.close()
