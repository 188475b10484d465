"""The tracer-to-denoiser workflow on the GPU: pairs traced by the library
(1e6-ray input, 3e7-ray target, jittered layered phantoms), a short training
run, and the held-out check that the denoised channel data is closer to a
1e8-ray reference than the network's own 1e6-ray input (each scene by 8 %, on average by 15 %)
and than the plain tracer given the same wall time.  Training runs with FP32 atomics, so the
trained network varies slightly from run to run; the margins allow for that."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_denoiser_beats_its_input_on_held_out_scenes():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05828_gb300 as ur
    from paper_2501_05828_gb300 import denoise as dz
    import phantoms
    sim = ur.Simulator(0)
    xr, xq, tr, tq, _ = dz.make_pairs(sim, phantoms.batched_variant, range(1, 33), 1e6, 3e7)
    assert xr.shape == (32, 128, 3200)
    net = ur.Denoiser(0, max_batch=8, n_el=128, n_s=3200, width=32, seed=1)
    net.set_scale(dz.channel_scale(tr, tq))
    hist = dz.train(net, xr, xq, tr, tq, epochs=25, batch=8, lr=1e-3)
    assert hist[-1] < hist[0]
    rows = dz.evaluate(sim, net, phantoms.batched_variant, [2001, 2002], 1e6, 1e8)
    for r in rows:
        print(r)
        assert np.isfinite(r["err_denoised"])
        assert r["err_denoised"] < 0.92 * r["err_input"]          # every scene improves
        assert r["err_denoised"] < r["err_equal_time"]             # and beats the tracer given its time
        assert r["n_equal_time"] >= 1_000_000
    assert np.mean([r["err_denoised"] / r["err_input"] for r in rows]) < 0.85
