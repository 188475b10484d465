"""Path-replay adjoint through the C ABI: against the FP64 oracle's dual-number
gradient on the same rays, against central finite differences of the GPU
forward (relative step 1e-3, branch sampling frozen at the unperturbed media),
and through torch autograd.  Loss: squared L2 distance between the simulated
channel data and a target simulated with speeds +2 %, impedances +5 % and
attenuation +10 % (same seed)."""
import numpy as np
import pytest

import oracle
import phantoms
from _parity import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ur():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05828_gb300 as ur
    ur.lib()
    return ur


def target_media(media):
    t = np.array(media, np.float64)
    t[:, 0] *= 1.02
    t[:, 1] *= 1.05
    t[:, 2] *= 1.10
    return t.astype(np.float32)


def setup_loss(ur, w, n_rays):
    import torch
    sim = ur.Simulator(0)
    sim.load(w)
    med0 = np.array(w["scene"]["media"], np.float32)
    sim.set_media(target_media(med0))
    trf, tq = sim.trace(n_rays, w["seed"], w["max_bounces"], w["max_path"])
    sim.set_media(med0)
    rf, q = sim.trace(n_rays, w["seed"], w["max_bounces"], w["max_path"])
    g_rf, g_q = 2 * (rf - trf), 2 * (q - tq)
    return sim, med0, (trf, tq), (rf, q), (g_rf, g_q)


def loss_of(sim, w, n_rays, tgt, media=None, sampling=None, amp=None):
    import torch
    if media is not None:
        sim.set_media(media, sampling=sampling)
    if amp is not None:
        sim.set_amplitudes(amp)
    rf, q = sim.trace(n_rays, w["seed"], w["max_bounces"], w["max_path"])
    return float(((rf.double() - tgt[0].double()) ** 2).sum() + ((q.double() - tgt[1].double()) ** 2).sum())


@pytest.mark.parametrize("name", ["tiny", "layered"])
def test_adjoint_matches_oracle_gradient(ur, name):
    w = phantoms.tiny(n_rays=100_000) if name == "tiny" else phantoms.layered(n_rays=100_000)
    if name == "tiny":
        w["angles"] = np.deg2rad(np.array([0.0, 9.0])).astype(np.float32)
    N = w["n_rays"]
    sim, med0, tgt, cur, (g_rf, g_q) = setup_loss(ur, w, N)
    n_med, n_scat = len(med0), len(w["scene"]["scatterers"])
    gm, ga = sim.trace_adjoint(N, w["seed"], w["max_bounces"], g_rf, g_q, w["max_path"], n_med=n_med, n_scat=n_scat)
    om, oa = oracle.grad(w["scene"], w["array"], w["angles"], N, w["seed"], w["max_bounces"],
                         g_rf.double().cpu().numpy(), g_q.double().cpu().numpy(), w["max_path"])
    gm = gm.double().cpu().numpy()
    assert rel_l2(gm, om) <= 2e-3, (gm, om)
    big = np.abs(om) > 1e-3 * np.abs(om).max()
    assert np.all(np.abs(gm - om)[big] <= 1e-2 * np.abs(om)[big] + 1e-4 * np.abs(om).max())
    assert rel_l2(ga.double().cpu().numpy(), oa) <= 2e-3


def test_adjoint_matches_central_differences(ur):
    """12 media parameters and the 8 largest scatterer-amplitude gradients, relative step 1e-3."""
    import torch
    w = phantoms.layered(n_rays=100_000)
    N = w["n_rays"]
    sim, med0, tgt, cur, (g_rf, g_q) = setup_loss(ur, w, N)
    n_med, n_scat = len(med0), len(w["scene"]["scatterers"])
    gm, ga = sim.trace_adjoint(N, w["seed"], w["max_bounces"], g_rf, g_q, w["max_path"], n_med=n_med, n_scat=n_scat)
    gm = gm.double().cpu().numpy()
    ga = ga.double().cpu().numpy()
    fd_m = np.zeros_like(gm)
    for m in range(n_med):
        for col in range(3):
            base = float(med0[m, col])
            # central difference; one-sided at alpha = 0 (attenuation cannot go negative)
            h, signs = (1e-3 * base, (1.0, -1.0)) if base != 0.0 else (1e-3, (1.0, 0.0))
            vals = []
            for sgn in signs:
                med = med0.astype(np.float64).copy()
                med[m, col] = base + sgn * h
                med = med.astype(np.float32)
                vals.append((loss_of(sim, w, N, tgt, media=med, sampling=med0), float(med[m, col])))
            fd_m[m, col] = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
    sim.set_media(med0)
    scale = np.abs(fd_m).max()
    for m in range(n_med):
        for col in range(3):
            tol = 0.05 * abs(fd_m[m, col]) + 0.01 * scale
            assert abs(gm[m, col] - fd_m[m, col]) <= tol, (m, col, gm[m, col], fd_m[m, col])
    amp0 = np.array(w["scene"]["scatterers"][:, 3], np.float32)
    top = np.argsort(-np.abs(ga))[:8]
    for j in top:
        h = 1e-3 * max(abs(float(amp0[j])), 1e-2)
        vals = []
        for sgn in (1.0, -1.0):
            a = amp0.astype(np.float64).copy()
            a[j] += sgn * h
            a = a.astype(np.float32)
            vals.append((loss_of(sim, w, N, tgt, amp=a), float(a[j])))
        fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
        assert abs(ga[j] - fd) <= 0.02 * abs(fd) + 1e-3 * np.abs(ga).max(), (j, ga[j], fd)
    sim.set_amplitudes(amp0)


def test_autograd_backward_equals_adjoint(ur):
    import torch
    w = phantoms.tiny(n_rays=50_000)
    N = w["n_rays"]
    sim, med0, tgt, cur, (g_rf, g_q) = setup_loss(ur, w, N)
    media = torch.tensor(med0, requires_grad=True)
    amp = torch.tensor(np.array(w["scene"]["scatterers"][:, 3], np.float32), device="cuda", requires_grad=True)
    rf, q = ur.trace_differentiable(sim, media, amp, N, w["seed"], w["max_bounces"], w["max_path"])
    loss = ((rf - tgt[0]) ** 2).sum() + ((q - tgt[1]) ** 2).sum()
    loss.backward()
    gm, ga = sim.trace_adjoint(N, w["seed"], w["max_bounces"], g_rf, g_q, w["max_path"], n_med=len(med0),
                               n_scat=len(amp))
    assert torch.allclose(media.grad[:, :3], gm.cpu(), rtol=1e-5, atol=0)
    assert torch.all(media.grad[:, 3] == 0)
    assert torch.allclose(amp.grad, ga, rtol=1e-5, atol=0)
    # a small step along the negative gradient of the speeds lowers the loss
    with torch.no_grad():
        g = media.grad[:, 0].clone()
        step = 0.2 / g.abs().max()
        new = media.detach().clone()
        new[:, 0] -= step * g
    rf2, q2 = ur.trace_differentiable(sim, new, amp.detach(), N, w["seed"], w["max_bounces"], w["max_path"])
    loss2 = ((rf2 - tgt[0]) ** 2).sum() + ((q2 - tgt[1]) ** 2).sum()
    assert float(loss2.detach()) < float(loss.detach())


def test_adjoint_replays_only_depositing_rays_consistently(ur):
    """Only paths that deposit carry a gradient, so the adjoint replays one thread per arrival
    of the forward trace: first from arrivals it records itself, then from those recorded by a
    matching ur_trace; a forward trace with other settings must not be reused.  All three
    gradients agree (up to FP32 summation order), and against the oracle as in the tests above."""
    w = phantoms.layered(n_rays=200_000)
    N = w["n_rays"]
    sim, med0, tgt, cur, (g_rf, g_q) = setup_loss(ur, w, N)
    n_med, n_scat = len(med0), len(w["scene"]["scatterers"])
    args = (N, w["seed"], w["max_bounces"], g_rf, g_q, w["max_path"])
    gm1, ga1 = sim.trace_adjoint(*args, n_med=n_med, n_scat=n_scat)            # records its own arrivals
    sim.trace(N, w["seed"], w["max_bounces"], w["max_path"])                  # records as it traces
    gm2, ga2 = sim.trace_adjoint(*args, n_med=n_med, n_scat=n_scat)            # reuses it
    sim.trace(N, w["seed"] + 1, w["max_bounces"], w["max_path"])              # other seed: not reusable
    gm3, ga3 = sim.trace_adjoint(*args, n_med=n_med, n_scat=n_scat)
    for gm, ga in ((gm2, ga2), (gm3, ga3)):
        assert rel_l2(gm.double().cpu().numpy(), gm1.double().cpu().numpy()) <= 1e-5
        assert rel_l2(ga.double().cpu().numpy(), ga1.double().cpu().numpy()) <= 1e-5
    om, oa = oracle.grad(w["scene"], w["array"], w["angles"], N, w["seed"], w["max_bounces"],
                         g_rf.double().cpu().numpy(), g_q.double().cpu().numpy(), w["max_path"])
    assert rel_l2(gm2.double().cpu().numpy(), om) <= 2e-3
    assert rel_l2(ga2.double().cpu().numpy(), oa) <= 2e-3
