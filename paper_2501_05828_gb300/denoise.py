"""Channel-data denoising workflow around the library's U-Net (``Denoiser``).

The tracer generates its own training data: for a scene seed s it traces the
same transmit twice, with few rays (the network input) and with many rays (the
target), under independent Philox seeds.  Because every ray starts with weight
cos(theta) / N (Eq. 6, N = rays per transmit), both are unbiased estimates of
the same expected channel data and differ only in Monte Carlo noise, so the
network learns E[channel data] from a noisy sample.  Evaluation compares, on
held-out scenes and against a much higher-ray reference, (a) the noisy input,
(b) the denoised input, (c) the plain tracer given the same wall time as
trace + network and (d) the rays and wall time the plain tracer needs to reach
the denoised error; the plain tracer is also the fallback when no trained
network exists.

Everything here is orchestration: tracing runs in ur_trace, the network in
ur_nn_*; errors for reporting are computed on the host in float64.
"""
from __future__ import annotations

import time

import numpy as np

from . import Denoiser, Simulator


def _load(sim, workload, angle):
    s = workload["scene"]
    sim.upload_scene(s["media"], s["boundaries"], s["med_array"], s["z_max"], s["scatterers"], s["r_s"])
    sim.set_array(workload["array"])
    sim.set_plane_waves(np.asarray([angle], np.float32))


def transmit_angle(workload, scene_seed):
    """The plane-wave angle used for a scene: one of the workload's angles, by seed."""
    a = np.asarray(workload["angles"], np.float32).reshape(-1)
    return float(a[scene_seed % a.size])


def make_pairs(sim, scene_fn, scene_seeds, n_in, n_tgt, max_bounces=8, ray_seed_offset=0):
    """Trace (input, target) channel data for every scene seed.

    scene_fn(seed) -> workload dict (scene, array, angles).  Returns device
    tensors x_rf, x_quad, t_rf, t_quad of shape [P, n_el, n_s] and the seconds
    spent tracing."""
    torch = sim._torch
    xs, ts = [], []
    t0 = time.perf_counter()
    for s in scene_seeds:
        w = scene_fn(int(s))
        _load(sim, w, transmit_angle(w, int(s)))
        xr, xq = sim.trace(int(n_in), 2 * int(s) + ray_seed_offset, max_bounces)
        tr, tq = sim.trace(int(n_tgt), 2 * int(s) + 1 + ray_seed_offset, max_bounces)
        xs.append((xr[0], xq[0]))
        ts.append((tr[0], tq[0]))
    torch.cuda.synchronize(sim.device)
    secs = time.perf_counter() - t0
    st = lambda L, k: torch.stack([p[k] for p in L]).contiguous()
    return st(xs, 0), st(xs, 1), st(ts, 0), st(ts, 1), secs


def channel_scale(t_rf, t_quad, n=8):
    """RMS of the first n targets (host float64): the network's input/output unit."""
    a = t_rf[:n].double().cpu().numpy()
    b = t_quad[:n].double().cpu().numpy()
    return float(np.sqrt(0.5 * (np.mean(a * a) + np.mean(b * b))))


def train(net, x_rf, x_quad, t_rf, t_quad, epochs, batch, lr, seed=0, lr_final=None, log=None):
    """Adam over contiguous batches of the pair tensors, batch order shuffled
    each epoch; cosine decay from lr to lr_final.  Returns the loss history."""
    P = int(x_rf.shape[0])
    nb = P // batch
    rng = np.random.default_rng(seed)
    lr_final = lr * 0.05 if lr_final is None else lr_final
    total, step, hist = epochs * nb, 0, []
    for ep in range(epochs):
        order = rng.permutation(nb)
        ep_loss = 0.0
        for b in order:
            sl = slice(int(b) * batch, int(b) * batch + batch)
            cur = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * step / max(1, total)))
            ep_loss += net.train_step(x_rf[sl], x_quad[sl], t_rf[sl], t_quad[sl], float(cur))
            step += 1
        hist.append(ep_loss / max(1, nb))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return hist


def rel_err(a_rf, a_quad, r_rf, r_quad):
    """Relative L2 error of channel data (rf and quad together), float64."""
    a = np.concatenate([a_rf.double().cpu().numpy().ravel(), a_quad.double().cpu().numpy().ravel()])
    r = np.concatenate([r_rf.double().cpu().numpy().ravel(), r_quad.double().cpu().numpy().ravel()])
    return float(np.linalg.norm(a - r) / np.linalg.norm(r))


def _timed(torch, fn, reps=3):
    """Median CUDA-event time of fn() in seconds (fn may synchronise itself)."""
    out, ts = None, []
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s.record()
        out = fn()
        e.record()
        torch.cuda.synchronize()
        ts.append(s.elapsed_time(e) * 1e-3)
    return out, float(np.median(ts))


def evaluate(sim, net, scene_fn, scene_seeds, n_in, n_ref, max_bounces=8, ray_seed_offset=0):
    """Held-out comparison per scene: errors of the noisy input, the denoised
    input and the plain tracer at equal wall time, all against an n_ref-ray
    reference, and the rays and time the plain tracer needs for the denoised
    error.  Returns a list of dicts."""
    torch = sim._torch
    rows = []
    for s in scene_seeds:
        w = scene_fn(int(s))
        _load(sim, w, transmit_angle(w, int(s)))
        seed_in = 2 * int(s) + ray_seed_offset
        rr, rq = sim.trace(int(n_ref), 10_000_000 + int(s), max_bounces)
        (xr, xq), t_trace = _timed(torch, lambda: sim.trace(int(n_in), seed_in, max_bounces))
        (yr, yq), t_nn = _timed(torch, lambda: net.forward(xr, xq))
        # plain tracer with the same time budget: rays grow until its time matches trace + network
        n_eq = int(n_in * (t_trace + t_nn) / t_trace)
        for _ in range(3):
            _, t_eq = _timed(torch, lambda: sim.trace(n_eq, seed_in + 1, max_bounces), reps=1)
            n_eq = max(int(n_in), int(n_eq * (t_trace + t_nn) / t_eq))
        (er, eq), t_eq = _timed(torch, lambda: sim.trace(n_eq, seed_in + 1, max_bounces))
        err_den = rel_err(yr, yq, rr, rq)
        # plain tracer at equal error: Monte Carlo error falls as n^-1/2, so n is rescaled by
        # (err(n) / err_denoised)^2 until the traced error is within 2 % of the denoised one
        n_ee, err_ee = int(n_in), rel_err(xr, xq, rr, rq)
        for _ in range(8):
            if abs(err_ee / err_den - 1.0) <= 0.02:
                break
            n_ee = int(min(max(n_ee * (err_ee / err_den) ** 2, 1e4), 0.5 * n_ref))
            r_ee, q_ee = sim.trace(n_ee, seed_in + 2, max_bounces)
            err_ee = rel_err(r_ee, q_ee, rr, rq)
        _, t_ee = _timed(torch, lambda: sim.trace(n_ee, seed_in + 2, max_bounces))
        rows.append({"seed": int(s), "err_input": rel_err(xr, xq, rr, rq), "err_denoised": err_den,
                     "err_equal_time": rel_err(er, eq, rr, rq), "n_equal_time": n_eq,
                     "t_trace_s": t_trace, "t_net_s": t_nn, "t_equal_time_s": t_eq,
                     "n_equal_error": n_ee, "err_equal_error": err_ee, "t_equal_error_s": t_ee})
    return rows


def main(argv=None):
    """Command line: trace pairs from jittered layered phantoms, train, evaluate on held-out scenes.

    Run from the repository root (the seeded phantom generators live in phantoms/ there)."""
    import argparse
    import json

    import phantoms

    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--pairs", type=int, default=256, help="training scenes (seeds 1..pairs)")
    ap.add_argument("--n-in", type=float, default=1e6, help="rays of the network input")
    ap.add_argument("--n-tgt", type=float, default=3e8, help="rays of the training target")
    ap.add_argument("--n-ref", type=float, default=1e9, help="rays of the evaluation reference")
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval", type=int, default=8, help="held-out scenes (seeds 2001..)")
    ap.add_argument("--out", default=None, help="JSON report path")
    a = ap.parse_args(argv)
    sim = Simulator(0)
    print("tracing %d pairs (%.0e / %.0e rays)" % (a.pairs, a.n_in, a.n_tgt), flush=True)
    xr, xq, tr, tq, gen_s = make_pairs(sim, phantoms.batched_variant, range(1, a.pairs + 1), a.n_in, a.n_tgt)
    print("pairs traced in %.1f s" % gen_s, flush=True)
    net = Denoiser(0, max_batch=a.batch, n_el=int(xr.shape[1]), n_s=int(xr.shape[2]), width=32, seed=1)
    net.set_scale(channel_scale(tr, tq))
    t0 = time.perf_counter()
    hist = train(net, xr, xq, tr, tq, a.epochs, a.batch, a.lr, log=lambda m: print(m, flush=True))
    train_s = time.perf_counter() - t0
    rows = evaluate(sim, net, phantoms.batched_variant, range(2001, 2001 + a.eval), a.n_in, a.n_ref)
    keys = ("err_input", "err_denoised", "err_equal_time", "err_equal_error", "n_equal_error", "t_equal_error_s",
            "t_trace_s", "t_net_s")
    rep = {"args": vars(a), "generation_s": gen_s, "training_s": train_s, "loss": hist, "eval": rows,
           "mean": {k: float(np.mean([r[k] for r in rows])) for k in keys}}
    for r in rows:
        print(json.dumps(r), flush=True)
    print(json.dumps(rep["mean"]))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rep, f, indent=1)


if __name__ == "__main__":
    main()
