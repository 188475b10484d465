"""Diverging, focused and synthetic-aperture transmits and per-ray transmit
mixing on the CUDA path against the FP64 oracle, through the C ABI: path
topology, arrivals and channel data of mixed sets of transmits, their
delay-and-sum images, and the calls that refuse them.  Bars as in
test_gpu_trace.py."""
import numpy as np
import pytest

import oracle
import phantoms
from _parity import rel_l2
from test_gpu_trace import PATH_FRAC, check_trace_parity, run_gpu

pytestmark = pytest.mark.gpu

# (kind, x, z) in the oracle's form; angles carry the plane wave's steering
MIXED = [(oracle.TX_DIVERGING, -2e-3, -10e-3), (oracle.TX_FOCUSED, 1e-3, 20e-3), (oracle.TX_PLANE, 0.0, 0.0),
         (oracle.TX_DIVERGING, 3e-3, -4e-3), (oracle.TX_FOCUSED, -2e-3, 12e-3)]
ANGLES = np.deg2rad([0.0, 0.0, 5.0, 0.0, 0.0]).astype(np.float32)


@pytest.fixture(scope="module")
def ur():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05828_gb300 as ur
    ur.lib()
    return ur


def mixed_workload(n_rays):
    w = phantoms.tiny(n_rays=n_rays)
    w["angles"] = ANGLES
    # the binding takes (kind, angle, 0) for plane waves and (kind, x, z) otherwise
    w["transmits"] = [(k, float(a), 0.0) if k == oracle.TX_PLANE else (k, x, z) for (k, x, z), a in zip(MIXED, ANGLES)]
    return w


def test_mixed_transmits_parity(ur):
    w = mixed_workload(30_000)
    G = run_gpu(ur, w)
    assert G["stats"]["rays"] == len(MIXED) * w["n_rays"]
    arr, topo, _ = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], w["seed"], w["max_bounces"],
                                w["max_path"], topo=True, transmits=MIXED)
    res = check_trace_parity(w, G, arr, topo, "mixed transmits")
    assert res["n_matched"] >= 0.999 * len(arr)
    per_tx = np.bincount(arr["tx"], minlength=len(MIXED))
    assert np.all(per_tx > 0)                     # every transmit produces echoes


def test_beamform_transmit_kinds(ur):
    """Same float32 channel data into both beamformers, compounding all five transmits."""
    import torch
    w = mixed_workload(30_000)
    arr, _, _ = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], w["seed"], w["max_bounces"],
                             w["max_path"], transmits=MIXED)
    orf, oq = oracle.deposit(w["array"], len(MIXED), arr)
    rf32, q32 = orf.astype(np.float32), oq.astype(np.float32)
    sim = ur.Simulator(0)
    sim.load(w)
    iq, env, db = sim.beamform(torch.from_numpy(rf32).cuda(), torch.from_numpy(q32).cuda(), w["x_px"], w["z_px"],
                               w["dyn_range_db"])
    oiq = oracle.beamform(w["array"], w["angles"], rf32.astype(np.float64), q32.astype(np.float64), w["x_px"],
                          w["z_px"], transmits=MIXED)
    giq = iq.double().cpu().numpy()
    giq = giq[..., 0] + 1j * giq[..., 1]
    assert rel_l2(giq, oiq) <= 1e-5
    # a plane-wave beamformer on the same data gives another image: the kinds are used
    opw = oracle.beamform(w["array"], w["angles"], rf32.astype(np.float64), q32.astype(np.float64), w["x_px"],
                          w["z_px"])
    assert rel_l2(giq, opw) > 0.1
    sim.close()


def test_transmit_kinds_refused_where_unsupported(ur):
    import torch
    w = mixed_workload(1000)
    sim = ur.Simulator(0)
    sim.load(w)
    g = torch.zeros((len(MIXED), 32, 1536), dtype=torch.float32, device="cuda")
    with pytest.raises(ur.URError):
        sim.trace_adjoint(1000, 0, 4, g, g, n_med=3, n_scat=200)
    out = torch.empty((w["z_px"].size, w["x_px"].size), dtype=torch.float32, device="cuda")
    with pytest.raises(ur.URError):
        sim.beamform_noalloc(g, g, w["x_px"], w["z_px"], 60.0, env=out)
    for bad in ([(ur.TX_DIVERGING, 0.0, 5e-3)], [(ur.TX_FOCUSED, 0.0, -5e-3)], [(9, 0.0, 1e-2)],
                [(ur.TX_PLANE, 1.2, 0.0)]):
        with pytest.raises(ur.URError):
            sim.set_transmits(bad)
    sim.close()


SYNTH = [(oracle.TX_SYNTHETIC, 5.0, 0.0), (oracle.TX_PLANE, 0.0, 0.0), (oracle.TX_SYNTHETIC, 26.0, 0.0),
         (oracle.TX_DIVERGING, 1e-3, -6e-3)]
SYNTH_ANGLES = np.deg2rad([0.0, -6.0, 0.0, 0.0]).astype(np.float32)


def synthetic_workload(n_rays, mix=False):
    w = phantoms.tiny(n_rays=n_rays)
    # a wider step directivity (f_d = 1 up to 12 degrees) for more echoes of oblique rays; a ramp would
    # need the amplitude floor of the convex tests
    w["array"] = dict(w["array"], alpha_m_deg=12.0, alpha_c_deg=12.0)
    w["angles"] = SYNTH_ANGLES
    w["transmits"] = [(k, float(a), 0.0) if k == oracle.TX_PLANE else (k, x, z) for (k, x, z), a in zip(SYNTH, SYNTH_ANGLES)]
    w["mix"] = mix
    return w


def test_synthetic_aperture_parity(ur):
    w = synthetic_workload(30_000)
    G = run_gpu(ur, w, capacity=4 * len(SYNTH) * w["n_rays"])
    assert G["stats"]["rays"] == len(SYNTH) * w["n_rays"]
    arr, topo, ost = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], w["seed"], w["max_bounces"],
                                  w["max_path"], topo=True, transmits=SYNTH)
    res = check_trace_parity(w, G, arr, topo, "synthetic aperture")
    assert res["n_matched"] >= 0.999 * len(arr)
    per_tx = np.bincount(arr["tx"], minlength=len(SYNTH))
    assert np.all(per_tx > 0)
    assert abs(G["stats"]["segments"] - ost["segments"]) <= 10


def picks(seed, n, n_tx):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    x0 = np.array([int(oracle.philox4x32_10([i, 0, 0, 1], key)[0]) for i in range(n)], np.uint64)
    return (((x0 >> np.uint64(8)) * np.uint64(n_tx)) >> np.uint64(24)).astype(np.int64)


def test_transmit_mixing_parity(ur):
    """Per-ray transmit mixing over plane, diverging and synthetic-aperture transmits: the same
    draws, paths and arrivals as the oracle's mixed sequence."""
    w = synthetic_workload(8_000, mix=True)
    n_tx, N = len(SYNTH), w["n_rays"]
    G = run_gpu(ur, w, capacity=4 * n_tx * N)
    assert G["stats"]["rays"] == n_tx * N
    arr, topo, _ = oracle.trace(w["scene"], w["array"], w["angles"], N, w["seed"], w["max_bounces"], w["max_path"],
                                topo=True, transmits=SYNTH, mix=True)
    assert G["hash"].shape == topo.shape == (n_tx * N,)
    assert np.mean(G["hash"] == topo) >= PATH_FRAC
    # hashes by (drawn transmit, ray) so that mismatching rays are dropped from the right channel rows
    k = picks(w["seed"], n_tx * N, n_tx)
    hg = np.zeros((n_tx, n_tx * N), np.uint64)
    ho = np.zeros_like(hg)
    hg[k, np.arange(n_tx * N)] = G["hash"]
    ho[k, np.arange(n_tx * N)] = topo
    assert np.array_equal(np.unique(arr["tx"]), np.arange(n_tx))
    assert np.all(k[arr["ray"]] == arr["tx"])                 # the oracle's rays carry the draws computed here
    res = check_trace_parity(w, dict(G, hash=hg), arr, ho, "mixed transmits")
    assert res["n_matched"] >= 0.999 * len(arr) and len(arr) > 300
    G["sim"].close()


def test_beamform_synthetic_aperture(ur):
    import torch
    w = synthetic_workload(20_000)
    arr, _, _ = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], w["seed"], w["max_bounces"],
                             w["max_path"], transmits=SYNTH)
    orf, oq = oracle.deposit(w["array"], len(SYNTH), arr)
    rf32, q32 = orf.astype(np.float32), oq.astype(np.float32)
    sim = ur.Simulator(0)
    sim.load(w)
    iq, env, db = sim.beamform(torch.from_numpy(rf32).cuda(), torch.from_numpy(q32).cuda(), w["x_px"], w["z_px"],
                               w["dyn_range_db"])
    oiq = oracle.beamform(w["array"], w["angles"], rf32.astype(np.float64), q32.astype(np.float64), w["x_px"],
                          w["z_px"], transmits=SYNTH)
    giq = iq.double().cpu().numpy()
    assert rel_l2(giq[..., 0] + 1j * giq[..., 1], oiq) <= 1e-5
    sim.close()


def test_synthetic_aperture_and_mixing_refused_where_unsupported(ur):
    import torch
    w = synthetic_workload(1000, mix=True)
    sim = ur.Simulator(0)
    sim.load(w)
    g = torch.zeros((len(SYNTH), 32, 1536), dtype=torch.float32, device="cuda")
    sim.set_transmits([(ur.TX_PLANE, 0.0, 0.0)] * len(SYNTH))
    with pytest.raises(ur.URError):                       # plane waves, but mixed
        sim.trace_adjoint(1000, 0, 4, g, g, n_med=3, n_scat=200)
    with pytest.raises(ur.URError):
        sim._call(ur.lib().ur_set_transmit_mixing(sim._ctx, 2))
    for bad in ([(ur.TX_SYNTHETIC, 32.0, 0.0)], [(ur.TX_SYNTHETIC, -1.0, 0.0)], [(ur.TX_SYNTHETIC, 1.5, 0.0)]):
        with pytest.raises(ur.URError):
            sim.set_transmits(bad)
    with pytest.raises(ur.URError):                       # more than 2^32 mixed rays
        sim.trace((1 << 31), 0, 4)
    # frozen sampling media need plane waves without mixing
    sim.set_transmit_mixing(False)
    sim.set_transmits([(ur.TX_SYNTHETIC, 3.0, 0.0)])
    media = [list(m) for m in w["scene"]["media"]]
    samp = [list(m) for m in media]
    samp[1][0] *= 1.01
    sim.set_media(media, sampling=samp)
    with pytest.raises(ur.URError):
        sim.trace(1000, 0, 4)
    sim.close()


def test_transmit_mixing_many_transmits(ur):
    """400 transmits x 32 elements exceed the (transmit, element) bins of the ray-order sort, which
    then orders the mixed sequence by transmit alone: same paths as the oracle, every ray once."""
    w = phantoms.tiny(n_rays=100)
    w["array"] = dict(w["array"], alpha_m_deg=12.0, alpha_c_deg=12.0)
    w["angles"] = np.deg2rad(np.linspace(-20.0, 20.0, 400)).astype(np.float32)
    w["mix"] = True
    n_tx, N = w["angles"].size, w["n_rays"]
    G = run_gpu(ur, w, capacity=4 * n_tx * N)
    assert G["stats"]["rays"] == n_tx * N
    arr, topo, _ = oracle.trace(w["scene"], w["array"], w["angles"], N, w["seed"], w["max_bounces"], w["max_path"],
                                topo=True, mix=True)
    assert np.mean(G["hash"] == topo) >= PATH_FRAC
    from _parity import compare
    res = compare(G["rec"], arr)
    assert res["n_matched"] >= 0.999 * len(arr) and len(arr) > 50
    assert res["el_mismatch"] == 0 and res["max_dt"] <= 1e-3 and res["max_amp_rel"] <= 1e-4
    G["sim"].close()
