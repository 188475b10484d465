"""Convex arrays on the CUDA path against the FP64 oracle, through the C ABI:
path topology, arrivals and channel data (plane waves; diverging waves over a
rough bone sphere), images, the closed-form echo of a concentric shell, and the
calls that refuse convex arrays.  Bars as in test_gpu_trace.py, with per-arrival
amplitudes below 1 % of the largest compared against that level: these tests use
a directivity ramp (10 to 15 degrees) so that a convex array receives from many
directions, and near the cutoff f_d = (alpha_c - alpha) / (alpha_c - alpha_m) is
small while the FP32 angle error (about 2e-7 rad from acosf near 15 degrees) is not,
so a tail arrival with f_d ~ 1e-3 carries a relative error of a few 1e-3 (1e-9 of
the largest arrival); channel data stay at 1e-4.  With rough boundaries the time
bar of the paper-settings test applies (curved bounces in FP32)."""
import numpy as np
import pytest

import oracle
import phantoms
from _parity import rel_l2
from test_gpu_rough import with_roughness
from test_gpu_trace import check_trace_parity, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

CONVEX_AMP_FLOOR = 1e-2


@pytest.fixture(scope="module")
def ur():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05828_gb300 as ur
    ur.lib()
    return ur


def convex(w, radius=0.04, alpha_deg=None):
    w = dict(w)
    a = dict(w["array"])
    a["radius"] = float(np.float32(radius))
    if alpha_deg is not None:
        a["alpha_m_deg"], a["alpha_c_deg"] = float(alpha_deg), float(alpha_deg) + 5.0
    w["array"] = a
    return w


def test_convex_plane_waves_parity(ur):
    w = convex(phantoms.tiny(n_rays=100_000), alpha_deg=10.0)
    w["angles"] = np.deg2rad([0.0, 8.0]).astype(np.float32)
    G = run_gpu(ur, w)
    arr, topo, _ = run_oracle(w)
    res = check_trace_parity(w, G, arr, topo, "convex plane waves", amp_floor=CONVEX_AMP_FLOOR)
    assert res["n_matched"] >= 0.999 * len(arr) and len(arr) > 1000


def test_convex_diverging_rough_parity(ur):
    """Every extended feature at once: convex array, diverging waves, rough bone sphere."""
    w = with_roughness(convex(phantoms.tiny(n_rays=40_000), alpha_deg=10.0), 2, 0.5)
    w["angles"] = np.zeros(2, np.float32)
    tx = [(oracle.TX_DIVERGING, -2e-3, -0.04), (oracle.TX_DIVERGING, 3e-3, -0.03)]
    w["transmits"] = tx
    G = run_gpu(ur, w, capacity=4 * 2 * w["n_rays"])
    arr, topo, _ = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], w["seed"], w["max_bounces"],
                                w["max_path"], topo=True, transmits=tx)
    check_trace_parity(w, G, arr, topo, "convex diverging rough", amp_floor=CONVEX_AMP_FLOOR, dt_max=1e-2,
                       dt_q99=1e-3)


def test_convex_beamform_parity(ur):
    import torch
    w = convex(phantoms.tiny(n_rays=50_000), alpha_deg=10.0)
    arr, _, _ = run_oracle(w)
    orf, oq = oracle.deposit(w["array"], 1, arr)
    rf32, q32 = orf.astype(np.float32), oq.astype(np.float32)
    sim = ur.Simulator(0)
    sim.load(w)
    iq, env, db = sim.beamform(torch.from_numpy(rf32).cuda(), torch.from_numpy(q32).cuda(), w["x_px"], w["z_px"],
                               w["dyn_range_db"])
    oiq = oracle.beamform(w["array"], w["angles"], rf32.astype(np.float64), q32.astype(np.float64), w["x_px"],
                          w["z_px"])
    giq = iq.double().cpu().numpy()
    assert rel_l2(giq[..., 0] + 1j * giq[..., 1], oiq) <= 1e-5
    sim.close()


def test_concentric_shell_echo_on_the_gpu(ur):
    """Diverging wave from the centre of curvature, concentric bone shell d = 10 mm beyond the arc:
    every echo returns to its emitting element at 2 d fs / c."""
    R, d = 0.04, 10e-3
    w = {"scene": {"media": [(1540.0, 1.54, 0.0, 0.0), (3500.0, 7.8, 0.0, 0.0)],
                   "boundaries": [(oracle.CYL_Y, [0.0, -R, R + d, 0.0], 0, 1)], "med_array": 0, "z_max": 0.05,
                   "scatterers": np.zeros((0, 4), np.float32), "r_s": 1e-4},
         "array": phantoms.array_params(32, 2048, c_bf=1540.0, alpha_m_deg=10.0, alpha_c_deg=15.0),
         "angles": np.zeros(1, np.float32), "transmits": [(oracle.TX_DIVERGING, 0.0, -R)],
         "n_rays": 32 * 2000, "seed": 5, "max_bounces": 1, "max_path": 0.2}
    w["array"]["radius"] = float(np.float32(R))
    G = run_gpu(ur, w)
    rec = G["rec"]
    assert rec.size > 0.1 * w["n_rays"]                     # the reflected share of the rays
    d_in = float(np.float32(R + d)) - float(np.float32(R))
    assert np.abs(rec["t"] - 2 * d_in * w["array"]["fs"] / 1540.0).max() < 1e-3
    assert np.array_equal(rec["el"], rec["ray"] % 32)


def test_convex_refused_where_unsupported(ur):
    import torch
    w = convex(phantoms.tiny(n_rays=1000))
    sim = ur.Simulator(0)
    sim.load(w)
    g = torch.zeros((1, 32, 1536), dtype=torch.float32, device="cuda")
    with pytest.raises(ur.URError):
        sim.trace_adjoint(1000, 0, 4, g, g, n_med=3, n_scat=200)
    out = torch.empty((w["z_px"].size, w["x_px"].size), dtype=torch.float32, device="cuda")
    with pytest.raises(ur.URError):
        sim.beamform_noalloc(g, g, w["x_px"], w["z_px"], 60.0, env=out)
    for radius in (-0.01, 0.003):
        a = dict(w["array"])
        a["radius"] = radius
        with pytest.raises(ur.URError):
            sim.set_array(a)
    sim.close()


def test_paper_settings_on_the_convex_probe(ur):
    """The paper's acquisition with its probe geometry (128 elements over 70 degrees, R = 50 mm):
    all 25 plane waves against the oracle; time bar of the paper-settings test (rough curved bone,
    50 MHz), amplitude floor of the rough tests (the 2-degree directivity here is a step)."""
    from test_gpu_rough import ROUGH_AMP_FLOOR
    w = phantoms.paper_like(n_rays=4000, convex=True)
    G = run_gpu(ur, w, capacity=4 * 25 * w["n_rays"])
    assert G["stats"]["rays"] == 25 * w["n_rays"]
    arr, topo, _ = run_oracle(w)
    check_trace_parity(w, G, arr, topo, "paper settings, convex", amp_floor=ROUGH_AMP_FLOOR, dt_max=1e-2,
                       dt_q99=1e-3)
    assert len(arr) > 100


def test_convex_synthetic_aperture_parity(ur):
    """Synthetic-aperture transmits of a convex array: rays at angles to the local normal of an
    edge element and of an inner one."""
    w = convex(phantoms.tiny(n_rays=30_000), alpha_deg=10.0)
    tx = [(oracle.TX_SYNTHETIC, 0.0, 0.0), (oracle.TX_SYNTHETIC, 17.0, 0.0)]
    w["angles"] = np.zeros(len(tx), np.float32)
    w["transmits"] = tx
    G = run_gpu(ur, w, capacity=4 * len(tx) * w["n_rays"])
    arr, topo, _ = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], w["seed"], w["max_bounces"],
                                w["max_path"], topo=True, transmits=tx)
    res = check_trace_parity(w, G, arr, topo, "convex synthetic aperture", amp_floor=CONVEX_AMP_FLOOR)
    assert res["n_matched"] >= 0.999 * len(arr) and len(arr) > 200
