"""Rough (GGX, Eq. 12) boundaries on the CUDA path against the FP64 oracle, through
the C ABI: path topology, per-arrival time/amplitude/element (including the
secondary rays of rough vertices), channel data; the small-roughness limit
against the smooth trace; and the calls that refuse rough scenes.  Bars as in
test_gpu_trace.py, except that per-arrival amplitudes below 1e-4 of the largest are
compared against that floor: secondary rays of rough vertices reach far into the BSDF tails
(amplitudes down to 1e-6 of the peak), where FP32 cancellations in grazing Fresnel and
connection factors exceed 1e-4 relative while the channel data stay within 1e-4."""
import numpy as np
import pytest

import oracle
import phantoms
from _parity import rel_l2
from test_gpu_trace import check_trace_parity, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

ROUGH_AMP_FLOOR = 1e-4


@pytest.fixture(scope="module")
def ur():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05828_gb300 as ur
    ur.lib()
    return ur


def with_roughness(w, medium, alpha):
    w = dict(w)
    s = dict(w["scene"])
    med = [list(m) for m in s["media"]]
    med[medium][3] = float(np.float32(alpha))
    s["media"] = [tuple(m) for m in med]
    w["scene"] = s
    return w


def secondary(rec):
    return rec[((rec["event"] >> 31) == 1) & ((rec["event"] & 0xFFFFFF) != 0)]


def test_tiny_rough_sphere(ur):
    """Bone sphere with the paper's bone roughness 0.5; 1e5 rays."""
    w = with_roughness(phantoms.tiny(), 2, 0.5)
    G = run_gpu(ur, w)
    arr, topo, ost = run_oracle(w)
    res = check_trace_parity(w, G, arr, topo, "tiny rough", amp_floor=ROUGH_AMP_FLOOR)
    assert secondary(arr).size > 100                       # rough vertices send secondary rays
    assert res["n_matched"] >= 0.999 * len(arr)
    assert G["stats"]["connections"] > 0


def test_layered_rough_bone(ur):
    """Layered phantom with a rough bone cylinder (0.5) and rough fat (0.1): planes then
    take the fat's roughness, so every boundary is rough."""
    w = phantoms.layered(n_rays=20_000)
    w = with_roughness(with_roughness(w, 3, 0.5), 1, 0.1)
    G = run_gpu(ur, w)
    arr, topo, _ = run_oracle(w)
    check_trace_parity(w, G, arr, topo, "layered rough", amp_floor=ROUGH_AMP_FLOOR)
    assert secondary(arr).size > 0


def test_steered_rough_plane(ur):
    """A rough bone plane under a 50 degree transmit (shadowing matters) and a -20 degree one."""
    media = [(1540.0, 1.54, 0.0, 0.0), (3500.0, 7.8, 0.0, 0.8)]
    scene = {"media": media, "boundaries": [(oracle.PLANE_Z, [0.02, 0.0, 0.0, 0.0], 0, 1)], "med_array": 0,
             "z_max": 0.04, "scatterers": np.zeros((0, 4), np.float32), "r_s": 1e-4}
    arr_p = phantoms.array_params(32, 2048, elev_h=2e-3, c_bf=1540.0, alpha_m_deg=30.0, alpha_c_deg=60.0)
    x, z = phantoms.image_grid(arr_p, 64, 64)
    w = {"scene": scene, "array": arr_p, "angles": np.deg2rad([50.0, -20.0]).astype(np.float32),
         "n_rays": 200_000, "seed": 9, "max_bounces": 3, "max_path": 0.2, "x_px": x, "z_px": z,
         "dyn_range_db": 60.0}
    G = run_gpu(ur, w, capacity=3 * 2 * w["n_rays"])      # about one secondary-ray return per ray
    arr, topo, _ = run_oracle(w)
    check_trace_parity(w, G, arr, topo, "rough plane", amp_floor=ROUGH_AMP_FLOOR)
    assert secondary(arr).size > 1000


def test_small_roughness_matches_the_smooth_gpu_trace(ur):
    """alpha = 1e-9: microfacet normals within 1e-9 rad of the macro normal, the direct hits
    take the whole weight; the trace equals the smooth kernel's (rare FP32 threshold flips
    aside)."""
    w = phantoms.tiny(n_rays=50_000)
    smooth = run_gpu(ur, w)
    rough = run_gpu(ur, with_roughness(w, 2, 1e-9))
    assert np.mean(smooth["hash"] == rough["hash"]) >= 0.9999
    assert rel_l2(rough["rf"], smooth["rf"]) < 1e-3
    assert rel_l2(rough["quad"], smooth["quad"]) < 1e-3
    sec = secondary(rough["rec"])
    assert sec.size > 0 and np.abs(sec["amp"]).max() < 1e-9 * np.abs(smooth["rec"]["amp"]).max()


def test_rough_scenes_refused_where_unsupported(ur):
    import torch
    w = with_roughness(phantoms.tiny(n_rays=1000), 2, 0.5)
    sim = ur.Simulator(0)
    sim.load(w)
    g = torch.zeros((1, 32, 1536), dtype=torch.float32, device="cuda")
    with pytest.raises(ur.URError):
        sim.trace_adjoint(1000, 0, 4, g, g, n_med=3, n_scat=200)
    med = np.array(w["scene"]["media"], np.float32)
    with pytest.raises(ur.URError):
        sim.set_media(med, sampling=med)
    bad = med.copy()
    bad[2, 3] = -0.5
    with pytest.raises(ur.URError):
        sim.set_media(bad)
    sim.close()


def test_paper_settings_phantom(ur):
    """The paper's acquisition settings (25 plane waves over [-30, 30] degrees, fs 50 MHz, 10 bounces,
    2-degree directivity) on the rough vertebra stand-in: every transmit against the oracle.
    Time bar: FP32 hit points carry errors of a few nm; on a 10 mm sphere a normal then tilts by
    about 1e-7 rad per bounce, and over the tens of millimetres that follow the arrival moves by
    up to about 1e-8 m = 3e-4 samples at 50 MHz per curved bounce.  Paths with several bounces in the
    bone reach a few 1e-3 samples: bar 1e-3 samples for 99 % of the arrivals and 1e-2 for all."""
    w = phantoms.paper_like(n_rays=4000)
    G = run_gpu(ur, w, capacity=4 * 25 * w["n_rays"])
    assert G["stats"]["rays"] == 25 * w["n_rays"]
    arr, topo, _ = run_oracle(w)
    check_trace_parity(w, G, arr, topo, "paper settings", amp_floor=ROUGH_AMP_FLOOR, dt_max=1e-2, dt_q99=1e-3)
    assert secondary(arr).size > 0
