"""Triangle-mesh boundaries on the CUDA path (BVH traversal in the extended
tracer) against the FP64 oracle's brute force over every triangle, through the
C ABI: path topology, arrivals and channel data for a quad standing in for a
plane (smooth and rough), a closed lossy box, a rough bone icosphere with
scatterers, a convex array over a mesh, and the paper's acquisition with its bone
as meshes; plus the calls that refuse meshes.  Bars as in test_gpu_trace.py
(rough scenes: the amplitude floor of test_gpu_rough.py; curved rough bone at
50 MHz: the time bars of the paper-settings test)."""
import numpy as np
import pytest

import oracle
import phantoms
from _parity import rel_l2
from test_gpu_rough import ROUGH_AMP_FLOOR
from test_gpu_trace import check_trace_parity, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ur():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05828_gb300 as ur
    ur.lib()
    return ur


def quad_scene(roughness):
    w = phantoms.tiny(n_rays=30_000)
    w["array"] = dict(w["array"], alpha_m_deg=12.0, alpha_c_deg=12.0)   # a wider step directivity
    s = dict(w["scene"])
    med = [list(m) for m in s["media"]]
    (kind, p, m_neg, m_pos), rest = s["boundaries"][0], s["boundaries"][1:]
    med[m_pos][3] = roughness
    s["media"] = [tuple(m) for m in med]
    s["boundaries"] = rest
    s["triangles"] = phantoms.triangles((phantoms.mesh_quad(p[0], -0.1, 0.1, -0.1, 0.1), m_neg, m_pos))
    w["scene"] = s
    w["angles"] = np.deg2rad([-8.0, 5.0]).astype(np.float32)
    return w


@pytest.mark.parametrize("roughness", [0.0, 0.4])
def test_quad_mesh_parity(ur, roughness):
    w = quad_scene(roughness)
    G = run_gpu(ur, w, capacity=6 * 2 * w["n_rays"])
    arr, topo, _ = run_oracle(w)
    # rough: the muscle around the bone sphere is rough too, so the time bars of curved rough bounces apply
    bars = dict(amp_floor=ROUGH_AMP_FLOOR, dt_max=1e-2, dt_q99=1e-3) if roughness else {}
    res = check_trace_parity(w, G, arr, topo, "quad mesh", **bars)
    assert res["n_matched"] >= 0.999 * len(arr) and len(arr) > 1000
    assert G["stats"]["rays"] == 2 * w["n_rays"]


def test_closed_box_parity(ur):
    lossy = (1540.0, 1.54, 2.0, 0.0)
    w = phantoms.tiny(n_rays=20_000)
    s = dict(w["scene"])
    s["media"] = list(s["media"]) + [lossy]
    box = phantoms.mesh_box((-3e-3, -1e-3, 6e-3), (3e-3, 1e-3, 10e-3))
    s["triangles"] = phantoms.triangles((box, len(s["media"]) - 1, 0))
    w["scene"] = s
    w["max_bounces"] = 8
    G = run_gpu(ur, w)
    arr, topo, _ = run_oracle(w)
    res = check_trace_parity(w, G, arr, topo, "closed box")
    assert res["n_matched"] >= 0.999 * len(arr)


def icosphere_workload(n_rays, subdiv=3, rough=0.5, convex=False):
    """Water over a rough bone icosphere (r 4 mm at 20 mm) holding 300 scatterers, 3 steered plane
    waves, a 12-degree step directivity."""
    rng = np.random.default_rng(4)
    water, bone = (1540.0, 1.54, 0.0, 0.0), (3500.0, 7.8, 10.0, rough)
    ctr, r = np.array([1e-3, 0.0, 20e-3]), 4e-3
    d = rng.normal(size=(300, 3))
    pts = ctr + d / np.linalg.norm(d, axis=1)[:, None] * r * rng.uniform(0, 0.9, (300, 1))
    sc = np.column_stack([pts, rng.standard_normal(300)]).astype(np.float32)
    arr = phantoms.array_params(32, 1536, c_bf=1540.0, alpha_m_deg=12.0, alpha_c_deg=12.0)
    if convex:
        arr["radius"] = float(np.float32(0.04))
    scene = {"media": [water, bone], "boundaries": [], "med_array": 0, "z_max": 0.035, "scatterers": sc,
             "r_s": 1e-4, "triangles": phantoms.triangles((phantoms.mesh_icosphere(ctr, r, subdiv), 1, 0))}
    return {"scene": scene, "array": arr, "angles": np.deg2rad([-6.0, 0.0, 9.0]).astype(np.float32),
            "n_rays": n_rays, "seed": 2, "max_bounces": 6, "max_path": 0.2,
            "x_px": np.linspace(-4e-3, 4e-3, 64).astype(np.float32),
            "z_px": np.linspace(2e-3, 28e-3, 128).astype(np.float32), "dyn_range_db": 60.0}


@pytest.mark.parametrize("rough", [0.0, 0.5])
def test_icosphere_parity(ur, rough):
    w = icosphere_workload(20_000, rough=rough)
    G = run_gpu(ur, w, capacity=6 * 3 * w["n_rays"])
    arr, topo, _ = run_oracle(w)
    res = check_trace_parity(w, G, arr, topo, "icosphere", amp_floor=ROUGH_AMP_FLOOR if rough else 0.0,
                             dt_max=1e-2, dt_q99=1e-3)
    assert res["n_matched"] >= 0.999 * len(arr) and len(arr) > 500
    if rough:   # transducer sampling at the triangles (hit id + 1 >= 4 with no analytic boundaries)
        ev = arr["event"].astype(np.uint32)
        assert np.any(((ev >> np.uint32(31)) == 1) & ((ev & np.uint32(0xFFFFFF)) >= 4))


def test_convex_array_over_a_mesh(ur):
    w = icosphere_workload(20_000, convex=True)
    G = run_gpu(ur, w, capacity=6 * 3 * w["n_rays"])
    arr, topo, _ = run_oracle(w)
    res = check_trace_parity(w, G, arr, topo, "convex over icosphere", amp_floor=ROUGH_AMP_FLOOR, dt_max=1e-2,
                             dt_q99=1e-3)
    assert res["n_matched"] >= 0.999 * len(arr) and len(arr) > 200


def test_paper_settings_with_mesh_bone(ur):
    """The paper's acquisition (25 plane waves, 50 MHz, 10 bounces, rough bone) with the bone as
    triangle meshes: icosphere body and prism processes (1536 triangles at this size)."""
    w = phantoms.paper_mesh_like(n_rays=2000, subdiv=3, n_seg=32)
    G = run_gpu(ur, w, capacity=6 * 25 * w["n_rays"])
    assert G["stats"]["rays"] == 25 * w["n_rays"]
    arr, topo, _ = run_oracle(w)
    check_trace_parity(w, G, arr, topo, "paper settings, mesh bone", amp_floor=ROUGH_AMP_FLOOR, dt_max=1e-2,
                       dt_q99=1e-3)
    assert len(arr) > 100


def test_meshes_refused_where_unsupported(ur):
    import torch
    w = quad_scene(0.0)
    sim = ur.Simulator(0)
    sim.load(w)
    g = torch.zeros((2, 32, 1536), dtype=torch.float32, device="cuda")
    with pytest.raises(ur.URError):
        sim.trace_adjoint(1000, 0, 4, g, g, n_med=3, n_scat=200)
    q = phantoms.mesh_quad(0.01, -0.01, 0.01, -0.01, 0.01)
    for tri, med in ((q, np.array([[0, 5], [0, 1]], np.int32)), (np.zeros((1, 9), np.float32), np.array([[0, 1]])),
                     (np.full((1, 9), np.nan, np.float32), np.array([[0, 1]]))):
        with pytest.raises(ur.URError):
            sim.set_triangles(tri, med)
    with pytest.raises(ur.URError):                       # no scene in slot 3
        sim.set_triangles(q, np.array([[0, 1], [0, 1]]), slot=3)
    # removing the mesh gives the scene without it
    sim.set_triangles(np.zeros((0, 9), np.float32), np.zeros((0, 2), np.int32))
    rf0, q0, st0, _, _ = sim.trace_debug(2000, 1, 4, capacity=20_000)
    ref = ur.Simulator(0)
    ref.load(dict(w, scene=dict(w["scene"], triangles=None)))
    rf1, q1, st1, _, _ = ref.trace_debug(2000, 1, 4, capacity=20_000)
    assert st0 == st1
    assert rel_l2(rf0.double().cpu().numpy(), rf1.double().cpu().numpy()) <= 1e-6   # atomics' order aside
    sim.close()
    ref.close()


def test_contexts_release_mesh_and_mixing_buffers(ur):
    """Creating, using and destroying contexts with meshes and mixed traces returns the device memory
    (the hierarchy, the triangles, the mixed ray order)."""
    import torch
    w = icosphere_workload(20_000)
    w["mix"] = True

    def cycle():
        sim = ur.Simulator(0)
        sim.load(w)
        sim.trace(w["n_rays"], 1, 4)
        sim.close()
    cycle()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        cycle()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (16 << 20)
