"""Batches of (scene, transmit) items with uneven ray counts in one persistent
launch, their CUDA-graph replay, and the autotuner: every item must equal the
single-scene path (itself checked against the oracle), and items of a scene
other than slot 0 are also checked against the oracle directly."""
import numpy as np
import pytest

import oracle
import phantoms
from _parity import rel_l2

pytestmark = pytest.mark.gpu

ANGLES = np.deg2rad(np.array([-8.0, 0.0, 5.0, 11.0])).astype(np.float32)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05828_gb300 as ur
    a = phantoms.tiny(seed=0, n_rays=30_000)
    b = phantoms.tiny(seed=5, n_scat=1500, with_sphere=False, n_rays=30_000)
    for w in (a, b):
        w["angles"] = ANGLES
    # uneven rays per item; item streams = transmit index (as in ur_trace)
    items = [(0, 0, 20_000), (0, 2, 7_001), (1, 1, 33_333), (1, 3, 12_000), (0, 3, 9_000), (1, 0, 5_000)]
    return torch, ur, a, b, items


def single(ur, w, n, tx):
    sim = ur.Simulator(0)
    sim.load(w)
    rf, q = sim.trace(n, 0, w["max_bounces"], w["max_path"])
    sim.close()
    return rf[tx].double().cpu().numpy(), q[tx].double().cpu().numpy()


def planned(ur, a, b, items, capacity=0):
    sim = ur.Simulator(0)
    sim.load(a, slot=0)
    sim.load(b, slot=1)
    sim.batch_plan(items, a["x_px"], a["z_px"], capacity=capacity)
    return sim


def test_batch_items_equal_single_traces(env):
    torch, ur, a, b, items = env
    sim = planned(ur, a, b, items)
    rf, q = sim.batch_trace(0, 4)
    n, st = sim.batch_status()
    assert st["rays"] == sum(it[2] for it in items)
    for k, (scene, tx, nr) in enumerate(items):
        srf, sq = single(ur, a if scene == 0 else b, nr, tx)
        assert rel_l2(rf[k].double().cpu().numpy(), srf) <= 1e-6, (k, scene, tx)
        assert rel_l2(q[k].double().cpu().numpy(), sq) <= 1e-6


def test_large_items_trace_every_ray(env):
    """Items of 1e5-4e5 rays: tracer warps claim slot pools of consecutive items within one
    pass; every planned ray is traced and items still equal single traces."""
    torch, ur, a, b, items = env
    big = [(s, tx, 12 * n) for s, tx, n in items]
    sim = planned(ur, a, b, big)
    rf, q = sim.batch_trace(0, 4)
    n, st = sim.batch_status()
    assert st["rays"] == sum(it[2] for it in big)
    for k in (0, 2):
        scene, tx, nr = big[k]
        srf, sq = single(ur, a if scene == 0 else b, nr, tx)
        assert rel_l2(rf[k].double().cpu().numpy(), srf) <= 1e-6, (k, scene, tx)
        assert rel_l2(q[k].double().cpu().numpy(), sq) <= 1e-6


def test_batch_item_of_second_scene_matches_oracle(env):
    torch, ur, a, b, items = env
    sim = planned(ur, a, b, items)
    rf, q = sim.batch_trace(0, 4)
    k = 2                                     # scene 1, transmit 1, 33 333 rays
    scene, tx, nr = items[k]
    arr, _, _ = oracle.trace(b["scene"], b["array"], ANGLES, nr, 0, 4)
    arr = arr[arr["tx"] == tx]
    arr["tx"] = 0
    orf, oq = oracle.deposit(b["array"], 1, arr)
    assert rel_l2(rf[k].double().cpu().numpy(), orf[0]) <= 1e-4
    assert rel_l2(q[k].double().cpu().numpy(), oq[0]) <= 1e-4


def test_batch_images_equal_per_scene_compounding(env):
    torch, ur, a, b, items = env
    sim = planned(ur, a, b, items)
    rf, q = sim.batch_trace(0, 4)
    _, benv, bdb = sim.batch_beamform(rf, q, 60.0, env=True, db=True)
    assert benv.shape[0] == 2
    for img, (w, scene) in enumerate(((a, 0), (b, 1))):
        # same data through the single-context beamformer: stack this scene's items by transmit
        full_rf = torch.zeros((len(ANGLES), 32, w["array"]["n_s"]), device=rf.device)
        full_q = torch.zeros_like(full_rf)
        for k, (s, tx, _) in enumerate(items):
            if s == scene:
                full_rf[tx] += rf[k]
                full_q[tx] += q[k]
        ref = ur.Simulator(0)
        ref.load(w)
        _, renv, rdb = ref.beamform(full_rf, full_q, w["x_px"], w["z_px"], 60.0)
        assert rel_l2(benv[img].double().cpu().numpy(), renv.double().cpu().numpy()) <= 1e-5


def test_graph_replay_matches_direct_run(env):
    torch, ur, a, b, items = env
    side = torch.cuda.Stream()                     # the legacy default stream cannot be captured
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        _graph_replay(torch, ur, a, b, items)
    torch.cuda.synchronize()


def _graph_replay(torch, ur, a, b, items):
    sim = planned(ur, a, b, items)
    rf0, q0 = sim.batch_trace(0, 4)
    _, _, db0 = sim.batch_beamform(rf0, q0, 60.0)
    rf = torch.empty_like(rf0)
    q = torch.empty_like(q0)
    db = torch.empty_like(db0)
    torch.cuda.current_stream().synchronize()
    sim.graph_begin()
    sim.batch_trace(0, 4, rf=rf, quad=q)
    sim.batch_beamform(rf, q, 60.0, db=db)
    sim.graph_end()
    for _ in range(2):
        rf.zero_()
        db.fill_(1.0)
        sim.graph_launch()
        torch.cuda.current_stream().synchronize()
        assert rel_l2(rf.double().cpu().numpy(), rf0.double().cpu().numpy()) <= 1e-6
        strong = (db0 > -40).cpu().numpy()
        assert np.abs(db.cpu().numpy() - db0.cpu().numpy())[strong].max() <= 1e-3
    with pytest.raises(ur.URError) as e:          # synchronising calls are refused while capturing
        sim.graph_begin()
        try:
            sim.batch_status()
        finally:
            sim.graph_end()
    assert e.value.code == 6


def test_batch_overflow_is_reported(env):
    torch, ur, a, b, items = env
    sim = planned(ur, a, b, items, capacity=64)
    rf, q = sim.batch_trace(0, 4)
    with pytest.raises(ur.URError) as e:
        sim.batch_status()
    assert e.value.code == 4
    assert torch.isfinite(rf).all()


def test_autotune_keeps_parity(env):
    torch, ur, a, b, items = env
    w = phantoms.layered(n_rays=20_000)
    sim = ur.Simulator(0)
    sim.load(w)
    best = sim.autotune(200_000)
    assert best["cell_xy"] > 0 and best["cell_z"] > 0 and 1 <= best["resolve_batch"] <= 32
    rf, q = sim.trace(w["n_rays"], 0, w["max_bounces"], w["max_path"])
    arr, _, _ = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], 0, w["max_bounces"])
    orf, oq = oracle.deposit(w["array"], 1, arr)
    assert rel_l2(rf.double().cpu().numpy(), orf) <= 1e-3        # raw, all paths


def test_batch_with_rough_scene_and_point_source_transmits(env):
    """A batch whose scenes include a rough one and whose transmits include diverging and focused
    waves runs on the extended tracer; each item equals the single-scene trace."""
    torch, ur, a, b, items = env
    rough = dict(a)
    s = dict(a["scene"])
    med = [list(m) for m in s["media"]]
    med[2][3] = 0.5                                   # rough bone sphere
    s["media"] = [tuple(m) for m in med]
    rough["scene"] = s
    tx = [(ur.TX_DIVERGING, -2e-3, -10e-3), (ur.TX_PLANE, float(ANGLES[1]), 0.0), (ur.TX_FOCUSED, 1e-3, 20e-3),
          (ur.TX_PLANE, float(ANGLES[3]), 0.0)]
    for w in (rough, b):
        w["transmits"] = tx
    sim = ur.Simulator(0)
    sim.load(rough, slot=0)
    sim.load(b, slot=1)
    its = [(0, 0, 20_000), (1, 2, 15_000), (0, 2, 9_000), (1, 0, 12_000)]
    sim.batch_plan(its, a["x_px"], a["z_px"])
    rf, q = sim.batch_trace(0, 4)
    n, st = sim.batch_status()
    assert st["rays"] == sum(it[2] for it in its)
    for k, (scene, t, nr) in enumerate(its):
        srf, sq = single(ur, rough if scene == 0 else b, nr, t)
        assert rel_l2(rf[k].double().cpu().numpy(), srf) <= 1e-6, (k, scene, t)
        assert rel_l2(q[k].double().cpu().numpy(), sq) <= 1e-6
    sim.close()
