"""ur_beamform_noalloc: the allocation-free beamforming entry point for callers
that cannot let the library call cudaMalloc (real-time loops that forbid
allocation after start-up, hosts that give all device memory to their own pool,
plug-ins inside frameworks that own every device buffer).  Its output must equal
ur_beamform's on the same channel data, call after call, and a repeated call
must not change the device's free memory.  Collected last on purpose."""
import numpy as np
import pytest

import phantoms
from _parity import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05828_gb300 as ur
    w = phantoms.tiny(n_rays=50_000)
    w["angles"] = np.deg2rad(np.array([-6.0, 0.0, 4.0])).astype(np.float32)
    sim = ur.Simulator(0)
    sim.load(w)
    rf, quad = sim.trace(w["n_rays"], 0, w["max_bounces"], w["max_path"])
    iq, env, db = sim.beamform(rf, quad, w["x_px"], w["z_px"], 60.0)
    torch.cuda.synchronize()
    return torch, ur, w, sim, rf, quad, iq, env, db


def test_noalloc_matches_beamform_twice(setup):
    torch, ur, w, sim, rf, quad, iq_ref, env_ref, db_ref = setup
    nz, nx = env_ref.shape
    strong = (env_ref > 1e-3 * env_ref.max()).cpu().numpy()
    for call in range(2):
        iq = torch.full((nz, nx, 2), float("nan"), device=rf.device)
        env = torch.full((nz, nx), float("nan"), device=rf.device)
        db = torch.full((nz, nx), float("nan"), device=rf.device)
        free_before = torch.cuda.mem_get_info()[0]
        sim.beamform_noalloc(rf, quad, w["x_px"], w["z_px"], 60.0, iq=iq, env=env, db=db)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before
        a = iq.double().cpu().numpy()
        b = iq_ref.double().cpu().numpy()
        assert rel_l2(a[..., 0] + 1j * a[..., 1], b[..., 0] + 1j * b[..., 1]) <= 1e-5
        assert rel_l2(env.double().cpu().numpy(), env_ref.double().cpu().numpy()) <= 1e-5
        d = np.abs(db.double().cpu().numpy() - db_ref.double().cpu().numpy())
        assert d[strong].max() <= 1e-3


def test_noalloc_db_only_uses_its_own_envelope(setup):
    torch, ur, w, sim, rf, quad, iq_ref, env_ref, db_ref = setup
    nz, nx = env_ref.shape
    strong = (env_ref > 1e-3 * env_ref.max()).cpu().numpy()
    for call in range(2):
        db = torch.full((nz, nx), float("nan"), device=rf.device)
        sim.beamform_noalloc(rf, quad, torch.from_numpy(w["x_px"]).cuda(), torch.from_numpy(w["z_px"]).cuda(), 60.0,
                             db=db)
        torch.cuda.synchronize()
        d = np.abs(db.double().cpu().numpy() - db_ref.double().cpu().numpy())
        assert d[strong].max() <= 1e-3 and np.isfinite(db.cpu().numpy()).all()


def test_noalloc_rejects_oversized_requests(setup):
    torch, ur, w, sim, rf, quad, iq_ref, env_ref, db_ref = setup
    too_wide = np.linspace(-1e-3, 1e-3, 8193).astype(np.float32)
    out = torch.empty((w["z_px"].size, 8193), device=rf.device)
    with pytest.raises(ur.URError) as e:
        sim.beamform_noalloc(rf, quad, too_wide, w["z_px"], 60.0, env=out)
    assert e.value.code == 1
    big_x = np.linspace(-1e-3, 1e-3, 4096).astype(np.float32)
    big_z = np.linspace(1e-3, 2e-2, 512).astype(np.float32)      # 2^21 pixels, no caller envelope
    db = torch.empty((512, 4096), device=rf.device)
    with pytest.raises(ur.URError) as e:
        sim.beamform_noalloc(rf, quad, big_x, big_z, 60.0, db=db)
    assert e.value.code == 1
    with pytest.raises(ur.URError):                               # host outputs are refused
        sim.beamform_noalloc(rf, quad, w["x_px"], w["z_px"], 60.0, db=torch.empty(env_ref.shape))


def _cplx(t):
    a = t.double().cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def test_noalloc_single_outputs(setup):
    """Only the complex image, then only the envelope: each equals ur_beamform's."""
    torch, ur, w, sim, rf, quad, iq_ref, env_ref, db_ref = setup
    nz, nx = env_ref.shape
    for call in range(2):
        iq = torch.full((nz, nx, 2), float("nan"), device=rf.device)
        sim.beamform_noalloc(rf, quad, w["x_px"], w["z_px"], 60.0, iq=iq)
        env = torch.full((nz, nx), float("nan"), device=rf.device)
        sim.beamform_noalloc(rf, quad, w["x_px"], w["z_px"], 60.0, env=env)
        torch.cuda.synchronize()
        assert rel_l2(_cplx(iq), _cplx(iq_ref)) <= 1e-5
        assert rel_l2(env.double().cpu().numpy(), env_ref.double().cpu().numpy()) <= 1e-5


def test_noalloc_follows_changed_transmits(setup):
    """The per-transmit tables are rebuilt by every call: after new plane-wave angles the
    output equals ur_beamform's for the new angles, and after restoring them, for the old."""
    torch, ur, w, sim, rf, quad, iq_ref, env_ref, db_ref = setup
    nz, nx = env_ref.shape
    new = np.deg2rad(np.array([-11.0, 2.0, 9.0])).astype(np.float32)
    try:
        for angles in (new, w["angles"]):
            sim.set_plane_waves(angles)
            ref, _, _ = sim.beamform(rf, quad, w["x_px"], w["z_px"], 60.0, env=False, db=False)
            iq = torch.full((nz, nx, 2), float("nan"), device=rf.device)
            sim.beamform_noalloc(rf, quad, w["x_px"], w["z_px"], 60.0, iq=iq)
            torch.cuda.synchronize()
            assert rel_l2(_cplx(iq), _cplx(ref)) <= 1e-5
        assert rel_l2(_cplx(iq), _cplx(iq_ref)) <= 1e-5
    finally:
        sim.set_plane_waves(w["angles"])
