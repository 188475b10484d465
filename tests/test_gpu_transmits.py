"""Diverging and focused transmits on the CUDA path against the FP64 oracle,
through the C ABI: path topology, arrivals and channel data of a mixed set of
transmits, their delay-and-sum images, and the calls that refuse them.  Bars as
in test_gpu_trace.py."""
import numpy as np
import pytest

import oracle
import phantoms
from _parity import rel_l2
from test_gpu_trace import check_trace_parity, run_gpu

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
