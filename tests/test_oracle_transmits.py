"""Pins of the oracle's diverging and focused transmits (Sec. 2.3 "Ray Emission").

The paper names focused and diverging wavefronts beside plane waves without
formulas; the oracle's readings (lateral delays of a virtual source or a focus,
rays along the line from the source / toward the focus, Eq. 6 cosine weight)
are pinned against geometry: which rays meet a scatterer, when their echoes
arrive, and where the delay-and-sum image of a point target peaks.
"""
import math

import numpy as np
import pytest

import oracle
import phantoms

C = 1540.0
WATER = (C, 1.54, 0.0, 0.0)


def point_scene(p, r_s=1e-4):
    return {"media": [WATER], "boundaries": [], "med_array": 0, "z_max": 0.05,
            "scatterers": np.array([[p[0], 0.0, p[1], 1.0]], np.float32), "r_s": r_s}


def array(n_el=32, elev=5e-5, n_s=2048):
    a = phantoms.array_params(n_el, n_s, elev_h=elev, c_bf=C, alpha_m_deg=89.0, alpha_c_deg=89.0)
    return a


def element_x(a, e):
    return (e - 0.5 * (a["n_el"] - 1)) * a["pitch"]


def test_plane_kind_matches_the_angle_interface():
    w = phantoms.tiny(n_rays=5000)
    ang = np.deg2rad([-7.0, 4.0]).astype(np.float32)
    a0, t0, _ = oracle.trace(w["scene"], w["array"], ang, 5000, 3, 4, topo=True)
    a1, t1, _ = oracle.trace(w["scene"], w["array"], ang, 5000, 3, 4, topo=True,
                             transmits=[(oracle.TX_PLANE, 0.0, 0.0)] * 2)
    assert np.array_equal(t0, t1) and np.array_equal(a0, a1)


def test_focused_wave_passes_through_its_focus():
    """Every ray of a focused transmit passes the focus: a scatterer there is met by all rays
    (a plane wave meets it with about 2 r_s / aperture of them), and its echo at element e'
    arrives at (max_e |f - c_e| + |f - c_e'|) / c within the emission-point offset."""
    a = array()
    f = (2e-3, 20e-3)
    N = 4000
    tx = [(oracle.TX_FOCUSED, f[0], f[1])]
    arr, _, st = oracle.trace(point_scene(f), a, np.zeros(1, np.float32), N, 1, 0, mode=oracle.MODE_EXPECT,
                              transmits=tx)
    assert st["candidates"] == N * a["n_el"] // a["n_el"]        # every ray of the transmit
    _, _, st_pw = oracle.trace(point_scene(f), a, np.zeros(1, np.float32), N, 1, 0, mode=oracle.MODE_EXPECT)
    assert st_pw["candidates"] < 0.05 * N
    fs = a["fs"]
    dist = [math.hypot(element_x(a, e) - f[0], f[1]) for e in range(a["n_el"])]
    expect = (max(dist) + np.array(dist)[arr["el"]]) / C * fs
    bound = 0.5 * a["pitch"] / C * fs + 1e-6                   # emission point within half a pitch
    assert np.all(np.abs(arr["t"] - expect) <= bound)
    assert np.abs(arr["t"] - expect).mean() < 0.35 * bound     # offsets average out


def test_diverging_wave_comes_from_its_virtual_source():
    """A scatterer at s is met only by rays leaving the array where the line from the virtual
    source v through s crosses it; the echo at e' arrives at (|s - v| - min_e |c_e - v| +
    |s - c_e'|) / c within the emission-point offset."""
    a = array()
    v = (-3e-3, -10e-3)
    s = (4e-3, 25e-3)
    N = 32 * 3000
    arr, _, st = oracle.trace(point_scene(s), a, np.zeros(1, np.float32), N, 2, 0, mode=oracle.MODE_EXPECT,
                              transmits=[(oracle.TX_DIVERGING, v[0], v[1])])
    assert st["candidates"] > 0
    x_cross = v[0] + (s[0] - v[0]) * (-v[1]) / (s[1] - v[1])
    e_cross = int(round(x_cross / a["pitch"] + 0.5 * (a["n_el"] - 1)))
    emitters = np.unique(arr["ray"] % a["n_el"])
    assert set(emitters.tolist()) <= {e_cross - 1, e_cross, e_cross + 1}
    fs = a["fs"]
    mn = min(math.hypot(element_x(a, e) - v[0], v[1]) for e in range(a["n_el"]))
    rcv = np.array([math.hypot(element_x(a, e) - s[0], s[1]) for e in range(a["n_el"])])
    expect = (math.hypot(s[0] - v[0], s[1] - v[1]) - mn + rcv[arr["el"]]) / C * fs
    assert np.all(np.abs(arr["t"] - expect) <= 0.5 * a["pitch"] / C * fs + 1e-6)


@pytest.mark.parametrize("kind,pts", [(oracle.TX_DIVERGING, [(-5e-3, -8e-3), (0.0, -8e-3), (5e-3, -8e-3)]),
                                      (oracle.TX_FOCUSED, [(-3e-3, 30e-3), (0.0, 30e-3), (3e-3, 30e-3)])])
def test_das_images_a_point_target_where_it_is(kind, pts):
    a = array(n_el=64, elev=4e-3, n_s=2048)
    target = (1.5e-3, 18e-3)
    scene = point_scene(target, r_s=2e-4)
    ang = np.zeros(len(pts), np.float32)
    tx = [(kind, x, z) for x, z in pts]
    arr, _, _ = oracle.trace(scene, a, ang, 64 * 400, 4, 0, mode=oracle.MODE_EXPECT, transmits=tx)
    rf, quad = oracle.deposit(a, len(pts), arr)
    x = np.linspace(-4e-3, 6e-3, 101).astype(np.float32)
    z = np.linspace(14e-3, 22e-3, 81).astype(np.float32)
    img = oracle.beamform(a, ang, rf, quad, x, z, transmits=tx)
    iz, ix = np.unravel_index(np.argmax(np.abs(img)), img.shape)
    assert abs(x[ix] - target[0]) <= 2e-4 and abs(z[iz] - target[1]) <= 2e-4
    # with the transmit delays of plane waves instead, the same data focus elsewhere or blur
    img_pw = oracle.beamform(a, ang, rf, quad, x, z)
    assert np.abs(img_pw).max() < 0.8 * np.abs(img).max()


def test_invalid_transmits_are_rejected():
    a = array()
    for tx in ([(oracle.TX_DIVERGING, 0.0, 5e-3)], [(oracle.TX_FOCUSED, 0.0, -5e-3)], [(7, 0.0, 1.0)]):
        with pytest.raises(ValueError):
            oracle.trace(point_scene((0.0, 0.02)), a, np.zeros(1, np.float32), 100, 0, 0, transmits=tx)
