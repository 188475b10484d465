"""Pins of the oracle's triangle-mesh boundaries (the paper's bone is a CT-derived
mesh, Sec. 4; its triangles are surfaces like any other, Eqs. 7-12).

A two-triangle quad gives exactly the arrivals of the analytic plane it lies in
(intersection, sidedness, skipping, connections through it); a quad tilted by
beta under a plane wave steered by beta sends every ray back along itself
(triangle normals); a closed attenuating box in front of a reflector scales the
echo of every ray that crosses it by exp(-2 a h) (closed meshes, media on both
sides, entering and leaving).
"""
import math

import numpy as np
import pytest

import oracle
import phantoms

C = 1540.0
WATER = (C, 1.54, 0.0, 0.0)
DENSE = (C, 3.0, 0.0, 0.0)          # same sound speed: r = (Z2 - Z1) / (Z2 + Z1) at every angle


def f32(x):
    return float(np.float32(x))


def r_dense():
    z1, z2 = f32(1.54), f32(3.0)
    return (z2 - z1) / (z2 + z1)


def canonical_events(ev):
    """Transducer-sampling events of rough vertices carry the vertex's hit id + 1 in bits 0..23,
    which differ between a plane and the quad replacing it: map them to 1."""
    ev = ev.astype(np.uint32).copy()
    rough = ((ev >> np.uint32(31)) == 1) & ((ev & np.uint32(0xFFFFFF)) != 0)
    ev[rough] = (ev[rough] & np.uint32(0xFF000000)) | np.uint32(1)
    return ev


@pytest.mark.parametrize("roughness,radius", [(0.0, 0.0), (0.4, 0.0), (0.0, 0.04)])
def test_quad_mesh_equals_the_analytic_plane(roughness, radius):
    """Tiny phantom (plane at 15 mm, sphere, scatterers), steered plane waves, Monte Carlo mode: the
    plane replaced by a quad covering every ray's crossing gives the same arrivals bit for bit
    (times and amplitudes to rounding), smooth, with the medium below it rough (GGX), and under a
    convex array."""
    w = phantoms.tiny(n_rays=20_000)
    a = dict(w["array"], alpha_m_deg=10.0, alpha_c_deg=15.0, radius=float(np.float32(radius)))
    ang = np.deg2rad([-8.0, 5.0]).astype(np.float32)
    s = dict(w["scene"])
    med = [list(m) for m in s["media"]]
    med[s["boundaries"][0][2]][3] = roughness              # the medium below the plane
    s["media"] = [tuple(m) for m in med]
    (kind, p, m_neg, m_pos), rest = s["boundaries"][0], s["boundaries"][1:]
    assert kind == oracle.PLANE_Z
    mesh = dict(s, boundaries=rest, triangles=phantoms.triangles((phantoms.mesh_quad(p[0], -0.1, 0.1, -0.1, 0.1),
                                                                  m_neg, m_pos)))
    ref, _, rst = oracle.trace(s, a, ang, 20_000, 4, 4)
    got, _, gst = oracle.trace(mesh, a, ang, 20_000, 4, 4)
    assert got.size == ref.size > 1000
    for f in ("tx", "el", "ray"):
        assert np.array_equal(got[f], ref[f]), f
    assert np.array_equal(canonical_events(got["event"]), canonical_events(ref["event"]))
    if roughness:
        ev = ref["event"].astype(np.uint32)
        assert np.any(((ev >> np.uint32(31)) == 1) & ((ev & np.uint32(0xFFFFFF)) != 0))   # rough vertices sampled
        assert np.any(canonical_events(got["event"]) != got["event"])   # at the quad's triangles
    np.testing.assert_allclose(got["t"], ref["t"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(got["amp"], ref["amp"], rtol=1e-12, atol=0)
    assert gst["interactions"] == rst["interactions"] and gst["connections"] == rst["connections"]


@pytest.mark.parametrize("beta_deg", [0.0, 7.0, -12.0])
def test_tilted_quad_retroreflects_a_matching_plane_wave(beta_deg):
    """Quad through (0, D) with normal (sin b, 0, cos b) under the plane wave steered by b: each ray
    returns to its emission point along itself, at tau_e + 2 (D cos b - x sin b) / c with x within
    half a pitch of the element centre, weight r cos b / N."""
    beta = math.radians(beta_deg)
    D = 12e-3
    quad = phantoms.mesh_tilted_quad((0.0, D), beta, 0.03, 0.03)
    scene = {"media": [WATER, DENSE], "boundaries": [], "med_array": 0, "z_max": 0.04,
             "scatterers": np.zeros((0, 4), np.float32), "r_s": 1e-4,
             "triangles": phantoms.triangles((quad, 0, 1))}
    n_el, N = 64, 64 * 100
    a = phantoms.array_params(n_el, 2048, c_bf=C, alpha_m_deg=20.0, alpha_c_deg=20.0)
    ang = np.array([beta], np.float32)
    arr, _, st = oracle.trace(scene, a, ang, N, 9, 1, mode=oracle.MODE_EXPECT)
    assert arr.size == N                                   # every ray comes back
    assert np.array_equal(arr["el"], arr["ray"] % n_el)    # to the element it left
    b32 = float(np.float32(beta))
    np.testing.assert_allclose(arr["amp"], r_dense() * math.cos(b32) / N, rtol=1e-9)
    p, fs, c = a["pitch"], a["fs"], f32(C)
    xe = (arr["el"] - 0.5 * (n_el - 1)) * p
    xe_all = (np.arange(n_el) - 0.5 * (n_el - 1)) * p
    tau = (xe * math.sin(b32) - (xe_all * math.sin(b32)).min()) / a["c_bf"] * fs
    # the quad's plane: n . x = D cos b (float32 vertices: within 1e-9 m)
    expect = tau + 2 * (D * math.cos(b32) - xe * math.sin(b32)) / c * fs
    assert np.abs(arr["t"] - expect).max() <= p * abs(math.sin(b32)) / c * fs + 1e-4


def test_closed_box_attenuates_the_rays_that_cross_it():
    """A closed box (12 triangles) of lossy water (same c and Z, attenuation a) between the array and
    a reflecting plane: at normal incidence a ray under the box crosses its height h twice and
    returns with r exp(-2 a h) / N; rays beside it with r / N."""
    lossy = (C, 1.54, 2.0, 0.0)
    zp, h = f32(20e-3), 4e-3
    box = phantoms.mesh_box((-2e-3, -1e-3, 6e-3), (2e-3, 1e-3, 6e-3 + h))
    scene = {"media": [WATER, DENSE, lossy], "boundaries": [(oracle.PLANE_Z, [zp, 0, 0, 0], 0, 1)],
             "med_array": 0, "z_max": 0.04, "scatterers": np.zeros((0, 4), np.float32), "r_s": 1e-4,
             "triangles": phantoms.triangles((box, 2, 0))}
    a = phantoms.array_params(32, 2048, c_bf=C)
    N = 32 * 400
    # five interactions: into the box, out of it, the reflector, into the box and out again
    arr, _, _ = oracle.trace(scene, a, np.zeros(1, np.float32), N, 2, 5, mode=oracle.MODE_EXPECT)
    assert arr.size == N
    att = 2.0 * (a["f0"] * 1e-6) * 100.0 / (20.0 * math.log10(math.e))   # dB/cm/MHz at f0 -> Np/m
    h32 = f32(6e-3 + h) - f32(6e-3)
    ratio = arr["amp"] * N / r_dense()
    inside = ratio < 0.999
    assert 0.05 < inside.mean() < 0.5                      # the box covers part of the beam
    # only elements under the box (|x| <= 2 mm, within half a pitch) see attenuated echoes
    xe = (arr["el"] - 0.5 * (a["n_el"] - 1)) * a["pitch"]
    assert np.all(np.abs(xe[inside]) <= 2e-3 + 0.5 * a["pitch"])
    under = np.abs(xe) < 2e-3 - 0.5 * a["pitch"]
    assert 0.4 < inside[under].mean() < 0.6                # |y| <= 1 mm of the 4 mm elevation
    np.testing.assert_allclose(ratio[inside], math.exp(-2 * att * h32), rtol=1e-9)
    np.testing.assert_allclose(ratio[~inside], 1.0, rtol=1e-12)
    np.testing.assert_allclose(arr["t"], 2 * zp * a["fs"] / f32(C), rtol=1e-12)


def test_invalid_meshes_are_rejected():
    w = phantoms.tiny(n_rays=100)
    q = phantoms.mesh_quad(0.01, -0.01, 0.01, -0.01, 0.01)
    for tri, med in ((q, np.array([[0, 5], [0, 1]], np.int32)),              # medium out of range
                     (np.zeros((1, 9), np.float32), np.array([[0, 1]], np.int32))):   # degenerate
        s = dict(w["scene"], triangles=(tri, med))
        with pytest.raises(ValueError):
            oracle.trace(s, w["array"], w["angles"], 100, 0, 1)
