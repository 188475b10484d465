"""Pins of the oracle's convex array (Sec. 2.3: a transducer described by its
elements, elevation, radius and opening angle; the paper's probe is a 128-element
convex array with a 70-degree opening, Sec. 4).  The readings (elements `pitch`
apart on an arc about (0, 0, -R), radial normals, emission from the element's arc
face, the probe's cylinder as the receiving surface) are pinned by the flat
limit, a closed-form echo of a concentric shell and a point-target image.
"""
import math

import numpy as np
import pytest

import oracle
import phantoms

C = 1540.0
WATER = (C, 1.54, 0.0, 0.0)
BONE = (3500.0, 7.8, 0.0, 0.0)


def convex_array(radius, n_el=32, pitch=0.3e-3, elev=4e-3, n_s=2048, alpha_deg=10.0):
    a = phantoms.array_params(n_el, n_s, pitch=pitch, elev_h=elev, c_bf=C, alpha_m_deg=alpha_deg,
                              alpha_c_deg=alpha_deg + 5.0)
    a["radius"] = float(np.float32(radius))
    return a


def test_large_radius_recovers_the_linear_array():
    """With R = 1 km the arc departs from the plane by ~1e-8 m over the aperture: same paths,
    same arrivals, times within 1e-3 samples."""
    w = phantoms.tiny(n_rays=20_000)
    ang = np.deg2rad([0.0, 6.0]).astype(np.float32)
    a_lin, t_lin, _ = oracle.trace(w["scene"], w["array"], ang, 20_000, 1, 4, topo=True)
    arr = dict(w["array"])
    arr["radius"] = 1000.0
    a_cvx, t_cvx, _ = oracle.trace(w["scene"], arr, ang, 20_000, 1, 4, topo=True)
    assert np.mean(t_lin == t_cvx) >= 0.9999
    k_lin = {(int(t), int(r), int(e)): i for i, (t, r, e) in enumerate(zip(a_lin["tx"], a_lin["ray"], a_lin["event"]))}
    matched = [(k_lin[(int(t), int(r), int(e))], j) for j, (t, r, e) in
               enumerate(zip(a_cvx["tx"], a_cvx["ray"], a_cvx["event"])) if (int(t), int(r), int(e)) in k_lin]
    assert len(matched) >= 0.999 * len(a_lin)
    i, j = np.array(matched).T
    assert np.all(a_lin["el"][i] == a_cvx["el"][j])
    assert np.abs(a_lin["t"][i] - a_cvx["t"][j]).max() < 1e-3
    assert np.abs(a_lin["amp"][i] - a_cvx["amp"][j]).max() <= 1e-6 * np.abs(a_lin["amp"]).max()


@pytest.mark.parametrize("radius", [0.02, 0.05])
def test_concentric_shell_echo(radius):
    """A diverging wave from the centre of curvature leaves every point of the arc along its
    normal (weight 1/N), reflects at normal incidence on a concentric bone shell d beyond the arc
    and returns to the same element: each ray gives one echo at 2 d fs / c with amplitude r / N,
    r = (Z2 - Z1) / (Z2 + Z1)."""
    d = 10e-3
    a = convex_array(radius)
    scene = {"media": [WATER, BONE], "boundaries": [(oracle.CYL_Y, [0.0, -radius, radius + d, 0.0], 0, 1)],
             "med_array": 0, "z_max": 0.05, "scatterers": np.zeros((0, 4), np.float32), "r_s": 1e-4}
    N = 32 * 200
    arr, _, st = oracle.trace(scene, a, np.zeros(1, np.float32), N, 3, 1, mode=oracle.MODE_EXPECT,
                              transmits=[(oracle.TX_DIVERGING, 0.0, -radius)])
    z1, z2 = float(np.float32(1.54)), float(np.float32(7.8))   # the scene's float32 inputs
    r = (z2 - z1) / (z2 + z1)
    assert arr.size == N                                   # one echo per ray
    d_in = float(np.float32(radius + d)) - float(np.float32(radius))   # the shell as the float32 inputs place it
    np.testing.assert_allclose(arr["t"], 2 * d_in * a["fs"] / C, atol=1e-7)
    np.testing.assert_allclose(arr["amp"], r / N, rtol=1e-9)
    assert np.array_equal(arr["el"], arr["ray"] % a["n_el"])   # back to the emitting element


def test_convex_point_target_image():
    a = convex_array(0.04, n_el=64, pitch=0.4e-3)
    target = (5e-3, 20e-3)
    scene = {"media": [WATER], "boundaries": [], "med_array": 0, "z_max": 0.05,
             "scatterers": np.array([[target[0], 0.0, target[1], 1.0]], np.float32), "r_s": 2e-4}
    tx = [(oracle.TX_DIVERGING, x, -0.04) for x in (-6e-3, 0.0, 6e-3)]
    ang = np.zeros(3, np.float32)
    arr, _, _ = oracle.trace(scene, a, ang, 64 * 300, 4, 0, mode=oracle.MODE_EXPECT, transmits=tx)
    rf, quad = oracle.deposit(a, 3, arr)
    x = np.linspace(1e-3, 9e-3, 81).astype(np.float32)
    z = np.linspace(16e-3, 24e-3, 81).astype(np.float32)
    img = oracle.beamform(a, ang, rf, quad, x, z, transmits=tx)
    iz, ix = np.unravel_index(np.argmax(np.abs(img)), img.shape)
    assert abs(x[ix] - target[0]) <= 2e-4 and abs(z[iz] - target[1]) <= 2e-4
    flat = dict(a)
    flat["radius"] = 0.0                                   # element positions of a linear array
    assert np.abs(oracle.beamform(flat, ang, rf, quad, x, z, transmits=tx)).max() < 0.8 * np.abs(img).max()


def test_invalid_convex_arrays_are_rejected():
    w = phantoms.tiny(n_rays=100)
    for radius in (-0.01, 0.003):                          # negative; 32 x 0.3 mm over 3 mm > 170 degrees
        a = dict(w["array"])
        a["radius"] = radius
        with pytest.raises(ValueError):
            oracle.trace(w["scene"], a, w["angles"], 100, 0, 1)
