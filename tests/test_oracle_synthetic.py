"""Pins of the oracle's synthetic-aperture transmits and per-ray transmit mixing.

Synthetic aperture is named among the acquisition schemes (Sec. 1) without
formulas; the oracle's reading (one element fires at t = 0, its rays leave
uniform points of its face at an angle to the normal drawn uniformly in
(-pi/2, pi/2), Eq. 6 weight cos / N) is pinned by image-source echoes of a
plane and of a concentric shell (times, weights and receiving elements in closed
form), by the angle distribution and by a point-target image.  Transmit mixing
(Sec. 2.3: rays of several acquisition events leave together, each with a
randomly selected transmit) is pinned against the per-transmit traces through
the Philox draw that selects the transmit, and by the binomial ray counts and
the weights it gives each transmit.
"""
import math

import numpy as np

import oracle
import phantoms

C = 1540.0
WATER = (C, 1.54, 0.0, 0.0)
# same sound speed, other impedance: straight transmission, r = (Z2 - Z1) / (Z2 + Z1) at every angle
DENSE = (C, 3.0, 0.0, 0.0)


def f32(x):
    return float(np.float32(x))


def wide_array(n_el, pitch=0.3e-3, n_s=4096):
    """Directivity open to 89 degrees: f_d = 1 for every returning ray used here."""
    return phantoms.array_params(n_el, n_s, pitch=pitch, elev_h=4e-3, c_bf=C, alpha_m_deg=89.0, alpha_c_deg=89.0)


def r_dense():
    z1, z2 = f32(1.54), f32(3.0)
    return (z2 - z1) / (z2 + z1)


def test_synthetic_aperture_plane_echo_and_angles():
    """Element f fires alone at t = 0; a ray at angle theta returns from the plane z = d after a
    path 2 d / cos(theta) with weight r cos(theta) / N, landing 2 d tan(theta) from its emission
    point (within half a pitch of the element centre); theta is uniform on (-pi/2, pi/2)."""
    n_el, f, N = 128, 40, 200_000
    a = wide_array(n_el)
    d = f32(5e-3)
    scene = {"media": [WATER, DENSE], "boundaries": [(oracle.PLANE_Z, [d, 0, 0, 0], 0, 1)], "med_array": 0,
             "z_max": 0.02, "scatterers": np.zeros((0, 4), np.float32), "r_s": 1e-4}
    arr, _, st = oracle.trace(scene, a, np.zeros(1, np.float32), N, 11, 1, mode=oracle.MODE_EXPECT,
                              transmits=[(oracle.TX_SYNTHETIC, float(f), 0.0)])
    assert st["rays"] == N
    fs, c, p = a["fs"], f32(C), a["pitch"]
    L = arr["t"] * c / fs                                  # path length of each echo
    cos_t = 2 * d / L
    assert np.all(cos_t <= 1.0 + 1e-12)
    np.testing.assert_allclose(arr["amp"], r_dense() * cos_t / N, rtol=1e-9)
    tan_t = np.sqrt(np.maximum(1.0 - cos_t ** 2, 0.0)) / cos_t
    xe = (arr["el"] - 0.5 * (n_el - 1)) * p
    xf = (f - 0.5 * (n_el - 1)) * p
    off = np.minimum(np.abs(xe - xf - 2 * d * tan_t), np.abs(xe - xf + 2 * d * tan_t))
    assert off.max() <= p * (1 + 1e-9)                     # emission and landing within half a pitch each
    # every ray with |theta| <= 45 deg lands inside the aperture: their count is N / 2 for a uniform angle
    # (a cosine-distributed angle would give N sin(45 deg) = 0.71 N)
    n45 = int(np.sum(cos_t >= math.cos(math.pi / 4)))
    assert abs(n45 - N / 2) <= 5 * math.sqrt(N / 4)
    assert arr.size == np.unique(arr["ray"]).size          # one echo per ray at most


def test_synthetic_aperture_concentric_shell_on_a_convex_array():
    """Convex array of radius R, shell of radius R2 = R + d about the same centre: a ray leaving the
    arc at angle theta to the local normal travels L with R2^2 = R^2 + L^2 + 2 R L cos(theta) to the
    shell and L back, reaching the arc at angle theta again: weight r cos(theta) / N at time 2 L / c."""
    R, dd, n_el, f, N = 0.04, 10e-3, 64, 20, 100_000
    a = wide_array(n_el, pitch=0.4e-3)
    a["radius"] = f32(R)
    scene = {"media": [WATER, DENSE], "boundaries": [(oracle.CYL_Y, [0.0, -R, R + dd, 0.0], 0, 1)],
             "med_array": 0, "z_max": 0.06, "scatterers": np.zeros((0, 4), np.float32), "r_s": 1e-4}
    arr, _, _ = oracle.trace(scene, a, np.zeros(1, np.float32), N, 5, 1, mode=oracle.MODE_EXPECT,
                             transmits=[(oracle.TX_SYNTHETIC, float(f), 0.0)])
    assert arr.size > 0.2 * N
    Rf, R2 = f32(R), f32(R + dd)                           # the scene's float32 radii
    L = 0.5 * arr["t"] * f32(C) / a["fs"]
    cos_t = (R2 ** 2 - Rf ** 2 - L ** 2) / (2 * Rf * L)
    assert np.all((cos_t > 0) & (cos_t <= 1 + 1e-9))
    np.testing.assert_allclose(arr["amp"], r_dense() * cos_t / N, rtol=1e-7)
    # the echo returns to elements near the firing one and farther out for oblique rays
    assert np.abs(arr["el"] - f).min() == 0
    # the angle is taken to the local normal: from an edge element (30 degrees off the axis here) every
    # ray leaves the face, each tracing one segment in an empty scene (an angle to the z axis would
    # aim a sixth of them into the probe)
    empty = dict(scene, boundaries=[])
    a["pitch"] = f32(R * math.radians(60.0) / n_el)
    _, _, st = oracle.trace(empty, a, np.zeros(1, np.float32), 20_000, 6, 1, mode=oracle.MODE_EXPECT,
                            transmits=[(oracle.TX_SYNTHETIC, 0.0, 0.0)])
    assert st["rays"] == st["segments"] == 20_000


def test_synthetic_aperture_images_a_point_target():
    a = phantoms.array_params(64, 2048, pitch=0.3e-3, elev_h=4e-3, c_bf=C, alpha_m_deg=89.0, alpha_c_deg=89.0)
    target = (1.5e-3, 12e-3)
    scene = {"media": [WATER], "boundaries": [], "med_array": 0, "z_max": 0.05,
             "scatterers": np.array([[target[0], 0.0, target[1], 1.0]], np.float32), "r_s": 2e-4}
    tx = [(oracle.TX_SYNTHETIC, float(e), 0.0) for e in (8, 24, 40, 56)]
    ang = np.zeros(len(tx), np.float32)
    arr, _, _ = oracle.trace(scene, a, ang, 40_000, 2, 0, mode=oracle.MODE_EXPECT, transmits=tx)
    assert np.all(np.bincount(arr["tx"], minlength=len(tx)) > 0)
    rf, quad = oracle.deposit(a, len(tx), arr)
    x = np.linspace(-2e-3, 5e-3, 71).astype(np.float32)
    z = np.linspace(9e-3, 15e-3, 61).astype(np.float32)
    img = oracle.beamform(a, ang, rf, quad, x, z, transmits=tx)
    iz, ix = np.unravel_index(np.argmax(np.abs(img)), img.shape)
    assert abs(x[ix] - target[0]) <= 2e-4 and abs(z[iz] - target[1]) <= 2e-4
    img_pw = oracle.beamform(a, ang, rf, quad, x, z)       # plane-wave transmit delays on the same data
    assert np.abs(img_pw).max() < 0.8 * np.abs(img).max()


def picks(seed, n, n_tx):
    """Transmit drawn by ray i: ((x0 >> 8) * n_tx) >> 24 with x = Philox(counter (i, 0, 0, 1), seed)."""
    key = [seed & 0xFFFFFFFF, seed >> 32]
    x0 = np.array([int(oracle.philox4x32_10([i, 0, 0, 1], key)[0]) for i in range(n)], np.uint64)
    return ((x0 >> np.uint64(8)) * np.uint64(n_tx)) >> np.uint64(24)


def test_mixed_rays_are_the_per_transmit_rays_they_drew():
    """Ray i of the mixed sequence is ray i of the transmit it draws, with weight over N instead of
    over the n_tx N rays of a per-transmit trace of the same length: same events, times, elements
    and path hashes, amplitudes n_tx times larger."""
    w = phantoms.tiny(n_rays=3000)
    a = dict(w["array"], alpha_m_deg=10.0, alpha_c_deg=15.0)   # a wider directivity: more echoes
    tx = [(oracle.TX_PLANE, 0.0, 0.0), (oracle.TX_DIVERGING, -2e-3, -8e-3), (oracle.TX_SYNTHETIC, 9.0, 0.0)]
    ang = np.deg2rad([-5.0, 0.0, 0.0]).astype(np.float32)
    N, n_tx, seed = 3000, 3, 17
    mixed, mtopo, mst = oracle.trace(w["scene"], a, ang, N, seed, 4, topo=True, transmits=tx, mix=True)
    full, ftopo, _ = oracle.trace(w["scene"], a, ang, n_tx * N, seed, 4, topo=True, transmits=tx)
    assert mst["rays"] == n_tx * N and mtopo.shape == (n_tx * N,)
    k = picks(seed, n_tx * N, n_tx).astype(np.int64)
    assert np.array_equal(mtopo, ftopo[k, np.arange(n_tx * N)])
    sel = full[k[full["ray"]] == full["tx"]]
    assert sel.size == mixed.size > 100
    for f in ("tx", "ray", "event", "el"):
        assert np.array_equal(sel[f], mixed[f]), f
    assert np.array_equal(sel["t"], mixed["t"])
    np.testing.assert_allclose(mixed["amp"], n_tx * sel["amp"], rtol=1e-12)
    assert np.all(np.bincount(k, minlength=n_tx) > 0)


def test_mixing_gives_each_transmit_its_expected_weight():
    """Normal-incidence echo of a plane (expectation mode, no scatterers): every ray that draws
    transmit k returns with weight r / N, so transmit k's total is r n_k / N with n_k binomial
    (n_tx N, 1 / n_tx); the total over transmits is r n_tx."""
    d = f32(10e-3)
    a = phantoms.array_params(32, 2048, c_bf=C)
    scene = {"media": [WATER, DENSE], "boundaries": [(oracle.PLANE_Z, [d, 0, 0, 0], 0, 1)], "med_array": 0,
             "z_max": 0.03, "scatterers": np.zeros((0, 4), np.float32), "r_s": 1e-4}
    N, n_tx = 20_000, 5
    arr, _, _ = oracle.trace(scene, a, np.zeros(n_tx, np.float32), N, 3, 1, mode=oracle.MODE_EXPECT, mix=True)
    n_k = np.bincount(arr["tx"], minlength=n_tx)
    assert n_k.sum() == n_tx * N                           # every ray returns once
    sums = np.bincount(arr["tx"], weights=arr["amp"], minlength=n_tx)
    np.testing.assert_allclose(sums, r_dense() * n_k / N, rtol=1e-9)
    sd = math.sqrt(n_tx * N * (1 / n_tx) * (1 - 1 / n_tx))
    assert np.all(np.abs(n_k - N) <= 5 * sd)
    np.testing.assert_allclose(arr["t"], 2 * d * a["fs"] / f32(C), rtol=1e-12)


def test_invalid_synthetic_aperture_and_mixing_are_rejected():
    w = phantoms.tiny(n_rays=100)
    import pytest
    for tx in ([(oracle.TX_SYNTHETIC, 32.0, 0.0)], [(oracle.TX_SYNTHETIC, -1.0, 0.0)],
               [(oracle.TX_SYNTHETIC, 2.5, 0.0)]):
        with pytest.raises(ValueError):
            oracle.trace(w["scene"], w["array"], np.zeros(1, np.float32), 100, 0, 1, transmits=tx)
    with pytest.raises(ValueError):                        # past the end of the mixed sequence
        oracle.trace(w["scene"], w["array"], np.zeros(2, np.float32), 100, 0, 1, ray_end=201, mix=True)
