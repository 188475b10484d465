"""Closed-form pins of the oracle's curved boundaries (Sec. 2.3 "Ray Traversal",
Eqs. 7-11, applied to the bone sphere and the bone cylinder of the phantoms).

Every ray of these scenes is followed a second time here, by geometry written from
first principles: the emission point is the ray's Philox draw (the generator is
pinned by known-answer vectors), each intersection is a root of the surface's
implicit quadratic (numpy's polynomial roots; the near root when arriving from
outside, the far root when leaving from inside), each normal is the gradient of
the implicit function, refraction is built from the tangential component and
Snell's law, and the reflection coefficient is the Kinsler-Frey form
(Z2/cos_t - Z1/cos_i)/(Z2/cos_t + Z1/cos_i).  Expectation mode makes each branch
deterministic, so every echo the oracle records must equal the closed-form one in
element, time (1e-9 samples) and amplitude (1e-10 relative), and no echo may be
missing or extra.

Oracle mistakes each test catches (``test_planted_mistakes_are_caught`` plants
them in a copy of the oracle and checks that they are):
  * near and far roots swapped (entry at the far root, exit at the near one);
  * inside and outside media of a sphere or cylinder swapped;
  * a y component in the cylinder's normal;
  * a ray leaving a sphere or cylinder at the near root (its own start point);
  * transmit delays referred to element 0 rather than to the first element that
    fires (breaks the mirror symmetry of opposite steering angles).
CPU only.
"""
import os
import re
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
import phantoms

EXPECT = oracle.MODE_EXPECT
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _f(x):
    """The float32 value an input carries, promoted to double."""
    return float(np.float32(x))


def _np_per_m(alpha_db_cm_mhz, f0):
    """dB/cm/MHz at f0 -> amplitude attenuation in Np/m (1 Np = 20 log10(e) dB)."""
    return _f(alpha_db_cm_mhz) * (_f(f0) * 1e-6) * 100.0 / (20.0 * np.log10(np.e))


# ------------------------------------------------------------ closed-form geometry

def emission_points(array, n_rays, seed, k=0):
    """Emission point of every ray of transmit k: element i mod n_el, uniform on its face,
    from the ray's Philox4x32-10 block (counter (i, k, 0, 0), key = seed; top 24 bits)."""
    n_el, p, H = array["n_el"], _f(array["pitch"]), _f(array["elev_h"])
    x0 = -0.5 * (n_el - 1) * p
    key = [seed & 0xFFFFFFFF, seed >> 32]
    pts = np.zeros((n_rays, 3))
    for i in range(n_rays):
        x = oracle.philox4x32_10([i, k, 0, 0], key)
        u0, u1 = (int(x[0]) >> 8) / 2.0 ** 24, (int(x[1]) >> 8) / 2.0 ** 24
        pts[i] = (x0 + (i % n_el) * p + (u0 - 0.5) * p, (u1 - 0.5) * H, 0.0)
    return pts


class Sphere:
    """|p - c|^2 - R^2 = 0."""

    def __init__(self, cx, cy, cz, R):
        self.c = np.array([_f(cx), _f(cy), _f(cz)])
        self.R = _f(R)

    def poly(self, o, d):
        oc = o - self.c
        return [d @ d, 2.0 * (oc @ d), oc @ oc - self.R ** 2]

    def grad(self, h):
        return 2.0 * (h - self.c)


class CylinderY:
    """(x - xc)^2 + (z - zc)^2 - R^2 = 0 (infinite along y)."""

    def __init__(self, xc, zc, R):
        self.xc, self.zc, self.R = _f(xc), _f(zc), _f(R)

    def poly(self, o, d):
        ox, oz = o[0] - self.xc, o[2] - self.zc
        return [d[0] ** 2 + d[2] ** 2, 2.0 * (ox * d[0] + oz * d[2]), ox * ox + oz * oz - self.R ** 2]

    def grad(self, h):
        return np.array([2.0 * (h[0] - self.xc), 0.0, 2.0 * (h[2] - self.zc)])


def real_roots(poly):
    if poly[0] == 0.0:
        return []
    r = np.roots(poly)
    return sorted(float(v.real) for v in r if abs(v.imag) <= 1e-12 * max(1.0, abs(v.real)))


def enter(surf, o, d):
    """First intersection of o + t d with a surface the point lies outside of (near root)."""
    r = [t for t in real_roots(surf.poly(o, d)) if t > 1e-7]
    return r[0] if r else None


def leave(surf, o, d):
    """Intersection of a ray starting on the surface and heading inside: the far root."""
    r = real_roots(surf.poly(o, d))
    return r[-1] if r and r[-1] > 1e-7 else None


def unit(v):
    return v / np.linalg.norm(v)


def interface(d, n, c1, Z1, c2, Z2):
    """Smooth fluid-fluid interface, written from Snell's law and the Kinsler-Frey
    reflection coefficient.  n is any unit normal of the surface.  Returns
    (reflected dir, transmitted dir or None on total reflection, r)."""
    nf = n if d @ n < 0 else -n             # normal on the incident side
    cos_i = -(d @ nf)
    tan = d + cos_i * nf                    # tangential part of d, |tan| = sin_i
    sin_i = np.linalg.norm(tan)
    d_r = tan + cos_i * nf
    sin_t = sin_i * c2 / c1
    if sin_t > 1.0:
        return d_r, None, 1.0
    cos_t = np.sqrt(1.0 - sin_t * sin_t)
    d_t = (sin_t * tan / sin_i if sin_i > 0 else 0.0 * tan) - cos_t * nf
    r = (Z2 / cos_t - Z1 / cos_i) / (Z2 / cos_t + Z1 / cos_i)
    return d_r, d_t, r


def directivity(alpha, am, ac):
    """Eq. 13: 1 inside the main beam, linear to 0 at the cutoff."""
    if alpha <= am:
        return 1.0
    return max(0.0, (ac - alpha) / (ac - am)) if ac > am else 0.0


def aperture(array, h, d):
    """Element receiving an upward ray at h on z = 0, with its directivity, or None."""
    n_el, p, H = array["n_el"], _f(array["pitch"]), _f(array["elev_h"])
    xl = -0.5 * (n_el - 1) * p - 0.5 * p
    if abs(h[1]) > 0.5 * H or not (xl <= h[0] < xl + n_el * p):
        return None
    e = min(int(np.floor((h[0] - xl) / p)), n_el - 1)
    fd = directivity(np.arccos(-d[2]), np.deg2rad(_f(array["alpha_m_deg"])), np.deg2rad(_f(array["alpha_c_deg"])))
    return (e, fd) if fd > 0 else None


def to_array_plane(h, d):
    """Straight travel from h to z = 0 (d pointing up); returns (distance, landing point)."""
    s = -h[2] / d[2]
    return s, h + s * d


# ------------------------------------------------------- a quadric in water

WATER = (1480.0, 1.48, 0.0, 0.0)
BONE = (3500.0, 7.8, 10.0, 0.0)


def quadric_scene(kind, zc=25e-3, R=3e-3, xc=0.0):
    """Water with a bone sphere or cylinder (bone inside, water outside), no scatterers."""
    arr = phantoms.array_params(32, 2048, c_bf=1480.0, alpha_m_deg=40.0, alpha_c_deg=60.0)
    if kind == "sphere":
        bnd = [(oracle.SPHERE, [xc, 0.0, zc, R], 1, 0)]
    else:
        bnd = [(oracle.CYL_Y, [xc, zc, R, 0.0], 1, 0)]
    sc = {"media": np.asarray([WATER, BONE], np.float32), "boundaries": bnd, "med_array": 0, "z_max": 0.040,
          "scatterers": np.zeros((0, 4), np.float32), "r_s": 1e-4}
    surf = Sphere(xc, 0.0, zc, R) if kind == "sphere" else CylinderY(xc, zc, R)
    return sc, arr, surf


def quadric_echoes(surf, array, o, N):
    """Closed-form echoes of one plane-wave ray (0 degrees) off a bone body in water:
    {1: front wall (reflection at entry), 3: back wall (transmit in, reflect at the far
    wall, transmit out)} -> (element, time in samples, amplitude)."""
    fs = _f(array["fs"])
    c1, Z1 = _f(WATER[0]), _f(WATER[1])
    c2, Z2 = _f(BONE[0]), _f(BONE[1])
    a2 = _np_per_m(BONE[2], array["f0"])
    d = np.array([0.0, 0.0, 1.0])
    out = {}
    t1 = enter(surf, o, d)
    if t1 is None:
        return out
    h1 = o + t1 * d
    n1 = unit(surf.grad(h1))
    d_r, d_t, r12 = interface(d, n1, c1, Z1, c2, Z2)
    if d_r[2] < 0:                                       # front-wall echo
        s, land = to_array_plane(h1, d_r)
        hit = aperture(array, land, d_r)
        if hit:
            out[1] = (hit[0], (t1 + s) / c1 * fs, r12 * hit[1] / N)
    if d_t is None:
        return out
    t2 = leave(surf, h1, d_t)                            # across the bone to the far wall
    h2 = h1 + t2 * d_t
    n2 = unit(surf.grad(h2))
    d_r2, _, r21 = interface(d_t, n2, c2, Z2, c1, Z1)
    t3 = leave(surf, h2, d_r2)                           # back across the bone
    h3 = h2 + t3 * d_r2
    n3 = unit(surf.grad(h3))
    _, d_out, r23 = interface(d_r2, n3, c2, Z2, c1, Z1)
    if d_out is None or d_out[2] >= 0:
        return out
    s, land = to_array_plane(h3, d_out)
    hit = aperture(array, land, d_out)
    if hit:
        amp = np.sqrt(1 - r12 ** 2) * r21 * np.sqrt(1 - r23 ** 2) * np.exp(-a2 * (t2 + t3)) * hit[1] / N
        out[3] = (hit[0], ((t1 + s) / c1 + (t2 + t3) / c2) * fs, amp)
    return out


def _aperture_by_ray(arr):
    ap = arr[(arr["event"] >> 31) == 1]
    b = (ap["event"] >> 24) & 0x7F
    got = {}
    for a, bb in zip(ap, b):
        got.setdefault((int(a["ray"]), int(bb)), []).append(a)
    return got


def check_quadric(kind, n_rays=32 * 400, seed=3, **geo):
    """Oracle echoes of the sphere / cylinder scene == the closed form, ray by ray.
    Returns the number of (front, back) echoes compared."""
    sc, arr, surf = quadric_scene(kind, **geo)
    got_arr, _, _ = oracle.trace(sc, arr, np.zeros(1, np.float32), n_rays, seed, 3, mode=EXPECT)
    got = _aperture_by_ray(got_arr)
    pts = emission_points(arr, n_rays, seed)
    n = {1: 0, 3: 0}
    expected = set()
    for i in range(n_rays):
        for b, (e, t, amp) in quadric_echoes(surf, arr, pts[i], n_rays).items():
            expected.add((i, b))
            g = got.get((i, b), [])
            assert len(g) == 1, "ray %d bounce %d: %d oracle echoes" % (i, b, len(g))
            g = g[0]
            assert int(g["el"]) == e, (i, b)
            assert abs(g["t"] - t) < 1e-9, (i, b, g["t"], t)
            assert g["amp"] == pytest.approx(amp, rel=1e-10, abs=1e-300), (i, b)
            n[b] += 1
    extra = set(got) - expected
    assert not extra, "oracle echoes without a closed-form path: %s" % sorted(extra)[:5]
    return n


def test_sphere_front_and_back_wall_echoes():
    """Bone sphere r = 5 mm at 10 mm in water.  Front wall: entry at the near root,
    r12(theta_i) of water -> bone; back wall: transmit in, far root, reflect with
    r21 of bone -> water, far root again, transmit out, bone attenuation on the
    chord.  Catches swapped roots, swapped inside/outside media, a wrong normal."""
    n = check_quadric("sphere", n_rays=32 * 1500, zc=10e-3, R=5e-3)
    assert n[1] > 1000 and n[3] > 100


def test_cylinder_front_and_back_wall_echoes():
    """Bone cylinder along y (r = 3 mm, 25 mm deep, 1.5 mm off axis) in water.  Rays
    leave the elements at |y| up to 2 mm: a y component in the normal would tilt
    every echo out of the xz plane.  Also catches swapped roots and swapped media."""
    n = check_quadric("cylinder", xc=1.5e-3)
    assert n[1] > 500 and n[3] > 100


def test_central_ray_limits():
    """The closed form itself against the textbook values: a central ray's front echo
    at 2 (z_c - R)/c1 with amplitude r12 = (Z2 - Z1)/(Z2 + Z1), its back-wall echo
    at 2 (z_c - R)/c1 + 4 R/c2 with amplitude (1 - r12^2) r21 exp(-2 a 2R)."""
    for surf in (Sphere(0, 0, 25e-3, 3e-3), CylinderY(0, 25e-3, 3e-3)):
        arr = phantoms.array_params(1, 2048, alpha_m_deg=40.0, alpha_c_deg=60.0)
        e = quadric_echoes(surf, arr, np.zeros(3), 1)
        zc, R, fs = _f(25e-3), _f(3e-3), _f(40e6)
        Z1, Z2 = _f(1.48), _f(7.8)
        r12 = (Z2 - Z1) / (Z2 + Z1)
        a2 = _np_per_m(10.0, 5e6)
        assert e[1][1] == pytest.approx(2 * (zc - R) / 1480.0 * fs, abs=1e-9)
        assert e[1][2] == pytest.approx(r12, rel=1e-12)
        assert e[3][1] == pytest.approx((2 * (zc - R) / 1480.0 + 4 * R / 3500.0) * fs, abs=1e-9)
        assert e[3][2] == pytest.approx((1 - r12 ** 2) * (-r12) * np.exp(-a2 * 4 * R), rel=1e-12)


# --------------------------------------------------- V12: layered bone-top echo

def bone_top_echo(array, o, N, z_skin=2e-3, z_fat=10e-3, bone=(0.0, 30e-3, 6e-3)):
    """Closed-form bone-top echo of a 0-degree ray in the layered phantom: transmit
    through skin/fat and fat/muscle at normal incidence, reflect off the bone cylinder,
    refract back up through both planes (obliquely) to the array.  Returns
    (element, time in samples, amplitude, attenuation in dB) or None."""
    fs = _f(array["fs"])
    skin, fat, muscle, bonem = phantoms.SKIN, phantoms.FAT, phantoms.MUSCLE, phantoms.BONE
    cs, Zs = _f(skin[0]), _f(skin[1])
    cf, Zf, af = _f(fat[0]), _f(fat[1]), _np_per_m(fat[2], array["f0"])
    cm, Zm, am = _f(muscle[0]), _f(muscle[1]), _np_per_m(muscle[2], array["f0"])
    cb, Zb = _f(bonem[0]), _f(bonem[1])
    z1, z2 = _f(z_skin), _f(z_fat)
    zn = np.array([0.0, 0.0, 1.0])
    cyl = CylinderY(*bone)
    d = zn.copy()
    _, _, r_sf = interface(d, zn, cs, Zs, cf, Zf)
    _, _, r_fm = interface(d, zn, cf, Zf, cm, Zm)
    h0 = np.array([o[0], o[1], z2])
    t_m = enter(cyl, h0, d)
    if t_m is None:
        return None
    h = h0 + t_m * d
    d_r, _, r_mb = interface(d, unit(cyl.grad(h)), cm, Zm, cb, Zb)
    if d_r[2] >= 0:
        return None
    s_m = (z2 - h[2]) / d_r[2]                      # up through muscle to the fat/muscle plane
    p2 = h + s_m * d_r
    _, d_f, r_mf = interface(d_r, zn, cm, Zm, cf, Zf)
    if d_f is None:
        return None
    s_f = (z1 - z2) / d_f[2]                        # up through fat to the skin/fat plane
    p1 = p2 + s_f * d_f
    _, d_s, r_fs = interface(d_f, zn, cf, Zf, cs, Zs)
    if d_s is None:
        return None
    s_s, land = to_array_plane(p1, d_s)
    hit = aperture(array, land, d_s)
    if hit is None:
        return None
    t = (z1 / cs + (z2 - z1) / cf + t_m / cm + s_m / cm + s_f / cf + s_s / cs) * fs
    att = af * ((z2 - z1) + s_f) + am * (t_m + s_m)
    tr = np.sqrt((1 - r_sf ** 2) * (1 - r_fm ** 2) * (1 - r_mf ** 2) * (1 - r_fs ** 2))
    return hit[0], t, tr * r_mb * np.exp(-att) * hit[1] / N, 20 * np.log10(np.exp(att))


def test_layered_bone_top_echo_v12():
    """Layered phantom with its bone cylinder: every ray's bone-top echo (five
    interactions) equals the closed form; the central ray's echo is the printed one:
    31.233 us, r_mb = +0.6421, 18.8 dB round-trip attenuation."""
    w = phantoms.layered(n_scat=0, n_rays=128 * 24)
    arr = dict(w["array"])
    arr["alpha_m_deg"], arr["alpha_c_deg"] = _f(20.0), _f(30.0)   # wide enough for the curved echo
    N, seed = w["n_rays"], 5
    # the central ray: closed form against the printed values
    e, t, amp, att_db = bone_top_echo(arr, np.array([1e-12, 0.0, 0.0]), 1)
    assert t / _f(40e6) * 1e6 == pytest.approx(31.233, abs=1e-3)
    assert att_db == pytest.approx(18.8, abs=1e-6)
    Zs, Zf, Zm, Zb = _f(1.99), _f(1.38), _f(1.70), _f(7.8)
    r_mb = (Zb - Zm) / (Zb + Zm)
    assert r_mb == pytest.approx(0.6421, abs=5e-5)
    tr = (1 - ((Zf - Zs) / (Zf + Zs)) ** 2) * (1 - ((Zm - Zf) / (Zm + Zf)) ** 2)
    assert amp == pytest.approx(tr * r_mb * 10 ** (-18.8 / 20), rel=1e-6)
    # every ray against the oracle
    got_arr, _, _ = oracle.trace(w["scene"], arr, w["angles"], N, seed, 5, mode=EXPECT)
    got = _aperture_by_ray(got_arr)
    pts = emission_points(arr, N, seed)
    n = 0
    for i in range(N):
        ref = bone_top_echo(arr, pts[i], N)
        if ref is None:
            continue
        cand = got.get((i, 5), [])
        assert cand, "ray %d: no five-interaction echo" % i
        j = int(np.argmin([abs(c["t"] - ref[1]) for c in cand]))
        g = cand[j]
        assert abs(g["t"] - ref[1]) < 1e-9, (i, g["t"], ref[1])
        assert int(g["el"]) == ref[0]
        assert g["amp"] == pytest.approx(ref[2], rel=1e-10)
        n += 1
    assert n > 200


# ------------------------------------------------------------ V4: mirror symmetry

def _mirror_scene(xc, theta_deg):
    """Layered planes, a bone cylinder at x = xc and 100 scatterers on its side (capture
    radius 0.4 mm, so that hits are frequent), a 64-element array, steering theta."""
    w = phantoms.layered(n_scat=0, n_rays=64 * 600, bone_r=4e-3, bone_z=25e-3)
    sc = dict(w["scene"])
    b = list(sc["boundaries"])
    k, p, m0, m1 = b[2]
    b[2] = (k, [_f(xc), p[1], p[2], p[3]], m0, m1)
    rng = np.random.default_rng(9)
    s = phantoms.uniform_scatterers(rng, 100, ((2e-3, 12e-3), (-2e-3, 2e-3), (12e-3, 35e-3)))
    if xc < 0:
        s[:, 0] = -s[:, 0]
    sc["boundaries"], sc["scatterers"], sc["r_s"] = b, s, _f(4e-4)
    arr = phantoms.array_params(64, 2400, c_bf=1540.0)
    return sc, arr, np.deg2rad(np.array([theta_deg], np.float64)).astype(np.float32), w["n_rays"]


def test_mirror_symmetry_v4():
    """A scene mirrored in x (bone cylinder and scatterers at -x) imaged with the mirrored
    steering angle gives channel data mirrored across the elements.  Emission points are
    random, so the check is statistical: the mirrored pair differs by no more than two
    independent runs of the same scene do.  Catches transmit delays that treat the two
    steering directions differently (e.g. referred to element 0)."""
    sc_p, arr, ang_p, N = _mirror_scene(+6e-3, +8.0)
    sc_m, _, ang_m, _ = _mirror_scene(-6e-3, -8.0)

    def rf(sc, ang, seed):
        a, _, _ = oracle.trace(sc, arr, ang, N, seed, 4, mode=EXPECT)
        return oracle.deposit(arr, 1, a)[0][0]

    a1, a2 = rf(sc_p, ang_p, 11), rf(sc_p, ang_p, 12)
    m1, m2 = rf(sc_m, ang_m, 13)[::-1], rf(sc_m, ang_m, 14)[::-1]
    scale = np.linalg.norm(a1)
    noise = max(np.linalg.norm(a1 - a2), np.linalg.norm(m1 - m2)) / scale
    mirror = max(np.linalg.norm(a1 - m1), np.linalg.norm(a2 - m2)) / scale
    assert noise < 0.3                                # the comparison has resolving power
    assert mirror < 1.6 * noise, (mirror, noise)
    # an unmirrored pair (same scene, opposite angle) is far apart: the test can fail
    assert np.linalg.norm(a1 - rf(sc_p, ang_m, 15)[::-1]) / scale > 3 * noise


def test_mirror_symmetry_v4_beamformer():
    """Delay-and-sum of channel data flipped across the elements at the opposite angle is
    the mirror image (x -> -x on a symmetric grid), exactly."""
    arr = phantoms.array_params(32, 800, c_bf=1540.0)
    rng = np.random.default_rng(2)
    rf, q = rng.standard_normal((2, 1, 32, 800))
    x = np.linspace(-4e-3, 4e-3, 33).astype(np.float32)
    z = np.linspace(2e-3, 14e-3, 40).astype(np.float32)
    ang = np.deg2rad(np.array([9.0], np.float32)).astype(np.float32)
    img = oracle.beamform(arr, ang, rf, q, x, z)
    img_m = oracle.beamform(arr, -ang, rf[:, ::-1].copy(), q[:, ::-1].copy(), x, z)
    np.testing.assert_allclose(img_m[:, ::-1], img, rtol=1e-9, atol=1e-9 * np.abs(img).max())


# ------------------------------------------------------------ planted mistakes

MUTATIONS = {
    # entry at the far root: t = -b + s instead of -b - s for spheres and cylinders
    "swapped_roots": (r"t = -b - s;\n(\s*)if \(!\(t > OR_TMIN\)\) t = -b \+ s;",
                      r"t = -b + s;\n\1if (!(t > OR_TMIN)) t = -b - s;"),
    # medium on the far side of a quadric swapped (inside <-> outside)
    "swapped_media": (r"return dot3\(d, n_out\) > 0\.0 \? m\[1\] : m\[0\];",
                      r"if (p < C->sc->n_bnd && C->sc->bnd_kind[p] != OR_PLANE_Z) "
                      r"return dot3(d, n_out) > 0.0 ? m[0] : m[1];\n"
                      r"    return dot3(d, n_out) > 0.0 ? m[1] : m[0];"),
    # the cylinder's normal picks up the y offset of the hit point
    "cylinder_normal_y": (r"n\[0\] = h\[0\] - q\[0\]; n\[1\] = 0\.0; n\[2\] = h\[2\] - q\[1\];",
                          r"n[0] = h[0] - q[0]; n[1] = 0.3 * h[1]; n[2] = h[2] - q[1];"),
    # a ray leaving a sphere or cylinder from inside takes the near root (its own start point)
    "exit_near_root": (r"t = -2\.0 \* b;", r"t = 0.0;"),
    # transmit delays referred to element 0 instead of the first element to fire
    "delay_reference": (r"\(len\[e\] - mn\) / \(double\)ar->c_bf", r"(len[e] - len[0]) / (double)ar->c_bf"),
}

CATCHES = {
    "swapped_roots": ["test_sphere_front_and_back_wall_echoes", "test_cylinder_front_and_back_wall_echoes"],
    "swapped_media": ["test_sphere_front_and_back_wall_echoes", "test_layered_bone_top_echo_v12"],
    "cylinder_normal_y": ["test_cylinder_front_and_back_wall_echoes", "test_layered_bone_top_echo_v12"],
    "exit_near_root": ["test_sphere_front_and_back_wall_echoes", "test_cylinder_front_and_back_wall_echoes"],
    "delay_reference": ["test_mirror_symmetry_v4"],
}


@pytest.mark.parametrize("mutation", sorted(MUTATIONS))
def test_planted_mistakes_are_caught(mutation, tmp_path):
    """Builds a copy of the oracle with one plausible mistake and runs the pins above
    against it in a child process: each named pin must fail."""
    src = open(os.path.join(ROOT, "oracle", "ur_oracle.c")).read()
    pat, rep = MUTATIONS[mutation]
    bad, n = re.subn(pat, rep, src)
    assert n >= 1, "mutation %s no longer applies to the oracle source" % mutation
    (tmp_path / "ur_oracle.c").write_text(bad)
    (tmp_path / "ur_oracle.h").write_text(open(os.path.join(ROOT, "oracle", "ur_oracle.h")).read())
    so = tmp_path / "liburoracle.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-o", str(so), str(tmp_path / "ur_oracle.c"), "-lm"])
    for test in CATCHES[mutation]:
        script = textwrap.dedent("""
            import sys
            sys.path[:0] = [%r, %r]
            import oracle
            oracle._LIB_PATH = %r
            oracle.build = lambda force=False: oracle._LIB_PATH
            import test_oracle_quadrics as T
            try:
                getattr(T, %r)()
            except AssertionError:
                sys.exit(3)
            sys.exit(0)
        """ % (ROOT, HERE, str(so), test))
        r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=600)
        assert r.returncode == 3, "%s survived %s (rc %d): %s" % (mutation, test, r.returncode, r.stderr[-400:])
