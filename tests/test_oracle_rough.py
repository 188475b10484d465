"""Pins of the oracle's rough (GGX) boundaries, Sec. 2.3 and Eq. 12.

The paper prints only the microfacet density D; sampling, shadowing, the
amplitude-form BSDF, the transducer sampling at rough vertices and its balance
heuristic follow the microfacet model it cites (Walter et al. 2007).  Each test
pins a piece against something other than the oracle's own formula:
quadrature of D, the closed-form CDF of the sampled angle, BSDF reciprocity,
normalisation of the sampling density over all directions, the smooth limit of
the whole trace, and agreement of the two estimators of the same returns.
"""
import math

import numpy as np
import pytest

import oracle
import phantoms

WATER = (1540.0, 1.54, 0.0, 0.0)


@pytest.mark.parametrize("alpha", [0.05, 0.2, 0.5, 1.0, 2.0])
def test_ggx_density_is_normalised(alpha):
    """Eq. 12 projected onto the macro surface integrates to one over the hemisphere."""
    from scipy.integrate import quad
    f = lambda u: 2.0 * math.pi * oracle.ggx_d(u, alpha) * u     # u = cos(theta_m), d omega = 2 pi du
    pts = [1.0 - 10 * alpha * alpha] if alpha < 0.3 else None
    total = quad(f, 0.0, 1.0, points=pts, limit=400, epsabs=1e-12, epsrel=1e-10)[0]
    assert total == pytest.approx(1.0, abs=1e-7)
    assert oracle.ggx_d(1.0, alpha) == pytest.approx(1.0 / (math.pi * alpha * alpha), rel=1e-12)
    assert oracle.ggx_d(1e-9, alpha) == pytest.approx(alpha * alpha / math.pi, rel=1e-9)
    assert oracle.ggx_d(-0.1, alpha) == 0.0


@pytest.mark.parametrize("n", [(0.0, 0.0, 1.0), (0.0, 0.0, -1.0), (0.3, -0.2, 0.93), (-0.8, 0.0, -0.6)])
@pytest.mark.parametrize("alpha", [0.1, 0.5, 1.3])
def test_ggx_sampling_follows_its_density(n, alpha):
    """Sampled normals are unit, around n, with P(cos theta_m >= u) equal to the integral of
    2 pi D(u') u' over [u, 1], and a uniform azimuth."""
    from scipy.integrate import quad
    n = np.asarray(n) / np.linalg.norm(n)
    rng = np.random.default_rng(7)
    xi = rng.random((8000, 2))
    ms = np.array([oracle.ggx_sample(n, alpha, a, b) for a, b in xi])
    np.testing.assert_allclose(np.linalg.norm(ms, axis=1), 1.0, atol=1e-12)
    cos_m = ms @ n
    assert cos_m.min() > 0.0
    for u in (0.5, 0.8, 0.9, 0.95, 0.99):
        expect = quad(lambda x: 2.0 * math.pi * oracle.ggx_d(x, alpha) * x, u, 1.0, limit=200)[0]
        assert np.mean(cos_m >= u) == pytest.approx(expect, abs=0.02)
    # azimuth around n: uniform on [0, 2 pi)
    a = np.cross(n, [1.0, 0.0, 0.0] if abs(n[0]) < 0.9 else [0.0, 1.0, 0.0])
    a /= np.linalg.norm(a)
    b = np.cross(n, a)
    phi = np.mod(np.arctan2(ms @ b, ms @ a), 2 * math.pi)
    hist = np.histogram(phi, bins=8, range=(0, 2 * math.pi))[0] / len(phi)
    np.testing.assert_allclose(hist, 1.0 / 8, atol=0.02)


def _unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


def test_rough_reflection_is_reciprocal():
    """f(i, o) = f(o, i) for the reflection lobe (eval returns f |o.n|)."""
    rng = np.random.default_rng(3)
    n = np.array([0.0, 0.0, -1.0])
    for _ in range(200):
        i = _unit(rng.normal(size=3)); i[2] = -abs(i[2]) - 0.05; i = _unit(i)   # on the n side
        o = _unit(rng.normal(size=3)); o[2] = -abs(o[2]) - 0.05; o = _unit(o)
        for c2, Z2 in ((3500.0, 7.8), (1450.0, 1.38)):
            f_io, _ = oracle.rough_eval(-i, n, o, 0.4, 1540.0, 1.54, c2, Z2)
            f_oi, _ = oracle.rough_eval(-o, n, i, 0.4, 1540.0, 1.54, c2, Z2)
            assert f_io / abs(o @ n) == pytest.approx(f_oi / abs(i @ n), rel=1e-9, abs=1e-300)


def _sphere_integral(fun, n_theta=600, n_phi=600):
    """Integral over the unit sphere of fun(o) (midpoint rule in cos(theta) and phi)."""
    u = (np.arange(n_theta) + 0.5) / n_theta * 2.0 - 1.0
    ph = (np.arange(n_phi) + 0.5) / n_phi * 2 * math.pi
    du, dph = 2.0 / n_theta, 2 * math.pi / n_phi
    tot = 0.0
    for uu in u:
        s = math.sqrt(max(0.0, 1.0 - uu * uu))
        for p in ph:
            tot += fun(np.array([s * math.cos(p), s * math.sin(p), uu]))
    return tot * du * dph


@pytest.mark.parametrize("alpha,theta_deg", [(0.5, 20.0), (0.8, 40.0)])
def test_sampling_density_covers_both_lobes(alpha, theta_deg):
    """The solid-angle densities of reflected and transmitted directions (with their Jacobians
    and branch probabilities) integrate to the admissible fraction of microfacet samples: at
    most one, and close to it for moderate incidence."""
    n = np.array([0.0, 0.0, -1.0])                        # incident side: z < 0
    th = math.radians(theta_deg)
    d = np.array([math.sin(th), 0.0, math.cos(th)])         # travelling toward +z
    media = (1540.0, 1.54, 1450.0, 1.38)                    # no total internal reflection at these angles

    def pdf(o):
        return oracle.rough_eval(d, n, o, alpha, *media)[1]

    tot = _sphere_integral(pdf, 300, 300)
    # admissible fraction by direct Monte Carlo over microfacets: c_im > 0 and the new
    # direction on the right side (computed with the oracle's sampler and Snell step)
    rng = np.random.default_rng(11)
    ok = 0.0
    K = 20000
    for a, b, y in rng.random((K, 3)):
        m = oracle.ggx_sample(n, alpha, a, b)
        ci = -(d @ m)
        if ci <= 0:
            continue
        dr, dt, r, R, tir = _interface(d, m, *media)
        if tir:
            ok += (dr @ n > 0)
        else:
            ok += R * (dr @ n > 0) + (1 - R) * (dt @ n < 0)
    frac = ok / K
    assert tot == pytest.approx(frac, abs=0.02)
    assert tot <= 1.0 + 0.01 and tot > 0.85


def _interface(d, m, c1, Z1, c2, Z2):
    dr, dt = np.zeros(3), np.zeros(3)
    r, R = np.zeros(1), np.zeros(1)
    import ctypes as C
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    dd, mm = np.ascontiguousarray(d, float), np.ascontiguousarray(m, float)
    tir = oracle.lib().or_interface(dp(dd), dp(mm), c1, Z1, c2, Z2, dp(dr), dp(dt), dp(r), dp(R))
    return dr, dt, float(r[0]), float(R[0]), bool(tir)


def _rough_copy(w, alpha, media_index):
    s = dict(w["scene"])
    med = [list(m) for m in s["media"]]
    med[media_index][3] = alpha
    s["media"] = [tuple(m) for m in med]
    return s


def test_small_roughness_recovers_the_smooth_trace():
    """As alpha -> 0 microfacet sampling returns the smooth interface, the direct hits take the
    whole balance-heuristic weight and transducer sampling at the rough vertex vanishes: the
    channel data of the tiny phantom (bone sphere rough) equal the smooth ones."""
    w = phantoms.tiny(n_rays=20000)
    smooth_arr, smooth_topo, _ = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], 0, 4, topo=True)
    rough_scene = _rough_copy(w, 1e-6, 2)
    arr, topo, st = oracle.trace(rough_scene, w["array"], w["angles"], w["n_rays"], 0, 4, topo=True)
    assert np.array_equal(topo, smooth_topo)
    rf0, q0 = oracle.deposit(w["array"], 1, smooth_arr)
    rf1, q1 = oracle.deposit(w["array"], 1, arr)
    rel = np.linalg.norm(np.concatenate([(rf1 - rf0).ravel(), (q1 - q0).ravel()])) / \
        np.linalg.norm(np.concatenate([rf0.ravel(), q0.ravel()]))
    assert rel < 1e-6
    nee = arr[(arr["event"] >> 31 == 1) & ((arr["event"] & 0xFFFFFF) != 0)]
    assert nee.size > 0 and np.abs(nee["amp"]).max() < 1e-9 * np.abs(smooth_arr["amp"]).max()   # O(alpha^2)


def _rough_plane_scene(alpha):
    """Water over a rough bone half-space at 20 mm; 32 elements with a 2 mm elevation (3 degrees seen
    from the plane) so that the element-centre connections stand for the element faces."""
    media = [WATER, (3500.0, 7.8, 0.0, alpha)]
    scene = {"media": media, "boundaries": [(oracle.PLANE_Z, [0.02, 0.0, 0.0, 0.0], 0, 1)], "med_array": 0,
             "z_max": 0.04, "scatterers": np.zeros((0, 4), np.float32), "r_s": 1e-4}
    arr = phantoms.array_params(32, 2048, elev_h=2e-3, c_bf=1540.0)
    arr["alpha_c_deg"] = 60.0
    arr["alpha_m_deg"] = 30.0
    return scene, arr


@pytest.mark.parametrize("alpha,steer_deg,more", [(0.3, 0.0, 4), (0.5, 0.0, 4), (0.8, 50.0, 16)])
def test_transducer_sampling_agrees_with_bsdf_sampling(alpha, steer_deg, more):
    """The method (transducer sampling at the rough vertex combined with the direct hits by the
    balance heuristic) and plain BSDF sampling estimate the same returns of a rough plane: the
    summed amplitude per element agrees within the Monte Carlo error.  The steered case makes the
    shadowing term matter (G1 of the incident direction about 0.84)."""
    scene, arr = _rough_plane_scene(alpha)
    ang = np.asarray([math.radians(steer_deg)], np.float32)
    N = 400_000          # each estimate is normalised by its own ray count (weights cos/N, Eq. 6)
    a_mis, _, st = oracle.trace(scene, arr, ang, N, 5, 1)
    a_bsdf, _, _ = oracle.trace(scene, arr, ang, more * N, 5, 1, rough_bsdf_only=True)   # few direct hits: more rays
    assert st["connections"] > 0

    def per_element(a):
        return np.bincount(a["el"], weights=a["amp"], minlength=32)

    def per_element_sq(a):
        return np.bincount(a["el"], weights=a["amp"] ** 2, minlength=32)

    m, b = per_element(a_mis), per_element(a_bsdf)
    sd = np.sqrt(per_element_sq(a_mis) + per_element_sq(a_bsdf))   # std of the difference of the sums
    sigma = math.sqrt((sd ** 2).sum())
    assert sigma < 0.03 * abs(b.sum())                 # precise enough to see a wrong factor
    assert abs(m.sum() - b.sum()) < 4 * sigma
    mid = slice(8, 24)
    assert np.all(np.abs(m[mid] - b[mid]) < 5 * sd[mid])
    # the method's estimate is the less noisy one
    assert per_element_sq(a_mis).sum() < per_element_sq(a_bsdf).sum()


def test_rough_scenes_outside_the_supported_modes_are_rejected():
    scene, arr = _rough_plane_scene(0.5)
    ang = np.zeros(1, np.float32)
    with pytest.raises(ValueError):
        oracle.trace(scene, arr, ang, 100, 0, 1, mode=oracle.MODE_EXPECT)
    g = np.zeros((1, 32, 2048))
    with pytest.raises(ValueError):
        oracle.grad(scene, arr, ang, 100, 0, 1, g, g)
    bad = dict(scene)
    bad["media"] = [WATER, (3500.0, 7.8, 0.0, -0.1)]
    with pytest.raises(ValueError):
        oracle.trace(bad, arr, ang, 100, 0, 1)
