"""Pins for the FP64 oracle: each test checks the oracle against something other
than itself (published vectors, closed forms, textbook acoustics, invariants,
statistics of the Monte Carlo estimator).  CPU only."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
import phantoms

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EXPECT = oracle.MODE_EXPECT


def _f(x):
    """The float32 value an input carries, promoted to double."""
    return float(np.float32(x))


# ----------------------------------------------------------------- Philox

def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_philox_matches_triton_interpreter(tmp_path):
    """Random counters and keys against triton.language.philox in Triton's CPU interpreter."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=2, dtype=np.uint64).astype(np.uint32)
    np.save(tmp_path / "ctr.npy", ctr)
    script = textwrap.dedent("""
        import os, sys
        os.environ["TRITON_INTERPRET"] = "1"
        import numpy as np, torch, triton, triton.language as tl
        @triton.jit
        def k(out_ptr, c_ptr, seed, N: tl.constexpr):
            off = tl.arange(0, N)
            c0 = tl.load(c_ptr + off * 4 + 0)
            c1 = tl.load(c_ptr + off * 4 + 1)
            c2 = tl.load(c_ptr + off * 4 + 2)
            c3 = tl.load(c_ptr + off * 4 + 3)
            a, b, c, d = tl.philox(seed, c0, c1, c2, c3, n_rounds=10)
            tl.store(out_ptr + off * 4 + 0, a)
            tl.store(out_ptr + off * 4 + 1, b)
            tl.store(out_ptr + off * 4 + 2, c)
            tl.store(out_ptr + off * 4 + 3, d)
        d = sys.argv[1]
        ctr = np.load(d + "/ctr.npy")
        out = torch.zeros(ctr.size, dtype=torch.int32)
        k[(1,)](out, torch.from_numpy(ctr.view(np.int32).reshape(-1).copy()), int(sys.argv[2]), N=ctr.shape[0])
        np.save(d + "/out.npy", out.numpy().view(np.uint32).reshape(ctr.shape))
    """)
    seed = int(key[0]) | (int(key[1]) << 32)
    try:
        subprocess.run([sys.executable, "-c", script, str(tmp_path), str(seed)], check=True, timeout=600,
                       capture_output=True)
    except subprocess.CalledProcessError as e:  # triton present but its interpreter unusable here
        pytest.skip("triton interpreter unavailable: %s" % e.stderr[-300:])
    ref = np.load(tmp_path / "out.npy")
    for q in range(ctr.shape[0]):
        assert list(oracle.philox4x32_10(ctr[q], key)) == list(ref[q])


# ------------------------------------------------- interface (Eqs. 7-11)

def _angle_dir(theta):
    return np.array([np.sin(theta), 0.0, np.cos(theta)])


def test_normal_incidence_reflection_coefficient():
    """Normal incidence: r = (Z2 - Z1)/(Z2 + Z1), straight-through transmission."""
    for (c1, Z1, c2, Z2) in [(1480, 1.48, 1580, 1.70), (1615, 1.99, 1450, 1.38), (1580, 1.70, 3500, 7.8)]:
        tir, dr, dt, r, R = oracle.interface([0, 0, 1], [0, 0, 1], c1, Z1, c2, Z2)
        assert not tir
        assert r == pytest.approx((Z2 - Z1) / (Z2 + Z1), rel=1e-14)
        assert np.allclose(dr, [0, 0, -1], atol=1e-15) and np.allclose(dt, [0, 0, 1], atol=1e-15)
    # values quoted for the layered phantom: skin/fat -0.1810, fat/muscle +0.1039, muscle/bone +0.6421
    assert oracle.interface([0, 0, 1], [0, 0, 1], 1615, 1.99, 1450, 1.38)[3] == pytest.approx(-0.1810, abs=5e-5)
    assert oracle.interface([0, 0, 1], [0, 0, 1], 1450, 1.38, 1580, 1.70)[3] == pytest.approx(0.1039, abs=5e-5)
    assert oracle.interface([0, 0, 1], [0, 0, 1], 1580, 1.70, 3500, 7.8)[3] == pytest.approx(0.6421, abs=5e-5)


def test_snell_law_and_mirror_reflection():
    rng = np.random.default_rng(1)
    for _ in range(200):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        c1, c2 = rng.uniform(1400, 3600, 2)
        Z1, Z2 = rng.uniform(1.3, 8.0, 2)
        tir, dr, dt, r, R = oracle.interface(d, n, c1, Z1, c2, Z2)
        sin_i = np.linalg.norm(np.cross(d, n))
        assert np.linalg.norm(dr) == pytest.approx(1.0, abs=1e-13)
        # reflection: same angle to the normal, mirrored normal component, in the plane of incidence
        assert abs(np.dot(dr, n)) == pytest.approx(abs(np.dot(d, n)), abs=1e-12)
        assert np.dot(dr, n) * np.dot(d, n) <= 0
        assert abs(np.dot(dr, np.cross(d, n))) < 1e-12
        if sin_i * c2 / c1 > 1.0 + 1e-12:
            assert tir and r == 1.0
            continue
        if sin_i * c2 / c1 > 1.0 - 1e-9:
            continue
        assert not tir
        sin_t = np.linalg.norm(np.cross(dt, n))
        assert sin_t / c2 == pytest.approx(sin_i / c1, rel=1e-10, abs=1e-14)   # acoustic Snell law
        assert np.dot(dt, n) * np.dot(d, n) > 0                               # continues across
        assert abs(np.dot(dt, np.cross(d, n))) < 1e-12
        assert np.linalg.norm(dt) == pytest.approx(1.0, abs=1e-13)


def test_critical_angle():
    c1, c2 = 1580.0, 3500.0            # muscle -> bone: critical angle asin(c1/c2) = 26.83 deg
    th_c = np.arcsin(c1 / c2)
    assert oracle.interface(_angle_dir(th_c - 1e-6), [0, 0, 1], c1, 1.7, c2, 7.8)[0] is False
    tir, dr, dt, r, R = oracle.interface(_angle_dir(th_c + 1e-6), [0, 0, 1], c1, 1.7, c2, 7.8)
    assert tir and r == 1.0 and R == 1.0


def test_intromission_angle_has_no_reflection():
    """Fluid-fluid interface: r = 0 at sin^2(theta) = (m^2 - n^2)/(m^2 - 1),
    m = rho2/rho1, n = c1/c2 (Rayleigh's angle of intromission)."""
    c1, rho1, c2, rho2 = 1540.0, 1000.0, 1400.0, 1500.0
    m, n = rho2 / rho1, c1 / c2
    th = np.arcsin(np.sqrt((m * m - n * n) / (m * m - 1.0)))
    r = oracle.interface(_angle_dir(th), [0, 0, 1], c1, rho1 * c1 * 1e-6, c2, rho2 * c2 * 1e-6)[3]
    assert abs(r) < 1e-12
    # and the sign flips across it
    r_lo = oracle.interface(_angle_dir(th - 0.05), [0, 0, 1], c1, rho1 * c1 * 1e-6, c2, rho2 * c2 * 1e-6)[3]
    r_hi = oracle.interface(_angle_dir(th + 0.05), [0, 0, 1], c1, rho1 * c1 * 1e-6, c2, rho2 * c2 * 1e-6)[3]
    assert r_lo * r_hi < 0


def test_grazing_incidence_total_reflection_limit():
    r = oracle.interface(_angle_dir(np.pi / 2 - 1e-7), [0, 0, 1], 1580, 1.70, 1450, 1.38)[3]
    assert r == pytest.approx(-1.0, abs=1e-5)


def test_reflection_reciprocity():
    """R for 1->2 at theta_i equals R for 2->1 at the refracted angle theta_t."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        c1, c2 = rng.uniform(1400, 3600, 2)
        Z1, Z2 = rng.uniform(1.3, 8.0, 2)
        th = rng.uniform(0, np.pi / 2 * 0.99)
        tir, dr, dt, r, R = oracle.interface(_angle_dir(th), [0, 0, 1], c1, Z1, c2, Z2)
        if tir:
            continue
        tir2, _, dt2, r2, R2 = oracle.interface(dt, [0, 0, 1], c2, Z2, c1, Z1)
        assert not tir2
        assert R2 == pytest.approx(R, rel=1e-9, abs=1e-15)
        assert r2 == pytest.approx(-r, rel=1e-9, abs=1e-15)
        assert np.allclose(dt2, _angle_dir(th), atol=1e-9)   # path reverses exactly


def test_textbook_impedance_over_cosine_form():
    """Kinsler & Frey form R = (Z2/cos_t - Z1/cos_i)/(Z2/cos_t + Z1/cos_i)."""
    rng = np.random.default_rng(4)
    for _ in range(100):
        c1, c2 = rng.uniform(1400, 3600, 2)
        Z1, Z2 = rng.uniform(1.3, 8.0, 2)
        th = rng.uniform(0, 1.4)
        st = np.sin(th) * c2 / c1
        if st >= 1:
            continue
        ct = np.sqrt(1 - st * st)
        ref = (Z2 / ct - Z1 / np.cos(th)) / (Z2 / ct + Z1 / np.cos(th))
        assert oracle.interface(_angle_dir(th), [0, 0, 1], c1, Z1, c2, Z2)[3] == pytest.approx(ref, rel=1e-10, abs=1e-14)


# ------------------------------------------ directivity, pulse, attenuation

def test_directivity_eq13():
    am, ac = np.deg2rad(10.0), np.deg2rad(30.0)
    assert oracle.directivity(0.0, am, ac) == 1.0
    assert oracle.directivity(am, am, ac) == 1.0
    assert oracle.directivity(-am, am, ac) == 1.0
    assert oracle.directivity(0.5 * (am + ac), am, ac) == pytest.approx(0.5, abs=1e-15)
    assert oracle.directivity(ac, am, ac) == pytest.approx(0.0, abs=1e-15)
    assert oracle.directivity(ac + 1e-9, am, ac) == 0.0
    # degenerate main-beam = cutoff (2 deg / 2 deg): a step
    a2 = np.deg2rad(2.0)
    assert oracle.directivity(a2 * (1 - 1e-12), a2, a2) == 1.0
    assert oracle.directivity(a2 * (1 + 1e-12), a2, a2) == 0.0


def test_pulse_eq14():
    f0, nc = 5e6, 5.0
    s = nc / (4 * f0)
    for tau in np.linspace(-3 * s, 3 * s, 41):
        re, im = oracle.pulse(tau, f0, nc)
        assert re * re + im * im == pytest.approx(np.exp(-tau * tau / (s * s)), rel=1e-12)   # envelope
    for m in range(-4, 5):                                         # zero crossings of the carrier
        assert oracle.pulse(m / (2 * f0), f0, nc)[0] == pytest.approx(0.0, abs=1e-12)
    assert oracle.pulse(0.0, f0, nc)[1] == pytest.approx(-1.0)
    # +-2 s spans exactly n_cycles periods and the envelope there is exp(-2)
    re, im = oracle.pulse(2 * s, f0, nc)
    assert np.hypot(re, im) == pytest.approx(np.exp(-2.0), rel=1e-12)
    assert 4 * s * f0 == pytest.approx(nc)


def test_attenuation_conversion():
    assert oracle.np_per_m(1.0, 5e6) == pytest.approx(500.0 * np.log(10) / 20.0, rel=1e-12)
    assert oracle.np_per_m(1.0, 5e6) == pytest.approx(57.565, abs=5e-4)


def test_deposit_reproduces_pulse():
    arr = phantoms.array_params(4, 200)
    a = np.zeros(1, oracle.ARRIVAL_DTYPE)
    a["tx"], a["el"], a["t"], a["amp"] = 0, 2, 87.3125, -0.75
    rf, quad = oracle.deposit(arr, 1, a)
    fs = _f(arr["fs"])
    K = 5 * 5 / (4 * _f(arr["f0"])) * fs
    for n in range(200):
        tau = n - 87.3125
        if abs(tau) <= K:
            re, im = oracle.pulse(tau / fs, _f(arr["f0"]), _f(arr["n_cycles"]))
            assert rf[0, 2, n] == pytest.approx(-0.75 * re, abs=1e-15)
            assert quad[0, 2, n] == pytest.approx(-0.75 * im, abs=1e-15)
        else:
            assert rf[0, 2, n] == 0.0 and quad[0, 2, n] == 0.0
    assert np.all(rf[0, [0, 1, 3]] == 0.0)


# --------------------------------------------------------- closed-form echoes

def _aperture(arr):
    return arr[(arr["event"] >> 31) == 1]


def _bounces(arr):
    return (arr["event"] >> 24) & 0x7F


@pytest.mark.parametrize("alpha_upper", [0.0, 1.0])
def test_normal_incidence_planar_echo_expectation(alpha_upper):
    """Echo of a flat interface at depth d, 0 deg: t = 2 d/c, amplitude r exp(-2 a d)."""
    upper = (1480.0, 1.48, alpha_upper, 0.0)
    w = phantoms.single_plane(depth=0.015, upper=upper, n_rays=3200)
    arr, _, st = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], 1, 4, mode=EXPECT)
    ap = _aperture(arr)
    assert ap.size == w["n_rays"]                       # every ray's echo lands on its own element
    d, fs, f0 = _f(0.015), _f(40e6), _f(5e6)
    t_ref = 2 * d / 1480.0 * fs
    a = alpha_upper * f0 * 1e-6 * 100 / (20 / np.log(10))
    r = (1.70 - _f(1.48)) / (1.70 + _f(1.48))
    r = (_f(1.70) - _f(1.48)) / (_f(1.70) + _f(1.48))
    assert np.allclose(ap["t"], t_ref, rtol=0, atol=1e-9)
    assert np.allclose(ap["amp"], r * np.exp(-2 * a * d) / w["n_rays"], rtol=1e-12)
    assert t_ref == pytest.approx(810.81, abs=5e-3)
    per_el = np.bincount(ap["el"], weights=ap["amp"], minlength=32)
    assert np.allclose(per_el, r * np.exp(-2 * a * d) / 32, rtol=1e-12)


def test_normal_incidence_planar_echo_monte_carlo():
    """MC branch weights: the per-ray estimator is unbiased for r (within 5 sigma)."""
    w = phantoms.single_plane(depth=0.015, n_rays=320_000)
    arr, _, _ = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], 11, 4)
    ap = _aperture(arr)
    ap1 = ap[_bounces(ap) == 1]
    r = (_f(1.70) - _f(1.48)) / (_f(1.70) + _f(1.48))
    N = w["n_rays"]
    assert np.allclose(ap1["amp"], 1.0 / (N * r), rtol=1e-12)     # reflect weight w r/R = w/r
    total = ap1["amp"].sum()
    sigma = np.sqrt(N * r * r * (1 - r * r)) / (N * r)
    assert abs(total - r) < 5 * sigma


def test_layered_echo_times_and_amplitudes():
    """Skin 0-2 mm / fat 2-10 mm / muscle: first two echoes in closed form."""
    w = phantoms.layered(n_scat=0, n_rays=1280)
    sc = dict(w["scene"])
    sc["boundaries"] = sc["boundaries"][:2]                 # drop the bone cylinder
    arr, _, _ = oracle.trace(sc, w["array"], w["angles"], w["n_rays"], 2, 8, mode=EXPECT)
    ap = _aperture(arr)
    b = _bounces(ap)
    fs, f0 = _f(40e6), _f(5e6)
    d1, d2 = _f(2e-3), _f(10e-3) - _f(2e-3)
    cs, cf = 1615.0, 1450.0
    Zs, Zf, Zm = _f(1.99), _f(1.38), _f(1.70)
    r_sf = (Zf - Zs) / (Zf + Zs)
    r_fm = (Zm - Zf) / (Zm + Zf)
    a_f = _f(0.6) * f0 * 1e-6 * 100 * np.log(10) / 20
    e1, e3 = ap[b == 1], ap[b == 3]
    assert e1.size == w["n_rays"] and e3.size == w["n_rays"]
    assert np.allclose(e1["t"], 2 * d1 / cs * fs, atol=1e-9, rtol=0)
    assert np.allclose(e1["amp"], r_sf / w["n_rays"], rtol=1e-12)
    t3 = 2 * (d1 / cs + (_f(10e-3) - _f(2e-3)) / cf) * fs
    assert np.allclose(e3["t"], t3, atol=1e-9, rtol=0)
    assert np.allclose(e3["amp"], (1 - r_sf ** 2) * r_fm * np.exp(-2 * a_f * d2) / w["n_rays"], rtol=1e-11)
    assert t3 / fs * 1e6 == pytest.approx(13.511, abs=1e-3)
    assert 20 * np.log10(np.exp(-2 * a_f * d2)) == pytest.approx(-2 * 0.6 * 5 * 0.8, rel=1e-9)


def test_single_scatterer_time_amplitude_and_hit_rate():
    """A point scatterer in water: t_e = z/c + |p - c_e|/c, amplitude f_d(alpha_e)/N per hit,
    hit probability pi r_s^2 / aperture area (binomial, 5 sigma)."""
    pos = (0.05e-3, 0.3e-3, 10e-3)
    w = phantoms.single_scatterer(pos, n_rays=1_000_000, alpha_m_deg=10.0, alpha_c_deg=30.0)
    arr, _, st = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], 5, 4, mode=EXPECT)
    sa = arr[(arr["event"] >> 31) == 0]
    N, n_el, pitch, H = w["n_rays"], 32, _f(0.3e-3), _f(4e-3)
    p = np.array([_f(v) for v in pos])
    fs, c = _f(40e6), 1480.0
    am, ac = np.deg2rad(_f(10.0)), np.deg2rad(_f(30.0))
    hits = st["candidates"]
    for e in range(n_el):
        xe = (e - 15.5) * pitch
        D = np.sqrt((p[0] - xe) ** 2 + p[1] ** 2 + p[2] ** 2)
        alpha = np.arccos(p[2] / D)
        fd = 1.0 if alpha <= am else max(0.0, (ac - alpha) / (ac - am))
        mine = sa[sa["el"] == e]
        if fd == 0.0:
            assert mine.size == 0
            continue
        assert mine.size == hits
        assert np.allclose(mine["t"], (p[2] + D) / c * fs, atol=1e-9, rtol=0)
        assert np.allclose(mine["amp"], fd / N, rtol=1e-12)
    p_hit = np.pi * _f(1e-4) ** 2 / (n_el * pitch * H)
    assert abs(hits - N * p_hit) < 5 * np.sqrt(N * p_hit * (1 - p_hit))


def test_connection_through_plane_closed_form():
    """Straight connection from below an interface to the element centre above it."""
    w = phantoms.single_plane(depth=0.015, lower=(1580.0, 1.70, 1.0, 0.0))
    Z1, Z2 = _f(1.48), _f(1.70)
    fs, f0 = _f(40e6), _f(5e6)
    a2 = f0 * 1e-6 * 100 * np.log(10) / 20
    xe = 3.5 * _f(0.3e-3)
    fac, t, att = oracle.connection(w["scene"], w["array"], [xe, 0.0, 0.025], 1, xe)
    assert fac == pytest.approx(2 * np.sqrt(Z1 * Z2) / (Z1 + Z2), rel=1e-12)
    assert t == pytest.approx((_f(0.015) / 1480.0 + (0.025 - _f(0.015)) / 1580.0) * fs, rel=1e-12)
    assert att == pytest.approx(a2 * (0.025 - _f(0.015)), rel=1e-12)
    # oblique: factor sqrt(1 - R) at the crossing angle, and reciprocity of R under reversal
    p = np.array([xe + 4e-3, 1e-3, 0.030])
    fac, t, att = oracle.connection(w["scene"], w["array"], p, 1, xe)
    v = np.array([xe, 0, 0]) - p
    v /= np.linalg.norm(v)
    ci = abs(v[2])
    st = np.sqrt(1 - ci * ci) * 1480.0 / 1580.0
    ct = np.sqrt(1 - st * st)
    r = (Z1 / ct - Z2 / ci) / (Z1 / ct + Z2 / ci)
    assert fac == pytest.approx(np.sqrt(1 - r * r), rel=1e-10)


def test_connection_blocked_by_total_internal_reflection():
    """Leaving bone (fast) for muscle (slow) never reflects totally, the reverse can."""
    w = phantoms.single_plane(depth=0.015, upper=(1580.0, 1.70, 0.0, 0.0), lower=(3500.0, 7.8, 0.0, 0.0))
    # from muscle (above the plane) looking down is impossible; put the fast medium above instead
    w2 = phantoms.single_plane(depth=0.015, upper=(3500.0, 7.8, 0.0, 0.0), lower=(1580.0, 1.70, 0.0, 0.0))
    xe = 0.0
    # steep enough: sin(theta) > c1/c2 with c1 = 1580 (below) going into 3500 (above)
    p = np.array([0.02, 0.0, 0.020])
    assert oracle.connection(w2["scene"], w2["array"], p, 1, xe)[0] == 0.0
    assert oracle.connection(w["scene"], w["array"], p, 1, xe)[0] > 0.0


# ------------------------------------------------ MC estimator vs expectation

def test_monte_carlo_matches_expectation():
    """Per seed, the MC estimate minus the expectation-mode value (same emission
    points) has zero mean over the branch and element choices."""
    w = phantoms.tiny(n_scat=3000, n_rays=20_000)
    sc = w["scene"]
    diffs = []
    for s in range(40):
        tot = []
        for mode in (oracle.MODE_MC, EXPECT):
            arr, _, _ = oracle.trace(sc, w["array"], w["angles"], w["n_rays"], 100 + s, 3, mode=mode)
            kind = (arr["event"] >> 31).astype(np.int64)
            key = arr["el"].astype(np.int64) * 2 + kind
            tot.append(np.bincount(key, weights=arr["amp"], minlength=64))
        diffs.append(tot[0] - tot[1])
    D = np.array(diffs)
    m = D.mean(0)
    se = D.std(0, ddof=1) / np.sqrt(D.shape[0])
    ok = se > 0
    assert ok.sum() > 40
    assert np.all(np.abs(m[ok]) < 6 * se[ok])
    # aggregate over elements (much tighter)
    for kind in (0, 1):
        agg = D[:, kind::2].sum(1)
        assert abs(agg.mean()) < 5 * agg.std(ddof=1) / np.sqrt(agg.size)


# ---------------------------------------------------------------- imaging

@pytest.mark.parametrize("theta_deg", [0.0, 10.0])
def test_das_focuses_point_target(theta_deg):
    """Channel data of a point target built from closed-form plane-wave delays
    beamforms to an envelope peak at the target."""
    arr = phantoms.array_params(64, 2048, c_bf=1540.0)
    xs, zs = 1.2e-3, 20e-3
    th = np.deg2rad(theta_deg)
    ang = np.array([th], np.float32)
    th = float(ang[0])
    pitch = _f(arr["pitch"])
    xe = (np.arange(64) - 31.5) * pitch
    c, fs = _f(1540.0), _f(40e6)
    mn = np.min(xe * np.sin(th))
    t = (xs * np.sin(th) + zs * np.cos(th) - mn + np.sqrt(zs ** 2 + (xs - xe) ** 2)) / c * fs
    a = np.zeros(64, oracle.ARRIVAL_DTYPE)
    a["el"], a["t"], a["amp"] = np.arange(64), t, 1.0
    rf, quad = oracle.deposit(arr, 1, a)
    x = (xs + np.arange(-20, 21) * 0.05e-3).astype(np.float32)
    z = (zs + np.arange(-20, 21) * 0.01e-3).astype(np.float32)
    iq = oracle.beamform(arr, ang, rf, quad, x, z)
    env, db = oracle.envelope_log(iq, 60.0)
    iz, ix = np.unravel_index(np.argmax(env), env.shape)
    assert abs(x[ix] - xs) <= 0.0501e-3 and abs(z[iz] - zs) <= 0.0101e-3   # within one pixel
    assert env.max() > 0.9 * 64          # coherent sum; linear interpolation of the phasor costs < 8%
    assert db.max() == 0.0 and db.min() >= -60.0


def test_envelope_log_compression():
    iq = np.array([[3 + 4j, 0.0, 0.3 + 0.4j, 1e-6]])
    env, db = oracle.envelope_log(iq, 60.0)
    assert np.allclose(env, [[5.0, 0.0, 0.5, 1e-6]])
    assert np.allclose(db, [[0.0, -60.0, -20.0, -60.0]])


# ------------------------------------------------------------ bookkeeping

def test_path_hashes_deterministic_and_seed_dependent():
    w = phantoms.tiny(n_rays=2000)
    a1, h1, _ = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], 0, 4, topo=True)
    a2, h2, _ = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], 0, 4, topo=True, threads=3)
    a3, h3, _ = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], 1, 4, topo=True)
    assert np.array_equal(h1, h2) and np.array_equal(a1, a2)
    assert not np.array_equal(h1, h3)
    # a sub-range reproduces the same rays
    a4, h4, _ = oracle.trace(w["scene"], w["array"], w["angles"], w["n_rays"], 0, 4, ray_begin=500,
                             ray_end=900, topo=True)
    assert np.array_equal(h4[0], h1[0, 500:900])
    sel = a1[(a1["ray"] >= 500) & (a1["ray"] < 900)]
    assert np.array_equal(sel, a4)
