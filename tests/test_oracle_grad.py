"""Pins for the oracle's FP64 dual-number gradient: finite differences of the
oracle's own forward with the branch sampling frozen at the unperturbed media
(the reading under which the pathwise gradient is taken), and closed forms for
the normal-incidence planar echo."""
import copy

import numpy as np
import pytest

import oracle
import phantoms


def linear_loss(w, G_rf, G_q, seed, n_rays, scene=None):
    sc = scene or w["scene"]
    arr, _, _ = oracle.trace(sc, w["array"], w["angles"], n_rays, seed, w["max_bounces"], w["max_path"])
    rf, q = oracle.deposit(w["array"], len(w["angles"]), arr)
    return float(np.sum(G_rf * rf) + np.sum(G_q * q))


def perturbed(w, m, col, h):
    sc = copy.deepcopy(w["scene"])
    sc["media_sampling"] = np.array(w["scene"]["media"], np.float32)
    med = np.array(sc["media"], np.float64)
    med[m, col] += h
    sc["media"] = med.astype(np.float32)
    return sc, float(np.float32(med[m, col])) - float(np.float32(w["scene"]["media"][m, col]))


@pytest.mark.parametrize("angle_deg", [0.0, 9.0])
def test_media_gradient_matches_finite_differences(angle_deg):
    w = phantoms.tiny(n_scat=400, n_rays=6000)
    w["angles"] = np.array([np.deg2rad(angle_deg)], np.float32)
    shape = (1, 32, w["array"]["n_s"])
    rng = np.random.default_rng(3)
    G_rf, G_q = rng.standard_normal(shape), rng.standard_normal(shape)
    gm, _ = oracle.grad(w["scene"], w["array"], w["angles"], w["n_rays"], 4, w["max_bounces"], G_rf, G_q)
    med = w["scene"]["media"]
    checked = 0
    for m in range(3):
        for col in range(3):
            base = float(med[m, col])
            if col == 2 and base == 0.0:
                h = 1e-3                          # alpha = 0: step from zero
            else:
                h = base * 1e-4
            sp, hp = perturbed(w, m, col, h)
            sm, hm = perturbed(w, m, col, -h)
            Lp = linear_loss(w, G_rf, G_q, 4, w["n_rays"], sp)
            Lm = linear_loss(w, G_rf, G_q, 4, w["n_rays"], sm)
            fd = (Lp - Lm) / (hp - hm)
            tol = 2e-3 * abs(fd) + 1e-6 * np.abs(gm).max()
            assert abs(gm[m, col] - fd) <= tol, (m, col, gm[m, col], fd)
            checked += abs(fd) > 0
    assert checked >= 6


def test_amplitude_gradient_is_exact():
    w = phantoms.tiny(n_scat=300, n_rays=20_000)
    shape = (1, 32, w["array"]["n_s"])
    rng = np.random.default_rng(5)
    G_rf, G_q = rng.standard_normal(shape), rng.standard_normal(shape)
    _, ga = oracle.grad(w["scene"], w["array"], w["angles"], w["n_rays"], 2, w["max_bounces"], G_rf, G_q)
    nz = np.flatnonzero(ga)
    assert nz.size >= 3
    for j in nz[:4]:
        sc = copy.deepcopy(w["scene"])
        s = np.array(sc["scatterers"], np.float64)
        h = 0.25
        s[j, 3] += h
        sc["scatterers"] = s.astype(np.float32)
        sc2 = copy.deepcopy(w["scene"])
        s2 = np.array(sc2["scatterers"], np.float64)
        s2[j, 3] -= h
        sc2["scatterers"] = s2.astype(np.float32)
        fd = (linear_loss(w, G_rf, G_q, 2, w["n_rays"], sc) - linear_loss(w, G_rf, G_q, 2, w["n_rays"], sc2)) / (
            float(np.float32(s[j, 3])) - float(np.float32(s2[j, 3])))
        assert ga[j] == pytest.approx(fd, rel=1e-9, abs=1e-12)


def test_planar_echo_gradient_closed_form():
    """Reflected rays of a flat interface at normal incidence: amplitude (1/N) r / R_fixed and
    time 2 d fs / c1, so dL/dZ2 = sum (1/N) (dr/dZ2)/r^2 S(t) and dL/dc1 = sum g_t (-2 d fs / c1^2)."""
    w = phantoms.single_plane(depth=0.015, n_rays=64_000)
    N, fs, f0 = w["n_rays"], float(np.float32(40e6)), float(np.float32(5e6))
    shape = (1, 32, w["array"]["n_s"])
    rng = np.random.default_rng(8)
    G_rf, G_q = rng.standard_normal(shape), rng.standard_normal(shape)
    gm, _ = oracle.grad(w["scene"], w["array"], w["angles"], N, 6, 4, G_rf, G_q)
    arr, _, _ = oracle.trace(w["scene"], w["array"], w["angles"], N, 6, 4)
    ap = arr[(arr["event"] >> 31) == 1]
    Z1, Z2, c1 = float(np.float32(1.48)), float(np.float32(1.70)), 1480.0
    r = (Z2 - Z1) / (Z2 + Z1)
    d = float(np.float32(0.015))
    t = 2 * d / c1 * fs
    s_n = 5.0 / (4 * f0) * fs
    om = 2 * np.pi * f0 / fs
    n = np.arange(w["array"]["n_s"])
    tau = n - t
    win = np.abs(tau) <= 5 * s_n
    g = np.exp(-tau ** 2 / (2 * s_n ** 2)) * win
    p_re, p_im = g * np.sin(om * tau), -g * np.cos(om * tau)
    dp_re = g * (om * np.cos(om * tau) - tau / s_n ** 2 * np.sin(om * tau))
    dp_im = g * (om * np.sin(om * tau) + tau / s_n ** 2 * np.cos(om * tau))
    dZ2 = 0.0
    dc1 = 0.0
    for a in ap:
        S = np.sum(G_rf[0, a["el"]] * p_re + G_q[0, a["el"]] * p_im)
        St = -np.sum(G_rf[0, a["el"]] * dp_re + G_q[0, a["el"]] * dp_im)
        dZ2 += (1.0 / N) * (2 * Z1 / (Z1 + Z2) ** 2) / r ** 2 * S
        dc1 += a["amp"] * St * (-2 * d * fs / c1 ** 2)
    assert ap.size > 100
    assert gm[1, 1] == pytest.approx(dZ2, rel=1e-9)
    assert gm[0, 0] == pytest.approx(dc1, rel=1e-9)
