"""FP64 CPU oracle (test infrastructure only).

This package is the slow, obviously correct reference implementation of the
UltraRay hot path (arXiv 2501.05828): plane-wave ray emission (Sec. 2.3, Eq. 6),
traversal with reflection/refraction (Eqs. 7-11), transducer sampling with the
receive directivity (Eq. 13), pulse deposit (Eq. 14), delay-and-sum, envelope
and log compression (Sec. 2.3, last paragraph).  The arithmetic lives in
``ur_oracle.c``; this module only builds it and marshals numpy arrays.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It never imports the CUDA package, and the CUDA
package never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ur_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liburoracle.so")
_lock = threading.Lock()
_lib = None

PLANE_Z, SPHERE, CYL_Y = 0, 1, 2
TX_PLANE, TX_DIVERGING, TX_FOCUSED, TX_SYNTHETIC = 0, 1, 2, 3
MODE_MC, MODE_EXPECT = 0, 1
END_APERTURE, END_ARRAY_MISS, END_BOTTOM, END_PATH, END_TIME, END_MAXB, END_ROUGH = 1, 2, 3, 4, 5, 6, 7


def build(force: bool = False) -> str:
    """Compile ur_oracle.c into _build/liburoracle.so with gcc (OpenMP, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(os.path.join(_HERE, "ur_oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Scene(C.Structure):
    _fields_ = [("n_med", C.c_int32), ("med", C.POINTER(C.c_float)),
                ("n_bnd", C.c_int32), ("bnd_kind", C.POINTER(C.c_int32)),
                ("bnd_p", C.POINTER(C.c_float)), ("bnd_med", C.POINTER(C.c_int32)),
                ("med_array", C.c_int32), ("z_max", C.c_float),
                ("n_scat", C.c_int32), ("scat", C.POINTER(C.c_float)), ("r_s", C.c_float),
                ("med_sampling", C.POINTER(C.c_float)),
                ("n_tri", C.c_int32), ("tri", C.POINTER(C.c_float)), ("tri_med", C.POINTER(C.c_int32))]


class Array(C.Structure):
    _fields_ = [("n_el", C.c_int32), ("pitch", C.c_float), ("elev_h", C.c_float),
                ("f0", C.c_float), ("fs", C.c_float), ("n_s", C.c_int32),
                ("n_cycles", C.c_float), ("alpha_m_deg", C.c_float), ("alpha_c_deg", C.c_float),
                ("c_bf", C.c_float), ("tcut_sigmas", C.c_float), ("radius", C.c_float)]


class TraceCfg(C.Structure):
    _fields_ = [("n_tx", C.c_int32), ("angles", C.POINTER(C.c_float)),
                ("n_rays", C.c_uint64), ("ray_begin", C.c_uint64), ("ray_end", C.c_uint64),
                ("seed", C.c_uint64), ("max_bounces", C.c_int32), ("max_path", C.c_float),
                ("mode", C.c_int32), ("rough_bsdf_only", C.c_int32),
                ("tx_kind", C.POINTER(C.c_int32)), ("tx_x", C.POINTER(C.c_float)), ("tx_z", C.POINTER(C.c_float)),
                ("mix", C.c_int32)]


class Arrival(C.Structure):
    _fields_ = [("tx", C.c_int32), ("el", C.c_int32), ("ray", C.c_uint32), ("event", C.c_uint32),
                ("t", C.c_double), ("amp", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("rays", C.c_uint64), ("segments", C.c_uint64), ("interactions", C.c_uint64),
                ("candidates", C.c_uint64), ("connections", C.c_uint64), ("arrivals", C.c_uint64)]


ARRIVAL_DTYPE = np.dtype([("tx", "<i4"), ("el", "<i4"), ("ray", "<u4"), ("event", "<u4"),
                          ("t", "<f8"), ("amp", "<f8")])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
            L.or_trace.restype = C.c_int64
            L.or_trace.argtypes = [C.POINTER(Scene), C.POINTER(Array), C.POINTER(TraceCfg),
                                   C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(Stats), C.c_int]
            L.or_deposit.argtypes = [C.POINTER(Array), C.c_int32, C.c_void_p, C.c_int64, dp, dp]
            L.or_beamform.argtypes = [C.POINTER(Array), C.c_int32, C.POINTER(C.c_float), dp, dp,
                                      C.POINTER(C.c_float), C.c_int32, C.POINTER(C.c_float), C.c_int32,
                                      dp, dp, C.c_int]
            L.or_envelope_log.argtypes = [dp, dp, C.c_int64, C.c_double, dp, dp]
            L.or_beamform_tx.argtypes = [C.POINTER(Array), C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_int32),
                                         C.POINTER(C.c_float), C.POINTER(C.c_float), dp, dp,
                                         C.POINTER(C.c_float), C.c_int32, C.POINTER(C.c_float), C.c_int32,
                                         dp, dp, C.c_int]
            L.or_interface.restype = C.c_int
            L.or_interface.argtypes = [dp, dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                       dp, dp, dp, dp]
            L.or_directivity.restype = C.c_double
            L.or_directivity.argtypes = [C.c_double] * 3
            L.or_pulse.restype = C.c_double
            L.or_pulse.argtypes = [C.c_double, C.c_double, C.c_double, dp]
            L.or_np_per_m.restype = C.c_double
            L.or_np_per_m.argtypes = [C.c_double, C.c_double]
            L.or_connection.restype = C.c_double
            L.or_connection.argtypes = [C.POINTER(Scene), C.POINTER(Array), dp, C.c_int32,
                                        C.c_double, dp, dp]
            L.or_ggx_d.restype = C.c_double
            L.or_ggx_d.argtypes = [C.c_double, C.c_double]
            L.or_ggx_g1.restype = C.c_double
            L.or_ggx_g1.argtypes = [C.c_double, C.c_double]
            L.or_ggx_sample.argtypes = [dp, C.c_double, C.c_double, C.c_double, dp]
            L.or_rough_eval.restype = C.c_double
            L.or_rough_eval.argtypes = [dp, dp, dp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, dp]
            L.or_grad.restype = C.c_int
            L.or_grad.argtypes = [C.POINTER(Scene), C.POINTER(Array), C.POINTER(TraceCfg), dp, dp, dp, dp, C.c_int]
            _lib = L
    return _lib


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


class _Keep:
    """Holds the numpy buffers a ctypes struct points into."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def make_scene(scene):
    med = np.ascontiguousarray(scene["media"], dtype=np.float32).reshape(-1, 4)
    kinds = np.ascontiguousarray([b[0] for b in scene["boundaries"]], dtype=np.int32)
    bp = np.ascontiguousarray([b[1] for b in scene["boundaries"]], dtype=np.float32).reshape(-1, 4)
    bm = np.ascontiguousarray([[b[2], b[3]] for b in scene["boundaries"]], dtype=np.int32).reshape(-1, 2)
    sc = np.ascontiguousarray(scene["scatterers"], dtype=np.float32).reshape(-1, 4)
    if kinds.size == 0:
        kinds = np.zeros(1, np.int32)
        bp = np.zeros((1, 4), np.float32)
        bm = np.zeros((1, 2), np.int32)
    if sc.size == 0:
        sc_buf = np.zeros((1, 4), np.float32)
    else:
        sc_buf = sc
    ms = scene.get("media_sampling")
    ms = None if ms is None else np.ascontiguousarray(ms, dtype=np.float32).reshape(-1, 4)
    tris = scene.get("triangles")   # (vertices [n, 9] float32, media [n, 2]: behind, in front)
    tv = tm = None
    if tris is not None:
        tv = np.ascontiguousarray(tris[0], dtype=np.float32).reshape(-1, 9)
        tm = np.ascontiguousarray(tris[1], dtype=np.int32).reshape(-1, 2)
    s = Scene(med.shape[0], _fp(med), len(scene["boundaries"]), _ip(kinds), _fp(bp), _ip(bm),
              int(scene["med_array"]), float(scene["z_max"]), sc.shape[0], _fp(sc_buf),
              float(scene["r_s"]), _fp(ms) if ms is not None else None,
              0 if tv is None else tv.shape[0], _fp(tv) if tv is not None else None,
              _ip(tm) if tm is not None else None)
    return s, _Keep(med=med, kinds=kinds, bp=bp, bm=bm, sc=sc_buf, ms=ms, tv=tv, tm=tm)


def make_array(arr):
    return Array(int(arr["n_el"]), arr["pitch"], arr["elev_h"], arr["f0"], arr["fs"], int(arr["n_s"]),
                 arr["n_cycles"], arr["alpha_m_deg"], arr["alpha_c_deg"], arr["c_bf"],
                 arr["tcut_sigmas"], float(arr.get("radius", 0.0)))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    P = C.POINTER(C.c_uint32)
    lib().or_philox4x32_10(c.ctypes.data_as(P), k.ctypes.data_as(P), out.ctypes.data_as(P))
    return out


def _transmit_arrays(transmits, n_tx):
    """transmits: None (plane waves of `angles`) or a sequence of (kind, x, z) per transmit
    (TX_SYNTHETIC: x = the firing element's index)."""
    if transmits is None:
        return None
    t = list(transmits)
    assert len(t) == n_tx
    kind = np.ascontiguousarray([int(k) for k, _, _ in t], np.int32)
    tx = np.ascontiguousarray([x for _, x, _ in t], np.float32)
    tz = np.ascontiguousarray([z for _, _, z in t], np.float32)
    return kind, tx, tz


def trace(scene, array, angles, n_rays, seed, max_bounces, max_path=0.2, ray_begin=0, ray_end=None,
          mode=MODE_MC, topo=False, threads=None, rough_bsdf_only=False, transmits=None, mix=False):
    """Trace rays [ray_begin, ray_end) of every transmit; with mix, rays [ray_begin, ray_end) of
    one sequence of n_tx * n_rays rays that draw their transmits.

    Returns (arrivals structured array, topology hashes [n_tx, n_sub] ([n_sub] with mix) or None,
    stats dict)."""
    L = lib()
    ang = np.ascontiguousarray(angles, dtype=np.float32).reshape(-1)
    if ray_end is None:
        ray_end = n_rays * (ang.size if mix else 1)
    s, keep_s = make_scene(scene)
    a = make_array(array)
    txa = _transmit_arrays(transmits, ang.size)
    cfg = TraceCfg(ang.size, _fp(ang), int(n_rays), int(ray_begin), int(ray_end), int(seed),
                   int(max_bounces), float(max_path), int(mode), int(bool(rough_bsdf_only)),
                   _ip(txa[0]) if txa else None, _fp(txa[1]) if txa else None, _fp(txa[2]) if txa else None,
                   int(bool(mix)))
    n_sub = int(ray_end) - int(ray_begin)
    topo_arr = (np.zeros(n_sub, np.uint64) if mix else np.zeros((ang.size, n_sub), np.uint64)) if topo else None
    threads = threads or (os.cpu_count() or 1)
    cap = max(1024, n_sub * ang.size // 2)
    while True:
        out = np.zeros(cap, ARRIVAL_DTYPE)
        st = Stats()
        n = L.or_trace(C.byref(s), C.byref(a), C.byref(cfg), out.ctypes.data, cap,
                       topo_arr.ctypes.data if topo else None, C.byref(st), int(threads))
        if n < 0:
            raise ValueError("or_trace rejected its arguments")
        if n <= cap:
            break
        cap = int(n)
    del keep_s
    stats = {f: int(getattr(st, f)) for f, _ in Stats._fields_}
    return out[:n].copy(), topo_arr, stats


def grad(scene, array, angles, n_rays, seed, max_bounces, g_rf, g_q, max_path=0.2, ray_begin=0, ray_end=None,
         threads=None):
    """Pathwise gradient of L (given dL/drf, dL/dquad) w.r.t. the media (c, Z, alpha) and the
    scatterer amplitudes: returns (grad_media [n_med, 3], grad_amp [n_scat])."""
    if ray_end is None:
        ray_end = n_rays
    s, keep = make_scene(scene)
    a = make_array(array)
    ang = np.ascontiguousarray(angles, dtype=np.float32).reshape(-1)
    cfg = TraceCfg(ang.size, _fp(ang), int(n_rays), int(ray_begin), int(ray_end), int(seed), int(max_bounces),
                   float(max_path), MODE_MC, 0, None, None, None)
    gr = np.ascontiguousarray(g_rf, dtype=np.float64)
    gq = np.ascontiguousarray(g_q, dtype=np.float64)
    n_med = len(scene["media"])
    gm = np.zeros((n_med, 3), np.float64)
    n_scat = len(scene["scatterers"])
    ga = np.zeros(max(n_scat, 1), np.float64)
    rc = lib().or_grad(C.byref(s), C.byref(a), C.byref(cfg), _dp(gr), _dp(gq), _dp(gm), _dp(ga),
                       int(threads or (os.cpu_count() or 1)))
    del keep
    if rc != 0:
        raise ValueError("or_grad rejected its arguments")
    return gm, ga[:n_scat]


def deposit(array, n_tx, arrivals):
    """Eq. 14 deposit: returns (rf, quad) float64 [n_tx, n_el, n_s]."""
    a = make_array(array)
    shape = (int(n_tx), int(array["n_el"]), int(array["n_s"]))
    rf = np.zeros(shape, np.float64)
    quad = np.zeros(shape, np.float64)
    arr = np.ascontiguousarray(arrivals, dtype=ARRIVAL_DTYPE)
    lib().or_deposit(C.byref(a), int(n_tx), arr.ctypes.data if arr.size else None, arr.size,
                     _dp(rf), _dp(quad))
    return rf, quad


def beamform(array, angles, rf, quad, x_px, z_px, threads=None, transmits=None):
    """DAS with coherent compounding (plane waves of `angles`, or the kinds of `transmits`):
    returns complex128 [nz, nx]."""
    a = make_array(array)
    ang = np.ascontiguousarray(angles, dtype=np.float32).reshape(-1)
    txa = _transmit_arrays(transmits, ang.size)
    rf = np.ascontiguousarray(rf, dtype=np.float64)
    quad = np.ascontiguousarray(quad, dtype=np.float64)
    xp = np.ascontiguousarray(x_px, dtype=np.float32)
    zp = np.ascontiguousarray(z_px, dtype=np.float32)
    re = np.zeros((zp.size, xp.size), np.float64)
    im = np.zeros_like(re)
    lib().or_beamform_tx(C.byref(a), ang.size, _fp(ang), _ip(txa[0]) if txa else None,
                         _fp(txa[1]) if txa else None, _fp(txa[2]) if txa else None, _dp(rf), _dp(quad),
                         _fp(xp), xp.size, _fp(zp), zp.size, _dp(re), _dp(im), int(threads or (os.cpu_count() or 1)))
    return re + 1j * im


def envelope_log(iq, dyn_range_db):
    """Envelope and log compression: returns (env, dB) float64 arrays like iq."""
    re = np.ascontiguousarray(iq.real, dtype=np.float64)
    im = np.ascontiguousarray(iq.imag, dtype=np.float64)
    env = np.zeros_like(re)
    db = np.zeros_like(re)
    lib().or_envelope_log(_dp(re), _dp(im), re.size, float(dyn_range_db), _dp(env), _dp(db))
    return env, db


def interface(d, n, c1, Z1, c2, Z2):
    """Eqs. 7-11 at one boundary: returns (tir, d_r, d_t, r, R)."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    dr = np.zeros(3)
    dt = np.zeros(3)
    r = C.c_double()
    R = C.c_double()
    tir = lib().or_interface(_dp(d), _dp(n), c1, Z1, c2, Z2, _dp(dr), _dp(dt), C.byref(r), C.byref(R))
    return bool(tir), dr, dt, r.value, R.value


def directivity(alpha, alpha_m, alpha_c):
    return lib().or_directivity(float(alpha), float(alpha_m), float(alpha_c))


def pulse(tau, f0, n_cycles):
    im = C.c_double()
    re = lib().or_pulse(float(tau), float(f0), float(n_cycles), C.byref(im))
    return re, im.value


def np_per_m(alpha_db_cm_mhz, f0):
    return lib().or_np_per_m(float(alpha_db_cm_mhz), float(f0))


def ggx_d(cos_m, alpha):
    """Eq. 12 at n.h = cos_m."""
    return lib().or_ggx_d(float(cos_m), float(alpha))


def ggx_g1(c, alpha):
    return lib().or_ggx_g1(float(c), float(alpha))


def ggx_sample(n, alpha, xi1, xi2):
    nn = np.ascontiguousarray(n, np.float64)
    m = np.zeros(3)
    lib().or_ggx_sample(_dp(nn), float(alpha), float(xi1), float(xi2), _dp(m))
    return m


def rough_eval(d, n, o, alpha, c1, Z1, c2, Z2):
    """(f |o.n| in the amplitude form, solid-angle density of o under the method's sampling)."""
    dd, nn, oo = (np.ascontiguousarray(v, np.float64) for v in (d, n, o))
    pdf = np.zeros(1)
    f = lib().or_rough_eval(_dp(dd), _dp(nn), _dp(oo), float(alpha), float(c1), float(Z1), float(c2), float(Z2),
                            _dp(pdf))
    return f, float(pdf[0])


def connection(scene, array, p, med, x_e):
    """Straight connection ray p -> (x_e, 0, 0): returns (factor, t_samples, atten_np)."""
    s, keep = make_scene(scene)
    a = make_array(array)
    pp = np.ascontiguousarray(p, dtype=np.float64)
    t = C.c_double()
    at = C.c_double()
    f = lib().or_connection(C.byref(s), C.byref(a), _dp(pp), int(med), float(x_e), C.byref(t), C.byref(at))
    del keep
    return f, t.value, at.value


def simulate(scene, array, angles, n_rays, seed, max_bounces, x_px, z_px, dyn_range_db=60.0,
             max_path=0.2, ray_begin=0, ray_end=None, threads=None, transmits=None, mix=False):
    """Whole chain for one frame: trace, deposit, beamform, envelope, log."""
    arr, _, st = trace(scene, array, angles, n_rays, seed, max_bounces, max_path, ray_begin, ray_end,
                       threads=threads, transmits=transmits, mix=mix)
    rf, quad = deposit(array, len(np.atleast_1d(angles)), arr)
    iq = beamform(array, angles, rf, quad, x_px, z_px, threads=threads, transmits=transmits)
    env, db = envelope_log(iq, dyn_range_db)
    return {"arrivals": arr, "stats": st, "rf": rf, "quad": quad, "iq": iq, "env": env, "db": db}
