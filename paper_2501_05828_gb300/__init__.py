"""GB300 (sm_103a) full-path acoustic ray tracer for plane-wave ultrasound.

Python binding of the C ABI in ``include/ultraray.h`` (UltraRay, arXiv
2501.05828, Sec. 2.3): argument marshalling only.  Every step of the
simulation (emission, traversal, transducer sampling, pulse deposit,
beamforming, envelope, log compression) runs in the CUDA library
``_build/libultraray.so``; PyTorch only provides device memory and the stream.
There is no CPU fallback: if the library is missing the import of
:func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libultraray.so")

PLANE_Z, SPHERE, CYL_Y = 0, 1, 2
STATUS = {0: "UR_OK", 1: "UR_ERR_INVALID_ARG", 2: "UR_ERR_CUDA", 3: "UR_ERR_OOM", 4: "UR_ERR_OVERFLOW",
          5: "UR_ERR_TIMEOUT", 6: "UR_ERR_STATE"}

# every entry point include/ultraray.h declares
EXPORTS = ("ur_create", "ur_destroy", "ur_last_error", "ur_scene_upload", "ur_set_array", "ur_set_plane_waves",
           "ur_trace", "ur_trace_debug", "ur_beamform", "ur_set_tuning", "ur_set_profiling", "ur_get_profile",
           "ur_sync", "ur_beamform_noalloc", "ur_scene_upload_slot", "ur_batch_plan", "ur_batch_trace",
           "ur_batch_status", "ur_batch_beamform", "ur_graph_begin", "ur_graph_end", "ur_graph_launch", "ur_autotune",
           "ur_scene_set_media", "ur_scene_set_amplitudes", "ur_trace_adjoint", "ur_nn_create", "ur_nn_destroy",
           "ur_nn_last_error", "ur_nn_param_count", "ur_nn_launch_count", "ur_nn_params", "ur_nn_set_scale", "ur_nn_forward",
           "ur_nn_train_step", "ur_set_transmits", "ur_set_transmit_mixing",
           "ur_scene_set_triangles")
PHASES = ("grid", "trace", "sort", "deposit", "das", "log", "adjoint")


class URError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class Medium(C.Structure):
    _fields_ = [("c", C.c_float), ("Z", C.c_float), ("alpha_db_cm_mhz", C.c_float), ("roughness", C.c_float)]


class Boundary(C.Structure):
    _fields_ = [("kind", C.c_int32), ("med_neg", C.c_int32), ("med_pos", C.c_int32), ("p", C.c_float * 4)]


class Array(C.Structure):
    _fields_ = [("n_el", C.c_int32), ("pitch", C.c_float), ("elev_h", C.c_float), ("f0", C.c_float),
                ("fs", C.c_float), ("n_s", C.c_int32), ("n_cycles", C.c_float), ("alpha_m_deg", C.c_float),
                ("alpha_c_deg", C.c_float), ("c_bf", C.c_float), ("tcut_sigmas", C.c_float), ("radius", C.c_float)]


class Stats(C.Structure):
    _fields_ = [("rays", C.c_uint64), ("segments", C.c_uint64), ("interactions", C.c_uint64),
                ("candidates", C.c_uint64), ("connections", C.c_uint64), ("arrivals", C.c_uint64)]


class Debug(C.Structure):
    _fields_ = [("capacity", C.c_uint64), ("count", C.c_uint64), ("ray", C.c_void_p), ("event", C.c_void_p),
                ("row", C.c_void_p), ("t_hi", C.c_void_p), ("t_lo", C.c_void_p), ("amp", C.c_void_p),
                ("path_hash", C.c_void_p)]


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 8), ("launches", C.c_uint64 * 8), ("calls", C.c_uint64 * 8)]


class BatchItem(C.Structure):
    _fields_ = [("scene", C.c_int32), ("tx", C.c_int32), ("stream", C.c_uint32), ("reserved", C.c_uint32),
                ("n_rays", C.c_uint64)]


TX_PLANE, TX_DIVERGING, TX_FOCUSED, TX_SYNTHETIC = 0, 1, 2, 3


class Transmit(C.Structure):
    _fields_ = [("kind", C.c_int32), ("angle", C.c_float), ("x", C.c_float), ("z", C.c_float)]


class Tuning(C.Structure):
    _fields_ = [("cell_xy", C.c_float), ("cell_z", C.c_float), ("block", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("resolve_batch", C.c_int32), ("cell_y", C.c_float)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError("CUDA library %s not built: run python -m paper_2501_05828_gb300.build" % LIB_PATH)
            L = C.CDLL(LIB_PATH)
            vp, u64, i32, f32 = C.c_void_p, C.c_uint64, C.c_int, C.c_float
            L.ur_create.argtypes = [C.POINTER(vp), i32, vp]
            L.ur_destroy.argtypes = [vp]
            L.ur_last_error.restype = C.c_char_p
            L.ur_last_error.argtypes = [vp]
            L.ur_scene_upload.argtypes = [vp, C.POINTER(Medium), i32, C.POINTER(Boundary), i32, i32, f32, vp, i32, f32]
            L.ur_set_array.argtypes = [vp, C.POINTER(Array)]
            L.ur_set_plane_waves.argtypes = [vp, vp, i32]
            L.ur_set_transmits.argtypes = [vp, C.POINTER(Transmit), i32]
            L.ur_set_transmit_mixing.argtypes = [vp, i32]
            L.ur_scene_set_triangles.argtypes = [vp, i32, vp, vp, i32]
            L.ur_trace.argtypes = [vp, u64, u64, i32, f32, vp, vp, C.POINTER(Stats)]
            L.ur_trace_debug.argtypes = [vp, u64, u64, i32, f32, vp, vp, C.POINTER(Stats), C.POINTER(Debug)]
            L.ur_beamform.argtypes = [vp, vp, vp, vp, i32, vp, i32, f32, vp, vp, vp]
            L.ur_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
            L.ur_sync.argtypes = [vp]
            L.ur_set_profiling.argtypes = [vp, i32]
            L.ur_beamform_noalloc.argtypes = [vp, vp, vp, vp, i32, vp, i32, f32, vp, vp, vp]
            L.ur_scene_upload_slot.argtypes = [vp, i32, C.POINTER(Medium), i32, C.POINTER(Boundary), i32, i32, f32,
                                               vp, i32, f32]
            L.ur_batch_plan.argtypes = [vp, C.POINTER(BatchItem), i32, u64, vp, i32, vp, i32]
            L.ur_batch_trace.argtypes = [vp, u64, i32, f32, vp, vp]
            L.ur_batch_status.argtypes = [vp, C.POINTER(C.c_uint64), C.POINTER(Stats)]
            L.ur_batch_beamform.argtypes = [vp, vp, vp, f32, vp, vp, vp]
            L.ur_graph_begin.argtypes = [vp]
            L.ur_graph_end.argtypes = [vp]
            L.ur_graph_launch.argtypes = [vp]
            L.ur_autotune.argtypes = [vp, i32, u64, u64, i32, f32, C.POINTER(Tuning)]
            L.ur_scene_set_media.argtypes = [vp, i32, C.POINTER(Medium), i32, C.POINTER(Medium)]
            L.ur_scene_set_amplitudes.argtypes = [vp, i32, vp, i32]
            L.ur_trace_adjoint.argtypes = [vp, u64, u64, i32, f32, vp, vp, vp, vp]
            L.ur_nn_create.argtypes = [C.POINTER(vp), i32, vp, i32, i32, i32, i32, u64]
            L.ur_nn_destroy.argtypes = [vp]
            L.ur_nn_last_error.restype = C.c_char_p
            L.ur_nn_last_error.argtypes = [vp]
            L.ur_nn_param_count.argtypes = [vp, C.POINTER(C.c_uint64)]
            L.ur_nn_launch_count.argtypes = [vp, C.POINTER(C.c_uint64)]
            L.ur_nn_params.argtypes = [vp, vp, vp]
            L.ur_nn_set_scale.argtypes = [vp, f32]
            L.ur_nn_forward.argtypes = [vp, vp, vp, i32, vp, vp]
            L.ur_nn_train_step.argtypes = [vp, vp, vp, vp, vp, i32, f32, C.POINTER(C.c_float), vp]
            L.ur_get_profile.argtypes = [vp, C.POINTER(Profile)]
            for name in EXPORTS:
                if name not in ("ur_last_error", "ur_nn_last_error"):
                    getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _ptr(x):
    """Raw address of a torch tensor or numpy array (host or device)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


class Simulator:
    """One library context bound to a CUDA device and stream.

    Inputs may be numpy arrays (host) or torch tensors (host or device);
    outputs are torch CUDA tensors allocated here unless passed in."""

    def __init__(self, device=0, stream=None):
        import torch
        self._torch = torch
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self._ctx = C.c_void_p()
        # torch's default stream has handle 0: hand the library cudaStreamLegacy (1) so that its
        # work stays ordered with torch's instead of going to a private stream
        handle = stream.cuda_stream or 1
        self._call(lib().ur_create(C.byref(self._ctx), int(device), C.c_void_p(handle)), ctx=False)
        self.n_tx = 0
        self.array = None

    def _call(self, code, ctx=True):
        if code != 0:
            msg = lib().ur_last_error(self._ctx).decode() if ctx else ""
            raise URError(code, msg)

    def close(self):
        if self._ctx:
            lib().ur_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up -------------------------------------------------------------
    def upload_scene(self, media, boundaries, med_array, z_max, scatterers, r_s, slot=0):
        med = np.ascontiguousarray(media, np.float32).reshape(-1, 4)
        M = (Medium * len(med))(*[Medium(*map(float, m)) for m in med])
        B = (Boundary * max(1, len(boundaries)))()
        for q, (kind, p, neg, pos) in enumerate(boundaries):
            B[q] = Boundary(int(kind), int(neg), int(pos), (C.c_float * 4)(*[float(v) for v in p]))
        if hasattr(scatterers, "data_ptr"):
            sc, n = scatterers, int(scatterers.shape[0])
        else:
            sc = np.ascontiguousarray(scatterers, np.float32).reshape(-1, 4)
            n = sc.shape[0]
        if slot == 0:
            self._call(lib().ur_scene_upload(self._ctx, M, len(med), B, len(boundaries), int(med_array), float(z_max),
                                             _ptr(sc) if n else None, n, float(r_s)))
        else:
            self._call(lib().ur_scene_upload_slot(self._ctx, int(slot), M, len(med), B, len(boundaries),
                                                  int(med_array), float(z_max), _ptr(sc) if n else None, n,
                                                  float(r_s)))

    def set_array(self, arr):
        self.array = dict(arr)
        a = Array(int(arr["n_el"]), arr["pitch"], arr["elev_h"], arr["f0"], arr["fs"], int(arr["n_s"]),
                  arr["n_cycles"], arr["alpha_m_deg"], arr["alpha_c_deg"], arr["c_bf"], arr["tcut_sigmas"],
                  float(arr.get("radius", 0.0)))
        self._call(lib().ur_set_array(self._ctx, C.byref(a)))

    def set_plane_waves(self, angles_rad):
        a = np.ascontiguousarray(angles_rad, np.float32).reshape(-1)
        self._call(lib().ur_set_plane_waves(self._ctx, _ptr(a), a.size))
        self.n_tx = a.size

    def set_transmits(self, transmits):
        """transmits: sequence of (kind, x, z) with kind TX_DIVERGING / TX_FOCUSED (virtual source /
        focus at (x, z) in metres), (TX_SYNTHETIC, element, 0) or (TX_PLANE, angle_rad, 0)."""
        t = list(transmits)
        arr = (Transmit * len(t))()
        for k, (kind, a, b) in enumerate(t):
            arr[k] = Transmit(int(kind), float(a) if int(kind) == TX_PLANE else 0.0,
                              float(a) if int(kind) != TX_PLANE else 0.0, float(b) if int(kind) != TX_PLANE else 0.0)
        self._call(lib().ur_set_transmits(self._ctx, arr, len(t)))
        self.n_tx = len(t)

    def set_triangles(self, tri, tri_med, slot=0):
        """Triangle-mesh boundaries: tri [n, 9] vertices (m), tri_med [n, 2] (behind, in front)."""
        v = np.ascontiguousarray(tri, np.float32).reshape(-1, 9)
        m = np.ascontiguousarray(tri_med, np.int32).reshape(-1, 2)
        self._call(lib().ur_scene_set_triangles(self._ctx, int(slot), _ptr(v), _ptr(m), v.shape[0]))

    def set_transmit_mixing(self, enabled):
        """True: trace() and trace_debug() trace n_tx * n_rays rays, each drawing its transmit."""
        self._call(lib().ur_set_transmit_mixing(self._ctx, int(bool(enabled))))
        self.mix = bool(enabled)

    def set_tuning(self, cell_xy=0.0, cell_z=0.0, block=0, blocks_per_sm=0, resolve_batch=0, cell_y=0.0):
        """Grid cell sizes along x (cell_xy), y and z in metres, launch shape; 0 keeps a default."""
        t = Tuning(cell_xy, cell_z, block, blocks_per_sm, resolve_batch, cell_y)
        self._call(lib().ur_set_tuning(self._ctx, C.byref(t)))

    def load(self, workload, slot=0):
        """Scene, array and transmits of a phantoms.* workload dictionary."""
        s = workload["scene"]
        self.upload_scene(s["media"], s["boundaries"], s["med_array"], s["z_max"], s["scatterers"], s["r_s"], slot)
        if s.get("triangles") is not None:
            self.set_triangles(s["triangles"][0], s["triangles"][1], slot)
        self.set_array(workload["array"])
        if workload.get("transmits") is not None:
            self.set_transmits(workload["transmits"])
        else:
            self.set_plane_waves(workload["angles"])
        if workload.get("mix") is not None or getattr(self, "mix", False):
            self.set_transmit_mixing(bool(workload.get("mix")))

    # -- simulation ---------------------------------------------------------
    def _channel_shape(self):
        return (self.n_tx, int(self.array["n_el"]), int(self.array["n_s"]))

    def trace(self, n_rays, seed, max_bounces, max_path=0.2, rf=None, quad=None, stats=False):
        torch = self._torch
        shape = self._channel_shape()
        if rf is None:
            rf = torch.empty(shape, dtype=torch.float32, device=self.device)
        if quad is None:
            quad = torch.empty(shape, dtype=torch.float32, device=self.device)
        st = Stats()
        self._call(lib().ur_trace(self._ctx, int(n_rays), int(seed), int(max_bounces), float(max_path),
                                  _ptr(rf), _ptr(quad), C.byref(st)))
        if stats:
            return rf, quad, {f: int(getattr(st, f)) for f, _ in Stats._fields_}
        return rf, quad

    def trace_debug(self, n_rays, seed, max_bounces, max_path=0.2, capacity=None, path_hash=True):
        """Trace plus every arrival record and per-path hashes (device tensors; [n_tx, n_rays], with
        transmit mixing [n_tx * n_rays] indexed by the ray)."""
        torch = self._torch
        shape = self._channel_shape()
        rf = torch.empty(shape, dtype=torch.float32, device=self.device)
        quad = torch.empty(shape, dtype=torch.float32, device=self.device)
        if capacity is None:
            capacity = max(4096, int(n_rays) * self.n_tx)
        dev = self.device
        out = {k: torch.empty(capacity, dtype=torch.int32, device=dev) for k in ("ray", "event", "row")}
        out.update({k: torch.empty(capacity, dtype=torch.float32, device=dev) for k in ("t_hi", "t_lo", "amp")})
        hs = (self.n_tx * int(n_rays),) if getattr(self, "mix", False) else (self.n_tx, int(n_rays))
        ph = torch.empty(hs, dtype=torch.int64, device=dev) if path_hash else None
        dbg = Debug(capacity, 0, _ptr(out["ray"]), _ptr(out["event"]), _ptr(out["row"]), _ptr(out["t_hi"]),
                    _ptr(out["t_lo"]), _ptr(out["amp"]), _ptr(ph))
        st = Stats()
        self._call(lib().ur_trace_debug(self._ctx, int(n_rays), int(seed), int(max_bounces), float(max_path),
                                        _ptr(rf), _ptr(quad), C.byref(st), C.byref(dbg)))
        n = int(dbg.count)
        rec = {k: v[:n] for k, v in out.items()}
        return rf, quad, {f: int(getattr(st, f)) for f, _ in Stats._fields_}, rec, ph

    def beamform(self, rf, quad, x_px, z_px, dyn_range_db=60.0, iq=True, env=True, db=True):
        torch = self._torch
        xp = x_px if hasattr(x_px, "data_ptr") else np.ascontiguousarray(x_px, np.float32)
        zp = z_px if hasattr(z_px, "data_ptr") else np.ascontiguousarray(z_px, np.float32)
        nx, nz = int(xp.shape[0]), int(zp.shape[0])
        dev = self.device
        def out(spec, shape):
            if spec is True:
                return torch.empty(shape, dtype=torch.float32, device=dev)
            return None if spec is None or spec is False else spec

        o_iq, o_env, o_db = out(iq, (nz, nx, 2)), out(env, (nz, nx)), out(db, (nz, nx))
        self._call(lib().ur_beamform(self._ctx, _ptr(rf), _ptr(quad), _ptr(xp), nx, _ptr(zp), nz, float(dyn_range_db),
                                     _ptr(o_iq), _ptr(o_env), _ptr(o_db)))
        return o_iq, o_env, o_db

    def beamform_noalloc(self, rf, quad, x_px, z_px, dyn_range_db=60.0, iq=None, env=None, db=None):
        """ur_beamform_noalloc: outputs are caller-allocated device tensors (or None); nothing is allocated."""
        xp = x_px if hasattr(x_px, "data_ptr") else np.ascontiguousarray(x_px, np.float32)
        zp = z_px if hasattr(z_px, "data_ptr") else np.ascontiguousarray(z_px, np.float32)
        code = lib().ur_beamform_noalloc(self._ctx, _ptr(rf), _ptr(quad), _ptr(xp), int(xp.shape[0]), _ptr(zp),
                                         int(zp.shape[0]), float(dyn_range_db), _ptr(iq), _ptr(env), _ptr(db))
        if code != 0:
            raise URError(code, "ur_beamform_noalloc rejected the call")
        return iq, env, db

    # -- differentiation ----------------------------------------------------
    def set_media(self, media, sampling=None, slot=0):
        med = np.ascontiguousarray(media, np.float32).reshape(-1, 4)
        M = (Medium * len(med))(*[Medium(*map(float, m)) for m in med])
        Ms = None
        if sampling is not None:
            sm = np.ascontiguousarray(sampling, np.float32).reshape(-1, 4)
            Ms = (Medium * len(sm))(*[Medium(*map(float, m)) for m in sm])
        self._call(lib().ur_scene_set_media(self._ctx, int(slot), M, len(med), Ms))

    def set_amplitudes(self, amp, slot=0):
        a = amp if hasattr(amp, "data_ptr") else np.ascontiguousarray(amp, np.float32)
        self._call(lib().ur_scene_set_amplitudes(self._ctx, int(slot), _ptr(a), int(a.shape[0])))

    def trace_adjoint(self, n_rays, seed, max_bounces, g_rf, g_quad, max_path=0.2, n_med=None, n_scat=None):
        """dL/d(c, Z, alpha) per medium [n_med, 3] and dL/d(amplitude) [n_scat] (torch CUDA tensors)."""
        torch = self._torch
        n_med = n_med or 4
        gm = torch.zeros((n_med, 3), dtype=torch.float32, device=self.device)
        ga = torch.zeros((n_scat,), dtype=torch.float32, device=self.device) if n_scat else None
        g_rf, g_quad = g_rf.contiguous(), g_quad.contiguous()
        self._call(lib().ur_trace_adjoint(self._ctx, int(n_rays), int(seed), int(max_bounces), float(max_path),
                                          _ptr(g_rf), _ptr(g_quad), _ptr(gm), _ptr(ga)))
        return gm, ga

    # -- batches, graphs, autotuning ---------------------------------------
    def batch_plan(self, items, x_px, z_px, capacity=0):
        """items: iterable of (scene, tx, n_rays[, stream]); stream defaults to tx."""
        its = list(items)
        arr = (BatchItem * len(its))()
        for q, it in enumerate(its):
            scene, tx, n = it[0], it[1], it[2]
            stream = it[3] if len(it) > 3 else tx
            arr[q] = BatchItem(int(scene), int(tx), int(stream), 0, int(n))
        xp = x_px if hasattr(x_px, "data_ptr") else np.ascontiguousarray(x_px, np.float32)
        zp = z_px if hasattr(z_px, "data_ptr") else np.ascontiguousarray(z_px, np.float32)
        self._call(lib().ur_batch_plan(self._ctx, arr, len(its), int(capacity), _ptr(xp), int(xp.shape[0]), _ptr(zp),
                                       int(zp.shape[0])))
        self.batch_items = its
        self.batch_images = sorted({int(it[0]) for it in its})
        self.batch_grid = (int(zp.shape[0]), int(xp.shape[0]))

    def batch_trace(self, seed, max_bounces, max_path=0.2, rf=None, quad=None):
        torch = self._torch
        shape = (len(self.batch_items), int(self.array["n_el"]), int(self.array["n_s"]))
        rf = torch.empty(shape, dtype=torch.float32, device=self.device) if rf is None else rf
        quad = torch.empty(shape, dtype=torch.float32, device=self.device) if quad is None else quad
        self._call(lib().ur_batch_trace(self._ctx, int(seed), int(max_bounces), float(max_path), _ptr(rf), _ptr(quad)))
        return rf, quad

    def batch_status(self):
        n = C.c_uint64()
        st = Stats()
        self._call(lib().ur_batch_status(self._ctx, C.byref(n), C.byref(st)))
        return int(n.value), {f: int(getattr(st, f)) for f, _ in Stats._fields_}

    def batch_beamform(self, rf, quad, dyn_range_db=60.0, iq=None, env=None, db=True):
        torch = self._torch
        nz, nx = self.batch_grid
        shape = (len(self.batch_images), nz, nx)

        def out(spec, sh):
            if spec is True:
                return torch.empty(sh, dtype=torch.float32, device=self.device)
            return None if spec is None or spec is False else spec

        o_iq, o_env, o_db = out(iq, shape + (2,)), out(env, shape), out(db, shape)
        self._call(lib().ur_batch_beamform(self._ctx, _ptr(rf), _ptr(quad), float(dyn_range_db), _ptr(o_iq),
                                           _ptr(o_env), _ptr(o_db)))
        return o_iq, o_env, o_db

    def graph_begin(self):
        self._call(lib().ur_graph_begin(self._ctx))

    def graph_end(self):
        self._call(lib().ur_graph_end(self._ctx))

    def graph_launch(self):
        self._call(lib().ur_graph_launch(self._ctx))

    def autotune(self, n_rays, seed=0, max_bounces=8, max_path=0.2, scene=0):
        t = Tuning()
        self._call(lib().ur_autotune(self._ctx, int(scene), int(n_rays), int(seed), int(max_bounces), float(max_path),
                                     C.byref(t)))
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def set_profiling(self, on=True):
        self._call(lib().ur_set_profiling(self._ctx, 1 if on else 0))

    def profile(self):
        """{phase: (device ms, kernel launches, calls)} accumulated while profiling."""
        p = Profile()
        self._call(lib().ur_get_profile(self._ctx, C.byref(p)))
        return {name: (p.ms[q], int(p.launches[q]), int(p.calls[q])) for q, name in enumerate(PHASES)}

    def sync(self):
        self._call(lib().ur_sync(self._ctx))


def build_library(force=False):
    """Compile the CUDA library in-tree (see build.py)."""
    from .build import build as _build
    return _build(force=force)


def _trace_function():
    import torch

    class TraceFunction(torch.autograd.Function):
        """Differentiable ur_trace on scene slot 0: (media [n_med, 4] = c, Z, alpha, roughness;
        scatterer amplitudes [n_scat]) -> (rf, quad).  Backward calls the path-replay adjoint
        (ur_trace_adjoint); roughness gets no gradient."""

        @staticmethod
        def forward(ctx, media, amplitudes, sim, n_rays, seed, max_bounces, max_path):
            sim.set_media(media.detach().cpu().numpy())
            sim.set_amplitudes(amplitudes.detach().to(sim.device, torch.float32).contiguous())
            rf, quad = sim.trace(n_rays, seed, max_bounces, max_path)
            ctx.sim, ctx.cfg = sim, (n_rays, seed, max_bounces, max_path)
            ctx.shapes = (media.shape, amplitudes.shape[0], media.device, amplitudes.device)
            return rf, quad

        @staticmethod
        def backward(ctx, g_rf, g_quad):
            n_rays, seed, max_bounces, max_path = ctx.cfg
            mshape, n_scat, mdev, adev = ctx.shapes
            if g_rf is None:
                g_rf = torch.zeros_like(g_quad)
            if g_quad is None:
                g_quad = torch.zeros_like(g_rf)
            gm, ga = ctx.sim.trace_adjoint(n_rays, seed, max_bounces, g_rf, g_quad, max_path, n_med=mshape[0],
                                           n_scat=n_scat)
            grad_media = torch.zeros(mshape, dtype=torch.float32, device=mdev)
            grad_media[:, :3] = gm.to(mdev)
            return grad_media, ga.to(adev), None, None, None, None, None

    return TraceFunction


def trace_differentiable(sim, media, amplitudes, n_rays, seed, max_bounces, max_path=0.2):
    """rf, quad = ur_trace with autograd support for media and scatterer amplitudes."""
    return _trace_function().apply(media, amplitudes, sim, n_rays, seed, max_bounces, max_path)


NN_LAYERS = ("e1a", "e1b", "e2a", "e2b", "e3a", "e3b", "e4a", "e4b", "d3a", "d3b", "d2a", "d2b", "d1a", "d1b")


def nn_layout(width=32):
    """Offsets of the packed parameter vector documented in ultraray.h:
    {name: (w_offset, (9, c_out, c_in), b_offset, c_out)} plus ('head': ...)."""
    C = width
    cin = (32, C, C, 2 * C, 2 * C, 4 * C, 4 * C, 8 * C, 12 * C, 4 * C, 6 * C, 2 * C, 3 * C, C)
    cout = (C, C, 2 * C, 2 * C, 4 * C, 4 * C, 8 * C, 8 * C, 4 * C, 4 * C, 2 * C, 2 * C, C, C)
    lay, off = {}, 0
    for name, ci, co in zip(NN_LAYERS, cin, cout):
        w_off = off
        off += 9 * ci * co
        b_off = off
        off += co
        off = (off + 7) // 8 * 8
        lay[name] = (w_off, (9, co, ci), b_off, co)
    lay["head"] = (off, (1, 2, C), off + 2 * C, 2)
    return lay


class Denoiser:
    """The library's U-Net denoiser of channel data (ur_nn_* entry points)."""

    def __init__(self, device=0, max_batch=4, n_el=128, n_s=3200, width=32, seed=0, stream=None):
        import torch
        self._torch = torch
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self._h = C.c_void_p()
        code = lib().ur_nn_create(C.byref(self._h), int(device), C.c_void_p(stream.cuda_stream or 1), int(max_batch),
                                  int(n_el), int(n_s), int(width), int(seed))
        if code != 0:
            raise URError(code, "ur_nn_create failed")
        n = C.c_uint64()
        lib().ur_nn_param_count(self._h, C.byref(n))
        self.n_params = int(n.value)
        self.shape = (int(n_el), int(n_s))
        self.width = width

    def launch_count(self):
        """Kernels the network has enqueued since creation."""
        n = C.c_uint64()
        self._call(lib().ur_nn_launch_count(self._h, C.byref(n)))
        return int(n.value)

    def _call(self, code):
        if code != 0:
            raise URError(code, lib().ur_nn_last_error(self._h).decode())

    def close(self):
        if self._h:
            lib().ur_nn_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.zeros(self.n_params, np.float32)
        self._call(lib().ur_nn_params(self._h, _ptr(out), None))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.n_params
        self._call(lib().ur_nn_params(self._h, None, _ptr(p)))

    def set_scale(self, scale):
        self._call(lib().ur_nn_set_scale(self._h, float(scale)))

    def forward(self, rf, quad):
        torch = self._torch
        rf, quad = rf.contiguous(), quad.contiguous()
        o_rf, o_q = torch.empty_like(rf), torch.empty_like(quad)
        self._call(lib().ur_nn_forward(self._h, _ptr(rf), _ptr(quad), int(rf.shape[0]), _ptr(o_rf), _ptr(o_q)))
        return o_rf, o_q

    def train_step(self, rf, quad, t_rf, t_quad, lr, grad=False):
        torch = self._torch
        rf, quad, t_rf, t_quad = (t.contiguous() for t in (rf, quad, t_rf, t_quad))
        loss = C.c_float()
        g = torch.empty(self.n_params, dtype=torch.float32, device=self.device) if grad else None
        self._call(lib().ur_nn_train_step(self._h, _ptr(rf), _ptr(quad), _ptr(t_rf), _ptr(t_quad), int(rf.shape[0]),
                                          float(lr), C.byref(loss), _ptr(g)))
        return (float(loss.value), g) if grad else float(loss.value)
