"""Seeded synthetic workloads for the UltraRay hot path.

Inputs only: media tables, analytic boundaries, scatterer clouds, array and
imaging-grid parameters, drawn with numpy from a seed.  None of the method's
arithmetic (delays, Fresnel, pulse, beamforming) lives here, so both the CUDA
library and the CPU oracle can be fed from it.  The paper's own scenes (a
CT-derived spine mesh, Sec. 4) are not available; these phantoms follow the
sizes and tissue parameters of the workloads the library is measured on.

All geometric quantities are in metres, sound speeds in m/s, impedances in
MRayl, attenuation in dB/cm/MHz.  Every array handed out is float32: the exact
values both implementations consume.
"""
from __future__ import annotations

import numpy as np

PLANE_Z, SPHERE, CYL_Y = 0, 1, 2

WATER = (1480.0, 1.48, 0.0, 0.0)
MUSCLE = (1580.0, 1.70, 1.0, 0.0)
BONE = (3500.0, 7.8, 10.0, 0.0)
SKIN = (1615.0, 1.99, 0.0, 0.0)
FAT = (1450.0, 1.38, 0.6, 0.0)


def array_params(n_el, n_s, pitch=0.3e-3, elev_h=4e-3, f0=5e6, fs=40e6, n_cycles=5.0,
                 alpha_m_deg=2.0, alpha_c_deg=2.0, c_bf=1540.0, tcut_sigmas=5.0):
    """Linear array: n_el elements of width `pitch` (no kerf), elevation height elev_h."""
    return {"n_el": int(n_el), "pitch": float(np.float32(pitch)), "elev_h": float(np.float32(elev_h)),
            "f0": float(np.float32(f0)), "fs": float(np.float32(fs)), "n_s": int(n_s),
            "n_cycles": float(np.float32(n_cycles)), "alpha_m_deg": float(np.float32(alpha_m_deg)),
            "alpha_c_deg": float(np.float32(alpha_c_deg)), "c_bf": float(np.float32(c_bf)),
            "tcut_sigmas": float(np.float32(tcut_sigmas))}


def image_grid(array, nx, nz, z0=1e-3, z1=None):
    """Pixel coordinates: x spans the element centres, z from z0 to the depth of the last sample."""
    half = 0.5 * (array["n_el"] - 1) * array["pitch"]
    if z1 is None:
        z1 = array["c_bf"] * array["n_s"] / (2.0 * array["fs"])
    x = np.linspace(-half, half, nx).astype(np.float32)
    z = np.linspace(z0, z1, nz).astype(np.float32)
    return x, z


def uniform_scatterers(rng, n, box):
    """n points uniform in box = ((x0, x1), (y0, y1), (z0, z1)) with N(0, 1) amplitudes."""
    (x0, x1), (y0, y1), (z0, z1) = box
    s = np.empty((n, 4), np.float64)
    s[:, 0] = rng.uniform(x0, x1, n)
    s[:, 1] = rng.uniform(y0, y1, n)
    s[:, 2] = rng.uniform(z0, z1, n)
    s[:, 3] = rng.standard_normal(n)
    return s.astype(np.float32)


def _scene(media, boundaries, med_array, z_max, scatterers, r_s):
    return {"media": np.asarray(media, np.float32).reshape(-1, 4),
            "boundaries": [(int(k), [float(np.float32(v)) for v in p], int(a), int(b))
                           for k, p, a, b in boundaries],
            "med_array": int(med_array), "z_max": float(np.float32(z_max)),
            "scatterers": np.asarray(scatterers, np.float32).reshape(-1, 4),
            "r_s": float(np.float32(r_s))}


def tiny(seed=0, n_scat=200, with_sphere=True, n_rays=100_000):
    """32-element array, water over muscle (interface at 15 mm), bone sphere r = 3 mm
    centred at 25 mm, 200 scatterers in x,y,z = [-10,10] x [-2.5,2.5] x [5,25] mm;
    one 0-degree plane wave, 1536 samples, 4 bounces, 128 x 256 image."""
    rng = np.random.default_rng(seed)
    media = [WATER, MUSCLE, BONE]
    bnd = [(PLANE_Z, [0.015, 0, 0, 0], 0, 1)]
    if with_sphere:
        bnd.append((SPHERE, [0.0, 0.0, 0.025, 0.003], 2, 1))
    sc = uniform_scatterers(rng, n_scat, ((-10e-3, 10e-3), (-2.5e-3, 2.5e-3), (5e-3, 25e-3)))
    arr = array_params(32, 1536, c_bf=1480.0)
    x, z = image_grid(arr, 128, 256)
    return {"name": "tiny", "scene": _scene(media, bnd, 0, 0.040, sc, 1e-4), "array": arr,
            "angles": np.zeros(1, np.float32), "n_rays": int(n_rays), "seed": 0, "max_bounces": 4,
            "max_path": 0.2, "x_px": x, "z_px": z, "dyn_range_db": 60.0}


def layered(seed=0, n_scat=50_000, n_rays=10_000_000, angles_deg=(0.0,), z_skin=2e-3, z_fat=10e-3,
            bone_r=6e-3, bone_z=30e-3):
    """128-element array; skin 0-2 mm, fat 2-10 mm, muscle 10-60 mm; bone cylinder
    r = 6 mm along elevation at 30 mm depth; 50k scatterers over
    x,y,z = [-19,19] x [-2.5,2.5] x [0,60] mm; 3200 samples, 8 bounces, 512 x 256 image."""
    rng = np.random.default_rng(seed)
    media = [SKIN, FAT, MUSCLE, BONE]
    bnd = [(PLANE_Z, [z_skin, 0, 0, 0], 0, 1),
           (PLANE_Z, [z_fat, 0, 0, 0], 1, 2),
           (CYL_Y, [0.0, bone_z, bone_r, 0], 3, 2)]
    sc = uniform_scatterers(rng, n_scat, ((-19e-3, 19e-3), (-2.5e-3, 2.5e-3), (0.0, 60e-3)))
    arr = array_params(128, 3200, c_bf=1540.0)
    x, z = image_grid(arr, 512, 256)
    ang = np.deg2rad(np.asarray(angles_deg, np.float64)).astype(np.float32)
    return {"name": "layered", "scene": _scene(media, bnd, 0, 0.060, sc, 1e-4), "array": arr,
            "angles": ang, "n_rays": int(n_rays), "seed": 0, "max_bounces": 8, "max_path": 0.2,
            "x_px": x, "z_px": z, "dyn_range_db": 60.0}


def batched_variant(scene_seed):
    """One jittered layered phantom of the batched workload: layer depths +/- 2 mm,
    bone radius U(3, 10) mm, scatterer count U{10k..200k}, rays per transmit
    log-uniform in [1e6, 3e7], 31 plane waves from -15 to +15 degrees."""
    rng = np.random.default_rng(1000 + int(scene_seed))
    z_skin = 2e-3 + rng.uniform(-2e-3, 2e-3) * 0.5      # keep the skin layer non-empty
    z_fat = 10e-3 + rng.uniform(-2e-3, 2e-3)
    bone_r = rng.uniform(3e-3, 10e-3)
    n_scat = int(rng.integers(10_000, 200_001))
    n_rays = int(np.exp(rng.uniform(np.log(1e6), np.log(3e7))))
    w = layered(seed=int(scene_seed), n_scat=n_scat, n_rays=n_rays,
                angles_deg=tuple(float(a) for a in range(-15, 16)),
                z_skin=z_skin, z_fat=z_fat, bone_r=bone_r)
    w["name"] = "batched-%d" % scene_seed
    return w


def paper_like(seed=0, n_scat=20_000, n_rays=512_000, convex=False):
    """The acquisition of the paper's experiments (Sec. 4) on a synthetic bone-surface stand-in
    (the CT spine mesh is not available): 128 elements, 5 MHz, fs 50 MHz, 5 cycles, 4 mm
    elevation, directivity 2 degrees, 25 plane waves over [-30, 30] degrees, 10 bounces, 20 cm
    paths, 90 dB.  Water (c 1540, Z 1.54) around bone (c 3500, Z 7.8, 10 dB/cm/MHz, GGX roughness
    0.5): a vertebral body (sphere r = 10 mm at 45 mm depth) and two processes (cylinders along
    elevation, r = 3 mm, at x = +-12 mm, 28 mm depth); n_scat scatterers uniform inside the bone,
    none in the water.  n_rays per transmit (25 x 512k = 12.8M rays per acquisition, the paper's
    128 elements x 100k rays).  convex: the paper's probe geometry, 128 elements over a 70-degree
    arc of radius 50 mm (arc pitch 0.477 mm), instead of a linear array with 0.3 mm pitch."""
    rng = np.random.default_rng(seed)
    water = (1540.0, 1.54, 0.0, 0.0)
    bone = (3500.0, 7.8, 10.0, 0.5)
    body = (0.0, 0.0, 45e-3, 10e-3)
    procs = ((-12e-3, 28e-3, 3e-3), (12e-3, 28e-3, 3e-3))
    bnd = [(SPHERE, list(body), 1, 0)] + [(CYL_Y, [x, z, r, 0.0], 1, 0) for x, z, r in procs]
    pts = []
    while sum(len(p) for p in pts) < n_scat:   # rejection sampling inside the bone primitives
        q = np.column_stack([rng.uniform(-15e-3, 15e-3, 4 * n_scat), rng.uniform(-10e-3, 10e-3, 4 * n_scat),
                             rng.uniform(25e-3, 55e-3, 4 * n_scat)])
        inside = np.sum((q - np.array(body[:3])) ** 2, axis=1) < body[3] ** 2
        for x, z, r in procs:
            inside |= (q[:, 0] - x) ** 2 + (q[:, 2] - z) ** 2 < r * r
        pts.append(q[inside])
    xyz = np.concatenate(pts)[:n_scat]
    sc = np.column_stack([xyz, rng.standard_normal(n_scat)]).astype(np.float32)
    if convex:
        radius = 0.05
        arr = array_params(128, 4096, pitch=np.deg2rad(70.0) * radius / 128, fs=50e6, c_bf=1540.0,
                           alpha_m_deg=2.0, alpha_c_deg=2.0)
        arr["radius"] = float(np.float32(radius))
    else:
        arr = array_params(128, 4096, fs=50e6, c_bf=1540.0, alpha_m_deg=2.0, alpha_c_deg=2.0)
    x, z = image_grid(arr, 512, 256, z0=1e-3, z1=60e-3)
    ang = np.deg2rad(np.linspace(-30.0, 30.0, 25)).astype(np.float32)
    return {"name": "paper_like", "scene": _scene([water, bone], bnd, 0, 0.080, sc, 1e-4), "array": arr,
            "angles": ang, "n_rays": int(n_rays), "seed": 0, "max_bounces": 10, "max_path": 0.2,
            "x_px": x, "z_px": z, "dyn_range_db": 90.0}


def single_plane(depth=0.015, upper=WATER, lower=MUSCLE, n_el=32, n_s=1536, n_rays=3200,
                 z_max=0.040, c_bf=1480.0, **arr_kw):
    """One planar interface, no scatterers (normal-incidence echo checks)."""
    arr = array_params(n_el, n_s, c_bf=c_bf, **arr_kw)
    sc = _scene([upper, lower], [(PLANE_Z, [depth, 0, 0, 0], 0, 1)], 0, z_max,
                np.zeros((0, 4), np.float32), 1e-4)
    return {"name": "plane", "scene": sc, "array": arr, "angles": np.zeros(1, np.float32),
            "n_rays": int(n_rays), "seed": 0, "max_bounces": 4, "max_path": 0.2}


def single_scatterer(pos, amp=1.0, medium=WATER, n_el=32, n_s=1536, n_rays=1_000_000,
                     r_s=1e-4, z_max=0.040, c_bf=1480.0, **arr_kw):
    """One point scatterer in a homogeneous medium."""
    arr = array_params(n_el, n_s, c_bf=c_bf, **arr_kw)
    sc = _scene([medium], [], 0, z_max, np.asarray([[pos[0], pos[1], pos[2], amp]], np.float32), r_s)
    return {"name": "scatterer", "scene": sc, "array": arr, "angles": np.zeros(1, np.float32),
            "n_rays": int(n_rays), "seed": 0, "max_bounces": 4, "max_path": 0.2}


# ------------------------------------------------------------------ triangle meshes
# Triangles are [n, 9] float32 vertex triples (v0, v1, v2) wound so that
# (v1 - v0) x (v2 - v0) points out of the enclosed region; with them goes an
# [n, 2] int32 table of (medium inside / behind, medium outside / in front).

def _outward(tris, inner):
    """Reorder each triangle's vertices so that its normal points away from inner(centroid)."""
    t = tris.reshape(-1, 3, 3).copy()
    n = np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0])
    c = t.mean(axis=1)
    flip = np.einsum("ij,ij->i", n, c - inner(c)) < 0
    t[flip, 1], t[flip, 2] = t[flip, 2].copy(), t[flip, 1].copy()
    return t.reshape(-1, 9)


def mesh_quad(z, x0, x1, y0, y1):
    """Rectangle z = const over [x0, x1] x [y0, y1] as two triangles, normal +z."""
    t = np.array([[x0, y0, z, x1, y0, z, x1, y1, z], [x0, y0, z, x1, y1, z, x0, y1, z]], np.float64)
    return t.astype(np.float32)


def mesh_tilted_quad(p0, beta, half_x, half_y):
    """Rectangle through p0 = (x, z) with unit normal (sin beta, 0, cos beta), 2 half_x along the
    tilted x direction and 2 half_y along y, as two triangles facing the normal."""
    u = np.array([np.cos(beta), 0.0, -np.sin(beta)]) * half_x
    v = np.array([0.0, half_y, 0.0])
    c = np.array([p0[0], 0.0, p0[1]])
    a, b, cc, d = c - u - v, c + u - v, c + u + v, c - u + v
    t = np.array([np.concatenate([a, b, cc]), np.concatenate([a, cc, d])])
    n = np.cross(t[:, 3:6] - t[:, 0:3], t[:, 6:9] - t[:, 0:3])
    want = np.array([np.sin(beta), 0.0, np.cos(beta)])
    flip = n @ want < 0
    t[flip, 3:6], t[flip, 6:9] = t[flip, 6:9].copy(), t[flip, 3:6].copy()
    return t.astype(np.float32)


def mesh_box(lo, hi):
    """Closed axis-aligned box, 12 triangles, outward normals."""
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    corner = lambda i: np.where([(i >> 0) & 1, (i >> 1) & 1, (i >> 2) & 1], hi, lo)
    faces = [(0, 1, 3, 2), (4, 5, 7, 6), (0, 1, 5, 4), (2, 3, 7, 6), (0, 2, 6, 4), (1, 3, 7, 5)]
    t = []
    for a, b, c, d in faces:
        t.append(np.concatenate([corner(a), corner(b), corner(c)]))
        t.append(np.concatenate([corner(a), corner(c), corner(d)]))
    mid = 0.5 * (lo + hi)
    return _outward(np.array(t), lambda c: mid).astype(np.float32)


def mesh_icosphere(centre, radius, subdiv):
    """Sphere approximated by a subdivided icosahedron (20 * 4^subdiv triangles, vertices on the
    sphere), outward normals."""
    g = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, g, 0), (1, g, 0), (-1, -g, 0), (1, -g, 0), (0, -1, g), (0, 1, g), (0, -1, -g), (0, 1, -g),
         (g, 0, -1), (g, 0, 1), (-g, 0, -1), (-g, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    for _ in range(subdiv):
        cache, nf = {}, []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    P = np.array(verts) * radius + np.asarray(centre, np.float64)
    t = np.array([np.concatenate([P[a], P[b], P[c]]) for a, b, c in f])
    ctr = np.asarray(centre, np.float64)
    return _outward(t, lambda c: ctr).astype(np.float32)


def mesh_cylinder_y(x, z, r, y0, y1, n_seg):
    """Closed prism with n_seg sides about the axis through (x, z) along y from y0 to y1 (vertices
    on the circle of radius r), with end caps; outward normals."""
    a = np.linspace(0.0, 2 * np.pi, n_seg, endpoint=False)
    ring = np.column_stack([x + r * np.cos(a), np.zeros(n_seg), z + r * np.sin(a)])
    t = []
    for i in range(n_seg):
        j = (i + 1) % n_seg
        p, q = ring[i], ring[j]
        lo_p, lo_q, hi_p, hi_q = p + [0, y0, 0], q + [0, y0, 0], p + [0, y1, 0], q + [0, y1, 0]
        t += [np.concatenate([lo_p, lo_q, hi_q]), np.concatenate([lo_p, hi_q, hi_p])]
        for yy in (y0, y1):
            t.append(np.concatenate([[x, yy, z], p + [0, yy, 0], q + [0, yy, 0]]))
    axis = lambda c: np.column_stack([np.full(len(c), x), c[:, 1], np.full(len(c), z)])
    tt = np.array(t)
    n = np.cross(tt[:, 3:6] - tt[:, 0:3], tt[:, 6:9] - tt[:, 0:3])
    cen = tt.reshape(-1, 3, 3).mean(axis=1)
    cap = np.abs(n[:, 1]) > 0.5 * np.linalg.norm(n, axis=1)
    out = np.where(cap[:, None], np.column_stack([np.zeros(len(cen)), cen[:, 1] - 0.5 * (y0 + y1),
                                                  np.zeros(len(cen))]), cen - axis(cen))
    flip = np.einsum("ij,ij->i", n, out) < 0
    tt[flip, 3:6], tt[flip, 6:9] = tt[flip, 6:9].copy(), tt[flip, 3:6].copy()
    return tt.astype(np.float32)


def triangles(*parts):
    """Concatenate (triangles, inside medium, outside medium) parts into a scene's mesh entry."""
    tri = np.concatenate([p[0] for p in parts]).astype(np.float32)
    med = np.concatenate([np.tile(np.array([[p[1], p[2]]], np.int32), (len(p[0]), 1)) for p in parts])
    return tri, med


def paper_mesh_like(seed=0, n_scat=20_000, n_rays=512_000, subdiv=4, n_seg=96):
    """paper_like with the bone as triangle meshes, as the paper's CT-derived bone is: the vertebral
    body an icosphere (20 * 4^subdiv triangles, 5120 by default), the processes closed prisms along
    elevation (n_seg sides, y in [-15, 15] mm); same acquisition, media and scatterers."""
    w = paper_like(seed=seed, n_scat=n_scat, n_rays=n_rays)
    body = mesh_icosphere((0.0, 0.0, 45e-3), 10e-3, subdiv)
    procs = [mesh_cylinder_y(x, 28e-3, 3e-3, -15e-3, 15e-3, n_seg) for x in (-12e-3, 12e-3)]
    s = dict(w["scene"])
    s["boundaries"] = []
    s["triangles"] = triangles((body, 1, 0), *[(p, 1, 0) for p in procs])
    w["scene"] = s
    w["name"] = "paper_mesh_like"
    return w
