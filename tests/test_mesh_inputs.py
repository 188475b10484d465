"""The triangle-mesh inputs are what the mesh tests assume: closed surfaces (every
edge shared by exactly two triangles, traversed in opposite directions), normals
(v1 - v0) x (v2 - v0) pointing out of the enclosed region (positive enclosed
volume by the divergence theorem), vertices of the icosphere on its sphere."""
import numpy as np
import pytest

import phantoms


def edges_closed(tri):
    t = tri.reshape(-1, 3, 3).astype(np.float64)
    key = lambda p: tuple(np.round(p, 12))
    directed = {}
    for a, b, c in t:
        for u, v in ((a, b), (b, c), (c, a)):
            k = (key(u), key(v))
            directed[k] = directed.get(k, 0) + 1
    # each directed edge once, and its reverse once
    return all(n == 1 and directed.get((v, u), 0) == 1 for (u, v), n in directed.items())


def enclosed_volume(tri):
    t = tri.reshape(-1, 3, 3).astype(np.float64)
    return np.einsum("ij,ij->i", t[:, 0], np.cross(t[:, 1], t[:, 2])).sum() / 6.0


@pytest.mark.parametrize("make,volume", [
    (lambda: phantoms.mesh_box((-1.0, -2.0, 0.5), (2.0, 1.0, 1.5)), 3.0 * 3.0 * 1.0),
    (lambda: phantoms.mesh_icosphere((0.1, -0.2, 0.3), 2.0, 3), 4.0 / 3.0 * np.pi * 8.0),
    (lambda: phantoms.mesh_cylinder_y(0.5, 1.0, 1.5, -2.0, 3.0, 64), np.pi * 2.25 * 5.0),
])
def test_closed_and_outward(make, volume):
    tri = make()
    assert tri.dtype == np.float32 and tri.shape[1] == 9
    assert edges_closed(tri)
    v = enclosed_volume(tri)
    assert v > 0                                        # outward normals
    assert abs(v - volume) < 0.03 * volume              # faceting: within 3 % of the smooth solid


def test_icosphere_vertices_on_the_sphere():
    c, r = np.array([1e-3, 0.0, 20e-3]), 4e-3
    tri = phantoms.mesh_icosphere(c, r, 3).reshape(-1, 3).astype(np.float64)
    assert len(tri) == 3 * 20 * 4 ** 3
    np.testing.assert_allclose(np.linalg.norm(tri - c, axis=1), r, rtol=1e-6)


def test_quads_face_their_normal():
    q = phantoms.mesh_quad(0.01, -0.02, 0.02, -0.01, 0.01).reshape(-1, 3, 3).astype(np.float64)
    n = np.cross(q[:, 1] - q[:, 0], q[:, 2] - q[:, 0])
    assert np.all(n[:, 2] > 0) and np.allclose(n[:, :2], 0)
    for beta in (0.0, 0.3, -0.5):
        t = phantoms.mesh_tilted_quad((0.0, 0.01), beta, 0.02, 0.02).reshape(-1, 3, 3).astype(np.float64)
        n = np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0])
        n /= np.linalg.norm(n, axis=1)[:, None]
        np.testing.assert_allclose(n, np.tile([np.sin(beta), 0.0, np.cos(beta)], (2, 1)), atol=1e-6)
