"""Pins of the isosurface oracle (Sec. 3.4: density field at grid corners, marching cubes).

Against mathematics, not against itself: linear interpolation puts every vertex of a
linear field exactly on its level plane and the mesh of a plane has the plane's area; a
closed level set gives a closed, consistently oriented mesh (every edge in exactly two
triangles, traversed in opposite directions) whose Euler characteristic is 2 for a sphere
and whose enclosed volume is the ball's; the field of one particle is m W(r); the field
integrates to the particles' mass.
"""
from collections import Counter

import numpy as np
import pytest

import oracle
from oracle import iso


def _grid_points(dims, origin, cube):
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (np.asarray(origin, np.float64)[None, None, None, :]
            + cube * np.stack([i, j, k], -1).astype(np.float64))


def _edges_closed(vid):
    """Every undirected mesh edge in exactly two triangles, in opposite directions."""
    directed = Counter()
    for a, b, c in vid:
        for u, v in ((a, b), (b, c), (c, a)):
            directed[(u, v)] += 1
    for (u, v), n in directed.items():
        if n != 1 or directed.get((v, u), 0) != 1:
            return False
    return True


def _normals(t):
    return np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0])


def test_plane_vertices_on_level_and_area():
    dims, cube = (9, 7, 8), 0.1
    origin = np.array([0.05, -0.3, 0.2])
    p = _grid_points(dims, origin, cube)
    z0 = 0.537
    f = z0 - p[..., 2]                    # inside below z0; outward is +z
    t, vid = iso.polygonize(f, origin, cube, 0.0)
    assert np.abs(t[..., 2] - z0).max() < 1e-12
    n = _normals(t)
    assert np.all(n[:, 2] > 0)
    area = 0.5 * np.linalg.norm(n, axis=1).sum()
    assert area == pytest.approx((dims[0] - 1) * (dims[1] - 1) * cube * cube, rel=1e-12)


def test_tilted_plane_vertices_on_level_and_orientation():
    dims, cube = (10, 11, 9), 0.05
    origin = np.zeros(3)
    p = _grid_points(dims, origin, cube)
    nrm = np.array([0.3, -0.5, 0.81])
    nrm /= np.linalg.norm(nrm)
    f = 0.1 - p @ nrm                     # inside where n.x < 0.1; outward is +n
    t, _ = iso.polygonize(f, origin, cube, 0.0)
    assert len(t) > 50
    assert np.abs(t @ nrm - 0.1).max() < 1e-12
    n = _normals(t)
    big = np.linalg.norm(n, axis=1) > 1e-12
    assert np.all(n[big] @ nrm > 0)


def test_sphere_closed_genus_zero_and_volume():
    dims, cube = (24, 24, 24), 0.05
    origin = np.zeros(3)
    p = _grid_points(dims, origin, cube)
    c, R = np.array([0.57, 0.61, 0.55]), 0.4
    f = R - np.linalg.norm(p - c, axis=-1)
    t, vid = iso.polygonize(f, origin, cube, 0.0)
    assert _edges_closed(vid)
    V = len(np.unique(vid))
    E = len({tuple(sorted(e)) for a, b, cc in vid for e in ((a, b), (b, cc), (cc, a))})
    assert V - E + len(vid) == 2
    vol = np.einsum("ij,ij->i", t[:, 0], np.cross(t[:, 1], t[:, 2])).sum() / 6.0
    assert vol == pytest.approx(4.0 / 3.0 * np.pi * R ** 3, rel=0.02)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_fields_give_closed_surfaces(seed):
    # random corner values (every ambiguous face and cube case occurs); the outer layer
    # is outside, so the level set is closed and every mesh edge must pair up
    rng = np.random.default_rng(seed)
    f = rng.uniform(-1.0, 1.0, (10, 11, 12))
    f[0], f[-1], f[:, 0], f[:, -1], f[:, :, 0], f[:, :, -1] = -1, -1, -1, -1, -1, -1
    t, vid = iso.polygonize(f, np.zeros(3), 1.0, 0.0)
    assert len(t) > 500
    assert _edges_closed(vid)


def test_field_of_one_particle_is_m_W():
    h = 0.02
    dims, origin = iso.grid((0.0, 0.0, 0.0), (0.2, 0.2, 0.2), 0.01)
    x = np.array([[0.1037, 0.0962, 0.1011]], np.float32)
    f = iso.field(x, np.array([0.008]), np.array([1]), h, dims, origin, np.float32(0.01))
    # corners at the FP32 value of origin + (i, j, k) cube
    p = _grid_points(dims, origin.astype(np.float64), float(np.float32(0.01)))
    p = p.astype(np.float32).astype(np.float64)
    r = np.linalg.norm(p - x[0].astype(np.float64), axis=-1)
    h32 = float(np.float32(h))                 # the method's h is an FP32 value
    want = np.array([0.008 * oracle.W(v, h32) for v in r.ravel()]).reshape(r.shape)
    np.testing.assert_allclose(f, want, rtol=1e-6, atol=1e-12)
    # boundary (is_fluid = 0) particles do not contribute
    f0 = iso.field(x, np.array([0.008]), np.array([0]), h, dims, origin, np.float32(0.01))
    assert np.all(f0 == 0)


def test_field_integrates_to_the_mass():
    # a Riemann sum of sum_j m_j W over corners a = h / 2 apart equals sum_j m_j (unit integral)
    h, s = 0.02, 0.02
    rng = np.random.default_rng(5)
    n = np.arange(4)
    pts = np.stack(np.meshgrid(n, n, n, indexing="ij"), -1).reshape(-1, 3) * s + 0.17
    x = (pts + rng.uniform(-0.003, 0.003, pts.shape)).astype(np.float32)
    m = np.full(len(x), 1000.0 * s ** 3)
    cube = np.float32(h / 2)
    dims, origin = iso.grid((0.0, 0.0, 0.0), (0.4, 0.4, 0.4), cube)
    f = iso.field(x, m, np.ones(len(x), np.int32), h, dims, origin, cube)
    assert f.sum() * float(cube) ** 3 == pytest.approx(m.sum(), rel=2e-3)
