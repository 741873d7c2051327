"""Pins of the envelope / initialisation / voxel oracle against closed forms,
brute force and independent formulations (CPU only)."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import envelope as E


def cube_points(s=4.0, n_inner=50, seed=0):
    rng = np.random.default_rng(seed)
    corners = np.array(list(itertools.product([0.0, s], repeat=3)))
    inner = rng.uniform(0.5, s - 0.5, size=(n_inner, 3))
    return np.vstack([inner[:10], corners, inner[10:]])


def fibonacci_sphere(n, r=10.0):
    k = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * k / n)
    th = np.pi * (1 + 5 ** 0.5) * k
    return r * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)


def test_hull_of_cube_is_the_cube():
    P = cube_points()
    V, T = E.envelope_mesh(P)
    assert T.shape == (12, 3)
    assert E.mesh_volume(V, T) == pytest.approx(64.0, rel=1e-13)
    assert set(np.unique(T)) == set(range(10, 18))  # the corners only


def test_hull_of_sphere_points():
    P = fibonacci_sphere(400)
    V, T = E.envelope_mesh(P)
    assert len(np.unique(T)) == 400  # every point is on the hull
    assert T.shape[0] == 2 * 400 - 4  # Euler: closed triangulated sphere
    vol = E.mesh_volume(V, T)
    assert 0.98 * 4 / 3 * np.pi * 1000 < vol < 4 / 3 * np.pi * 1000


def test_ray_parity_matches_half_spaces():
    from scipy.spatial import ConvexHull

    P = np.random.default_rng(1).normal(size=(60, 3)) * [3.0, 2.0, 1.0]
    V, T = E.envelope_mesh(P)
    eq = ConvexHull(P).equations
    rng = np.random.default_rng(2)
    X = rng.uniform(P.min(0) - 0.5, P.max(0) + 0.5, size=(300, 3))
    for x in X:
        s = eq[:, :3] @ x + eq[:, 3]
        if np.min(np.abs(s)) < 1e-9:
            continue
        assert (E.ray_crossings(V, T, x) % 2 == 1) == bool(np.all(s < 0))


def test_distance_inside_convex_is_nearest_plane():
    from scipy.spatial import ConvexHull

    P = np.random.default_rng(3).normal(size=(40, 3))
    V, T = E.envelope_mesh(P)
    eq = ConvexHull(P).equations
    X = np.random.default_rng(4).normal(size=(80, 3)) * 0.3
    for x in X:
        s = eq[:, :3] @ x + eq[:, 3]
        if np.any(s >= 0):
            continue
        assert E.point_triangle_distance(V, T, x) == pytest.approx(-np.max(s), rel=1e-12)


def test_distance_outside_cube_closed_forms():
    V, T = E.envelope_mesh(cube_points())
    assert E.point_triangle_distance(V, T, [2.0, 2.0, 7.0]) == pytest.approx(3.0)  # face
    assert E.point_triangle_distance(V, T, [5.0, 5.0, 2.0]) == pytest.approx(2 ** 0.5)  # edge
    assert E.point_triangle_distance(V, T, [5.0, 6.0, 7.0]) == pytest.approx(
        np.sqrt(1 + 4 + 9))  # corner


def test_unit_double_from_golden_splitmix():
    with open("tests/golden/splitmix64_seed1234567.txt") as f:
        vals = [int(line.split()[-1], 0) for line in f if line.strip() and not line.startswith("#")]
    for k, v in enumerate(vals[:5]):
        assert E.unit_double(1234567, k) == (v >> 11) / 2.0 ** 53


def test_sampling_is_uniform_in_the_inset_cube():
    V, T = E.envelope_mesh(cube_points(s=4.0))
    n_cand, inset = 1200, 0.5
    balls, idx = E.sample_cloud(V, T, 10 ** 6, seed=7, inset=inset, first=0,
                                n_candidates=n_cand)
    p = (3.0 / 4.0) ** 3  # (s - 2 inset)^3 / s^3
    sd = np.sqrt(n_cand * p * (1 - p))
    assert abs(len(idx) - n_cand * p) < 4 * sd
    c = balls[:3].astype(np.float64)
    assert np.all(c >= 0.5) and np.all(c <= 3.5)
    assert np.all(np.abs(c.mean(1) - 2.0) < 4 * np.sqrt(0.75 / len(idx)))  # U(0.5,3.5): var 0.75
    assert np.all((balls[3] >= 0.05) & (balls[3] <= 0.2))
    assert np.all((balls[4] >= 0.0) & (balls[4] <= 1.0))


def test_sampling_is_a_function_of_the_candidate_index():
    V, T = E.envelope_mesh(cube_points())
    a, ia = E.sample_cloud(V, T, 10 ** 6, seed=9, inset=0.2, first=0, n_candidates=200)
    b, ib = E.sample_cloud(V, T, 10 ** 6, seed=9, inset=0.2, first=100, n_candidates=100)
    keep = ia >= 100
    np.testing.assert_array_equal(ia[keep], ib)
    np.testing.assert_array_equal(a[:, keep], b)
    c, ic = E.sample_cloud(V, T, 5, seed=9, inset=0.2, first=0, n_candidates=200)
    np.testing.assert_array_equal(ic, ia[:5])


def test_voxelize_lattice_counts():
    dims = (9, 9, 9)
    h = 0.1
    origin = (0.0, 0.0, 0.0)
    centre = 4.5 * h  # the centre of voxel (4, 4, 4)
    for R, count in ((1.01 * h, 7), (1.5 * h, 19), (0.5 * h, 1)):
        b = np.array([[centre], [centre], [centre], [R], [2.0]], dtype=np.float64)
        vol = E.voxelize(b, origin, h, dims)
        assert np.count_nonzero(vol) == count
        assert vol.sum() == pytest.approx(2.0 * count)


def test_voxelize_brute_force_and_linearity():
    rng = np.random.default_rng(5)
    n = 12
    b = np.stack([rng.uniform(0.1, 1.1, n), rng.uniform(0.1, 0.9, n), rng.uniform(0.2, 0.7, n),
                  rng.uniform(0.03, 0.25, n), rng.uniform(-1, 1, n)])
    origin, h, dims = (0.05, -0.02, 0.1), 0.07, (17, 14, 10)
    vol = E.voxelize(b, origin, h, dims)
    brute = np.zeros((dims[2], dims[1], dims[0]))
    for k, j, i in itertools.product(range(dims[2]), range(dims[1]), range(dims[0])):
        x = origin[0] + (i + 0.5) * h
        y = origin[1] + (j + 0.5) * h
        z = origin[2] + (k + 0.5) * h
        for q in range(n):
            dx, dy, dz = x - b[0, q], y - b[1, q], z - b[2, q]
            if (dx * dx + dy * dy) + dz * dz < b[3, q] * b[3, q]:
                brute[k, j, i] += b[4, q]
    np.testing.assert_allclose(vol, brute, rtol=0, atol=1e-12)
    half = E.voxelize(b[:, :6], origin, h, dims) + E.voxelize(b[:, 6:], origin, h, dims)
    np.testing.assert_allclose(vol, half, rtol=0, atol=1e-12)
    vals = rng.uniform(0, 3, n)
    np.testing.assert_allclose(E.voxelize(b, origin, h, dims, values=vals),
                               E.voxelize(np.vstack([b[:4], vals]), origin, h, dims), atol=0)
