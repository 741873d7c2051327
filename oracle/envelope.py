"""FP64 CPU oracle for the entry and exit of Algorithm 1: envelope mesh,
ray-casting initialisation and the point cloud -> voxel grid conversion.

TEST INFRASTRUCTURE ONLY: only `tests/`, `__graft_entry__.smoke()` and the
CPU legs of `bench.py` may import this module. The product library never
calls it and shares no code with it.

What the paper states (Section 4.1, Algorithm 1, Section 2.1) and the
readings taken where it is silent:

* Envelope mesh. A closed polygonal envelope is built from the array
  coordinates. The paper names no construction; the reading is the convex
  hull of the sensor positions (closed, polygonal, defined for any array
  that is not flat). scipy's Qhull serves as the library primitive.
* Reconstruction region. The region is the envelope pulled a small distance
  inward along its normals. The reading: points inside the mesh whose
  distance to the mesh surface is at least `inset`.
* Initialisation. N points are placed uniformly at random inside the mesh,
  with ray casting deciding inside / outside (an odd number of crossings of
  a ray from the point). Candidates are drawn uniformly from the mesh's
  bounding box by a counter-based generator (SplitMix64 at stream positions
  5k .. 5k+4 for candidate k: x, y, z, R, p0) and accepted in candidate
  order, so the first N accepted are a deterministic function of the seed.
* Voxel grid. The paper converts the final cloud with a point-cloud-to-voxel
  shader and gives no formula. The reading, consistent with the uniform
  sphere model of the radiator: voxel v with centre x_v takes the sum of
  the values (p0 by default) of the balls with |x_v - c| < R. Grid layout
  [nz][ny][nx], x_v = origin + (index + 1/2) spacing.

All geometry is float64.
"""
from __future__ import annotations

import numpy as np

from . import splitmix64_at

# a fixed generic direction for the casting ray (not parallel to any axis or
# coordinate plane, so rays through axis-aligned edges are unlikely)
RAY_DIR = np.array([0.8017837257372732, 0.5345224838248488, 0.2672612419124244])


def envelope_mesh(points):
    """Convex hull of the sensor positions (M, 3) -> (vertices (M, 3) float64,
    triangles (F, 3) int64 with outward orientation). Raises for a flat or
    degenerate array."""
    from scipy.spatial import ConvexHull

    P = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    hull = ConvexHull(P)
    tri = hull.simplices.astype(np.int64).copy()
    # orient every triangle so that its normal agrees with the outward plane
    for f in range(tri.shape[0]):
        a, b, c = P[tri[f]]
        nrm = np.cross(b - a, c - a)
        if np.dot(nrm, hull.equations[f, :3]) < 0:
            tri[f, [1, 2]] = tri[f, [2, 1]]
    return P, tri


def mesh_volume(vertices, triangles) -> float:
    """Volume enclosed by a closed outward-oriented triangle mesh (sum of the
    signed tetrahedra against the origin)."""
    V = np.asarray(vertices, dtype=np.float64)
    a, b, c = V[triangles[:, 0]], V[triangles[:, 1]], V[triangles[:, 2]]
    return float(np.sum(np.einsum("ij,ij->i", a, np.cross(b, c))) / 6.0)


def ray_crossings(vertices, triangles, x, direction=RAY_DIR) -> int:
    """Number of triangles crossed by the ray x + t d, t > 0 (Moller-Trumbore
    intersection, closed triangles)."""
    V = np.asarray(vertices, dtype=np.float64)
    v0, v1, v2 = V[triangles[:, 0]], V[triangles[:, 1]], V[triangles[:, 2]]
    e1, e2 = v1 - v0, v2 - v0
    d = np.asarray(direction, dtype=np.float64)
    pvec = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, pvec)
    ok = np.abs(det) > 1e-300
    inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
    tvec = np.asarray(x, dtype=np.float64) - v0
    u = np.einsum("ij,ij->i", tvec, pvec) * inv
    qvec = np.cross(tvec, e1)
    v = (qvec @ d) * inv
    t = np.einsum("ij,ij->i", e2, qvec) * inv
    hit = ok & (u >= 0.0) & (u <= 1.0) & (v >= 0.0) & (u + v <= 1.0) & (t > 0.0)
    return int(np.count_nonzero(hit))


def point_triangle_distance(vertices, triangles, x) -> float:
    """Distance from x to the nearest point of the mesh surface: per
    triangle, the closest point by the Voronoi regions of its vertices, edges
    and face (the standard region test), minimised over triangles."""
    V = np.asarray(vertices, dtype=np.float64)
    p = np.asarray(x, dtype=np.float64)
    best = np.inf
    for f in range(triangles.shape[0]):
        a, b, c = V[triangles[f, 0]], V[triangles[f, 1]], V[triangles[f, 2]]
        ab, ac, ap = b - a, c - a, p - a
        d1, d2 = ab @ ap, ac @ ap
        if d1 <= 0 and d2 <= 0:
            q = a
        else:
            bp = p - b
            d3, d4 = ab @ bp, ac @ bp
            if d3 >= 0 and d4 <= d3:
                q = b
            else:
                vc = d1 * d4 - d3 * d2
                if vc <= 0 and d1 >= 0 and d3 <= 0:
                    q = a + (d1 / (d1 - d3)) * ab
                else:
                    cp = p - c
                    d5, d6 = ab @ cp, ac @ cp
                    if d6 >= 0 and d5 <= d6:
                        q = c
                    else:
                        vb = d5 * d2 - d1 * d6
                        if vb <= 0 and d2 >= 0 and d6 <= 0:
                            q = a + (d2 / (d2 - d6)) * ac
                        else:
                            va = d3 * d6 - d5 * d4
                            if va <= 0 and (d4 - d3) >= 0 and (d5 - d6) >= 0:
                                q = b + ((d4 - d3) / ((d4 - d3) + (d5 - d6))) * (c - b)
                            else:
                                den = 1.0 / (va + vb + vc)
                                q = a + ab * (vb * den) + ac * (vc * den)
        best = min(best, float(np.linalg.norm(p - q)))
    return best


def in_region(vertices, triangles, x, inset: float) -> bool:
    """Inside the mesh (odd number of crossings) and at least `inset` from
    its surface."""
    if ray_crossings(vertices, triangles, x) % 2 == 0:
        return False
    return inset <= 0.0 or point_triangle_distance(vertices, triangles, x) >= inset


def unit_double(seed: int, k: int) -> float:
    """The k-th uniform in [0, 1) of the stream: the top 53 bits of
    SplitMix64 output k, times 2^-53."""
    return float(splitmix64_at(seed, k) >> 11) * (1.0 / 9007199254740992.0)


def candidate(seed: int, k: int, lo, hi, R_range, p_range):
    """Candidate k: centre lo + (hi - lo) u (per axis), R and p0 likewise from
    their ranges; every value computed in double and rounded to float32."""
    u = [unit_double(seed, 5 * k + j) for j in range(5)]
    c = [np.float32(lo[a] + (hi[a] - lo[a]) * u[a]) for a in range(3)]
    R = np.float32(R_range[0] + (R_range[1] - R_range[0]) * u[3])
    p0 = np.float32(p_range[0] + (p_range[1] - p_range[0]) * u[4])
    return c, R, p0


def sample_cloud(vertices, triangles, n: int, seed: int, inset: float, first: int,
                 n_candidates: int, R_range=(0.05, 0.2), p_range=(0.0, 1.0)):
    """Ray-casting initialisation: tests candidates first .. first +
    n_candidates - 1 of the seeded stream in order and keeps the first n inside
    the region. Returns (balls (5, m) float32, accepted candidate indices)."""
    V = np.asarray(vertices, dtype=np.float64)
    lo, hi = V.min(axis=0), V.max(axis=0)
    out, idx = [], []
    for k in range(first, first + n_candidates):
        if len(out) == n:
            break
        c, R, p0 = candidate(seed, k, lo, hi, R_range, p_range)
        if in_region(V, triangles, np.array(c, dtype=np.float64), inset):
            out.append([c[0], c[1], c[2], R, p0])
            idx.append(k)
    balls = np.array(out, dtype=np.float32).T.reshape(5, -1)
    return balls, np.array(idx, dtype=np.int64)


def voxel_centres(origin, spacing: float, n: int, axis: int) -> np.ndarray:
    return float(origin[axis]) + (np.arange(n, dtype=np.float64) + 0.5) * float(spacing)


def voxelize(balls, origin, spacing: float, dims, values=None) -> np.ndarray:
    """Voxel v (centre x_v) = sum of values[i] over balls i with
    |x_v - c_i|^2 < R_i^2 (squares and sums in double, in that order).
    dims = (nx, ny, nz); returns float64 [nz][ny][nx]."""
    b = np.asarray(balls, dtype=np.float64).reshape(5, -1)
    vals = b[4] if values is None else np.asarray(values, dtype=np.float64)
    nx, ny, nz = (int(v) for v in dims)
    vol = np.zeros((nz, ny, nx))
    cx, cy, cz = (voxel_centres(origin, spacing, n, a) for a, n in enumerate((nx, ny, nz)))
    for i in range(b.shape[1]):
        x, y, z, R = b[0, i], b[1, i], b[2, i], b[3, i]
        if not (R > 0.0):
            continue
        sel = []
        for a, (n, centre) in enumerate(((nx, x), (ny, y), (nz, z))):
            lo = max(0, int(np.floor((centre - R - float(origin[a])) / spacing)) - 1)
            hi = min(n - 1, int(np.ceil((centre + R - float(origin[a])) / spacing)) + 1)
            sel.append((lo, hi))
        (x0, x1), (y0, y1), (z0, z1) = sel
        if x0 > x1 or y0 > y1 or z0 > z1:
            continue
        dx = cx[x0:x1 + 1] - x
        dy = cy[y0:y1 + 1] - y
        dz = cz[z0:z1 + 1] - z
        d2 = (dx[None, None, :] * dx[None, None, :] + dy[None, :, None] * dy[None, :, None]) \
            + dz[:, None, None] * dz[:, None, None]
        vol[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1] += np.where(d2 < R * R, vals[i], 0.0)
    return vol
