"""Seeded synthetic workloads shaped like the SlingBAG Pro experiments.

This module only draws inputs: sensor arrays, point clouds and vessel-tree
phantoms. It holds none of the radiator's arithmetic, so both the FP64 oracle
(`oracle/`) and the CUDA path (`paper_2601_00551_gb300`) can take their inputs
from here without sharing any of the method.

Units are mm and microseconds; the speed of sound is 1.5 mm/us (1500 m/s, as
in Section 2.1 of the paper). The paper's own data (hand-vessel simulation,
Section 2.1; in vivo rat, Section 2.2) is not available, so these seeded
stand-ins keep its shapes: irregular arrays of a few hundred to two thousand
oriented sensors, 40 MHz sampling, records of 1024-4096 samples, and initial
clouds of 10^3-10^5 random balls (Section 2.1 uses 200,000).

Every array is float32 (the CUDA path's storage type). Seeds: 0 ground truth,
1 initial cloud, 2 sensors, 3 noise (fixed per workload below).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_MM_PER_US = 1.5  # 1500 m/s (Section 2.1)


@dataclasses.dataclass
class Sensors:
    """Sensor array: positions (M,3) and unit inward normals (M,3), float32."""

    pos: np.ndarray
    normal: np.ndarray

    @property
    def M(self) -> int:
        return int(self.pos.shape[0])


@dataclasses.dataclass
class Balls:
    """Point cloud in structure-of-arrays form, float32 each of length n."""

    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    R: np.ndarray
    p0: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def stack(self) -> np.ndarray:
        """(5, n) float32 array in the order x, y, z, R, p0."""
        return np.stack([self.x, self.y, self.z, self.R, self.p0]).astype(np.float32)

    @staticmethod
    def from_stack(a: np.ndarray) -> "Balls":
        a = np.asarray(a, dtype=np.float32)
        return Balls(a[0].copy(), a[1].copy(), a[2].copy(), a[3].copy(), a[4].copy())

    def take(self, idx) -> "Balls":
        return Balls(self.x[idx], self.y[idx], self.z[idx], self.R[idx], self.p0[idx])

    def concat(self, other: "Balls") -> "Balls":
        return Balls(*(np.concatenate([a, b]) for a, b in zip(
            (self.x, self.y, self.z, self.R, self.p0),
            (other.x, other.y, other.z, other.R, other.p0))))


# --------------------------------------------------------------------------
# geometry helpers (random directions, jittered normals)
# --------------------------------------------------------------------------

def _random_unit(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _jitter_normals(rng: np.random.Generator, nrm: np.ndarray, max_deg: float) -> np.ndarray:
    """Rotate each unit vector by an angle ~U(0, max_deg) about a random
    perpendicular axis."""
    n = nrm.shape[0]
    a = _random_unit(rng, n)
    perp = a - np.sum(a * nrm, axis=1, keepdims=True) * nrm
    bad = np.linalg.norm(perp, axis=1) < 1e-6
    while bad.any():
        a[bad] = _random_unit(rng, int(bad.sum()))
        perp = a - np.sum(a * nrm, axis=1, keepdims=True) * nrm
        bad = np.linalg.norm(perp, axis=1) < 1e-6
    perp /= np.linalg.norm(perp, axis=1, keepdims=True)
    ang = np.deg2rad(rng.uniform(0.0, max_deg, size=(n, 1)))
    out = np.cos(ang) * nrm + np.sin(ang) * perp
    return out / np.linalg.norm(out, axis=1, keepdims=True)


def spherical_cap(M: int, radius: float = 20.0, max_polar_deg: float = 60.0,
                  jitter_deg: float = 10.0, seed: int = 2) -> Sensors:
    """M sensors uniform (by area) on a spherical cap about +z, normals
    pointing at the centre and jittered by up to `jitter_deg`."""
    rng = np.random.default_rng(seed)
    cos_t = rng.uniform(math.cos(math.radians(max_polar_deg)), 1.0, size=M)
    phi = rng.uniform(0.0, 2 * math.pi, size=M)
    sin_t = np.sqrt(1.0 - cos_t ** 2)
    pos = radius * np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)
    nrm = -pos / np.linalg.norm(pos, axis=1, keepdims=True)
    nrm = _jitter_normals(rng, nrm, jitter_deg)
    return Sensors(pos.astype(np.float32), nrm.astype(np.float32))


def ellipsoid_cap(M: int, axes=(30.0, 30.0, 20.0), jitter_deg: float = 15.0,
                  seed: int = 2, z_min: float = 0.0) -> Sensors:
    """M sensors on the z >= z_min part of an ellipsoid with semi-axes `axes`,
    drawn uniformly by area (rejection on the surface element), normals along
    the inward gradient of the implicit surface, jittered by up to
    `jitter_deg`."""
    rng = np.random.default_rng(seed)
    a, b, c = axes
    pts = []
    need = M
    gmax = max(b * c, a * c, a * b)
    while need > 0:
        u = _random_unit(rng, 4 * need + 64)
        u = u[u[:, 2] * c >= z_min]
        p = u * np.array([a, b, c])
        # surface element of the map sphere -> ellipsoid: |grad| scaling
        g = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2)
        keep = rng.uniform(0.0, gmax, size=g.shape[0]) < g
        p = p[keep][:need]
        pts.append(p)
        need -= p.shape[0]
    pos = np.concatenate(pts, axis=0)[:M]
    grad = pos / np.array([a * a, b * b, c * c])
    nrm = -grad / np.linalg.norm(grad, axis=1, keepdims=True)
    nrm = _jitter_normals(rng, nrm, jitter_deg)
    return Sensors(pos.astype(np.float32), nrm.astype(np.float32))


# --------------------------------------------------------------------------
# point clouds
# --------------------------------------------------------------------------

def uniform_balls(n: int, half: float, r_lo: float, r_hi: float, p_lo: float = 0.0,
                  p_hi: float = 1.0, seed: int = 1) -> Balls:
    """n balls with centres uniform in [-half, half]^3, R ~ U(r_lo, r_hi),
    p0 ~ U(p_lo, p_hi)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-half, half, size=(n, 3))
    R = rng.uniform(r_lo, r_hi, size=n)
    p0 = rng.uniform(p_lo, p_hi, size=n)
    f = np.float32
    return Balls(c[:, 0].astype(f), c[:, 1].astype(f), c[:, 2].astype(f), R.astype(f), p0.astype(f))


def morton_order(b: Balls, half: float, bits: int = 10) -> np.ndarray:
    """Permutation that sorts balls by the Morton (Z-order) code of their
    centre in a 2^bits grid over [-half, half]^3. Used only to lay a cloud
    out so that neighbouring indices are neighbouring in space."""
    g = (1 << bits) - 1
    q = [np.clip(((v.astype(np.float64) + half) / (2 * half) * g).round(), 0, g).astype(np.uint64)
         for v in (b.x, b.y, b.z)]

    def spread(v):
        out = np.zeros_like(v)
        for i in range(bits):
            out |= ((v >> np.uint64(i)) & np.uint64(1)) << np.uint64(3 * i)
        return out

    code = spread(q[0]) | (spread(q[1]) << np.uint64(1)) | (spread(q[2]) << np.uint64(2))
    return np.argsort(code, kind="stable")


def vessel_tree(n_balls: int, half: float = 10.0, root_radius: float = 0.4,
                shrink: float = 0.8, min_radius: float = 0.05, seg_len=(2.0, 5.0),
                branch_deg=(20.0, 60.0), p_range=(0.5, 1.0), seed: int = 0) -> Balls:
    """Seeded branching-tube phantom sampled as balls.

    A root tube of radius `root_radius` starts near the bottom of the cube
    [-half, half]^3 and grows upward; each segment has length ~U(seg_len) and
    ends in two children whose directions turn by ~U(branch_deg) from the
    parent about random axes, with radius multiplied by `shrink`, until the
    radius falls below `min_radius` or the segment leaves the cube. Balls are
    drawn on segments with probability proportional to length x radius^2, at
    a uniform position along the axis plus an offset uniform in the disc of
    radius 0.5 r; their R is the local radius times U(0.8, 1.2), clipped to
    [0.05, 0.4] mm, and p0 ~ U(p_range).
    """
    rng = np.random.default_rng(seed)
    segs = []  # (start(3), end(3), radius)
    stack = [(np.array([0.0, 0.0, -0.9 * half]), np.array([0.0, 0.0, 1.0]), root_radius)]
    while stack:
        start, d, r = stack.pop()
        if r < min_radius:
            continue
        length = rng.uniform(*seg_len)
        end = start + length * d
        if np.any(np.abs(end) > half):
            # clip the segment to the cube and stop this branch
            t_hi = length
            for ax in range(3):
                if abs(d[ax]) > 1e-12:
                    for bound in (-half, half):
                        t = (bound - start[ax]) / d[ax]
                        if 0 < t < t_hi:
                            t_hi = t
            end = start + t_hi * d
            if t_hi > 1e-3:
                segs.append((start, end, r))
            continue
        segs.append((start, end, r))
        for _ in range(2):
            axis = _random_unit(rng, 1)[0]
            axis -= np.dot(axis, d) * d
            axis /= np.linalg.norm(axis)
            ang = math.radians(rng.uniform(*branch_deg))
            nd = math.cos(ang) * d + math.sin(ang) * axis
            nd /= np.linalg.norm(nd)
            stack.append((end, nd, r * shrink))
    S = np.array([s[0] for s in segs])
    E = np.array([s[1] for s in segs])
    rad = np.array([s[2] for s in segs])
    L = np.linalg.norm(E - S, axis=1)
    w = L * rad ** 2
    seg = rng.choice(len(segs), size=n_balls, p=w / w.sum())
    t = rng.uniform(0.0, 1.0, size=(n_balls, 1))
    axis_pt = S[seg] + t * (E[seg] - S[seg])
    dirs = (E[seg] - S[seg]) / L[seg][:, None]
    # offset uniform in a disc perpendicular to the axis
    a = _random_unit(rng, n_balls)
    a -= np.sum(a * dirs, axis=1, keepdims=True) * dirs
    a /= np.maximum(np.linalg.norm(a, axis=1, keepdims=True), 1e-12)
    rr = 0.5 * rad[seg] * np.sqrt(rng.uniform(0.0, 1.0, size=n_balls))
    c = axis_pt + rr[:, None] * a
    c = np.clip(c, -half, half)
    R = np.clip(rad[seg] * rng.uniform(0.8, 1.2, size=n_balls), 0.05, 0.4)
    p0 = rng.uniform(*p_range, size=n_balls)
    f = np.float32
    return Balls(c[:, 0].astype(f), c[:, 1].astype(f), c[:, 2].astype(f), R.astype(f), p0.astype(f))


def add_noise(y: np.ndarray, rel: float = 0.01, seed: int = 3) -> np.ndarray:
    """y + N(0, (rel * max|y|)^2), float32 (the "1% Gaussian noise" reading)."""
    rng = np.random.default_rng(seed)
    sigma = rel * float(np.max(np.abs(y))) if y.size else 0.0
    return (y + rng.normal(0.0, sigma, size=y.shape)).astype(np.float32)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    sensors: Sensors
    init: Balls          # initial cloud to reconstruct from
    truth: Balls | None  # ground-truth cloud used to synthesise measurements
    fs_mhz: float
    T: int               # samples at the finest level
    levels: tuple        # downsampling factors f_k, coarse to fine
    c: float = C_MM_PER_US
    half: float = 2.0


def tiny(n_init: int = 2000, n_truth: int = 500, M: int = 64, T: int = 1024,
         sort: bool = False) -> Workload:
    """The small plain-method case: balls in a 4 mm cube, R ~ U(0.05, 0.2) mm,
    p0 ~ U(0, 1); 64 sensors on a 20 mm spherical cap (polar angle <= 60 deg),
    inward normals jittered by up to 10 deg; 40 MHz, T = 1024."""
    sens = spherical_cap(M, 20.0, 60.0, 10.0, seed=2)
    init = uniform_balls(n_init, 2.0, 0.05, 0.2, 0.0, 1.0, seed=1)
    truth = uniform_balls(n_truth, 2.0, 0.05, 0.2, 0.0, 1.0, seed=0)
    if sort:
        init = init.take(morton_order(init, 2.0))
    return Workload("tiny: 2000 balls x 64 sensors, 40 MHz, T=1024", sens, init, truth,
                    40.0, T, (1,), half=2.0)


def vessel(n_init: int = 200_000, n_truth: int = 150_000, M: int = 512, T: int = 4096,
           sort: bool = True) -> Workload:
    """The full plain-method case: a seeded vessel-tree phantom (radii
    0.05-0.4 mm) sampled as 150k balls in a 20 mm cube, an initial cloud of
    200k uniform random balls (R ~ U(0.05, 0.2), p0 ~ U(0, 1)), 512 sensors
    on the z >= 0 half of a (30, 30, 20) mm ellipsoid with normals jittered by
    up to 15 deg, and hierarchical sampling 10 -> 20 -> 40 MHz (f = 4, 2, 1)
    with T = 1024 / 2048 / 4096. The initial cloud is laid out in Morton
    order so that index neighbours are spatial neighbours."""
    sens = ellipsoid_cap(M, (30.0, 30.0, 20.0), 15.0, seed=2)
    init = uniform_balls(n_init, 10.0, 0.05, 0.2, 0.0, 1.0, seed=1)
    if sort:
        init = init.take(morton_order(init, 10.0))
    truth = vessel_tree(n_truth, half=10.0, seed=0)
    return Workload("vessel: 200k balls x 512 sensors, 10/20/40 MHz, T=1024/2048/4096",
                    sens, init, truth, 40.0, T, (4, 2, 1), half=10.0)


@dataclasses.dataclass
class FrameWorkload:
    """Dynamic imaging: one sensor array, F frames of a moving phantom, each
    reconstructed from its own initial cloud."""
    name: str
    sensors: Sensors
    inits: list           # initial cloud per frame (Balls)
    truths: list          # ground truth per frame (Balls), the phantom shifted
    shifts: np.ndarray    # (F, 3) displacement of frame f from frame 0, mm
    fs_mhz: float
    T: int
    levels: tuple
    c: float = C_MM_PER_US
    half: float = 10.0

    @property
    def F(self) -> int:
        return len(self.inits)


def frames(n_frames: int = 32, n_lo: int = 20_000, n_hi: int = 200_000, n_truth: int = 150_000,
           M: int = 256, T: int = 2048, max_step: float = 0.5, levels=(4, 2, 1),
           sort: bool = True) -> FrameWorkload:
    """The batched dynamic-imaging case: the vessel-tree phantom of `vessel`
    moved rigidly from frame to frame (step f has length ~U(0, max_step) mm
    along a seeded random direction, seed 4), measured by 256 sensors of the
    same ellipsoidal cap at 40 MHz with T = 2048; frame f starts from its own
    uniform random cloud whose size is drawn uniformly from {n_lo..n_hi}
    (seed 4), laid out in Morton order."""
    sens = ellipsoid_cap(M, (30.0, 30.0, 20.0), 15.0, seed=2)
    rng = np.random.default_rng(4)
    counts = rng.integers(n_lo, n_hi + 1, size=n_frames)
    steps = _random_unit(rng, n_frames) * rng.uniform(0.0, max_step, size=(n_frames, 1))
    steps[0] = 0.0
    shifts = np.cumsum(steps, axis=0)
    base = vessel_tree(n_truth, half=10.0, seed=0)
    truths, inits = [], []
    for f in range(n_frames):
        s = shifts[f].astype(np.float32)
        truths.append(Balls(base.x + s[0], base.y + s[1], base.z + s[2], base.R.copy(),
                            base.p0.copy()))
        b = uniform_balls(int(counts[f]), 10.0, 0.05, 0.2, 0.0, 1.0, seed=1000 + f)
        if sort:
            b = b.take(morton_order(b, 10.0))
        inits.append(b)
    name = (f"frames: {n_frames} frames x {n_lo // 1000}k-{n_hi // 1000}k balls x {M} sensors, "
            f"10/20/40 MHz, T={T // levels[0]}/{T // levels[1]}/{T}")
    return FrameWorkload(name, sens, inits, truths, shifts, 40.0, T, tuple(levels))


@dataclasses.dataclass
class EnvelopeWorkload:
    """A closed irregular array around an imaging region, the initial cloud
    size and inset, and the voxel grid of the region."""
    name: str
    sensors: Sensors
    n_init: int
    inset: float
    R_range: tuple
    p_range: tuple
    seed: int
    origin: tuple
    spacing: float
    dims: tuple


def envelope(M: int = 2006, axes=(48.0, 60.0, 26.0), n_init: int = 200_000,
             inset: float = 2.0) -> EnvelopeWorkload:
    """Stand-in for the hand-vessel setup (Section 2.1): M sensors drawn
    uniformly by area on a closed ellipsoid (semi-axes 48 / 60 / 26 mm, around
    an 80 x 104 x 40 mm imaging region), normals inward jittered by up to
    15 deg; 200,000 initial balls inside the envelope pulled 2 mm inward
    (R ~ U(0.05, 0.2) mm, p0 ~ U(0, 1), seed 1); the region voxelised at
    0.2 mm (400 x 520 x 200 voxels)."""
    sens = ellipsoid_cap(M, axes, 15.0, seed=2, z_min=-axes[2])
    return EnvelopeWorkload(
        f"envelope: {M} sensors on a closed {axes[0]:g}/{axes[1]:g}/{axes[2]:g} mm ellipsoid, "
        f"{n_init // 1000}k balls, 0.2 mm voxels over 80 x 104 x 40 mm",
        sens, n_init, inset, (0.05, 0.2), (0.0, 1.0), 1, (-40.0, -52.0, -20.0), 0.2,
        (400, 520, 200))


def large(n_truth: int = 1_000_000, n_init: int = 1_000_000, M: int = 1024, T: int = 8192,
          sort: bool = True) -> Workload:
    """The large case: a seeded vessel-tree phantom of 1M balls in a 40 mm
    cube, an initial cloud of 1M uniform balls (R ~ U(0.05, 0.2), p0 ~ U(0, 1),
    Morton order), 1024 sensors on the z >= 0 half of a (60, 60, 40) mm
    ellipsoid with normals jittered by up to 15 deg, and sampling at
    80 MHz with T = 8192 (levels f = 4, 2, 1: 20 / 40 / 80 MHz)."""
    sens = ellipsoid_cap(M, (60.0, 60.0, 40.0), 15.0, seed=2)
    init = uniform_balls(n_init, 20.0, 0.05, 0.2, 0.0, 1.0, seed=1)
    if sort:
        init = init.take(morton_order(init, 20.0))
    truth = vessel_tree(n_truth, half=20.0, seed=0)
    return Workload("large: 1M balls x 1024 sensors, 20/40/80 MHz, T=2048/4096/8192", sens,
                    init, truth, 80.0, T, (4, 2, 1), half=20.0)
