"""FP64 CPU oracle for the SlingBAG Pro hot path.

TEST INFRASTRUCTURE ONLY: only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline / reference legs of `bench.py` may import this package. The
product library never calls it and shares no code with it.

The radiator and its adjoint are plain double loops in C
(`slingbag_oracle.c`, compiled with gcc on first use); the light steps
(zero-gradient filter, growth, Adam, the reconstruction loop) are written
here in numpy, in the order the paper gives them:

* zero-gradient filtering -- Section 4.2 and Algorithm 1 (initialisation);
* hierarchical sampling and per-level loss -- Section 4.3;
* destroy / split / duplicate -- Section 4.1 and Algorithm 1 (the paper
  states the operations but not their thresholds or geometry; the rules
  below are this project's stated reading);
* Adam -- the paper names no optimizer (Section 2.1 only says the learning
  rates are the same for both methods); Adam is this project's reading.

Every function takes and returns float64 arrays; callers pass float32 inputs
that are converted exactly.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import shutil
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slingbag_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

W_MODES = {"clamp": 0, "none": 1, "cos": 2}
MASK_P0, MASK_R, MASK_XYZ = 1, 2, 4
MASK_ALL = 7
SOFTPLUS_R = 8  # optimise R through R = softplus(a) (Section 4.3)


def build(force: bool = False) -> str:
    """Compile the C part of the oracle into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("oracle: no C compiler found")
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = [cc, "-O2", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        L = ctypes.c_long
        lib.oracle_forward.restype = L
        lib.oracle_forward.argtypes = [L, d, d, d, d, d, L, d, d, ctypes.c_double,
                                       ctypes.c_double, L, ctypes.c_int, d, ctypes.c_int]
        lib.oracle_adjoint.restype = L
        lib.oracle_adjoint.argtypes = [L, d, d, d, d, d, L, d, d, ctypes.c_double,
                                       ctypes.c_double, L, ctypes.c_int, d, ctypes.c_int,
                                       d, d, d, d, d, d, ctypes.c_int]
        lib.oracle_forward_gauss.restype = L
        lib.oracle_forward_gauss.argtypes = lib.oracle_forward.argtypes
        lib.oracle_adjoint_gauss.restype = L
        lib.oracle_adjoint_gauss.argtypes = [L, d, d, d, d, d, L, d, d, ctypes.c_double,
                                             ctypes.c_double, L, ctypes.c_int, d, ctypes.c_int,
                                             d, d, d, d, d, ctypes.c_int]
        lib.oracle_downsample.restype = None
        lib.oracle_downsample.argtypes = [L, L, d, L, d]
        lib.oracle_num_procs.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_procs() -> int:
    return int(_load().oracle_num_procs())


# --------------------------------------------------------------------------
# radiator, adjoint, downsample (C)
# --------------------------------------------------------------------------

def forward(balls, pos, normal, c: float, dt: float, T: int, wmode: str = "clamp",
            threads: int = 1, return_inside: bool = False):
    """Cell-averaged traces S (M, T) of the N-wave radiator (Section 4.2,
    Simulate; Section 4.3 at sampling interval dt = f_k / fs).

    `balls` is a (5, n) array of x, y, z, R, p0; `pos`/`normal` are (M, 3)."""
    b = _f64(balls).reshape(5, -1)
    pos = _f64(pos).reshape(-1, 3)
    nrm = _f64(normal).reshape(-1, 3)
    n, M = b.shape[1], pos.shape[0]
    S = np.zeros((M, T), dtype=np.float64)
    rows = [np.ascontiguousarray(b[k]) for k in range(5)]
    inside = _load().oracle_forward(n, *(_ptr(r) for r in rows), M, _ptr(pos), _ptr(nrm),
                                    float(c), float(dt), int(T), W_MODES[wmode], _ptr(S),
                                    int(threads))
    return (S, int(inside)) if return_inside else S


def adjoint(balls, pos, normal, c: float, dt: float, T: int, G, mask: int = MASK_ALL,
            wmode: str = "clamp", threads: int = 1, with_abs: bool = False):
    """Per-ball gradients (5, n) in the order x, y, z, R, p0 of
    L(S) given G = dL/dS (M, T) -- the backpropagation step of Algorithm 1.
    With `with_abs` also returns sum_m |K A| per ball (the scale of dL/dp0)."""
    b = _f64(balls).reshape(5, -1)
    pos = _f64(pos).reshape(-1, 3)
    nrm = _f64(normal).reshape(-1, 3)
    G = _f64(G).reshape(pos.shape[0], T)
    n, M = b.shape[1], pos.shape[0]
    out = np.zeros((6, n), dtype=np.float64)
    rows = [np.ascontiguousarray(b[k]) for k in range(5)]
    outs = [np.zeros(n) for _ in range(6)]
    _load().oracle_adjoint(n, *(_ptr(r) for r in rows), M, _ptr(pos), _ptr(nrm), float(c),
                           float(dt), int(T), W_MODES[wmode], _ptr(G), int(mask),
                           *(_ptr(o) for o in outs), int(threads))
    for k in range(6):
        out[k] = outs[k]
    g = out[:5]
    return (g, out[5]) if with_abs else g


def forward_gauss(balls, pos, normal, c: float, dt: float, T: int, wmode: str = "clamp",
                  threads: int = 1, return_inside: bool = False):
    """Traces of the Gaussian-profile radiator (Section 4.1's Gaussian
    spherical sources; the R row holds the standard deviation a): cell
    averages of p0 w (d - ct) exp(-(d - ct)^2 / 2a^2) / (2d), on every cell.
    Pairs with d <= 6a are skipped (far-field reading) and counted."""
    b = _f64(balls).reshape(5, -1)
    pos = _f64(pos).reshape(-1, 3)
    nrm = _f64(normal).reshape(-1, 3)
    n, M = b.shape[1], pos.shape[0]
    S = np.zeros((M, T), dtype=np.float64)
    rows = [np.ascontiguousarray(b[k]) for k in range(5)]
    inside = _load().oracle_forward_gauss(n, *(_ptr(r) for r in rows), M, _ptr(pos), _ptr(nrm),
                                          float(c), float(dt), int(T), W_MODES[wmode], _ptr(S),
                                          int(threads))
    return (S, int(inside)) if return_inside else S


def adjoint_gauss(balls, pos, normal, c: float, dt: float, T: int, G, mask: int = MASK_ALL,
                  wmode: str = "clamp", threads: int = 1):
    """Per-ball gradients (5, n: x, y, z, a, p0) of the Gaussian-profile
    radiator for G = dL/dS."""
    b = _f64(balls).reshape(5, -1)
    pos = _f64(pos).reshape(-1, 3)
    nrm = _f64(normal).reshape(-1, 3)
    G = _f64(G).reshape(pos.shape[0], T)
    n, M = b.shape[1], pos.shape[0]
    rows = [np.ascontiguousarray(b[k]) for k in range(5)]
    outs = [np.zeros(n) for _ in range(5)]
    _load().oracle_adjoint_gauss(n, *(_ptr(r) for r in rows), M, _ptr(pos), _ptr(nrm), float(c),
                                 float(dt), int(T), W_MODES[wmode], _ptr(G), int(mask),
                                 *(_ptr(o) for o in outs), int(threads))
    return np.stack(outs)


def downsample(y, f: int) -> np.ndarray:
    """y_real^(k) = Downsample_f(y_real) (Section 4.3): block means of f
    samples, zero-padded to a multiple of f."""
    y = _f64(y)
    M, T = y.shape
    Tk = (T + f - 1) // f
    out = np.zeros((M, Tk))
    _load().oracle_downsample(M, T, _ptr(y), int(f), _ptr(out))
    return out


def loss_and_residual(S, y):
    """L = ||S - y||_2^2 (Section 4.2 and 4.3; a plain sum, no 1/2) and its
    gradient G = 2 (S - y)."""
    r = _f64(S) - _f64(y)
    return float(np.sum(r * r)), 2.0 * r


# --------------------------------------------------------------------------
# zero-gradient filtering (Section 4.2, Algorithm 1)
# --------------------------------------------------------------------------

KEEP_NEG, KEEP_NONPOS, DROP_ZERO = 0, 1, 2


def zero_gradient_filter(balls, pos, normal, c, dt, T, y_k, mode: int = KEEP_NEG,
                         wmode: str = "clamp", threads: int = 1, margin: float = 1e-5):
    """Zero-gradient filtering of Section 4.2 / Algorithm 1.

    Every p0 is set to zero, so the simulated signal is zero and the loss
    gradient wrt the traces is G = 2 (0 - y_k) = -2 y_k; one backpropagation
    gives g_i = dL/dp0_i at p0 = 0. Balls are kept by the sign rule (default
    g < 0, Algorithm 1; `KEEP_NONPOS` keeps g <= 0 as in the equations of
    Section 4.2; `DROP_ZERO` drops only g == 0) and keep their original p0.

    Returns (kept indices in original order, g, ambiguous indices) where a
    ball is ambiguous when |g| < margin * sum_m |K A| (a sign a rounding
    error of that relative size could flip)."""
    b = _f64(balls).reshape(5, -1).copy()
    zero = b.copy()
    zero[4] = 0.0
    G = -2.0 * _f64(y_k)
    g, gabs = adjoint(zero, pos, normal, c, dt, T, G, mask=MASK_P0, wmode=wmode,
                      threads=threads, with_abs=True)
    gp = g[4]
    if mode == KEEP_NEG:
        keep = gp < 0
    elif mode == KEEP_NONPOS:
        keep = gp <= 0
    elif mode == DROP_ZERO:
        keep = gp != 0
    else:
        raise ValueError(mode)
    amb = np.nonzero((np.abs(gp) < margin * gabs) & (gabs > 0))[0]
    return np.nonzero(keep)[0], gp, amb


# --------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood 2014; Vigna's splitmix64.c) as a
# counter-based generator: output k of the stream seeded with s is
# mix(s + (k + 1) * gamma).
# --------------------------------------------------------------------------

_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def splitmix64_mix(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def splitmix64_at(seed: int, k: int) -> int:
    return splitmix64_mix(seed + (k + 1) * _GAMMA)


def split_direction(seed: int, i: int) -> np.ndarray:
    """Unit vector for ball index i: three 24-bit draws k = 3i, 3i+1, 3i+2,
    each mapped to the odd lattice point (2u + 1 - 2^24) / 2^24 in (-1, 1),
    then normalised."""
    g = np.empty(3)
    for r in range(3):
        u = splitmix64_at(seed, 3 * i + r) >> 40
        g[r] = (2.0 * u + 1.0 - 16777216.0) / 16777216.0
    return g / np.sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2])


# --------------------------------------------------------------------------
# adaptive growth: destroy / split / duplicate (Section 4.1, Algorithm 1)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class GrowParams:
    """Thresholds of the growth step (the paper gives none; these are this
    project's readings). Ball i is, in this order of precedence:
      pruned     if `prune_zero` and every active gradient component is 0
                 (active = those in `grad_mask`);
      destroyed  if `destroy` and (p0 < p_min or R < R_min);
      split      if `split` and R > R_max, into two balls at c +- (R/2) v
                 with radius R 2^(-1/3) and the same p0;
      duplicated if `duplicate` and |dL/dc|^2 > g_dup^2, adding a clone at
                 c + (R/2) v after it;
    and kept otherwise. v is `split_direction(seed, i)`. New balls get zero
    gradients and zero optimizer state; kept balls keep theirs."""
    p_min: float = 1e-3
    R_min: float = 0.02
    R_max: float = 0.3
    g_dup: float = 1e30
    seed: int = 0
    grad_mask: int = MASK_ALL
    prune_zero: bool = True
    destroy: bool = True
    split: bool = True
    duplicate: bool = False


def grow(balls, grads, extra, gp: GrowParams):
    """One filter/grow pass. `balls` (5, n) float32, `grads` (5, n) float32
    (x, y, z, R, p0 order), `extra` (k, n) float32 carried state (e.g. Adam
    moments). Returns new (balls, grads, extra) as float32 arrays and the
    per-input-ball output count."""
    b = np.asarray(balls, dtype=np.float32).reshape(5, -1)
    g = np.asarray(grads, dtype=np.float32).reshape(5, -1)
    ex = np.asarray(extra, dtype=np.float32)
    ex = ex.reshape(ex.shape[0] if ex.size else 0, b.shape[1])
    n = b.shape[1]
    rows_b, rows_g, rows_e, counts = [], [], [], np.zeros(n, dtype=np.int64)
    shrink = np.float32(2.0 ** (-1.0 / 3.0))
    zero_g = np.zeros(5, dtype=np.float32)
    zero_e = np.zeros(ex.shape[0], dtype=np.float32)
    comp = [(MASK_XYZ, 0), (MASK_XYZ, 1), (MASK_XYZ, 2), (MASK_R, 3), (MASK_P0, 4)]
    for i in range(n):
        x, y, z, R, p0 = (b[k, i] for k in range(5))
        if gp.prune_zero:
            active = [g[k, i] for (bit, k) in comp if gp.grad_mask & bit]
            if active and all(a == 0.0 for a in active):
                continue
        if gp.destroy and (p0 < np.float32(gp.p_min) or R < np.float32(gp.R_min)):
            continue
        if gp.split and R > np.float32(gp.R_max):
            v = split_direction(gp.seed, i)
            for sgn in (1.0, -1.0):
                rows_b.append(np.array([x + sgn * 0.5 * R * v[0], y + sgn * 0.5 * R * v[1],
                                        z + sgn * 0.5 * R * v[2], R * float(shrink), p0]))
                rows_g.append(zero_g)
                rows_e.append(zero_e)
            counts[i] = 2
            continue
        rows_b.append(b[:, i].astype(np.float64))
        rows_g.append(g[:, i])
        rows_e.append(ex[:, i])
        counts[i] = 1
        if gp.duplicate:
            gx, gy, gz = (float(g[k, i]) for k in range(3))
            if gx * gx + gy * gy + gz * gz > float(np.float32(gp.g_dup)) ** 2:
                v = split_direction(gp.seed, i)
                rows_b.append(np.array([x + 0.5 * R * v[0], y + 0.5 * R * v[1],
                                        z + 0.5 * R * v[2], R, p0], dtype=np.float64))
                rows_g.append(zero_g)
                rows_e.append(zero_e)
                counts[i] = 2
    if rows_b:
        nb = np.stack(rows_b, axis=1).astype(np.float32)
        ng = np.stack(rows_g, axis=1).astype(np.float32)
        ne = np.stack(rows_e, axis=1).astype(np.float32) if ex.shape[0] else \
            np.zeros((0, nb.shape[1]), np.float32)
    else:
        nb = np.zeros((5, 0), np.float32)
        ng = np.zeros((5, 0), np.float32)
        ne = np.zeros((ex.shape[0], 0), np.float32)
    return nb, ng, ne, counts


# --------------------------------------------------------------------------
# spatial ordering (no counterpart in the paper: the library's sbp_sort_cloud)
# --------------------------------------------------------------------------

def morton_key(balls) -> np.ndarray:
    """The 30-bit Morton key of every ball, by its definition: lo = the
    componentwise minimum of the centres, span = the largest extent over the
    three axes, inv = 1024 / span, q = min(1023, floor((c - lo) * inv)) per
    axis (clamped below at 0), each operation in float32 rounded once, and
    the bits of (q_x, q_y, q_z) interleaved with x lowest."""
    b = np.asarray(balls, dtype=np.float32).reshape(5, -1)
    n = b.shape[1]
    if n == 0:
        return np.zeros(0, dtype=np.int64)
    lo = b[:3].min(axis=1)
    hi = b[:3].max(axis=1)
    ext = (hi - lo).astype(np.float32)
    span = np.float32(ext.max())
    inv = np.float32(np.float32(1024.0) / span) if span > 0 else np.float32(0.0)
    key = np.zeros(n, dtype=np.int64)
    for a in range(3):
        t = ((b[a] - lo[a]).astype(np.float32) * inv).astype(np.float32)
        q = np.clip(np.floor(t), 0, 1023).astype(np.int64)
        for bit in range(10):
            key |= ((q >> bit) & 1) << (3 * bit + a)
    return key


def morton_permutation(balls) -> np.ndarray:
    """Indices of the balls in ascending key order, equal keys in index
    order (a stable sort)."""
    return np.argsort(morton_key(balls), kind="stable")


# --------------------------------------------------------------------------
# Adam (reading: the paper names no optimizer)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class AdamParams:
    lr: tuple = (1e-3, 1e-3, 1e-3, 1e-3, 1e-2)  # x, y, z, R, p0
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8


def softplus(a):
    """log(1 + e^a) = max(a, 0) + log(1 + e^-|a|), without overflow."""
    a = np.asarray(a, dtype=np.float64)
    return np.maximum(a, 0.0) + np.log1p(np.exp(-np.abs(a)))


def softplus_inv(R):
    """The a with softplus(a) = R > 0: log(e^R - 1) = R + log(1 - e^-R)."""
    R = np.asarray(R, dtype=np.float64)
    return R + np.log(-np.expm1(-R))


def adam(balls, grads, m, v, t: int, ap: AdamParams, mask: int = MASK_ALL):
    """One Adam step (Kingma & Ba 2015) at step count t >= 1 on the
    parameters selected by `mask`; returns new (balls, m, v) in float64.
    With SOFTPLUS_R the radius is optimised as R = softplus(a) (the
    positivity-constrained refinement of Section 4.3): the moments follow
    dL/da = sigmoid(a) dL/dR and R becomes softplus(a - step)."""
    b = _f64(balls).reshape(5, -1).copy()
    g = _f64(grads).reshape(5, -1).copy()
    m = _f64(m).reshape(5, -1).copy()
    v = _f64(v).reshape(5, -1).copy()
    bits = [MASK_XYZ, MASK_XYZ, MASK_XYZ, MASK_R, MASK_P0]
    c1 = 1.0 - ap.beta1 ** t
    c2 = 1.0 - ap.beta2 ** t
    for k in range(5):
        if not (mask & bits[k]):
            continue
        sp = k == 3 and (mask & SOFTPLUS_R)
        p = b[k]
        if sp:
            p = softplus_inv(b[k])
            g[k] = g[k] / (1.0 + np.exp(-p))  # sigmoid(a) dL/dR
        m[k] = ap.beta1 * m[k] + (1.0 - ap.beta1) * g[k]
        v[k] = ap.beta2 * v[k] + (1.0 - ap.beta2) * g[k] * g[k]
        p = p - ap.lr[k] * (m[k] / c1) / (np.sqrt(v[k] / c2) + ap.eps)
        b[k] = softplus(p) if sp else p
    return b, m, v


# --------------------------------------------------------------------------
# the reconstruction loop (Algorithm 1)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Stage:
    level: int
    iterations: int
    grad_mask: int = MASK_ALL
    grow: bool = True
    duplicate: bool = False


def reconstruct(balls, pos, normal, c, fs_mhz, T, factors, y_full, stages,
                zero_grad_mode=KEEP_NEG, zero_grad_level=0, adam_params=None,
                grow_params=None, wmode="clamp", threads=1):
    """Algorithm 1: zero-gradient filtering at level `zero_grad_level`
    (Section 4.2), then for each stage `iterations` times: simulate at the
    stage's sampling level (Section 4.3), L = ||S - y_k||^2, backpropagate,
    one Adam step on the stage's components, then filter/grow (destroy,
    split, and duplicate in the fine stage; Section 4.1). The cloud, the Adam
    moments and the residual handed to the backpropagation are stored in
    float32 between steps, the precision of the arrays that carry the
    method's state; all arithmetic is float64. Returns (balls (5, n) float32, losses, counts)
    where counts[t] is the ball count entering iteration t."""
    ap = adam_params or AdamParams()
    gpar = grow_params or GrowParams()
    b = np.asarray(balls, dtype=np.float32).reshape(5, -1).copy()
    y_full = np.asarray(y_full, dtype=np.float32)
    m = np.zeros((5, b.shape[1]), np.float32)
    v = np.zeros((5, b.shape[1]), np.float32)

    def level_data(k):
        f = factors[k]
        return f / fs_mhz, (T + f - 1) // f, downsample(y_full, f)

    if zero_grad_mode is not None and zero_grad_mode >= 0:
        dt, Tk, yk = level_data(zero_grad_level)
        keep, _, _ = zero_gradient_filter(b, pos, normal, c, dt, Tk, yk, mode=zero_grad_mode,
                                          wmode=wmode, threads=threads)
        b, m, v = b[:, keep], m[:, keep], v[:, keep]
    losses, counts = [], []
    t = 0
    prev_sp = False
    for st in stages:
        dt, Tk, yk = level_data(st.level)
        sp = bool(st.grad_mask & SOFTPLUS_R)
        if sp and not prev_sp:  # the refinement's free variable starts with fresh moments
            m[3] = 0.0
            v[3] = 0.0
        prev_sp = sp
        gmask = st.grad_mask & MASK_ALL
        for _ in range(st.iterations):
            counts.append(b.shape[1])
            S = forward(b, pos, normal, c, dt, Tk, wmode=wmode, threads=threads)
            L, G = loss_and_residual(S, yk)
            losses.append(L)
            g = adjoint(b, pos, normal, c, dt, Tk, G.astype(np.float32), mask=gmask,
                        wmode=wmode, threads=threads)
            t += 1
            nb, nm, nv = adam(b, g, m, v, t, ap, mask=st.grad_mask)
            b, m, v = nb.astype(np.float32), nm.astype(np.float32), nv.astype(np.float32)
            if st.grow:
                gp = dataclasses.replace(gpar, seed=gpar.seed + t, grad_mask=gmask,
                                         duplicate=st.duplicate)
                b, _, ex, _ = grow(b, g.astype(np.float32), np.concatenate([m, v]), gp)
                m, v = ex[:5].copy(), ex[5:].copy()
    return b, np.array(losses), np.array(counts)


def _main():  # pragma: no cover - manual build helper
    print(build(force="--force" in sys.argv))


if __name__ == "__main__":  # pragma: no cover
    _main()
