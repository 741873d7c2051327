"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against something it does not compute itself:
exact integration of the N-wave in the time domain, the textbook N-wave
peak, closed-form orientation scaling, linearity, telescoping, exact level
consistency of block-mean downsampling, the adjoint identity, a dense
brute-force system matrix, complex-step derivatives of an independent
complex-arithmetic forward, central finite differences, numpy routines and a
published SplitMix64 test vector.
"""
import math
import os

import numpy as np
import pytest

import oracle

C = 1.5          # mm/us
FS = 40.0        # MHz
DT = 1.0 / FS    # us
H = C * DT       # mm per sample


def one_sensor(pos=(0.0, 0.0, 0.0), normal=(0.0, 0.0, 1.0)):
    return np.array([pos], float), np.array([normal], float)


def nwave_cell_average(d, R, p0, w, dt, T, c=C):
    """Cell averages of p(t) = p0 w (d - c t) / (2 d) on |d - c t| < R,
    integrated exactly in the time domain: the integrand is linear on the
    support, so its integral over [a, b] is (b - a) times its value at the
    midpoint."""
    out = np.zeros(T)
    lo, hi = (d - R) / c, (d + R) / c
    for j in range(T):
        a, b = max(j * dt, lo), min((j + 1) * dt, hi)
        if b > a:
            tm = 0.5 * (a + b)
            out[j] = p0 * w * (d - c * tm) / (2 * d) * (b - a) / dt
    return out


def balls_array(rows):
    return np.array(rows, float).T.copy()  # (5, n)


# ---------------------------------------------------------------- forward

@pytest.mark.parametrize("d,R,p0", [(20.0, 0.13, 0.7), (7.31, 0.05, 1.0),
                                    (33.3333, 0.4, 0.25), (12.0, 0.0374, 2.0),
                                    (3.0, 1.7, 0.5)])
def test_single_ball_matches_time_domain_integral(d, R, p0):
    pos, nrm = one_sensor()
    b = balls_array([[0.0, 0.0, d, R, p0]])   # straight ahead: w = 1
    T = int((d + R) / H) + 8
    S = oracle.forward(b, pos, nrm, C, DT, T)[0]
    ref = nwave_cell_average(d, R, p0, 1.0, DT, T)
    assert np.max(np.abs(S - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    assert np.count_nonzero(ref) > 0


def test_single_ball_matches_midpoint_quadrature():
    d, R, p0 = 15.2, 0.17, 0.9
    pos, nrm = one_sensor()
    b = balls_array([[0.0, 0.0, d, R, p0]])
    T = int((d + R) / H) + 4
    S = oracle.forward(b, pos, nrm, C, DT, T)[0]
    nq = 20000
    ref = np.zeros(T)
    for j in range(T):
        t = (j + (np.arange(nq) + 0.5) / nq) * DT
        e = d - C * t
        p = np.where(np.abs(e) < R, p0 * e / (2 * d), 0.0)
        ref[j] = p.mean()
    # a jump of height p0 R / (2 d) inside a cell costs at most that / nq
    assert np.max(np.abs(S - ref)) < 2 * p0 * R / (2 * d) / nq


def test_fine_sampling_tends_to_point_nwave_peak():
    """As dt -> 0 the cell average tends to the point-sampled N-wave, whose
    extremes are +-p0 w R / (2 d) (uniform sphere, textbook)."""
    d, R, p0 = 18.0, 0.2, 1.0
    pos, nrm = one_sensor()
    b = balls_array([[0.0, 0.0, d, R, p0]])
    fs = 4000.0
    dt = 1.0 / fs
    T = int((d + R) / (C * dt)) + 4
    S = oracle.forward(b, pos, nrm, C, dt, T)[0]
    peak = p0 * R / (2 * d)
    assert abs(S.max() - peak) < 2e-3 * peak
    assert abs(S.min() + peak) < 2e-3 * peak
    # positive lobe first (d - c t > 0 early), negative after
    assert np.argmax(S) < np.argmin(S)


@pytest.mark.parametrize("theta_deg", [0.0, 25.0, 60.0, 89.0, 91.0, 135.0])
def test_orientation_weight_scales_as_cosine(theta_deg):
    d, R, p0 = 20.0, 0.15, 1.0
    th = math.radians(theta_deg)
    ball = [0.0, d * math.sin(th), d * math.cos(th), R, p0]
    pos, nrm = one_sensor()
    T = int((d + R) / H) + 4
    S = oracle.forward(balls_array([ball]), pos, nrm, C, DT, T)[0]
    base = nwave_cell_average(d, R, p0, 1.0, DT, T)
    cos = math.cos(th)
    np.testing.assert_allclose(S, max(cos, 0.0) * base, atol=1e-14)
    Sc = oracle.forward(balls_array([ball]), pos, nrm, C, DT, T, wmode="cos")[0]
    np.testing.assert_allclose(Sc, cos * base, atol=1e-14)
    Sn = oracle.forward(balls_array([ball]), pos, nrm, C, DT, T, wmode="none")[0]
    np.testing.assert_allclose(Sn, base, atol=1e-14)


def _random_scene(rng, n, M, half=2.0, radius=20.0):
    b = np.stack([rng.uniform(-half, half, n), rng.uniform(-half, half, n),
                  rng.uniform(-half, half, n), rng.uniform(0.05, 0.2, n),
                  rng.uniform(0.0, 1.0, n)])
    u = rng.normal(size=(M, 3))
    u[:, 2] = np.abs(u[:, 2]) + 0.5
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    pos = radius * u
    nrm = -u + 0.15 * rng.normal(size=(M, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return b, pos, nrm


def test_linearity_and_superposition():
    rng = np.random.default_rng(11)
    b, pos, nrm = _random_scene(rng, 40, 6)
    T = 800
    S = oracle.forward(b, pos, nrm, C, DT, T)
    b2 = b.copy()
    b2[4] *= 2.5
    np.testing.assert_allclose(oracle.forward(b2, pos, nrm, C, DT, T), 2.5 * S,
                               rtol=1e-12, atol=1e-15)
    Sa = oracle.forward(b[:, :17], pos, nrm, C, DT, T)
    Sb = oracle.forward(b[:, 17:], pos, nrm, C, DT, T)
    np.testing.assert_allclose(Sa + Sb, S, rtol=1e-12, atol=1e-14)


def test_each_ball_trace_has_zero_mean():
    """The N-wave integrates to zero; with the whole window inside the
    record the cell sums telescope to exactly zero."""
    rng = np.random.default_rng(5)
    b, pos, nrm = _random_scene(rng, 25, 5)
    S = oracle.forward(b, pos, nrm, C, DT, 900)
    scale = np.max(np.abs(S))
    assert scale > 0
    assert np.max(np.abs(S.sum(axis=1))) < 1e-12 * scale * S.shape[1]


@pytest.mark.parametrize("f", [2, 4, 16])
def test_levels_are_block_means_of_the_finest_level(f):
    """Section 4.3: dt_k = f dt and T_k = T / f. Under the cell-average
    reading a coarse cell is exactly the mean of its f fine cells."""
    rng = np.random.default_rng(7)
    b, pos, nrm = _random_scene(rng, 30, 4)
    T = 1024
    S1 = oracle.forward(b, pos, nrm, C, DT, T)
    Sf = oracle.forward(b, pos, nrm, C, f * DT, T // f)
    np.testing.assert_allclose(Sf, oracle.downsample(S1, f), rtol=1e-10,
                               atol=1e-13 * np.max(np.abs(S1)))


def test_downsample_is_numpy_block_mean():
    rng = np.random.default_rng(3)
    y = rng.normal(size=(5, 64))
    np.testing.assert_allclose(oracle.downsample(y, 4), y.reshape(5, 16, 4).mean(axis=2),
                               rtol=1e-14, atol=1e-15)
    # ragged record: zero padded to a multiple of f
    yr = rng.normal(size=(3, 30))
    pad = np.concatenate([yr, np.zeros((3, 2))], axis=1)
    np.testing.assert_allclose(oracle.downsample(yr, 4), pad.reshape(3, 8, 4).mean(axis=2),
                               rtol=1e-14, atol=1e-15)


def test_record_clipping_and_inside_pairs():
    pos, nrm = one_sensor()
    # beyond the record: nothing
    far = balls_array([[0.0, 0.0, 50.0, 0.1, 1.0]])
    assert np.all(oracle.forward(far, pos, nrm, C, DT, 100) == 0)
    # sensor inside the ball: contributes nothing and is counted
    inside = balls_array([[0.0, 0.0, 0.05, 0.1, 1.0], [0.0, 0.0, 2.0, 0.1, 1.0]])
    S, cnt = oracle.forward(inside, pos, nrm, C, DT, 100, return_inside=True)
    assert cnt == 1
    ref = oracle.forward(inside[:, 1:], pos, nrm, C, DT, 100)
    np.testing.assert_array_equal(S, ref)


def test_window_covers_every_nonzero_cell():
    """Brute force over every cell of the record, in pure Python, with the
    clamp form of the cell integral: equal to the windowed oracle."""
    rng = np.random.default_rng(2)
    b, pos, nrm = _random_scene(rng, 4, 2)
    T = 700
    S = oracle.forward(b, pos, nrm, C, DT, T)
    ref = np.zeros((2, T))
    for m in range(2):
        for i in range(4):
            dv = b[:3, i] - pos[m]
            d = math.sqrt(float(dv @ dv))
            w = max(0.0, float(nrm[m] @ dv) / d)
            R = b[3, i]
            for j in range(T):
                ea, eb = d - j * H, d - (j + 1) * H
                qa, qb = min(max(ea, -R), R), min(max(eb, -R), R)
                ref[m, j] += b[4, i] * w * (qa * qa - qb * qb) / (4 * d * H)
    np.testing.assert_allclose(S, ref, rtol=1e-12, atol=1e-16)


# ---------------------------------------------------------------- adjoint

def test_adjoint_identity_for_amplitudes():
    """<A x, y> = <x, A^T y> with A = dS/dp0 (S is linear in p0)."""
    rng = np.random.default_rng(21)
    b, pos, nrm = _random_scene(rng, 60, 7)
    T = 900
    x = rng.normal(size=60)
    y = rng.normal(size=(7, T))
    bx = b.copy()
    bx[4] = x
    Ax = oracle.forward(bx, pos, nrm, C, DT, T)
    ATy = oracle.adjoint(b, pos, nrm, C, DT, T, y, mask=oracle.MASK_P0)[4]
    lhs, rhs = float(np.sum(Ax * y)), float(x @ ATy)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.sum(np.abs(Ax * y)))


def test_dense_system_matrix_brute_force():
    rng = np.random.default_rng(4)
    n, M, T = 6, 3, 64
    b, pos, nrm = _random_scene(rng, n, M, half=0.5, radius=1.0)
    A = np.zeros((M * T, n))
    for i in range(n):
        bi = b.copy()
        bi[4] = 0.0
        bi[4, i] = 1.0
        A[:, i] = oracle.forward(bi, pos, nrm, C, DT, T).ravel()
    S = oracle.forward(b, pos, nrm, C, DT, T)
    np.testing.assert_allclose(S.ravel(), A @ b[4], rtol=1e-12, atol=1e-15)
    G = rng.normal(size=(M, T))
    g = oracle.adjoint(b, pos, nrm, C, DT, T, G, mask=oracle.MASK_P0)[4]
    np.testing.assert_allclose(g, A.T @ G.ravel(), rtol=1e-12, atol=1e-14)
    assert np.count_nonzero(A) > 0


def _complex_forward(b, pos, nrm, T, wmode="clamp"):
    """Pure-Python forward in complex arithmetic for complex-step
    differentiation: clamps and window membership are decided on the real
    parts, the arithmetic is carried in complex numbers."""
    S = np.zeros((pos.shape[0], T), dtype=complex)
    for m in range(pos.shape[0]):
        for i in range(b.shape[1]):
            dv = [b[k, i] - pos[m, k] for k in range(3)]
            d = (dv[0] ** 2 + dv[1] ** 2 + dv[2] ** 2) ** 0.5
            R, p0 = b[3, i], b[4, i]
            cosv = (nrm[m, 0] * dv[0] + nrm[m, 1] * dv[1] + nrm[m, 2] * dv[2]) / d
            if wmode == "none":
                w = 1.0
            elif wmode == "cos":
                w = cosv
            else:
                w = cosv if cosv.real > 0 else 0.0
            for j in range(T):
                ea, eb = d - j * H, d - (j + 1) * H
                qa = R if ea.real > R.real else (-R if ea.real < -R.real else ea)
                qb = R if eb.real > R.real else (-R if eb.real < -R.real else eb)
                S[m, j] += p0 * w * (qa * qa - qb * qb) / (4 * d * H)
    return S


@pytest.mark.parametrize("wmode", ["clamp", "cos", "none"])
def test_gradients_match_complex_step(wmode):
    rng = np.random.default_rng(8)
    n, M, T = 2, 3, 48
    b, pos, nrm = _random_scene(rng, n, M, half=0.3, radius=0.9)
    b[3] = rng.uniform(0.06, 0.2, n)
    y = rng.normal(size=(M, T)) * 0.05
    S = oracle.forward(b, pos, nrm, C, DT, T, wmode=wmode)
    G = 2 * (S - y)
    g = oracle.adjoint(b, pos, nrm, C, DT, T, G, wmode=wmode)
    hstep = 1e-30
    for k in range(5):
        for i in range(n):
            bc = b.astype(complex)
            bc[k, i] += 1j * hstep
            Sc = _complex_forward(bc, pos, nrm, T, wmode)
            Lc = np.sum((Sc - y) ** 2)
            ref = Lc.imag / hstep
            assert abs(g[k, i] - ref) <= 1e-9 * max(1.0, abs(ref)) * 1e-0 + 1e-12, (k, i)


def _near_kink(b, pos, hstep):
    """True when some cell boundary sits within 2 hstep of d +- R for any
    pair, where the piecewise-quadratic loss has a kink."""
    for m in range(pos.shape[0]):
        for i in range(b.shape[1]):
            d = np.linalg.norm(b[:3, i] - pos[m])
            for e in (d - b[3, i], d + b[3, i]):
                r = (e / H) - round(e / H)
                if abs(r * H) < 2 * hstep * 4:
                    return True
    return False


def test_gradients_match_central_differences():
    rng = np.random.default_rng(12)
    n, M, T = 20, 6, 900
    b, pos, nrm = _random_scene(rng, n, M)
    y = oracle.forward(_random_scene(rng, n, M)[0], pos, nrm, C, DT, T)
    S = oracle.forward(b, pos, nrm, C, DT, T)
    g = oracle.adjoint(b, pos, nrm, C, DT, T, 2 * (S - y))
    # FP64 allows a step well below 1e-4 mm: the truncation error h^2 L'''/6
    # of a 1e-4 step already reaches 1e-4 of the smaller radius gradients
    hstep = 1e-5
    checked = 0
    for i in range(n):
        bi = b[:, i:i + 1]
        if _near_kink(bi, pos, hstep):
            continue
        for k in range(5):
            bp, bm = b.copy(), b.copy()
            bp[k, i] += hstep
            bm[k, i] -= hstep
            Lp = np.sum((oracle.forward(bp, pos, nrm, C, DT, T) - y) ** 2)
            Lm = np.sum((oracle.forward(bm, pos, nrm, C, DT, T) - y) ** 2)
            fd = (Lp - Lm) / (2 * hstep)
            scale = max(abs(fd), 1e-3 * np.max(np.abs(g[k])), 1e-12)
            assert abs(g[k, i] - fd) <= 1e-4 * scale, (k, i, g[k, i], fd)
            checked += 1
    assert checked >= 50


def test_grad_mask_zeroes_inactive_components():
    rng = np.random.default_rng(1)
    b, pos, nrm = _random_scene(rng, 10, 4)
    G = rng.normal(size=(4, 800))
    full = oracle.adjoint(b, pos, nrm, C, DT, 800, G)
    coarse = oracle.adjoint(b, pos, nrm, C, DT, 800, G, mask=oracle.MASK_P0 | oracle.MASK_R)
    np.testing.assert_array_equal(coarse[:3], 0.0)
    np.testing.assert_array_equal(coarse[3:], full[3:])


# ------------------------------------------------------- zero-grad filter

def test_zero_gradient_filter_is_sign_of_dense_backprojection():
    """Section 4.2: g_i = dL/dp0_i at p0 = 0 equals -2 <y, A e_i>; the kept set
    is {g < 0} (Algorithm 1), {g <= 0} (equations of Section 4.2) or {g != 0}."""
    rng = np.random.default_rng(9)
    n, M, T = 30, 4, 128
    b, pos, nrm = _random_scene(rng, n, M, half=0.6, radius=2.2)
    truth = _random_scene(rng, 8, M, half=0.6, radius=2.2)[0]
    y = oracle.forward(truth, pos, nrm, C, DT, T)
    A = np.zeros((M * T, n))
    for i in range(n):
        bi = b.copy()
        bi[4] = 0.0
        bi[4, i] = 1.0
        A[:, i] = oracle.forward(bi, pos, nrm, C, DT, T).ravel()
    g_ref = -2.0 * (A.T @ y.ravel())
    keep, g, amb = oracle.zero_gradient_filter(b, pos, nrm, C, DT, T, y)
    np.testing.assert_allclose(g, g_ref, rtol=1e-10, atol=1e-14)
    np.testing.assert_array_equal(keep, np.nonzero(g_ref < 0)[0])
    keep2, _, _ = oracle.zero_gradient_filter(b, pos, nrm, C, DT, T, y, mode=oracle.KEEP_NONPOS)
    np.testing.assert_array_equal(keep2, np.nonzero(g_ref <= 0)[0])
    keep3, _, _ = oracle.zero_gradient_filter(b, pos, nrm, C, DT, T, y, mode=oracle.DROP_ZERO)
    np.testing.assert_array_equal(keep3, np.nonzero(g_ref != 0)[0])
    assert 0 < keep.size < n
    assert amb.size == 0


def test_zero_gradient_filter_keeps_true_sources():
    """Balls placed on the true sources have negative zero-pressure gradient
    (their pressure would rise from zero), the premise of Section 4.2."""
    rng = np.random.default_rng(10)
    M, T = 16, 1024
    _, pos, nrm = _random_scene(rng, 1, M)
    truth = _random_scene(rng, 12, M)[0]
    truth[4] = rng.uniform(0.5, 1.0, 12)
    y = oracle.forward(truth, pos, nrm, C, DT, T)
    keep, g, _ = oracle.zero_gradient_filter(truth, pos, nrm, C, DT, T, y)
    assert keep.size == 12 and np.all(g < 0)


# ------------------------------------------------------------ growth, rng

def test_splitmix64_published_vector():
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")
    want = [int(s) for s in open(path) if s.strip() and not s.startswith("#")]
    assert [oracle.splitmix64_at(1234567, k) for k in range(5)] == want


def test_split_direction_is_unit_and_deterministic():
    v = np.array([oracle.split_direction(42, i) for i in range(200)])
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, rtol=1e-14)
    assert np.all(np.abs(v.mean(axis=0)) < 0.15)
    np.testing.assert_array_equal(v[17], oracle.split_direction(42, 17))
    assert not np.allclose(v[17], oracle.split_direction(43, 17))


def test_growth_rules():
    b = np.array([
        # x    y    z    R     p0
        [0.0, 0.0, 0.0, 0.10, 0.50],   # kept
        [1.0, 0.0, 0.0, 0.50, 0.80],   # split (R > 0.3)
        [2.0, 0.0, 0.0, 0.10, 1e-4],   # destroyed (p0 < 1e-3)
        [3.0, 0.0, 0.0, 0.01, 0.90],   # destroyed (R < 0.02)
        [4.0, 0.0, 0.0, 0.10, 0.70],   # pruned (all grads exactly 0)
        [5.0, 0.0, 0.0, 0.10, 0.70],   # duplicated
    ], np.float32).T
    g = np.array([[1, 1, 1, 1, 1], [1, 1, 1, 1, 1], [1, 1, 1, 1, 1], [1, 1, 1, 1, 1],
                  [0, 0, 0, 0, 0], [3, 4, 0, 1, 1]], np.float32).T
    ex = np.arange(12, dtype=np.float32).reshape(2, 6) + 1
    gp = oracle.GrowParams(seed=7, duplicate=True, g_dup=4.9)
    nb, ng, ne, counts = oracle.grow(b, g, ex, gp)
    np.testing.assert_array_equal(counts, [1, 2, 0, 0, 0, 2])
    assert nb.shape == (5, 5)
    # stable order: kept, two children, duplicated parent, its clone
    np.testing.assert_array_equal(nb[:, 0], b[:, 0])
    np.testing.assert_array_equal(nb[:, 3], b[:, 5])
    ch = nb[:, 1:3].astype(np.float64)
    R = 0.5
    np.testing.assert_allclose(2 * ch[3] ** 3, R ** 3, rtol=1e-6)           # volume kept
    np.testing.assert_allclose(ch[:3].mean(axis=1), b[:3, 1], atol=1e-6)   # centroid kept
    np.testing.assert_allclose(np.linalg.norm(ch[:3, 0] - ch[:3, 1]), R, rtol=1e-6)
    np.testing.assert_array_equal(ch[4], [np.float32(0.8)] * 2)
    v = oracle.split_direction(7, 5)
    np.testing.assert_allclose(nb[:3, 4], b[:3, 5] + 0.05 * v, atol=1e-6)
    # gradients and carried state: kept balls keep theirs, new balls get zeros
    np.testing.assert_array_equal(ng[:, 0], g[:, 0])
    np.testing.assert_array_equal(ng[:, 1:3], 0)
    np.testing.assert_array_equal(ne[:, 0], ex[:, 0])
    np.testing.assert_array_equal(ne[:, 3], ex[:, 5])
    np.testing.assert_array_equal(ne[:, 4], 0)


def test_growth_prune_respects_grad_mask():
    b = np.array([[0, 0, 0, 0.1, 0.5]], np.float32).T
    g = np.array([[2.0, 0, 0, 0, 0]], np.float32).T   # only x-gradient nonzero
    coarse = oracle.GrowParams(grad_mask=oracle.MASK_P0 | oracle.MASK_R)
    assert oracle.grow(b, g, np.zeros((0, 1)), coarse)[0].shape[1] == 0
    fine = oracle.GrowParams(grad_mask=oracle.MASK_ALL)
    assert oracle.grow(b, g, np.zeros((0, 1)), fine)[0].shape[1] == 1


def test_adam_first_step_is_signed_learning_rate():
    rng = np.random.default_rng(0)
    b = rng.normal(size=(5, 9))
    g = rng.normal(size=(5, 9))
    ap = oracle.AdamParams()
    nb, m, v = oracle.adam(b, g, np.zeros((5, 9)), np.zeros((5, 9)), 1, ap)
    lr = np.array(ap.lr)[:, None]
    # at t = 1 the bias corrections make m_hat = g and v_hat = g^2 exactly
    np.testing.assert_allclose(nb - b, -lr * g / (np.abs(g) + ap.eps), rtol=1e-9)
    assert np.all(np.abs(np.abs(nb - b) - lr) < 1e-4 * lr + ap.eps / np.abs(g) * lr)
    nb2, _, _ = oracle.adam(b, g, np.zeros((5, 9)), np.zeros((5, 9)), 1, ap,
                            mask=oracle.MASK_P0 | oracle.MASK_R)
    np.testing.assert_array_equal(nb2[:3], b[:3])


# ----------------------------------------------- softplus refinement (4.3)

def test_softplus_inverse_and_sigmoid_identity():
    R = np.array([1e-6, 1e-3, 0.05, 0.3, 1.0, 5.0, 30.0])
    a = oracle.softplus_inv(R)
    np.testing.assert_allclose(oracle.softplus(a), R, rtol=1e-12)
    # sigmoid(softplus^-1(R)) = 1 - exp(-R)
    np.testing.assert_allclose(1.0 / (1.0 + np.exp(-a)), -np.expm1(-R), rtol=1e-12)
    np.testing.assert_allclose(oracle.softplus(np.array([-800.0, 0.0, 800.0])),
                               [0.0, np.log(2.0), 800.0], rtol=1e-15, atol=1e-300)


def test_adam_softplus_first_step_and_positivity():
    rng = np.random.default_rng(3)
    b = np.abs(rng.normal(size=(5, 7))) + 0.01
    g = rng.normal(size=(5, 7))
    ap = oracle.AdamParams(lr=(1e-3, 1e-3, 1e-3, 0.05, 1e-2))
    mask = oracle.MASK_ALL | oracle.SOFTPLUS_R
    nb, _, _ = oracle.adam(b, g, np.zeros((5, 7)), np.zeros((5, 7)), 1, ap, mask=mask)
    step = ap.lr[3] * np.sign(g[3])  # first Adam step of the free variable: lr * sign
    np.testing.assert_allclose(nb[3], oracle.softplus(oracle.softplus_inv(b[3]) - step),
                               rtol=1e-6)
    # a step far larger than R still leaves R positive
    huge = oracle.AdamParams(lr=(0, 0, 0, 20.0, 0))
    nb2, _, _ = oracle.adam(b, np.abs(g) + 1, np.zeros((5, 7)), np.zeros((5, 7)), 1, huge,
                            mask=mask)
    assert np.all(nb2[3] > 0)
    np.testing.assert_allclose(nb2[3], oracle.softplus(oracle.softplus_inv(b[3]) - 20.0),
                               rtol=1e-6)


def test_softplus_chain_rule_matches_finite_difference():
    """dL/da = sigmoid(a) dL/dR through the radiator (oracle forward and
    adjoint), against a central difference in a."""
    rng = np.random.default_rng(4)
    b, pos, nrm = _random_scene(rng, 6, 4)
    T = 900
    y = oracle.forward(_random_scene(rng, 6, 4)[0], pos, nrm, C, DT, T)
    S = oracle.forward(b, pos, nrm, C, DT, T)
    gR = oracle.adjoint(b, pos, nrm, C, DT, T, 2 * (S - y), mask=oracle.MASK_R)[3]
    a = oracle.softplus_inv(b[3])
    h = 1e-6
    for i in range(6):
        bp, bm = b.copy(), b.copy()
        bp[3, i] = oracle.softplus(a[i] + h)
        bm[3, i] = oracle.softplus(a[i] - h)
        fd = (np.sum((oracle.forward(bp, pos, nrm, C, DT, T) - y) ** 2) -
              np.sum((oracle.forward(bm, pos, nrm, C, DT, T) - y) ** 2)) / (2 * h)
        an = gR[i] / (1.0 + np.exp(-a[i]))
        assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-8), (i, fd, an)
