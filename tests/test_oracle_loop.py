"""Pins of the oracle's optimizer and reconstruction loop (Algorithm 1).

Adam is checked against closed forms that follow from its definition
(Kingma & Ba 2015) over several steps: a constant gradient gives a constant
step once the bias corrections are applied, and a gradient that flips sign
gives a second step of known size that depends on the carried moments.

The loop is checked against compositions of independently pinned parts:
with no stages it returns the zero-gradient filter's survivors, computed
here from a dense system matrix and a numpy block mean; started at the truth
with noise-free traces every level's loss vanishes; one iteration equals the
first Adam step on the backprojected gradient; a softplus stage restarts
the radius moments (Section 4.3).
"""
import dataclasses

import numpy as np

import oracle

C = 1.5          # mm/us
FS = 40.0        # MHz
FACTORS = (4, 2, 1)
T = 256


def _scene(rng, n, M, half=0.6, radius=2.4):
    b = np.stack([rng.uniform(-half, half, n), rng.uniform(-half, half, n),
                  rng.uniform(-half, half, n), rng.uniform(0.05, 0.2, n),
                  rng.uniform(0.0, 1.0, n)])
    u = rng.normal(size=(M, 3))
    u[:, 2] = np.abs(u[:, 2]) + 0.5
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    pos = radius * u
    nrm = -u + 0.15 * rng.normal(size=(M, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return b.astype(np.float32), pos, nrm


def _block_mean(y, f):
    M, Tn = y.shape
    return y.reshape(M, Tn // f, f).mean(axis=2)


def _level(k):
    f = FACTORS[k]
    return f / FS, T // f


NO_GROW = dict(grow=False)


# ------------------------------------------------------------------ Adam

def test_adam_constant_gradient_gives_constant_step():
    """With g_t = g for every t, m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so
    the corrected moments are g and g^2 at every step: each step is
    -lr g / (|g| + eps). A missing or off-by-one bias correction changes the
    early steps by tens of per cent."""
    rng = np.random.default_rng(20)
    b = rng.normal(size=(5, 11))
    g = rng.normal(size=(5, 11))
    ap = oracle.AdamParams()
    lr = np.array(ap.lr)[:, None]
    m = np.zeros((5, 11))
    v = np.zeros((5, 11))
    for t in range(1, 7):
        nb, m, v = oracle.adam(b, g, m, v, t, ap)
        np.testing.assert_allclose(nb - b, -lr * g / (np.abs(g) + ap.eps), rtol=1e-9)
        b = nb


def test_adam_second_step_after_a_sign_flip():
    """Gradients g then -g: m_2 = -(1 - b1)^2 g and v_2 = (1 - b2^2) g^2, so
    m_hat = -(1 - b1) g / (1 + b1) and v_hat = g^2. The second step is
    +lr (1 - b1)/(1 + b1) g / (|g| + eps): about 0.053 lr for b1 = 0.9.
    Moments dropped between the steps would give about 0.74 lr instead."""
    rng = np.random.default_rng(21)
    b0 = rng.normal(size=(5, 13))
    g = rng.normal(size=(5, 13))
    ap = oracle.AdamParams()
    lr = np.array(ap.lr)[:, None]
    z = np.zeros((5, 13))
    b1, m1, v1 = oracle.adam(b0, g, z, z, 1, ap)
    b2, m2, v2 = oracle.adam(b1, -g, m1, v1, 2, ap)
    want = lr * (1 - ap.beta1) / (1 + ap.beta1) * g / (np.abs(g) + ap.eps)
    np.testing.assert_allclose(b2 - b1, want, rtol=1e-8, atol=1e-15)
    np.testing.assert_allclose(m2, -(1 - ap.beta1) ** 2 * g, rtol=1e-12)
    np.testing.assert_allclose(v2, (1 - ap.beta2 ** 2) * g * g, rtol=1e-12)
    # a reset of the moments at step 2 would be visibly different
    reset, _, _ = oracle.adam(b1, -g, z, z, 2, ap)
    assert np.min(np.abs(reset - b1) / np.abs(b2 - b1)) > 10


def test_adam_masked_components_keep_their_moments():
    rng = np.random.default_rng(22)
    b = rng.normal(size=(5, 4))
    g = rng.normal(size=(5, 4))
    m = rng.normal(size=(5, 4))
    v = np.abs(rng.normal(size=(5, 4)))
    nb, nm, nv = oracle.adam(b, g, m, v, 3, oracle.AdamParams(), mask=oracle.MASK_P0)
    np.testing.assert_array_equal(nb[:4], b[:4])
    np.testing.assert_array_equal(nm[:4], m[:4])
    np.testing.assert_array_equal(nv[:4], v[:4])
    assert np.all(nb[4] != b[4])


# ------------------------------------------------------------------ loop

def test_no_stages_returns_the_filter_survivors():
    """Algorithm 1 before its stage loops: zero-gradient filtering at the
    coarsest level. The survivors are {i : -2 <y_k, A e_i> < 0} with A the
    level's dense system matrix (columns = single-ball traces at p0 = 1) and
    y_k the numpy block mean of the record; order is kept."""
    rng = np.random.default_rng(30)
    n, M = 40, 5
    b, pos, nrm = _scene(rng, n, M)
    truth = _scene(rng, 10, M)[0]
    y = oracle.forward(truth, pos, nrm, C, 1.0 / FS, T).astype(np.float32)
    level = 0
    dt, Tk = _level(level)
    yk = _block_mean(y.astype(np.float64), FACTORS[level])
    A = np.zeros((M * Tk, n))
    for i in range(n):
        bi = b.astype(np.float64)
        bi[4] = 0.0
        bi[4, i] = 1.0
        A[:, i] = oracle.forward(bi, pos, nrm, C, dt, Tk).ravel()
    keep = np.nonzero(-2.0 * (A.T @ yk.ravel()) < 0)[0]
    assert 0 < keep.size < n
    out, losses, counts = oracle.reconstruct(b, pos, nrm, C, FS, T, FACTORS, y, [],
                                             zero_grad_level=level)
    np.testing.assert_array_equal(out, b[:, keep])
    assert losses.size == 0 and counts.size == 0


def test_truth_with_exact_traces_has_zero_loss_at_every_level():
    """Started at the truth with noise-free traces, the simulated traces at
    level k equal the block means of the record at every level (cell
    averages are exact block means), so every loss is zero up to the float32
    storage of the record. A stage given the wrong sampling interval or the
    wrong downsampled record would show a loss of the order of |y_k|^2."""
    rng = np.random.default_rng(31)
    truth, pos, nrm = _scene(rng, 25, 6)
    y = oracle.forward(truth, pos, nrm, C, 1.0 / FS, T).astype(np.float32)
    ap = oracle.AdamParams(lr=(0.0, 0.0, 0.0, 0.0, 0.0))
    stages = [oracle.Stage(0, 2, oracle.MASK_P0 | oracle.MASK_R, **NO_GROW),
              oracle.Stage(1, 2, oracle.MASK_P0 | oracle.MASK_R, **NO_GROW),
              oracle.Stage(2, 2, oracle.MASK_ALL, **NO_GROW),
              oracle.Stage(0, 1, oracle.MASK_ALL, **NO_GROW)]
    out, losses, counts = oracle.reconstruct(truth, pos, nrm, C, FS, T, FACTORS, y, stages,
                                             zero_grad_mode=None, adam_params=ap)
    assert losses.size == 7
    np.testing.assert_array_equal(counts, 25)
    np.testing.assert_array_equal(out, truth)
    for it, k in enumerate([0, 0, 1, 1, 2, 2, 0]):
        yk = _block_mean(y.astype(np.float64), FACTORS[k])
        assert losses[it] <= 1e-12 * np.sum(yk * yk), (it, losses[it])
    # the same stages against a record of another cloud do see a loss
    other = _scene(rng, 25, 6)[0]
    y2 = oracle.forward(other, pos, nrm, C, 1.0 / FS, T).astype(np.float32)
    _, l2, _ = oracle.reconstruct(truth, pos, nrm, C, FS, T, FACTORS, y2, stages[:1],
                                  zero_grad_mode=None, adam_params=ap)
    assert l2[0] > 1e-3 * np.sum(_block_mean(y2.astype(np.float64), 4) ** 2)


def _backprojected_gradient(b, pos, nrm, y, level, mask):
    dt, Tk = _level(level)
    yk = _block_mean(y.astype(np.float64), FACTORS[level])
    S = oracle.forward(b, pos, nrm, C, dt, Tk)
    G = (2.0 * (S - yk)).astype(np.float32)
    return oracle.adjoint(b, pos, nrm, C, dt, Tk, G, mask=mask)


def test_one_iteration_is_the_first_adam_step():
    """One iteration of a coarse stage (p0 and R): forward, L, backpropagate,
    and Adam's first step -lr g/(|g| + eps) on p0 and R only; the cloud is
    then stored in float32. x, y, z stay untouched."""
    rng = np.random.default_rng(32)
    b, pos, nrm = _scene(rng, 30, 5)
    y = oracle.forward(_scene(rng, 12, 5)[0], pos, nrm, C, 1.0 / FS, T).astype(np.float32)
    mask = oracle.MASK_P0 | oracle.MASK_R
    level = 1
    g = _backprojected_gradient(b.astype(np.float64), pos, nrm, y, level, mask)
    ap = oracle.AdamParams()
    lr = np.array(ap.lr)[:, None]
    want = (b.astype(np.float64) - lr * g / (np.abs(g) + ap.eps)).astype(np.float32)
    want[:3] = b[:3]
    out, losses, counts = oracle.reconstruct(
        b, pos, nrm, C, FS, T, FACTORS, y, [oracle.Stage(level, 1, mask, **NO_GROW)],
        zero_grad_mode=None)
    assert counts.tolist() == [30] and losses.size == 1
    assert np.count_nonzero(g[3:]) > 20
    np.testing.assert_array_equal(out, want)


def test_softplus_stage_restarts_the_radius_moments():
    """Section 4.3's refinement: when a softplus stage begins, the free
    variable a = softplus^-1(R) starts with zero moments while the step count
    t runs on. At t = 2 its step is lr (g_a / (1 + b1)) / (|g_a| / sqrt(1 + b2)
    + eps), g_a = sigmoid(a) dL/dR; p0 keeps its moments from the first stage."""
    rng = np.random.default_rng(33)
    b, pos, nrm = _scene(rng, 20, 5)
    y = oracle.forward(_scene(rng, 8, 5)[0], pos, nrm, C, 1.0 / FS, T).astype(np.float32)
    coarse = oracle.MASK_P0 | oracle.MASK_R
    ap = oracle.AdamParams(lr=(1e-3, 1e-3, 1e-3, 2e-2, 1e-2))
    s1 = oracle.Stage(2, 1, coarse, **NO_GROW)
    s2 = oracle.Stage(2, 1, coarse | oracle.SOFTPLUS_R, **NO_GROW)
    b1, _, _ = oracle.reconstruct(b, pos, nrm, C, FS, T, FACTORS, y, [s1],
                                  zero_grad_mode=None, adam_params=ap)
    b2, _, _ = oracle.reconstruct(b, pos, nrm, C, FS, T, FACTORS, y, [s1, s2],
                                  zero_grad_mode=None, adam_params=ap)
    g1 = _backprojected_gradient(b1.astype(np.float64), pos, nrm, y, 2, coarse)
    a = oracle.softplus_inv(b1[3].astype(np.float64))
    ga = g1[3] / (1.0 + np.exp(-a))
    b1c, b2c = ap.beta1, ap.beta2
    step = ap.lr[3] * (ga / (1 + b1c)) / (np.abs(ga) / np.sqrt(1 + b2c) + ap.eps)
    want = oracle.softplus(a - step).astype(np.float32)
    np.testing.assert_allclose(b2[3], want, rtol=2e-7, atol=0)
    # carrying stage 1's radius moments (taken in R, not a) would land elsewhere
    g0 = _backprojected_gradient(b.astype(np.float64), pos, nrm, y, 2, coarse)
    m = (1 - b1c) * g0[3]
    v = (1 - b2c) * g0[3] ** 2
    m = b1c * m + (1 - b1c) * ga
    v = b2c * v + (1 - b2c) * ga * ga
    carried = oracle.softplus(a - ap.lr[3] * (m / (1 - b1c ** 2)) /
                              (np.sqrt(v / (1 - b2c ** 2)) + ap.eps))
    assert np.max(np.abs(carried - want) / want) > 1e-3


def test_growth_in_the_loop_uses_the_step_count_as_seed():
    """Growth after iteration t draws its split directions from seed
    `GrowParams.seed + t`, so one iteration with splitting equals Adam's
    first step followed by `grow` with seed + 1."""
    rng = np.random.default_rng(34)
    b, pos, nrm = _scene(rng, 16, 4)
    b[3, :5] = 0.35   # above R_max: split
    y = oracle.forward(_scene(rng, 6, 4)[0], pos, nrm, C, 1.0 / FS, T).astype(np.float32)
    mask = oracle.MASK_P0 | oracle.MASK_R
    ap = oracle.AdamParams(lr=(0.0, 0.0, 0.0, 0.0, 0.0))
    gpar = oracle.GrowParams(seed=100)
    out, _, counts = oracle.reconstruct(b, pos, nrm, C, FS, T, FACTORS, y,
                                        [oracle.Stage(0, 1, mask, grow=True)],
                                        zero_grad_mode=None, adam_params=ap,
                                        grow_params=gpar)
    g = _backprojected_gradient(b.astype(np.float64), pos, nrm, y, 0, mask).astype(np.float32)
    want = oracle.grow(b, g, np.zeros((10, 16), np.float32),
                       dataclasses.replace(gpar, seed=101, grad_mask=mask))[0]
    assert out.shape[1] > 16
    np.testing.assert_array_equal(out, want)


# ------------------------------------------------------- spatial ordering

def test_morton_key_of_the_cube_corners_and_bits():
    """The corners of a 4 mm cube: a coordinate at the far side quantises to
    1023 (floor(4 * 1024 / 4) clamped), so corner (x, y, z) in {0, 1}^3 gets
    all ten bits of each set axis, x lowest: the octal digits of its key are
    all x + 2y + 4z. A point halfway along x alone is q_x = 512: bit 27."""
    corners = [(x, y, z) for z in (0, 1) for y in (0, 1) for x in (0, 1)]
    b = np.zeros((5, 8), np.float32)
    b[:3] = 4.0 * np.array(corners, np.float32).T
    want = [int(str(x + 2 * y + 4 * z) * 10, 8) for x, y, z in corners]
    np.testing.assert_array_equal(oracle.morton_key(b), want)
    b2 = np.zeros((5, 3), np.float32)
    b2[:3, 1] = [4.0, 4.0, 4.0]
    b2[:3, 2] = [2.0, 0.0, 0.0]
    k = oracle.morton_key(b2)
    assert k[0] == 0 and k[1] == (1 << 30) - 1 and k[2] == 1 << 27


def test_morton_permutation_is_stable_and_orders_the_keys():
    rng = np.random.default_rng(40)
    b = np.zeros((5, 500), np.float32)
    b[:3] = rng.integers(0, 4, size=(3, 500)).astype(np.float32)  # many equal keys
    b[3:] = rng.uniform(size=(2, 500))
    perm = oracle.morton_permutation(b)
    np.testing.assert_array_equal(np.sort(perm), np.arange(500))
    k = oracle.morton_key(b)[perm]
    assert np.all(np.diff(k) >= 0)
    for key in np.unique(k):  # equal keys keep their index order
        same = perm[k == key]
        assert np.all(np.diff(same) > 0)
    # the order depends on the centres only, and brute force agrees
    brute = sorted(range(500), key=lambda i: (int(oracle.morton_key(b)[i]), i))
    np.testing.assert_array_equal(perm, brute)
