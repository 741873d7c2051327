"""Pins of the CNN oracle: conv3d against scipy's correlate, identity and
shift kernels, linearity; bf16 rounding against torch's conversion."""
import numpy as np
import pytest

from oracle import cnn


def test_conv3d_matches_scipy_correlate():
    from scipy.ndimage import correlate

    rng = np.random.default_rng(0)
    x = rng.normal(size=(5, 6, 7, 1))
    k = rng.normal(size=(3, 3, 3))
    w = k.reshape(1, 27, 1)
    ref = correlate(x[..., 0], k, mode="constant", cval=0.0)
    np.testing.assert_allclose(cnn.conv3d(x, w)[..., 0], ref, rtol=1e-12, atol=1e-12)


def test_conv3d_identity_shift_and_linearity():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(4, 5, 6, 3))
    w = np.zeros((3, 27, 3))
    w[:, 13, :] = np.eye(3)  # centre tap
    np.testing.assert_allclose(cnn.conv3d(x, w), x, atol=0)
    w = np.zeros((3, 27, 3))
    w[:, 14, :] = np.eye(3)  # tap (dz, dy, dx) = (0, 0, +1): out[x] = in[x + 1]
    out = cnn.conv3d(x, w)
    np.testing.assert_allclose(out[:, :, :-1], x[:, :, 1:], atol=0)
    np.testing.assert_allclose(out[:, :, -1], 0.0, atol=0)
    w1, w2 = rng.normal(size=(2, 4, 27, 3))
    np.testing.assert_allclose(cnn.conv3d(x, w1 + w2), cnn.conv3d(x, w1) + cnn.conv3d(x, w2),
                               rtol=1e-12, atol=1e-12)
    b = rng.normal(size=4)
    np.testing.assert_allclose(cnn.conv3d(x, w1, b) - cnn.conv3d(x, w1), np.broadcast_to(b, (4, 5, 6, 4)),
                               rtol=1e-12, atol=1e-12)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    a = (rng.normal(size=10000) * 10.0 ** rng.integers(-5, 5, size=10000)).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(cnn.bf16_round(a), ref)


def test_das_single_sensor_impulse_closed_form():
    # one sensor at the origin looking along +z, a unit value in cell j: the
    # volume is w times the hat function of |tau/dt - 1/2 - j| on the shell
    pos = np.array([[0.0, 0.0, 0.0]])
    nrm = np.array([[0.0, 0.0, 1.0]])
    c, dt, T, j = 1.5, 0.1, 64, 20
    y = np.zeros((1, T))
    y[0, j] = 1.0
    origin, h, dims = (-1.6, -1.6, 0.2), 0.2, (16, 16, 16)
    vol = cnn.das_volume(y, pos, nrm, c, dt, origin, h, dims)
    cx = origin[0] + (np.arange(16) + 0.5) * h
    cz = origin[2] + (np.arange(16) + 0.5) * h
    Z, Y, X = np.meshgrid(cz, cx, cx, indexing="ij")
    d = np.sqrt(X * X + Y * Y + Z * Z)
    hat = np.maximum(1.0 - np.abs(d / (c * dt) - 0.5 - j), 0.0)
    np.testing.assert_allclose(vol, (Z / d) * hat, rtol=1e-12, atol=1e-14)


def test_das_linear_in_traces_and_weight_modes():
    rng = np.random.default_rng(3)
    pos = rng.normal(size=(5, 3)) * 10
    nrm = -pos / np.linalg.norm(pos, axis=1, keepdims=True)
    y1, y2 = rng.normal(size=(2, 5, 128))
    args = (1.5, 0.05, (-2.0, -2.0, -2.0), 0.5, (8, 8, 8))
    a = cnn.das_volume(y1 + 2 * y2, pos, nrm, *args)
    b = cnn.das_volume(y1, pos, nrm, *args) + 2 * cnn.das_volume(y2, pos, nrm, *args)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    # with w = 1 a constant trace gives the sensor count wherever every delay
    # falls inside the record
    ones = np.ones((5, 4096))
    v = cnn.das_volume(ones, pos, nrm, 1.5, 0.05, (-2.0, -2.0, -2.0), 0.5, (8, 8, 8),
                       wmode="none")
    np.testing.assert_allclose(v, 5.0, rtol=1e-12)


def random_params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for name, shape in cnn.PARAM_SHAPES:
        fan = shape[1] * shape[2] if len(shape) == 3 else shape[-1]
        out.append(rng.normal(size=shape).reshape(-1) * scale * np.sqrt(2.0 / fan)
                   if name.startswith("w") else rng.normal(size=shape) * 0.1)
    return np.concatenate(out).astype(np.float32)


def test_cnn_forward_two_implementations_agree():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    vol = rng.normal(size=(5, 6, 7))
    p = random_params(1)
    a = cnn.cnn_forward(p, vol, round_activations=False)
    # the same network through torch's conv3d (independent of cnn.conv3d)
    import torch.nn.functional as F

    P = cnn.unpack_params(p)
    x = torch.from_numpy(cnn.scaled_input(vol)[..., 0])[None, None]
    h = x
    for k in (1, 2, 3):
        w = cnn.bf16_round(P[f"w{k}"].astype(np.float32)).astype(np.float64)
        co, _, ci = w.shape
        kt = torch.from_numpy(w).permute(0, 2, 1).reshape(co, ci, 3, 3, 3)
        h = torch.relu(F.conv3d(h, kt, torch.from_numpy(P[f"b{k}"]), padding=1))
    out = h[0].permute(1, 2, 3, 0).reshape(-1, P["wh"].shape[1]).numpy() @ P["wh"].T + P["bh"]
    np.testing.assert_allclose(a, out, rtol=1e-10, atol=1e-10)


def test_cnn_gradient_matches_central_differences():
    pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    vol = rng.normal(size=(4, 4, 4))
    occ = (rng.uniform(size=64) < 0.3).astype(np.float64)
    p0 = rng.uniform(0.2, 1.0, size=64)
    p = random_params(2).astype(np.float64)
    # biases and the head enter without bf16 rounding: differentiate those
    names = [n for n, _ in cnn.PARAM_SHAPES]
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in cnn.PARAM_SHAPES])
    _, _, g = cnn.cnn_loss_grad(p, vol, occ, p0, 5.0)
    idx = [offs[names.index("b3")] + 3, offs[names.index("wh")] + 7,
           offs[names.index("bh")] + 0, offs[names.index("bh")] + 1,
           offs[names.index("b1")] + 2]
    for i in idx:
        e = np.zeros_like(p)
        e[i] = 1e-6
        lp = sum(cnn.cnn_loss_grad(p + e, vol, occ, p0, 5.0)[:2])
        lm = sum(cnn.cnn_loss_grad(p - e, vol, occ, p0, 5.0)[:2])
        assert g[i] == pytest.approx((lp - lm) / 2e-6, rel=1e-5, abs=1e-9)


def _bf16_forward_states(p, vol):
    """Hidden activations of the network with bf16 storage, from the pinned
    pieces (conv3d, bf16_round, scaled_input)."""
    P = cnn.unpack_params(p)
    r = lambda a: cnn.bf16_round(a.astype(np.float32)).astype(np.float64)
    h = cnn.scaled_input(vol)
    hs, pres = [h], []
    for k in (1, 2, 3):
        pre = cnn.conv3d(h, r(P[f"w{k}"]), P[f"b{k}"])
        h = r(np.maximum(pre, 0.0))
        pres.append(pre)
        hs.append(h)
    return P, hs, pres


def test_cnn_gradient_with_bf16_storage_head_and_last_convolution():
    """With bf16 storage the head's gradient is dout^T h3 with h3 the rounded
    activation, and the third convolution's weight gradient is
    sum_v g3[v][n] h2[v + off(tap)][c] with g3 = bf16([h3 > 0] (dout Wh)) and
    h2 rounded: both written out directly from the pinned forward pieces.
    Without storage rounding the same gradient differs from it."""
    pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    vol = rng.normal(size=(4, 5, 6))
    V = vol.size
    p = random_params(2)
    occ = (rng.uniform(size=V) < 0.3).astype(np.float64)
    q0 = rng.uniform(0.2, 1.0, size=V)
    pw = 5.0
    _, _, g = cnn.cnn_loss_grad(p, vol, occ, q0, pw, bf16_storage=True)
    P, hs, pres = _bf16_forward_states(p, vol)
    h3 = hs[3].reshape(V, -1)
    out = h3 @ P["wh"].T + P["bh"]
    z, q = out[:, 0], out[:, 1]
    sg = 1.0 / (1.0 + np.exp(-z))
    dout = np.stack([(pw * occ * (sg - 1.0) + (1.0 - occ) * sg) / V,
                     2.0 * occ * (q - q0) / V], axis=1)
    names = [n for n, _ in cnn.PARAM_SHAPES]
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in cnn.PARAM_SHAPES])
    blk = lambda n: g[offs[names.index(n)]:offs[names.index(n) + 1]]
    np.testing.assert_allclose(blk("wh"), (dout.T @ h3).reshape(-1), rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(blk("bh"), dout.sum(axis=0), rtol=1e-10, atol=1e-14)
    g3 = (dout @ P["wh"]) * (pres[2].reshape(V, -1) > 0)
    g3 = cnn.bf16_round(g3.astype(np.float32)).astype(np.float64)
    h2 = hs[2]
    nz, ny, nx, cin = h2.shape
    hp = np.zeros((nz + 2, ny + 2, nx + 2, cin))
    hp[1:-1, 1:-1, 1:-1] = h2
    dw3 = np.zeros(P["w3"].shape)
    for tap in range(27):
        dz, dy, dx = tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1
        sl = hp[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx].reshape(V, cin)
        dw3[:, tap, :] = g3.T @ sl
    np.testing.assert_allclose(blk("w3"), dw3.reshape(-1), rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(blk("b3"), g3.sum(axis=0), rtol=1e-9, atol=1e-14)
    _, _, g_exact = cnn.cnn_loss_grad(p, vol, occ, q0, pw)
    assert not np.allclose(g_exact, g, rtol=1e-6, atol=0)
