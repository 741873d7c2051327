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
