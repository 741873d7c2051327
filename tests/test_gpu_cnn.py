"""The tcgen05 implicit-GEMM convolution against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import cnn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    import __graft_entry__ as ge

    ge.build()
    from paper_2601_00551_gb300 import slingbag

    torch.cuda.set_device(0)
    return slingbag


def dyadic(rng, shape, scale=16):
    """Values k / scale with small integers k: exact in bf16, and their
    products and sums exact in FP32, so the tensor cores must match the
    FP64 oracle exactly."""
    return (rng.integers(-24, 25, size=shape) / scale).astype(np.float32)


@pytest.mark.parametrize("cin,cout", [(1, 16), (16, 32), (32, 32), (32, 16), (32, 64), (64, 32), (64, 64), (16, 16)])
def test_conv_exact_on_dyadic_values(sb, cin, cout):
    rng = np.random.default_rng(cin * 100 + cout)
    dims = (13, 9, 11)  # nx, ny, nz: 1287 voxels, a ragged last tile of 128
    nx, ny, nz = dims
    x = dyadic(rng, (nz, ny, nx, cin))
    w = dyadic(rng, (cout, 27, cin))
    b = dyadic(rng, (cout,))
    ref = cnn.conv3d(x, w, b)
    X = torch.from_numpy(x.reshape(-1, cin)).cuda().to(torch.bfloat16)
    W = sb.pack_conv_weights(torch.from_numpy(w).cuda())
    B = torch.from_numpy(b).cuda()
    got = sb.conv3d(X, dims, W, B, relu=False, out_f32=True)
    assert sb.cnn_status() == 0
    np.testing.assert_array_equal(got.cpu().numpy().reshape(nz, ny, nx, cout), ref)
    # ReLU and bf16 output: the oracle result rounded the same way
    got = sb.conv3d(X, dims, W, B, relu=True)
    refr = cnn.bf16_round(np.maximum(ref, 0.0).astype(np.float32))
    np.testing.assert_array_equal(got.float().cpu().numpy().reshape(nz, ny, nx, cout), refr)


def test_conv_tiles_span_the_volume(sb):
    """A volume of several halo tiles in every direction plus ragged ends
    (x = 8 k + 3, y = 16 k + 5): every voxel against the oracle, exactly."""
    rng = np.random.default_rng(11)
    dims = (19, 37, 6)
    nx, ny, nz = dims
    x = dyadic(rng, (nz, ny, nx, 32))
    w = dyadic(rng, (32, 27, 32))
    ref = cnn.conv3d(x, w)
    got = sb.conv3d(torch.from_numpy(x.reshape(-1, 32)).cuda().to(torch.bfloat16), dims,
                    sb.pack_conv_weights(torch.from_numpy(w).cuda()), out_f32=True)
    assert sb.cnn_status() == 0
    np.testing.assert_array_equal(got.cpu().numpy().reshape(nz, ny, nx, 32), ref)


@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 16)])
def test_conv_many_tiles_per_cta(sb, cin, cout):
    """A volume of 960 tiles of 8 x 16 x 1 voxels: the persistent kernel
    walks several tiles per CTA through its rotating halo slots and
    alternating accumulators. Exact on dyadic values, ReLU and bf16 output
    included."""
    rng = np.random.default_rng(cin + 3 * cout)
    dims = (64, 45, 40)  # ny = 16 k + 13: a ragged last tile row
    nx, ny, nz = dims
    x = dyadic(rng, (nz, ny, nx, cin))
    w = dyadic(rng, (cout, 27, cin))
    b = dyadic(rng, (cout,))
    ref = cnn.conv3d(x, w, b)
    X = torch.from_numpy(x.reshape(-1, cin)).cuda().to(torch.bfloat16)
    W = sb.pack_conv_weights(torch.from_numpy(w).cuda())
    B = torch.from_numpy(b).cuda()
    got = sb.conv3d(X, dims, W, B, relu=False, out_f32=True)
    assert sb.cnn_status() == 0
    np.testing.assert_array_equal(got.cpu().numpy().reshape(nz, ny, nx, cout), ref)
    got = sb.conv3d(X, dims, W, B, relu=True)
    refr = cnn.bf16_round(np.maximum(ref, 0.0).astype(np.float32))
    np.testing.assert_array_equal(got.float().cpu().numpy().reshape(nz, ny, nx, cout), refr)


def test_conv_random_values_within_fp32_accumulation(sb):
    rng = np.random.default_rng(7)
    dims = (32, 24, 20)
    nx, ny, nz = dims
    x = cnn.bf16_round(rng.normal(size=(nz, ny, nx, 32)).astype(np.float32))
    w = cnn.bf16_round((rng.normal(size=(64, 27, 32)) * 0.05).astype(np.float32))
    ref = cnn.conv3d(x, w)
    got = sb.conv3d(torch.from_numpy(x.reshape(-1, 32)).cuda().to(torch.bfloat16), dims,
                    sb.pack_conv_weights(torch.from_numpy(w).cuda()), out_f32=True)
    assert sb.cnn_status() == 0
    got = got.cpu().numpy().reshape(ref.shape)
    # FP32 accumulation of 864 terms: error below ~1e-6 of the sum of |terms|
    mag = cnn.conv3d(np.abs(x), np.abs(w))
    assert np.max(np.abs(got - ref) / (mag + 1e-30)) < 1e-5
