"""Delay-and-sum volume, the proposal CNN's forward pass, training step and
proposal on the GPU against the FP64 oracle."""
import numpy as np
import pytest
import torch

import workloads
from oracle import cnn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    import __graft_entry__ as ge

    ge.build()
    from paper_2601_00551_gb300 import slingbag

    torch.cuda.set_device(0)
    return slingbag


def test_das_matches_oracle(sb):
    wl = workloads.tiny()
    arr = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, (1,), n_cap=8)
    rng = np.random.default_rng(0)
    y = rng.normal(size=(wl.sensors.M, wl.T)).astype(np.float32)
    origin, h, dims = (-2.0, -2.0, -2.0), 4.0 / 20, (20, 20, 20)
    ref = cnn.das_volume(y, wl.sensors.pos, wl.sensors.normal, wl.c, 1.0 / wl.fs_mhz, origin, h,
                         dims)
    got = arr.das_volume(torch.from_numpy(y).cuda(), origin, h, dims).cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-4
    arr.close()


def init_params(seed):
    rng = np.random.default_rng(seed)
    out = []
    for name, shape in cnn.PARAM_SHAPES:
        fan = shape[1] * shape[2] if len(shape) == 3 else shape[-1]
        out.append(rng.normal(size=shape).reshape(-1) * np.sqrt(2.0 / fan)
                   if name.startswith("w") else rng.normal(size=shape) * 0.1)
    return np.concatenate(out).astype(np.float32)


def test_cnn_forward_matches_oracle(sb):
    dims = (12, 10, 9)
    rng = np.random.default_rng(1)
    vol = rng.normal(size=dims[::-1]).astype(np.float32)
    net = sb.VolumeCNN(dims)
    p = init_params(3)
    net.set_params(p)
    np.testing.assert_array_equal(net.params(), p)
    got = net.forward(torch.from_numpy(vol).cuda().reshape(-1)).cpu().numpy()
    assert sb.cnn_status() == 0
    ref = cnn.cnn_forward(p, vol)
    # activations are bf16 on both sides; a different rounding of a rare
    # near-tie propagates, so the bound is on the whole output
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-3
    net.close()


def test_cnn_training_step_follows_the_oracle_gradient(sb):
    dims = (10, 8, 8)
    V = 10 * 8 * 8
    rng = np.random.default_rng(2)
    vol = rng.normal(size=dims[::-1]).astype(np.float32)
    occ = (rng.uniform(size=V) < 0.2).astype(np.float32)
    p0 = rng.uniform(0.2, 1.0, size=V).astype(np.float32)
    net = sb.VolumeCNN(dims)
    p = init_params(4)
    net.set_params(p)
    loss = torch.zeros(2, dtype=torch.float64, device="cuda")
    lr = 1e-4
    net.train_step(torch.from_numpy(vol).cuda().reshape(-1), torch.from_numpy(occ).cuda(),
                   torch.from_numpy(p0).cuda(), lr=lr, pos_weight=5.0, loss=loss)
    l0, l1, g = cnn.cnn_loss_grad(p, vol, occ, p0, 5.0)
    assert loss.cpu().numpy() == pytest.approx([l0, l1], rel=2e-2)
    # the first Adam step moves every parameter by about -lr sign(g)
    step = net.params().astype(np.float64) - p
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    agree = np.mean(np.sign(step[big]) == -np.sign(g[big]))
    assert agree > 0.97
    assert np.allclose(np.abs(step[big]), lr, rtol=0.05)
    net.close()


@pytest.mark.parametrize("dims", [(10, 8, 8), (70, 9, 6)])
def test_cnn_gradient_matches_the_oracle_element_by_element(sb, dims):
    """sbp_cnn_grad (convolution weight gradients as tensor-core GEMMs over
    voxels, reduced in a fixed order) against torch autograd in float64 on the
    CPU, element by element per parameter block. Against the oracle that
    rounds to bf16 where the network stores bf16 (activations and their
    gradients) the bound is 5e-3 relative L2 per block: what is left is FP32
    against FP64 summation, and values rounding to a different bf16 near a
    tie. Against the oracle without any storage rounding it is 5e-2 (the
    first layer's gradient passes three bf16 data gradients). The second
    shape has rows longer than one 64-voxel K-step. Two calls give the same
    bits."""
    nx, ny, nz = dims
    V = nx * ny * nz
    rng = np.random.default_rng(5)
    vol = rng.normal(size=dims[::-1]).astype(np.float32)
    occ = (rng.uniform(size=V) < 0.2).astype(np.float32)
    p0 = rng.uniform(0.2, 1.0, size=V).astype(np.float32)
    net = sb.VolumeCNN(dims)
    p = init_params(6)
    net.set_params(p)
    args = (torch.from_numpy(vol).cuda().reshape(-1), torch.from_numpy(occ).cuda(),
            torch.from_numpy(p0).cuda())
    loss = torch.zeros(2, dtype=torch.float64, device="cuda")
    g1 = net.grad(*args, pos_weight=5.0, loss=loss).cpu().numpy()
    g2 = net.grad(*args, pos_weight=5.0).cpu().numpy()
    assert sb.cnn_status() == 0
    np.testing.assert_array_equal(g1, g2)
    np.testing.assert_array_equal(net.params(), p)  # unchanged
    net.close()
    _, _, ref_b = cnn.cnn_loss_grad(p, vol, occ, p0, 5.0, bf16_storage=True)
    l0, l1, ref = cnn.cnn_loss_grad(p, vol, occ, p0, 5.0)
    assert loss.cpu().numpy() == pytest.approx([l0, l1], rel=2e-2)
    errs, o = {}, 0
    for name, shape in cnn.PARAM_SHAPES:
        n = int(np.prod(shape))
        a = g1[o:o + n].astype(np.float64)
        e = lambda b: np.linalg.norm(a - b[o:o + n]) / max(np.linalg.norm(b[o:o + n]), 1e-30)
        errs[name] = (e(ref_b), e(ref))
        o += n
    assert all(eb <= 5e-3 and ex <= 5e-2 for eb, ex in errs.values()), errs


def test_cnn_training_is_reproducible(sb):
    """Two networks from the same parameters, trained three steps on the same
    data, end with the same parameters bit for bit."""
    dims = (12, 10, 9)
    V = 12 * 10 * 9
    rng = np.random.default_rng(7)
    vol = torch.from_numpy(rng.normal(size=V).astype(np.float32)).cuda()
    occ = torch.from_numpy((rng.uniform(size=V) < 0.2).astype(np.float32)).cuda()
    p0 = torch.from_numpy(rng.uniform(0.2, 1.0, size=V).astype(np.float32)).cuda()
    out = []
    for _ in range(2):
        net = sb.VolumeCNN(dims)
        net.set_params(init_params(8))
        for _ in range(3):
            net.train_step(vol, occ, p0, lr=1e-3, pos_weight=5.0)
        out.append(net.params())
        net.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_proposal_places_balls_in_marked_voxels(sb):
    dims = (8, 6, 5)
    V = 8 * 6 * 5
    net = sb.VolumeCNN(dims)
    p = np.zeros(net.n_params, dtype=np.float32)
    # zero convolutions: the head sees zero features, so its output is its
    # bias: logit 3 (probability 0.95) and pressure 0.7
    p[-2:] = [3.0, 0.7]
    net.set_params(p)
    origin, h = (1.0, -2.0, 0.5), 0.25
    vol = torch.rand(V, device="cuda")
    balls, n = net.propose(vol, origin, h, threshold=0.9, seed=5, R=0.1)
    assert int(n.item()) == V
    b = balls[:, :V].cpu().numpy()
    idx = np.arange(V)
    ix, iy, iz = idx % 8, (idx // 8) % 6, idx // 48
    for a, (o, i) in enumerate(zip(origin, (ix, iy, iz))):
        assert np.all(b[a] >= o + i * h - 1e-6) and np.all(b[a] < o + (i + 1) * h + 1e-6)
    assert np.all(b[3] == np.float32(0.1)) and np.allclose(b[4], 0.7)
    _, n = net.propose(vol, origin, h, threshold=0.99, seed=5, R=0.1)
    assert int(n.item()) == 0
    # three balls per marked voxel: every ball in its voxel, all 3 V
    # positions distinct
    balls3, n3 = net.propose(vol, origin, h, threshold=0.9, seed=5, R=0.1, per_voxel=3)
    assert int(n3.item()) == 3 * V
    b3 = balls3[:, :3 * V].cpu().numpy()
    for a, (o, i) in enumerate(zip(origin, (ix, iy, iz))):
        ii = np.repeat(i, 3)
        assert np.all(b3[a] >= o + ii * h - 1e-6) and np.all(b3[a] < o + (ii + 1) * h + 1e-6)
    assert len({tuple(c) for c in b3[:3].T.round(6)}) == 3 * V
    # a capacity below 3 V keeps the first n_cap balls
    small = torch.zeros((5, 100), device="cuda")
    _, n4 = net.propose(vol, origin, h, threshold=0.9, seed=5, R=0.1, per_voxel=3, out=small)
    assert int(n4.item()) == 100
    np.testing.assert_array_equal(small.cpu().numpy(), b3[:, :100])
    net.close()
