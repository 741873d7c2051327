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
    net.close()
