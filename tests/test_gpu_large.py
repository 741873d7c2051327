"""The large configuration (1M balls x 1024 sensors, T = 8192 at 80 MHz):
sampled sensors and balls against the FP64 oracle, in the launch
configuration the benchmark times."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    import __graft_entry__ as ge

    ge.build()
    from paper_2601_00551_gb300 import slingbag

    torch.cuda.set_device(0)
    return slingbag


@pytest.fixture(scope="module")
def large():
    return workloads.large()


# (level, forward tile): the default tile and the tiles the benchmark's tuner
# picks for the step (2048 balls per CTA, the wide window at 40 and 80 MHz)
CASES = [(2, 0), (2, 2048 | 0x10000), (1, 2048 | 0x10000), (0, 2048)]


@pytest.mark.parametrize("k,tile", CASES)
def test_large_forward_and_adjoint_sampled(sb, large, k, tile):
    wl = large
    n = wl.init.n
    arr = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, wl.levels,
                         n_cap=n)
    b = wl.init.stack()
    B = torch.from_numpy(b).cuda()
    f = wl.levels[k]
    Tk = wl.T // f
    arr.set_sampling_level(k)
    arr.set_tiles(k, tile, 0)
    S = arr.forward(B).cpu().numpy()
    assert arr.sync_status() == 0
    rng = np.random.default_rng(k)
    ms = rng.choice(wl.sensors.M, size=3, replace=False)
    ref = oracle.forward(b, wl.sensors.pos[ms], wl.sensors.normal[ms], wl.c, f / wl.fs_mhz,
                         Tk, threads=oracle.num_procs())
    for r, m in enumerate(ms):
        assert np.linalg.norm(S[m] - ref[r]) / np.linalg.norm(ref[r]) <= 1e-5
    if tile:  # every tile renders the default's traces bit for bit
        arr.set_tiles(k, 0, 0)
        assert np.array_equal(arr.forward(B).cpu().numpy(), S)
    G = rng.normal(size=(wl.sensors.M, Tk)).astype(np.float32)
    g = arr.adjoint(B, torch.from_numpy(G).cuda()).cpu().numpy()
    idx = rng.choice(n, size=64, replace=False)
    gref = oracle.adjoint(b[:, idx], wl.sensors.pos, wl.sensors.normal, wl.c, f / wl.fs_mhz,
                          Tk, G, threads=oracle.num_procs())
    for c in range(5):
        err = np.linalg.norm(g[c, idx] - gref[c]) / np.linalg.norm(gref[c])
        assert err <= 1e-4, (c, err)
    arr.close()
