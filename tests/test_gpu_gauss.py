"""The Gaussian-profile radiator and its adjoint on the GPU against the FP64
oracle."""
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


def gauss_cloud(n=1500, seed=21):
    b = workloads.uniform_balls(n, 2.0, 0.04, 0.15, 0.0, 1.0, seed=seed).stack()
    return b  # the R row is the standard deviation here


@pytest.mark.parametrize("level", [0, 1])
def test_forward_gauss_matches_oracle(sb, level):
    wl = workloads.tiny()
    arr = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, (1, 2),
                         n_cap=2000)
    b = gauss_cloud()
    arr.set_sampling_level(level)
    S = arr.forward_gauss(torch.from_numpy(b).cuda()).cpu().numpy()
    ref = oracle.forward_gauss(b, wl.sensors.pos, wl.sensors.normal, wl.c,
                               (1, 2)[level] / wl.fs_mhz, arr.Tk)
    assert np.linalg.norm(S - ref) / np.linalg.norm(ref) <= 1e-5
    # bitwise independent of the order of the balls
    perm = np.random.default_rng(0).permutation(b.shape[1])
    S2 = arr.forward_gauss(torch.from_numpy(np.ascontiguousarray(b[:, perm])).cuda()).cpu().numpy()
    np.testing.assert_array_equal(S, S2)
    arr.close()


def test_adjoint_gauss_matches_oracle(sb):
    wl = workloads.tiny()
    arr = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, (1,),
                         n_cap=2000)
    b = gauss_cloud(800, seed=22)
    G = np.random.default_rng(1).normal(size=(wl.sensors.M, wl.T)).astype(np.float32)
    g = arr.adjoint_gauss(torch.from_numpy(b).cuda(), torch.from_numpy(G).cuda()).cpu().numpy()
    ref = oracle.adjoint_gauss(b, wl.sensors.pos, wl.sensors.normal, wl.c, 1.0 / wl.fs_mhz,
                               wl.T, G)
    for k in range(5):
        err = np.linalg.norm(g[k] - ref[k]) / np.linalg.norm(ref[k])
        assert err <= 1e-4, (k, err)
    # masks zero the other components
    gm = arr.adjoint_gauss(torch.from_numpy(b).cuda(), torch.from_numpy(G).cuda(),
                           mask=sb.MASK_P0).cpu().numpy()
    assert np.all(gm[:4] == 0) and np.allclose(gm[4], g[4])
    arr.close()
