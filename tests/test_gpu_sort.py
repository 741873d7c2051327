"""Spatial ordering on the GPU (sbp_sort_cloud and sbp_reconstruct's
spatial_sort) against the oracle's definition of the Morton order, and the
reconstruction of a cloud in random order against the oracle's loop on the
same cloud in that order."""
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


@pytest.mark.parametrize("name", ["tiny", "vessel"])
def test_sort_cloud_is_the_oracle_order(sb, name):
    """Bit for bit: the live balls in the oracle's stable Morton order, the
    carried rows following them, everything past the live count untouched."""
    wl = workloads.tiny() if name == "tiny" else workloads.vessel(sort=False)
    b = wl.init.stack()
    n_cap = b.shape[1]
    n = n_cap - 37
    arr = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, wl.levels,
                         n_cap=n_cap)
    rng = np.random.default_rng(3)
    ex = rng.normal(size=(3, n_cap)).astype(np.float32)
    balls = torch.from_numpy(b).cuda()
    extra = torch.from_numpy(ex).cuda()
    arr.sort_cloud(balls, torch.tensor([n], dtype=torch.int32, device="cuda"), extra=[extra])
    assert arr.sync_status() == 0
    perm = oracle.morton_permutation(b[:, :n])
    got = balls.cpu().numpy()
    np.testing.assert_array_equal(got[:, :n], b[:, perm])
    np.testing.assert_array_equal(got[:, n:], b[:, n:])
    np.testing.assert_array_equal(extra.cpu().numpy()[:, :n], ex[:, perm])
    # sorting a sorted cloud changes nothing
    again = balls.clone()
    arr.sort_cloud(again, torch.tensor([n], dtype=torch.int32, device="cuda"))
    assert torch.equal(again, balls)
    arr.close()


def test_reconstruct_with_spatial_sort_matches_the_oracle_on_the_sorted_cloud(sb):
    """sbp_reconstruct with spatial_sort on the 2,000-ball cloud in random
    order equals the oracle's loop started from the same cloud in Morton
    order: ball counts per iteration, losses within float32 round-off and
    the final cloud."""
    wl = workloads.tiny()
    b = wl.init.stack()
    n = b.shape[1]
    y = workloads.add_noise(oracle.forward(wl.truth.stack(), wl.sensors.pos, wl.sensors.normal,
                                           wl.c, 1 / wl.fs_mhz, wl.T).astype(np.float32))
    factors = (4, 2, 1)
    arr = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, factors,
                         n_cap=2 * n)
    st_o = [oracle.Stage(0, 2, 3, True, False), oracle.Stage(1, 2, 7, True, False),
            oracle.Stage(2, 2, 7, True, True)]
    st_g = [sb.Stage(s.level, s.iterations, s.grad_mask, s.grow, s.duplicate) for s in st_o]
    grow = dict(p_min=1e-3, R_min=0.02, R_max=0.3, g_dup=5.0, seed=77)
    perm = oracle.morton_permutation(b)
    bo, losses, counts = oracle.reconstruct(b[:, perm], wl.sensors.pos, wl.sensors.normal, wl.c,
                                            wl.fs_mhz, wl.T, factors, y, st_o,
                                            grow_params=oracle.GrowParams(**grow),
                                            threads=max(1, oracle.num_procs()))
    balls = torch.zeros((5, 2 * n), device="cuda")
    balls[:, :n] = torch.from_numpy(b)
    n_dev = torch.tensor([n], dtype=torch.int32, device="cuda")
    loss = torch.zeros(6, dtype=torch.float64, device="cuda")
    n_log = torch.zeros(6, dtype=torch.int32, device="cuda")
    arr.reconstruct(torch.from_numpy(y).cuda(), balls, n_dev, st_g, grow=sb.GrowParams(**grow),
                    loss_log=loss, n_log=n_log, spatial_sort=True)
    assert arr.sync_status() == 0
    np.testing.assert_array_equal(n_log.cpu().numpy(), counts)
    np.testing.assert_allclose(loss.cpu().numpy(), losses, rtol=1e-4)
    assert int(n_dev.item()) == bo.shape[1]
    np.testing.assert_allclose(balls[:, :bo.shape[1]].cpu().numpy(), bo, rtol=0, atol=1e-4)
    arr.close()


def test_frames_reject_the_spatial_sort(sb):
    """The batched reconstruction does not sort: asking for it is an
    argument error, raised before anything runs."""
    import ctypes

    wl = workloads.tiny()
    arr = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, (1,),
                         n_cap=2048)
    arr.set_frames([1000, 1000])
    lib = sb.load_library()
    rp = sb._ReconParams()
    rp.zero_grad_mode = -1
    rp.spatial_sort = 1
    balls = torch.zeros((5, 2048), device="cuda")
    n_dev = torch.tensor([10, 10], dtype=torch.int32, device="cuda")
    y = torch.zeros((2, wl.sensors.M, wl.T), device="cuda")
    rc = lib.sbp_reconstruct_frames(arr._h, ctypes.c_void_p(y.data_ptr()), sb._rows(balls),
                                    ctypes.c_void_p(n_dev.data_ptr()), ctypes.byref(rp), None)
    assert rc == -1
    assert b"spatial_sort" in lib.sbp_last_error()
    arr.close()
