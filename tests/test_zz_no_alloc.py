"""sbp_forward_static, the forward for callers that cannot allocate device
memory (inside a stream capture or a host callback, or a host that borrows all
its buffers), against the regular sbp_forward through the C ABI.

Collected last on purpose: it uses the library's one static scratch array,
and the rest of the suite has already run if it fails."""

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-5


@pytest.fixture(scope="module")
def sb():
    import __graft_entry__ as ge

    ge.build()
    from paper_2601_00551_gb300 import slingbag

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    slingbag.load_library()
    return slingbag


def rel_l2(a, b):
    return float(np.linalg.norm(a.astype(np.float64) - b) / np.linalg.norm(b))


def sensors_6xM(pos, nrm):
    """[6][M] device layout with unit normals, normalised exactly as the array
    object does it (in double, then rounded to float32)."""
    n = nrm.astype(np.float64)
    n = n / np.sqrt(n[:, 0] * n[:, 0] + n[:, 1] * n[:, 1] + n[:, 2] * n[:, 2])[:, None]
    return np.concatenate([pos.T.astype(np.float32), n.T.astype(np.float32)]).copy()


def test_static_forward_matches_regular_forward_twice(sb):
    wl = workloads.tiny()
    b = wl.init.stack()
    n = b.shape[1]
    arr = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, (4, 1),
                         n_cap=n)
    balls = torch.from_numpy(b).cuda()
    sens = torch.from_numpy(sensors_6xM(wl.sensors.pos, wl.sensors.normal)).cuda()
    for k, f in enumerate((4, 1)):
        arr.set_sampling_level(k)
        ref = arr.forward(balls).cpu().numpy()
        Tk = wl.T // f
        for _ in range(2):  # two calls in a row share (and clear) the static scratch
            out = torch.full((wl.sensors.M, Tk), float("nan"), device="cuda")
            got = sb.forward_static(sens, wl.c, f / wl.fs_mhz, Tk, balls, out=out).cpu().numpy()
            assert np.all(np.isfinite(got))
            assert rel_l2(got, ref) <= TRACE_TOL


def test_static_forward_rejects_sizes_beyond_its_scratch(sb):
    """Through the C ABI directly: the error code and message."""
    lib = sb.load_library()
    dummy = torch.zeros((5, 4), device="cuda")
    sens = torch.zeros((6, 1024), device="cuda")
    out = torch.zeros(1, device="cuda")
    rc = lib.sbp_forward_static(sens.data_ptr(), 1024, 1.5, 0.025, 4096, 0, sb._rows(dummy),
                                None, 4, out.data_ptr(), None)
    assert rc == -1
    assert b"exceeds the static scratch" in lib.sbp_last_error()
