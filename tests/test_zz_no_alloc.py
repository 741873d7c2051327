"""sbp_forward_static, the forward for callers that cannot allocate device
memory (a process that borrows every buffer from a framework owning all
allocations, or one held to a fixed device-memory budget), against the
regular sbp_forward through the C ABI.

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


def level_dt(c, f, fs):
    """A sampling interval dt with c * dt equal, in double, to the array's own
    spacing c * f / fs, so that both entry points round the same h."""
    h = c * f / fs
    dt = h / c
    for _ in range(8):
        if c * dt == h:
            return dt
        dt = np.nextafter(dt, np.inf if c * dt < h else -np.inf)
    raise AssertionError("no dt reproduces the level spacing")


@pytest.mark.parametrize("wmode", ["clamp", "none", "cos"])
def test_static_forward_matches_regular_forward_twice(sb, wmode):
    """Both entry points run the same exact-integer kernels, so the traces
    agree bit for bit: for every weight mode, at two levels, with all balls
    and with a ragged live count held on the device, on two calls in a row
    (which share, and clear, the static scratch)."""
    wl = workloads.tiny()
    b = wl.init.stack()
    n = b.shape[1]
    arr = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, (4, 1),
                         n_cap=n, weight_mode=wmode)
    balls = torch.from_numpy(b).cuda()
    sens = torch.from_numpy(sensors_6xM(wl.sensors.pos, wl.sensors.normal)).cuda()
    ragged = torch.tensor([n - 37], dtype=torch.int32, device="cuda")
    for k, f in enumerate((4, 1)):
        arr.set_sampling_level(k)
        Tk = wl.T // f
        dt = level_dt(wl.c, f, wl.fs_mhz)
        for n_dev in (None, ragged):
            ref = arr.forward(balls, n=n_dev).cpu().numpy()
            assert np.count_nonzero(ref) > 0
            for _ in range(2):
                out = torch.full((wl.sensors.M, Tk), float("nan"), device="cuda")
                got = sb.forward_static(sens, wl.c, dt, Tk, balls, n=n_dev, out=out,
                                        weight_mode=wmode).cpu().numpy()
                np.testing.assert_array_equal(got, ref)
        # the ragged count leaves the last 37 balls out
        full = arr.forward(balls).cpu().numpy()
        part = arr.forward(balls, n=ragged).cpu().numpy()
        assert not np.array_equal(full, part)
        assert rel_l2(part, arr.forward(balls[:, :n - 37].contiguous()).cpu().numpy()) <= TRACE_TOL


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


def test_static_forward_binding_rejects_host_buffers(sb):
    """An output or a live count in host memory is refused before the
    library is called (the kernels would write through a host pointer)."""
    wl = workloads.tiny(M=8, T=64)
    sens = torch.from_numpy(sensors_6xM(wl.sensors.pos, wl.sensors.normal)).cuda()
    balls = torch.from_numpy(wl.init.stack()).cuda()
    with pytest.raises(ValueError):
        sb.forward_static(sens, wl.c, 0.025, 64, balls, out=torch.zeros((8, 64)))
    with pytest.raises(ValueError):
        sb.forward_static(sens, wl.c, 0.025, 64, balls, n=torch.tensor([3], dtype=torch.int32))
    with pytest.raises(ValueError):
        sb.forward_static(sens, wl.c, 0.025, 64, balls.cpu())
