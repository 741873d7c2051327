"""Stored-window adjoint (sbp_store_windows + sbp_adjoint_stored) against the
FP64 oracle adjoint and against the recomputing adjoint, and its autograd
Function against radiate()."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def sb():
    import __graft_entry__ as ge

    ge.build()
    from paper_2601_00551_gb300 import slingbag

    torch.cuda.set_device(0)
    return slingbag


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def threads():
    return max(1, oracle.num_procs())


@pytest.mark.parametrize("wmode", ["clamp", "cos", "none"])
def test_adjoint_stored_matches_the_oracle(sb, wmode):
    """All five components at two levels within the adjoint's bar, the p0-only
    mask, and the live count: balls past it keep their records empty and
    their gradients untouched."""
    wl = workloads.tiny(T=560)  # the record ends inside some windows
    b = wl.init.stack()
    n_cap = b.shape[1]
    n = n_cap - 37
    arr = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, (4, 1),
                         n_cap=n_cap, weight_mode=wmode)
    balls = torch.from_numpy(b).cuda()
    n_dev = torch.tensor([n], dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(11)
    for k, f in enumerate((4, 1)):
        Tk = -(-wl.T // f)
        arr.set_sampling_level(k)
        G = rng.normal(size=(wl.sensors.M, Tk)).astype(np.float32)
        Gd = torch.from_numpy(G).cuda()
        rec = arr.store_windows(balls, n=n_dev)
        assert torch.all(rec[3][:, n:] == -1)
        out = torch.full_like(balls, 7.0)
        g = arr.adjoint_stored(balls, Gd, rec, n=n_dev, out=out).cpu().numpy()
        assert arr.sync_status() == 0
        assert np.all(g[:, n:] == 7.0)
        ref = oracle.adjoint(b[:, :n], wl.sensors.pos, wl.sensors.normal, wl.c, f / wl.fs_mhz, Tk,
                             G.astype(np.float64), wmode=wmode, threads=threads())
        for c in range(5):
            assert rel_l2(g[c, :n], ref[c]) <= GRAD_TOL, (f, c)
        # the recomputing adjoint: the same gradients up to summation order
        gr = arr.adjoint(balls, Gd, n=n_dev).cpu().numpy()
        for c in range(5):
            assert rel_l2(g[c, :n], gr[c, :n]) <= 1e-5, (f, c, "recomputing")
        gp = arr.adjoint_stored(balls, Gd, rec, n=n_dev, mask=sb.MASK_P0).cpu().numpy()
        assert np.all(gp[:4, :n] == 0)
        assert rel_l2(gp[4, :n], ref[4]) <= GRAD_TOL


def test_radiate_stored_equals_radiate(sb):
    """The autograd Function with stored windows gives radiate()'s traces bit
    for bit and its gradients within float summation order."""
    wl = workloads.tiny()
    b = wl.init.stack()
    arr = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, (2, 1),
                         n_cap=b.shape[1])
    grads = []
    traces = []
    for fn in (sb.radiate, sb.radiate_stored):
        x, y, z, R, p0 = (torch.from_numpy(b[c]).cuda().requires_grad_(True) for c in range(5))
        S = fn(arr, x, y, z, R, p0, level=1)
        (S * S).sum().backward()
        traces.append(S.detach().clone())
        grads.append([t.grad.cpu().numpy() for t in (x, y, z, R, p0)])
    assert torch.equal(traces[0], traces[1])
    for c in range(5):
        assert rel_l2(grads[1][c], grads[0][c]) <= 1e-5, c


def test_store_windows_rejects_a_wrong_record(sb):
    wl = workloads.tiny()
    b = wl.init.stack()
    arr = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, (1,),
                         n_cap=b.shape[1])
    balls = torch.from_numpy(b).cuda()
    G = torch.zeros((wl.sensors.M, wl.T), device="cuda")
    with pytest.raises(ValueError):
        arr.adjoint_stored(balls, G, torch.zeros((5, 3, b.shape[1]), dtype=torch.int32,
                                                 device="cuda"))
