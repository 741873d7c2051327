"""Batched frames: every batched step equals the single-cloud step applied to
each frame, and every frame matches the FP64 oracle on its own (traces,
gradients, filter/grow and the whole reconstruction loop)."""
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


COUNTS = (1500, 300, 2000, 900)


def frame_clouds():
    return [workloads.uniform_balls(n, 2.0, 0.05, 0.35, 0.0, 1.0, seed=50 + f).stack()
            for f, n in enumerate(COUNTS)]


def setup(sb, levels=(2, 1)):
    wl = workloads.tiny()
    F = len(COUNTS)
    caps = [c + 700 for c in COUNTS]  # room to grow
    total = sum((c + 1023) // 1024 * 1024 for c in caps)
    arr = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, levels,
                         n_cap=total)
    off = arr.set_frames(caps)
    packed = torch.zeros((5, total), device="cuda")
    clouds = frame_clouds()
    for f, b in enumerate(clouds):
        packed[:, off[f]:off[f] + b.shape[1]] = torch.from_numpy(b)
    n_dev = torch.tensor(COUNTS, dtype=torch.int32, device="cuda")
    # a frame holds its padded capacity, so the single-cloud calls get the same
    single = sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, levels,
                            n_cap=max(off[f + 1] - off[f] for f in range(F)))
    return wl, arr, single, off, packed, n_dev, clouds


def test_forward_and_adjoint_frames_equal_single_cloud(sb):
    wl, arr, single, off, packed, n_dev, clouds = setup(sb)
    rng = np.random.default_rng(0)
    for k in range(2):
        arr.set_sampling_level(k)
        single.set_sampling_level(k)
        Tk = arr.Tk
        S = arr.forward_frames(packed, n_dev)
        G = torch.from_numpy(rng.normal(size=(len(COUNTS), wl.sensors.M, Tk))
                             .astype(np.float32)).cuda()
        g = arr.adjoint_frames(packed, n_dev, G)
        for f, b in enumerate(clouds):
            bf = torch.from_numpy(b).cuda()
            Sf = single.forward(bf)
            assert torch.equal(S[f], Sf)
            gf = single.adjoint(bf, G[f].contiguous())
            n = b.shape[1]
            assert torch.equal(g[:, off[f]:off[f] + n], gf[:, :n])
        # one frame against the oracle
        ref = oracle.forward(clouds[2], wl.sensors.pos, wl.sensors.normal, wl.c,
                             (2, 1)[k] / wl.fs_mhz, Tk)
        got = S[2].cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5


def test_filter_grow_and_adam_frames_equal_single_cloud(sb):
    wl, arr, single, off, packed, n_dev, clouds = setup(sb)
    rng = np.random.default_rng(1)
    total = packed.shape[1]
    grads = torch.from_numpy(rng.normal(size=(5, total)).astype(np.float32)).cuda()
    grads[:, ::7] = 0.0
    mom = torch.from_numpy(rng.normal(size=(10, total)).astype(np.float32)).cuda().abs()
    ap = sb.AdamParams()
    gp = sb.GrowParams(seed=9, R_max=0.3, duplicate=True, g_dup=1.5)
    # single-cloud reference, frame by frame
    ref = []
    for f, b in enumerate(clouds):
        n = b.shape[1]
        cap = off[f + 1] - off[f]
        B = torch.zeros((5, cap), device="cuda")
        Gd = torch.zeros((5, cap), device="cuda")
        Mm = torch.zeros((10, cap), device="cuda")
        B[:, :n] = packed[:, off[f]:off[f] + n]
        Gd[:, :n] = grads[:, off[f]:off[f] + n]
        Mm[:, :n] = mom[:, off[f]:off[f] + n]
        nd = torch.tensor([n], dtype=torch.int32, device="cuda")
        single.adam_step(B, Gd, Mm[:5], Mm[5:], 3, ap, n=nd, mask=7)
        single.filter_grow(B, Gd, nd, mode=sb.GROW, grow=gp, extra=[Mm])
        assert single.sync_status() == 0
        m = int(nd.item())
        ref.append((m, B[:, :m].clone(), Gd[:, :m].clone(), Mm[:, :m].clone()))
    arr.adam_step_frames(packed, grads, mom[:5], mom[5:], n_dev, 3, ap, mask=7)
    arr.filter_grow_frames(packed, grads, n_dev, mode=sb.GROW, grow=gp, extra=[mom])
    assert arr.sync_status() == 0
    counts = n_dev.cpu().numpy()
    for f, (m, B, Gd, Mm) in enumerate(ref):
        assert counts[f] == m
        assert torch.equal(packed[:, off[f]:off[f] + m], B)
        assert torch.equal(grads[:, off[f]:off[f] + m], Gd)
        assert torch.equal(mom[:, off[f]:off[f] + m], Mm)


def test_reconstruct_frames_equals_per_frame_reconstruct(sb):
    wl, arr, single, off, packed, n_dev, clouds = setup(sb)
    F = len(COUNTS)
    y_frames = []
    for f in range(F):
        truth = workloads.uniform_balls(200, 2.0, 0.05, 0.2, 0.5, 1.0, seed=70 + f).stack()
        y = oracle.forward(truth, wl.sensors.pos, wl.sensors.normal, wl.c, 1 / wl.fs_mhz, wl.T)
        y_frames.append(workloads.add_noise(y.astype(np.float32), seed=80 + f))
    Y = torch.from_numpy(np.stack(y_frames)).cuda()
    stages = [sb.Stage(0, 2, 3, True, False), sb.Stage(1, 3, 7, True, True)]
    gp = sb.GrowParams(seed=3, R_max=0.3, g_dup=2.0)
    loss = torch.zeros(5 * F, dtype=torch.float64, device="cuda")
    nlog = torch.zeros(5 * F, dtype=torch.int32, device="cuda")
    arr.reconstruct_frames(Y, packed, n_dev, stages, grow=gp, loss_log=loss, n_log=nlog)
    assert arr.sync_status() == 0
    loss = loss.cpu().numpy().reshape(5, F)
    nlog = nlog.cpu().numpy().reshape(5, F)
    for f, b in enumerate(clouds):
        cap = off[f + 1] - off[f]
        B = torch.zeros((5, cap), device="cuda")
        B[:, :b.shape[1]] = torch.from_numpy(b)
        nd = torch.tensor([b.shape[1]], dtype=torch.int32, device="cuda")
        lf = torch.zeros(5, dtype=torch.float64, device="cuda")
        nf = torch.zeros(5, dtype=torch.int32, device="cuda")
        single.reconstruct(Y[f].contiguous(), B, nd, stages, grow=gp, loss_log=lf, n_log=nf)
        assert single.sync_status() == 0
        np.testing.assert_array_equal(nlog[:, f], nf.cpu().numpy())
        np.testing.assert_allclose(loss[:, f], lf.cpu().numpy(), rtol=1e-12)
        m = int(nd.item())
        assert int(n_dev[f].item()) == m
        assert torch.equal(packed[:, off[f]:off[f] + m], B[:, :m])


def test_autotune_frames_keeps_results(sb):
    wl, arr, single, off, packed, n_dev, clouds = setup(sb)
    arr.set_sampling_level(1)
    S0 = arr.forward_frames(packed, n_dev).clone()
    chunk, split = arr.autotune_frames(packed, n_dev)
    assert chunk in (256, 512, 1024, 1024 | sb.TILE_WIDE) and split in (1, 2, 4, 8)
    assert torch.equal(arr.forward_frames(packed, n_dev), S0)


def test_frame_tiles_change_only_the_launch(sb):
    """Every forward tile of the batched path, narrow or wide, renders the
    default's traces bit for bit; every adjoint split gives the default's
    gradients within float summation order; invalid tiles are refused."""
    wl, arr, single, off, packed, n_dev, clouds = setup(sb)
    W = sb.TILE_WIDE
    with pytest.raises(sb.SlingbagError):
        arr.set_frame_tiles(2048, 0)  # a chunk would straddle two frames
    with pytest.raises(sb.SlingbagError):
        arr.set_frame_tiles(0, 3)
    rng = np.random.default_rng(5)
    for k in range(2):
        arr.set_sampling_level(k)
        arr.set_frame_tiles(0, 0)
        S0 = arr.forward_frames(packed, n_dev).clone()
        G = torch.from_numpy(rng.normal(size=(len(COUNTS), wl.sensors.M, arr.Tk))
                             .astype(np.float32)).cuda()
        g0 = arr.adjoint_frames(packed, n_dev, G).cpu().numpy()
        for tile in (32, 256, 1024, 32 | W, 1024 | W):
            arr.set_frame_tiles(tile, 0)
            assert arr.get_frame_tiles() == (tile, 0)
            assert torch.equal(arr.forward_frames(packed, n_dev), S0), (k, tile)
        for split in (1, 2, 4, 8):
            arr.set_frame_tiles(0, split)
            g = arr.adjoint_frames(packed, n_dev, G).cpu().numpy()
            for f in range(len(COUNTS)):
                sl = slice(off[f], off[f] + COUNTS[f])
                for c in range(5):
                    ref = g0[c, sl]
                    err = np.linalg.norm(g[c, sl] - ref) / max(np.linalg.norm(ref), 1e-30)
                    assert err <= 1e-5, (k, split, f, c)
    arr.set_frame_tiles(0, 0)


def test_reconstruct_frames_replays_in_cuda_graph(sb):
    wl, arr, single, off, packed, n_dev, clouds = setup(sb)
    F = len(COUNTS)
    y = np.stack([oracle.forward(workloads.uniform_balls(200, 2.0, 0.05, 0.2, 0.5, 1.0,
                                                         seed=90 + f).stack(),
                                 wl.sensors.pos, wl.sensors.normal, wl.c, 1 / wl.fs_mhz, wl.T)
                  for f in range(F)]).astype(np.float32)
    Y = torch.from_numpy(y).cuda()
    stages = [sb.Stage(0, 1, 3, True, False), sb.Stage(1, 2, 7, True, True)]
    gp = sb.GrowParams(seed=5, R_max=0.3, g_dup=2.0)
    init, n0 = packed.clone(), n_dev.clone()
    loss = torch.zeros(3 * F, dtype=torch.float64, device="cuda")

    def run():
        arr.reconstruct_frames(Y, packed, n_dev, stages, grow=gp, loss_log=loss)

    run()  # eager; also allocates the scratch
    torch.cuda.synchronize()
    eager = (packed.clone(), n_dev.clone(), loss.clone())
    g = torch.cuda.CUDAGraph()
    packed.copy_(init)
    n_dev.copy_(n0)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        run()
    for _ in range(2):  # replays start from the restored clouds
        packed.copy_(init)
        n_dev.copy_(n0)
        loss.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert arr.sync_status() == 0
        assert torch.equal(n_dev, eager[1])
        assert torch.equal(loss, eager[2])
        for f in range(F):
            m = int(n_dev[f].item())
            assert torch.equal(packed[:, off[f]:off[f] + m], eager[0][:, off[f]:off[f] + m])


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_frames_match_the_oracle_frame_by_frame(sb):
    """Every frame of the batched calls against the FP64 oracle on that
    frame alone (frames are independent reconstructions): traces and all
    five gradients at both levels, one filter/grow pass (counts, order, R,
    p0, gradients and carried state bit for bit, centres to 2e-6 mm), and a
    whole batched reconstruction (zero-gradient filtering, coarse and fine
    stages with growth): ball counts per iteration, losses and final clouds."""
    wl, arr, single, off, packed, n_dev, clouds = setup(sb)
    F, M = len(COUNTS), wl.sensors.M
    pos, nrm = wl.sensors.pos, wl.sensors.normal
    rng = np.random.default_rng(11)
    nt = max(1, oracle.num_procs())
    for k, f_k in enumerate((2, 1)):
        arr.set_sampling_level(k)
        Tk = arr.Tk
        dt = f_k / wl.fs_mhz
        S = arr.forward_frames(packed, n_dev).cpu().numpy()
        G = rng.normal(size=(F, M, Tk)).astype(np.float32)
        g = arr.adjoint_frames(packed, n_dev, torch.from_numpy(G).cuda()).cpu().numpy()
        for f, b in enumerate(clouds):
            ref = oracle.forward(b, pos, nrm, wl.c, dt, Tk, threads=nt)
            assert rel_l2(S[f], ref) <= 1e-5, (k, f)
            gref = oracle.adjoint(b, pos, nrm, wl.c, dt, Tk, G[f].astype(np.float64),
                                  threads=nt)
            n = b.shape[1]
            for c in range(5):
                assert rel_l2(g[c, off[f]:off[f] + n], gref[c]) <= 1e-4, (k, f, c)

    # one filter/grow pass with duplication, frame by frame against oracle.grow
    total = packed.shape[1]
    grads = rng.normal(size=(5, total)).astype(np.float32)
    grads[:, ::7] = 0.0
    extra = rng.normal(size=(4, total)).astype(np.float32)
    P0 = packed.clone()
    Gd = torch.from_numpy(grads).cuda()
    Ed = torch.from_numpy(extra).cuda()
    nd = n_dev.clone()
    gp = dict(seed=4321, R_max=0.3, duplicate=True, g_dup=1.5)
    arr.filter_grow_frames(P0, Gd, nd, mode=sb.GROW, grow=sb.GrowParams(**gp), extra=[Ed])
    assert arr.sync_status() == 0
    counts = nd.cpu().numpy()
    for f, b in enumerate(clouds):
        n = b.shape[1]
        s = slice(off[f], off[f] + n)
        nb, ng, ne, _ = oracle.grow(b, grads[:, s], extra[:, s], oracle.GrowParams(**gp))
        m = nb.shape[1]
        assert counts[f] == m, f
        t = slice(off[f], off[f] + m)
        Bo = P0[:, t].cpu().numpy()
        np.testing.assert_array_equal(Bo[3:], nb[3:])
        np.testing.assert_allclose(Bo[:3], nb[:3], rtol=0, atol=2e-6)
        np.testing.assert_array_equal(Gd[:, t].cpu().numpy(), ng)
        np.testing.assert_array_equal(Ed[:, t].cpu().numpy(), ne)

    # a whole batched reconstruction against the oracle's loop per frame
    y_frames = []
    for f in range(F):
        truth = workloads.uniform_balls(200, 2.0, 0.05, 0.2, 0.5, 1.0, seed=170 + f).stack()
        y = oracle.forward(truth, pos, nrm, wl.c, 1 / wl.fs_mhz, wl.T, threads=nt)
        y_frames.append(workloads.add_noise(y.astype(np.float32), seed=180 + f))
    Y = torch.from_numpy(np.stack(y_frames)).cuda()
    st_o = [oracle.Stage(0, 2, 3, True, False), oracle.Stage(1, 2, 7, True, True)]
    st_g = [sb.Stage(s.level, s.iterations, s.grad_mask, s.grow, s.duplicate) for s in st_o]
    grow = dict(p_min=1e-3, R_min=0.02, R_max=0.3, g_dup=2.0, seed=31)
    loss = torch.zeros(4 * F, dtype=torch.float64, device="cuda")
    nlog = torch.zeros(4 * F, dtype=torch.int32, device="cuda")
    arr.reconstruct_frames(Y, packed, n_dev, st_g, grow=sb.GrowParams(**grow), loss_log=loss,
                           n_log=nlog)
    assert arr.sync_status() == 0
    loss = loss.cpu().numpy().reshape(4, F)
    nlog = nlog.cpu().numpy().reshape(4, F)
    for f, b in enumerate(clouds):
        bo, losses, cnt = oracle.reconstruct(b, pos, nrm, wl.c, wl.fs_mhz, wl.T, (2, 1),
                                             y_frames[f], st_o,
                                             grow_params=oracle.GrowParams(**grow), threads=nt)
        np.testing.assert_array_equal(nlog[:, f], cnt, err_msg=f"frame {f}")
        np.testing.assert_allclose(loss[:, f], losses, rtol=1e-4, err_msg=f"frame {f}")
        m = int(n_dev[f].item())
        assert m == bo.shape[1], f
        np.testing.assert_allclose(packed[:, off[f]:off[f] + m].cpu().numpy(), bo, rtol=0,
                                   atol=1e-4, err_msg=f"frame {f}")
