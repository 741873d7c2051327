"""GPU parity: the sm_103a library, called through its C ABI, against the FP64
oracle on identical seeded inputs.

Bars (from the method's accuracy target): traces within relative L2 1e-5,
gradients within relative L2 1e-4 per component, integer decisions (which
balls survive filtering, which split or duplicate, in which order)
identical outside the oracle's list of sign-ambiguous balls.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-5
GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def sb():
    import __graft_entry__ as ge

    ge.build()
    from paper_2601_00551_gb300 import slingbag

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return slingbag


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def threads():
    return max(1, oracle.num_procs())


def make_array(sb, wl, factors, n_cap, wmode="clamp"):
    return sb.SensorArray(wl.sensors.pos, wl.sensors.normal, wl.c, wl.fs_mhz, wl.T, factors,
                          n_cap=n_cap, weight_mode=wmode)


def dt_of(wl, f):
    return f / wl.fs_mhz


# ------------------------------------------------------------------ forward

@pytest.mark.parametrize("wmode", ["clamp", "cos", "none"])
def test_forward_tiny_all_levels(sb, wmode):
    wl = workloads.tiny()
    b = wl.init.stack()
    arr = make_array(sb, wl, (4, 2, 1), b.shape[1], wmode)
    balls = torch.from_numpy(b).cuda()
    for k, f in enumerate((4, 2, 1)):
        arr.set_sampling_level(k)
        S = arr.forward(balls).cpu().numpy()
        ref = oracle.forward(b, wl.sensors.pos, wl.sensors.normal, wl.c, dt_of(wl, f),
                             wl.T // f, wmode=wmode, threads=threads())
        assert np.count_nonzero(ref) > 0
        e = rel_l2(S, ref)
        assert e <= TRACE_TOL, (f, e)
        # element-wise: no single sample far off
        assert np.max(np.abs(S - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_forward_is_bitwise_deterministic_and_order_independent(sb):
    wl = workloads.tiny()
    b = wl.init.stack()
    arr = make_array(sb, wl, (1,), b.shape[1])
    S1 = arr.forward(torch.from_numpy(b).cuda()).cpu().numpy()
    S2 = arr.forward(torch.from_numpy(b).cuda()).cpu().numpy()
    perm = np.random.default_rng(0).permutation(b.shape[1])
    S3 = arr.forward(torch.from_numpy(np.ascontiguousarray(b[:, perm])).cuda()).cpu().numpy()
    assert np.array_equal(S1, S2)
    assert np.array_equal(S1, S3)


def test_forward_edge_cases(sb):
    wl = workloads.tiny(M=8, T=600)
    pos, nrm = wl.sensors.pos, wl.sensors.normal
    cap = 1000
    arr = make_array(sb, wl, (3, 1), cap)   # 600 / 3 = 200 samples at level 0
    rng = np.random.default_rng(4)
    b = wl.init.stack()[:, :cap].copy()
    # a few balls beyond the record, one on top of sensor 0 (d <= R), one with p0 = 0
    b[:3, 0] = [0.0, 0.0, 60.0]
    b[:3, 1] = pos[0] + np.float32(0.01)
    b[3, 1] = 0.2
    b[4, 2] = 0.0
    balls = torch.from_numpy(b).cuda()
    for k, f in enumerate((3, 1)):
        arr.set_sampling_level(k)
        Tk = -(-600 // f)
        # ragged live count: garbage beyond n must be ignored
        for n in (0, 1, 37, 513, cap):
            junk = balls.clone()
            junk[:, n:] = torch.from_numpy(rng.normal(size=(5, cap - n)).astype(np.float32)).cuda()
            S = arr.forward(junk, n=n).cpu().numpy()
            ref, inside = oracle.forward(b[:, :n], pos, nrm, wl.c, dt_of(wl, f), Tk,
                                         return_inside=True)
            if n == 0:
                assert np.all(S == 0)
            else:
                assert rel_l2(S, ref) <= TRACE_TOL, (f, n)
    # the d <= R pair is counted (once per forward that sees it)
    assert arr.inside_pairs() > 0


def test_forward_latches_non_finite_balls(sb):
    """A live ball with a NaN or infinite value latches SBP_ERR_NUMERIC (read
    and cleared by sbp_sync_status); the same ball past the live count does
    not."""
    wl = workloads.tiny(M=8, T=256)
    b = wl.init.stack()[:, :300].copy()
    arr = make_array(sb, wl, (1,), b.shape[1])
    balls = torch.from_numpy(b).cuda()
    arr.forward(balls)
    assert arr.sync_status() == 0
    for row, bad in ((4, np.nan), (0, np.inf), (3, -np.inf)):
        b2 = b.copy()
        b2[row, 123] = bad
        bd = torch.from_numpy(b2).cuda()
        arr.forward(bd)
        assert arr.sync_status() == sb.SBP_ERR_NUMERIC, (row, bad)
        assert arr.sync_status() == 0  # cleared by the read
        arr.forward(bd, n=torch.tensor([100], dtype=torch.int32, device="cuda"))
        assert arr.sync_status() == 0


def test_forward_vessel_sampled_sensors(sb):
    """Full-size vessel workload (200k balls, 512 sensors, T = 4096 at 40 MHz and
    the 10 / 20 MHz levels) in the benchmark's launch configuration; the oracle
    evaluates a sample of sensors exactly."""
    wl = workloads.vessel()
    b = wl.init.stack()
    arr = make_array(sb, wl, wl.levels, b.shape[1])
    balls = torch.from_numpy(b).cuda()
    pick = np.array([0, 77, 255, 300, 511])
    for k, f in enumerate(wl.levels):
        arr.set_sampling_level(k)
        S = arr.forward(balls).cpu().numpy()
        ref = oracle.forward(b, wl.sensors.pos[pick], wl.sensors.normal[pick], wl.c,
                             dt_of(wl, f), wl.T // f, threads=threads())
        e = rel_l2(S[pick], ref)
        assert e <= TRACE_TOL, (f, e)


def test_unsorted_cloud_long_windows(sb):
    """A cloud in random order: a chunk's balls span the whole 20 mm cube, so
    the forward adds most impulses past its shared-memory window straight to
    the global accumulators, and the adjoint stages windows of up to ~930
    cells at 40 MHz, a few sensors per group (many groups per CTA)."""
    wl = workloads.vessel(n_init=20000, n_truth=2000, sort=False)
    b = wl.init.stack()
    arr = make_array(sb, wl, wl.levels, b.shape[1])
    balls = torch.from_numpy(b).cuda()
    pick_s = np.array([3, 200, 444])
    pick_b = np.random.default_rng(1).choice(b.shape[1], 200, replace=False)
    rng = np.random.default_rng(2)
    for k, f in enumerate(wl.levels):
        Tk = wl.T // f
        arr.set_sampling_level(k)
        S = arr.forward(balls).cpu().numpy()
        ref = oracle.forward(b, wl.sensors.pos[pick_s], wl.sensors.normal[pick_s], wl.c,
                             dt_of(wl, f), Tk, threads=threads())
        assert rel_l2(S[pick_s], ref) <= TRACE_TOL, (f, "forward")
        G = rng.normal(size=(wl.sensors.M, Tk)).astype(np.float32)
        g = arr.adjoint(balls, torch.from_numpy(G).cuda()).cpu().numpy()
        gref = oracle.adjoint(b[:, pick_b], wl.sensors.pos, wl.sensors.normal, wl.c,
                              dt_of(wl, f), Tk, G.astype(np.float64), threads=threads())
        for c in range(5):
            assert rel_l2(g[c, pick_b], gref[c]) <= GRAD_TOL, (f, c)


# ---------------------------------------------------------- residual, level

def test_downsample_and_residual(sb):
    wl = workloads.tiny(M=16, T=1000)
    rng = np.random.default_rng(1)
    y = rng.normal(size=(16, 1000)).astype(np.float32)
    arr = make_array(sb, wl, (8, 3, 1), 10)
    for k, f in enumerate((8, 3, 1)):
        yk = arr.set_sampling_level(k, torch.from_numpy(y).cuda()).cpu().numpy()
        np.testing.assert_allclose(yk, oracle.downsample(y, f), rtol=1e-6, atol=1e-6)
    arr.set_sampling_level(2)
    S = rng.normal(size=(16, 1000)).astype(np.float32)
    G, loss = arr.residual(torch.from_numpy(S).cuda(), torch.from_numpy(y).cuda())
    L_ref, G_ref = oracle.loss_and_residual(S, y)
    np.testing.assert_allclose(G.cpu().numpy(), G_ref, rtol=1e-6, atol=1e-6)
    assert abs(loss.item() - L_ref) <= 1e-9 * L_ref
    G0, _ = arr.residual(None, torch.from_numpy(y).cuda(), want_loss=False)
    np.testing.assert_array_equal(G0.cpu().numpy(), -2 * y)
    # reproducible loss
    _, loss2 = arr.residual(torch.from_numpy(S).cuda(), torch.from_numpy(y).cuda())
    assert loss2.item() == loss.item()


# ------------------------------------------------------------------ adjoint

_MEASURED = {}


def _measured(wl, f, noise=True):
    """'Measured' traces: the oracle's forward of the ground-truth cloud at the
    finest level, rounded to float32, plus 1% Gaussian noise."""
    key = (wl.name, noise)
    if key not in _MEASURED:
        y = oracle.forward(wl.truth.stack(), wl.sensors.pos, wl.sensors.normal, wl.c,
                           dt_of(wl, 1), wl.T, threads=threads())
        y = y.astype(np.float32)
        _MEASURED[key] = workloads.add_noise(y) if noise else y
    return _MEASURED[key]


@pytest.mark.parametrize("wmode", ["clamp", "cos"])
def test_adjoint_tiny_all_components(sb, wmode):
    wl = workloads.tiny()
    b = wl.init.stack()
    n = b.shape[1]
    arr = make_array(sb, wl, (4, 1), n, wmode)
    y = _measured(wl, 1)
    balls = torch.from_numpy(b).cuda()
    for k, f in enumerate((4, 1)):
        Tk = wl.T // f
        S = oracle.forward(b, wl.sensors.pos, wl.sensors.normal, wl.c, dt_of(wl, f), Tk,
                           wmode=wmode, threads=threads())
        yk = oracle.downsample(y, f)
        G = (2.0 * (S - yk)).astype(np.float32)
        arr.set_sampling_level(k)
        g = arr.adjoint(balls, torch.from_numpy(G).cuda()).cpu().numpy()
        ref = oracle.adjoint(b, wl.sensors.pos, wl.sensors.normal, wl.c, dt_of(wl, f), Tk,
                             G.astype(np.float64), wmode=wmode, threads=threads())
        for c in range(5):
            e = rel_l2(g[c], ref[c])
            assert e <= GRAD_TOL, (f, c, e)
        gc = arr.adjoint(balls, torch.from_numpy(G).cuda(), mask=sb.MASK_P0 | sb.MASK_R)
        gc = gc.cpu().numpy()
        assert np.all(gc[:3] == 0)
        np.testing.assert_array_equal(gc[3:], g[3:])


def test_adjoint_small_cloud_is_deterministic(sb):
    """Few balls (small chunks): bitwise reproducible and at parity."""
    wl = workloads.tiny(n_init=150)
    b = wl.init.stack()
    arr = make_array(sb, wl, (1,), b.shape[1])
    rng = np.random.default_rng(2)
    G = rng.normal(size=(wl.sensors.M, wl.T)).astype(np.float32)
    g1 = arr.adjoint(torch.from_numpy(b).cuda(), torch.from_numpy(G).cuda()).cpu().numpy()
    g2 = arr.adjoint(torch.from_numpy(b).cuda(), torch.from_numpy(G).cuda()).cpu().numpy()
    assert np.array_equal(g1, g2)
    ref = oracle.adjoint(b, wl.sensors.pos, wl.sensors.normal, wl.c, dt_of(wl, 1), wl.T,
                         G.astype(np.float64))
    for c in range(5):
        assert rel_l2(g1[c], ref[c]) <= GRAD_TOL, c


def test_adjoint_vessel_sampled_balls(sb):
    """Full-size vessel workload: gradients of a sample of balls at each level,
    against the oracle's, for G = -2 y_k (the zero-gradient pass)."""
    wl = workloads.vessel()
    b = wl.init.stack()
    arr = make_array(sb, wl, wl.levels, b.shape[1])
    y = _measured(wl, 1, noise=True)
    balls = torch.from_numpy(b).cuda()
    pick = np.random.default_rng(5).choice(b.shape[1], 300, replace=False)
    for k, f in enumerate(wl.levels):
        yk = arr.set_sampling_level(k, torch.from_numpy(y).cuda())
        G, _ = arr.residual(None, yk, want_loss=False)
        g = arr.adjoint(balls, G).cpu().numpy()
        Gref = -2.0 * oracle.downsample(y, f)
        ref = oracle.adjoint(b[:, pick], wl.sensors.pos, wl.sensors.normal, wl.c, dt_of(wl, f),
                             wl.T // f, Gref, threads=threads())
        for c in range(5):
            e = rel_l2(g[c, pick], ref[c])
            assert e <= GRAD_TOL, (f, c, e)


# --------------------------------------------------------- filtering, growth

@pytest.mark.parametrize("mode", [0, 1, 2])
def test_zero_gradient_filter_survivors(sb, mode):
    wl = workloads.tiny()
    b = wl.init.stack()
    n = b.shape[1]
    arr = make_array(sb, wl, (4, 1), n)
    y = _measured(wl, 1)
    yk = arr.set_sampling_level(0, torch.from_numpy(y).cuda())
    G, _ = arr.residual(None, yk, want_loss=False)
    balls = torch.from_numpy(b).cuda()
    g = arr.adjoint(balls, G, mask=sb.MASK_P0)
    n_dev = torch.tensor([n], dtype=torch.int32, device="cuda")
    arr.filter_grow(balls, g, n_dev, mode=mode)
    assert arr.sync_status() == 0
    n_new = int(n_dev.item())
    keep, gref, amb = oracle.zero_gradient_filter(
        b, wl.sensors.pos, wl.sensors.normal, wl.c, dt_of(wl, 4), wl.T // 4,
        oracle.downsample(y, 4), mode=mode)
    assert amb.size == 0, f"{amb.size} sign-ambiguous balls"
    assert n_new == keep.size
    np.testing.assert_array_equal(balls[:, :n_new].cpu().numpy(), b[:, keep])
    # roughly half the random balls survive (the paper retains 106,924 of 200,000)
    if mode == 0:
        assert 0.2 * n < n_new < 0.9 * n


def test_zero_gradient_filter_vessel(sb):
    wl = workloads.vessel()
    b = wl.init.stack()
    n = b.shape[1]
    arr = make_array(sb, wl, wl.levels, n)
    y = _measured(wl, 1)
    yk = arr.set_sampling_level(0, torch.from_numpy(y).cuda())
    G, _ = arr.residual(None, yk, want_loss=False)
    balls = torch.from_numpy(b).cuda()
    g = arr.adjoint(balls, G, mask=sb.MASK_P0)
    gp = g[4].cpu().numpy()
    n_dev = torch.tensor([n], dtype=torch.int32, device="cuda")
    arr.filter_grow(balls, g, n_dev, mode=sb.KEEP_NEG)
    n_new = int(n_dev.item())
    keep, gref, amb = oracle.zero_gradient_filter(
        b, wl.sensors.pos, wl.sensors.normal, wl.c, dt_of(wl, wl.levels[0]),
        wl.T // wl.levels[0], oracle.downsample(y, wl.levels[0]), threads=threads())
    amb_set = set(amb.tolist())
    gpu_keep = set(np.nonzero(gp < 0)[0].tolist())
    ref_keep = set(keep.tolist())
    assert (gpu_keep ^ ref_keep) <= amb_set
    assert n_new == len(gpu_keep)
    assert len(amb_set) <= 1e-3 * n
    # the compacted cloud, element by element and in order: the oracle's
    # survivors, with the GPU's own decision for the ambiguous balls
    order = np.array(sorted((ref_keep - amb_set) | (gpu_keep & amb_set)), dtype=np.int64)
    np.testing.assert_array_equal(balls[:, :n_new].cpu().numpy(), b[:, order])


def _grow_case(rng, n):
    b = np.stack([rng.uniform(-5, 5, n), rng.uniform(-5, 5, n), rng.uniform(-5, 5, n),
                  rng.uniform(0.0, 0.6, n), rng.uniform(-0.01, 1.0, n)]).astype(np.float32)
    g = rng.normal(size=(5, n)).astype(np.float32)
    g[:, rng.random(n) < 0.1] = 0.0
    g[:3, rng.random(n) < 0.1] = 0.0
    return b, g


@pytest.mark.parametrize("duplicate,mask", [(False, 3), (True, 7)])
def test_grow_matches_oracle(sb, duplicate, mask):
    rng = np.random.default_rng(7 + int(duplicate))
    n, cap = 3000, 7000
    b, g = _grow_case(rng, n)
    ex = rng.normal(size=(4, n)).astype(np.float32)
    gp = oracle.GrowParams(seed=12345, grad_mask=mask, duplicate=duplicate, g_dup=1.5)
    nb, ng, ne, counts = oracle.grow(b, g, ex, gp)
    wl = workloads.tiny(M=4, T=64)
    arr = make_array(sb, wl, (1,), cap)
    B = torch.zeros((5, cap), device="cuda")
    Gt = torch.zeros((5, cap), device="cuda")
    E = torch.zeros((4, cap), device="cuda")
    B[:, :n] = torch.from_numpy(b)
    Gt[:, :n] = torch.from_numpy(g)
    E[:, :n] = torch.from_numpy(ex)
    n_dev = torch.tensor([n], dtype=torch.int32, device="cuda")
    arr.filter_grow(B, Gt, n_dev, mode=sb.GROW,
                    grow=sb.GrowParams(seed=12345, grad_mask=mask, duplicate=duplicate,
                                       g_dup=1.5),
                    extra=[E])
    assert arr.sync_status() == 0
    m = int(n_dev.item())
    assert m == nb.shape[1]
    Bo, Go, Eo = B[:, :m].cpu().numpy(), Gt[:, :m].cpu().numpy(), E[:, :m].cpu().numpy()
    np.testing.assert_array_equal(Bo[3:], nb[3:])          # R, p0 bit-exact
    np.testing.assert_allclose(Bo[:3], nb[:3], rtol=0, atol=2e-6)
    np.testing.assert_array_equal(Go, ng)
    np.testing.assert_array_equal(Eo, ne)


def test_grow_capacity_overflow_is_latched(sb):
    rng = np.random.default_rng(3)
    n = 900
    b, g = _grow_case(rng, n)
    b[3] = 0.5  # every ball splits
    b[4] = 0.5
    g[:] = 1.0
    wl = workloads.tiny(M=4, T=64)
    arr = make_array(sb, wl, (1,), 1000)
    B = torch.zeros((5, 1000), device="cuda")
    B[:, :n] = torch.from_numpy(b)
    Gt = torch.ones((5, 1000), device="cuda")
    before = B.clone()
    n_dev = torch.tensor([n], dtype=torch.int32, device="cuda")
    arr.filter_grow(B, Gt, n_dev, mode=sb.GROW, grow=sb.GrowParams())
    assert arr.sync_status() == -3
    assert int(n_dev.item()) == n
    assert torch.equal(B, before)
    assert arr.sync_status() == 0


def test_adam_matches_oracle(sb):
    rng = np.random.default_rng(6)
    n = 1000
    b = rng.normal(size=(5, n)).astype(np.float32)
    g = rng.normal(size=(5, n)).astype(np.float32)
    m = (0.1 * rng.normal(size=(5, n))).astype(np.float32)
    v = (0.1 * rng.random(size=(5, n))).astype(np.float32)
    wl = workloads.tiny(M=4, T=64)
    arr = make_array(sb, wl, (1,), n)
    for mask in (3, 7):
        B, Gt = torch.from_numpy(b).cuda(), torch.from_numpy(g).cuda()
        Mt, Vt = torch.from_numpy(m).cuda(), torch.from_numpy(v).cuda()
        arr.adam_step(B, Gt, Mt, Vt, 3, sb.AdamParams(), mask=mask)
        rb, rm, rv = oracle.adam(b, g, m, v, 3, oracle.AdamParams(), mask=mask)
        # float32 moment updates cancel (beta1 m against (1 - beta1) g): compare
        # against the size of the operands, not of the result
        np.testing.assert_allclose(B.cpu().numpy(), rb, rtol=2e-6, atol=1e-7)
        np.testing.assert_allclose(Mt.cpu().numpy(), rm, rtol=0,
                                   atol=1e-7 * (np.abs(m).max() + np.abs(g).max()))
        np.testing.assert_allclose(Vt.cpu().numpy(), rv, rtol=0,
                                   atol=1e-7 * (np.abs(v).max() + (g * g).max()))


# ------------------------------------------------------------- reconstruct

def test_reconstruct_matches_oracle_loop(sb):
    """sbp_reconstruct (zero-gradient filter, then coarse and fine stages over
    three levels with Adam and growth) against the oracle's loop: identical
    ball counts and losses within float32 round-off, iteration by iteration."""
    wl = workloads.tiny()
    b = wl.init.stack()
    n = b.shape[1]
    y = _measured(wl, 1)
    factors = (4, 2, 1)
    arr = make_array(sb, wl, factors, 2 * n)
    st_o = [oracle.Stage(0, 2, 3, True, False), oracle.Stage(1, 2, 7, True, False),
            oracle.Stage(2, 2, 7, True, True)]
    st_g = [sb.Stage(s.level, s.iterations, s.grad_mask, s.grow, s.duplicate) for s in st_o]
    grow = dict(p_min=1e-3, R_min=0.02, R_max=0.3, g_dup=5.0, seed=77)
    bo, losses, counts = oracle.reconstruct(b, wl.sensors.pos, wl.sensors.normal, wl.c,
                                            wl.fs_mhz, wl.T, factors, y, st_o,
                                            grow_params=oracle.GrowParams(**grow),
                                            threads=threads())
    balls = torch.zeros((5, 2 * n), device="cuda")
    balls[:, :n] = torch.from_numpy(b)
    n_dev = torch.tensor([n], dtype=torch.int32, device="cuda")
    loss = torch.zeros(6, dtype=torch.float64, device="cuda")
    n_log = torch.zeros(6, dtype=torch.int32, device="cuda")
    arr.reconstruct(torch.from_numpy(y).cuda(), balls, n_dev, st_g,
                    grow=sb.GrowParams(**grow), loss_log=loss, n_log=n_log)
    assert arr.sync_status() == 0
    np.testing.assert_array_equal(n_log.cpu().numpy(), counts)
    np.testing.assert_allclose(loss.cpu().numpy(), losses, rtol=1e-4)
    assert int(n_dev.item()) == bo.shape[1]
    # within the first level the loss goes down (levels are not comparable)
    assert losses[1] < losses[0]
    out = balls[:, :bo.shape[1]].cpu().numpy()
    np.testing.assert_allclose(out, bo, rtol=0, atol=1e-4)


def test_fifty_iteration_run_matches_the_oracle_loop(sb):
    """The whole plain-method run of the 2,000-ball x 64-sensor case:
    zero-gradient filtering, then 50 Adam iterations of forward, adjoint and
    filter/grow at 40 MHz, through sbp_reconstruct against the oracle's loop.
    Ball counts per iteration are compared exactly; losses within 1e-3 (float32
    against float64 over 50 coupled iterations). The final cloud is compared
    in units of the learning rate (1e-3 mm for the position and radius, 1e-2
    for p0), the size of one Adam step, lr m_hat / sqrt(v_hat): where a
    component's gradient sits near zero, round-off can flip the sign of a
    step, so single elements may differ by a few steps (bound: five); the
    root-mean-square difference of every row stays within a tenth of one."""
    wl = workloads.tiny()
    b = wl.init.stack()
    n = b.shape[1]
    y = _measured(wl, 1)
    arr = make_array(sb, wl, (1,), 2 * n)
    st_o = [oracle.Stage(0, 50, 7, True, False)]
    st_g = [sb.Stage(0, 50, 7, True, False)]
    grow = dict(p_min=1e-3, R_min=0.02, R_max=0.3, g_dup=5.0, seed=5)
    bo, losses, counts = oracle.reconstruct(b, wl.sensors.pos, wl.sensors.normal, wl.c,
                                            wl.fs_mhz, wl.T, (1,), y, st_o,
                                            grow_params=oracle.GrowParams(**grow),
                                            threads=threads())
    balls = torch.zeros((5, 2 * n), device="cuda")
    balls[:, :n] = torch.from_numpy(b)
    n_dev = torch.tensor([n], dtype=torch.int32, device="cuda")
    loss = torch.zeros(50, dtype=torch.float64, device="cuda")
    n_log = torch.zeros(50, dtype=torch.int32, device="cuda")
    arr.reconstruct(torch.from_numpy(y).cuda(), balls, n_dev, st_g, grow=sb.GrowParams(**grow),
                    loss_log=loss, n_log=n_log)
    assert arr.sync_status() == 0
    np.testing.assert_array_equal(n_log.cpu().numpy(), counts)
    np.testing.assert_allclose(loss.cpu().numpy(), losses, rtol=1e-3)
    assert losses[-1] < 0.5 * losses[0]
    assert int(n_dev.item()) == bo.shape[1]
    out = balls[:, :bo.shape[1]].cpu().numpy()
    lr = np.array(sb.AdamParams().lr)
    for k in range(5):
        d = out[k].astype(np.float64) - bo[k]
        assert np.sqrt(np.mean(d * d)) <= 0.1 * lr[k], (k, np.sqrt(np.mean(d * d)))
        np.testing.assert_allclose(out[k], bo[k], rtol=0, atol=5 * lr[k])


# --------------------------------------------------------------- autograd

def test_autograd_function_matches_oracle_adjoint(sb):
    """torch.autograd through radiate(): L = ||S - y||^2 built from torch ops,
    gradients against the FP64 oracle's adjoint (itself pinned by central
    differences and complex-step derivatives); p0 also against a GPU finite
    difference, exact up to rounding because S is linear in p0."""
    wl = workloads.tiny(n_init=1000)
    b = wl.init.stack()
    arr = make_array(sb, wl, (2, 1), b.shape[1])
    y = _measured(wl, 1)
    for k, f in enumerate((2, 1)):
        Tk = wl.T // f
        yk = torch.from_numpy(oracle.downsample(y, f).astype(np.float32)).cuda()
        leaves = [torch.from_numpy(b[c].copy()).cuda().requires_grad_() for c in range(5)]
        S = sb.radiate(arr, *leaves, level=k)
        L = ((S - yk) ** 2).sum()
        L.backward()
        g = np.stack([t.grad.cpu().numpy() for t in leaves])
        S_ref = oracle.forward(b, wl.sensors.pos, wl.sensors.normal, wl.c, dt_of(wl, f), Tk)
        G = (2.0 * (S.detach().cpu().numpy().astype(np.float64) - yk.cpu().numpy()))
        ref = oracle.adjoint(b, wl.sensors.pos, wl.sensors.normal, wl.c, dt_of(wl, f), Tk, G,
                             threads=threads())
        assert rel_l2(S.detach().cpu().numpy(), S_ref) <= TRACE_TOL
        for c in range(5):
            assert rel_l2(g[c], ref[c]) <= GRAD_TOL, (f, c)
        # p0: finite difference on the GPU path along a random direction
        rng = np.random.default_rng(k)
        v = torch.from_numpy(rng.normal(size=b.shape[1]).astype(np.float32)).cuda()
        eps = 1e-2
        with torch.no_grad():
            def loss(p):
                return float(((sb.radiate(arr, *leaves[:4], p, level=k) - yk) ** 2)
                             .double().sum().item())
            fd = (loss(leaves[4] + eps * v) - loss(leaves[4] - eps * v)) / (2 * eps)
        an = float((leaves[4].grad.double() * v.double()).sum().item())
        assert abs(fd - an) <= 1e-3 * abs(an) + 1e-6


# ------------------------------------------- softplus refinement (Section 4.3)

def test_adam_softplus_matches_oracle(sb):
    rng = np.random.default_rng(11)
    n = 2000
    b = np.abs(rng.normal(size=(5, n))).astype(np.float32) + 0.02
    g = rng.normal(size=(5, n)).astype(np.float32)
    m = (0.1 * rng.normal(size=(5, n))).astype(np.float32)
    v = (0.1 * rng.random(size=(5, n))).astype(np.float32)
    wl = workloads.tiny(M=4, T=64)
    arr = make_array(sb, wl, (1,), n)
    ap = dict(lr=(1e-3, 1e-3, 1e-3, 5e-2, 1e-2))
    mask = sb.MASK_ALL | sb.SOFTPLUS_R
    B, Gt = torch.from_numpy(b).cuda(), torch.from_numpy(g).cuda()
    Mt, Vt = torch.from_numpy(m).cuda(), torch.from_numpy(v).cuda()
    arr.adam_step(B, Gt, Mt, Vt, 4, sb.AdamParams(**ap), mask=mask)
    rb, rm, rv = oracle.adam(b, g, m, v, 4, oracle.AdamParams(**ap), mask=mask)
    np.testing.assert_allclose(B.cpu().numpy(), rb, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(Mt.cpu().numpy(), rm, rtol=0,
                               atol=1e-6 * (np.abs(m).max() + np.abs(g).max()))
    assert np.all(B[3].cpu().numpy() > 0)


def test_reconstruct_with_softplus_refinement_matches_oracle(sb):
    wl = workloads.tiny()
    b = wl.init.stack()
    n = b.shape[1]
    y = _measured(wl, 1)
    factors = (2, 1)
    arr = make_array(sb, wl, factors, 2 * n)
    sp = 7 | oracle.SOFTPLUS_R
    st_o = [oracle.Stage(0, 2, 3, True, False), oracle.Stage(1, 2, 7, True, True),
            oracle.Stage(1, 3, sp, False, False)]
    st_g = [sb.Stage(s.level, s.iterations, s.grad_mask, s.grow, s.duplicate) for s in st_o]
    grow = dict(p_min=1e-3, R_min=0.02, R_max=0.3, g_dup=5.0, seed=5)
    ap = dict(lr=(1e-3, 1e-3, 1e-3, 5e-3, 1e-2))
    bo, losses, counts = oracle.reconstruct(b, wl.sensors.pos, wl.sensors.normal, wl.c,
                                            wl.fs_mhz, wl.T, factors, y, st_o,
                                            adam_params=oracle.AdamParams(**ap),
                                            grow_params=oracle.GrowParams(**grow),
                                            threads=threads())
    balls = torch.zeros((5, 2 * n), device="cuda")
    balls[:, :n] = torch.from_numpy(b)
    n_dev = torch.tensor([n], dtype=torch.int32, device="cuda")
    loss = torch.zeros(7, dtype=torch.float64, device="cuda")
    n_log = torch.zeros(7, dtype=torch.int32, device="cuda")
    arr.reconstruct(torch.from_numpy(y).cuda(), balls, n_dev, st_g, adam=sb.AdamParams(**ap),
                    grow=sb.GrowParams(**grow), loss_log=loss, n_log=n_log)
    assert arr.sync_status() == 0
    np.testing.assert_array_equal(n_log.cpu().numpy(), counts)
    np.testing.assert_allclose(loss.cpu().numpy(), losses, rtol=1e-4)
    out = balls[:, :bo.shape[1]].cpu().numpy()
    np.testing.assert_allclose(out, bo, rtol=0, atol=1e-4)
    assert np.all(out[3] > 0)


# ------------------------------------------------------------- tile choices

def test_tile_choices_and_autotune(sb):
    """The forward's balls per CTA and window shape change only the launch:
    every choice gives bitwise the same traces, also on the cloud in random
    order, where chunks span the whole region and impulses spill past the
    shared window of either shape. Every adjoint cluster split is at parity
    with the oracle. The autotuner keeps a valid choice per level and the
    results stay the same."""
    wl = workloads.vessel(n_init=20000, n_truth=2000)
    b = wl.init.stack()
    arr = make_array(sb, wl, wl.levels, b.shape[1])
    balls = torch.from_numpy(b).cuda()
    pick = np.random.default_rng(7).choice(b.shape[1], 150, replace=False)
    rng = np.random.default_rng(8)
    with pytest.raises(sb.SlingbagError):
        arr.set_tiles(0, 48, 0)
    with pytest.raises(sb.SlingbagError):
        arr.set_tiles(0, 0, 3)
    with pytest.raises(sb.SlingbagError):
        arr.set_tiles(len(wl.levels), 256, 2)
    with pytest.raises(sb.SlingbagError):
        arr.set_tiles(0, 4096 | sb.TILE_WIDE, 0)
    with pytest.raises(sb.SlingbagError):
        arr.set_tiles(0, 3072, 0)
    with pytest.raises(sb.SlingbagError):
        arr.set_tiles(0, 512 | sb.TILE_WIDE | 0x20000, 0)
    W = sb.TILE_WIDE
    shuffled = balls[:, torch.from_numpy(np.random.default_rng(9).permutation(b.shape[1])).cuda()]
    for k, f in enumerate(wl.levels):
        Tk = wl.T // f
        arr.set_sampling_level(k)
        S0 = arr.forward(balls).clone()
        for chunk in (32, 128, 256, 1024, 2048, 32 | W, 512 | W, 2048 | W):
            arr.set_tiles(k, chunk, 0)
            assert arr.get_tiles(k) == (chunk, 0)
            assert torch.equal(arr.forward(balls), S0), (f, chunk)
            assert torch.equal(arr.forward(shuffled), S0), (f, chunk, "random order")
        G = rng.normal(size=(wl.sensors.M, Tk)).astype(np.float32)
        Gd = torch.from_numpy(G).cuda()
        ref = oracle.adjoint(b[:, pick], wl.sensors.pos, wl.sensors.normal, wl.c, dt_of(wl, f),
                             Tk, G.astype(np.float64), threads=threads())
        for split in (1, 2, 8):
            arr.set_tiles(k, 0, split)
            assert arr.get_tiles(k) == (0, split)
            g = arr.adjoint(balls, Gd).cpu().numpy()
            for c in range(5):
                assert rel_l2(g[c, pick], ref[c]) <= GRAD_TOL, (f, split, c)
        arr.set_tiles(k, 0, 0)
        chunk, split = arr.autotune(balls, G=Gd)
        assert chunk in (0, 128, 256, 512, 1024, 2048, 1024 | W, 2048 | W) and \
            split in (0, 1, 2, 4, 8)
        assert arr.get_tiles(k) == (chunk, split)
        assert torch.equal(arr.forward(balls), S0)
        g = arr.adjoint(balls, Gd).cpu().numpy()
        for c in range(5):
            assert rel_l2(g[c, pick], ref[c]) <= GRAD_TOL, (f, "tuned", c)


def test_forward_tiles_with_a_ragged_sensor_group(sb):
    """20 sensors: one group of 32 lanes with 12 empty ones. Every tile shape
    gives the default's traces bit for bit, at parity with the oracle, also
    where windows spill past the record's end (T = 600)."""
    wl = workloads.tiny(M=20, T=600)
    b = wl.init.stack()
    arr = make_array(sb, wl, (2, 1), b.shape[1])
    balls = torch.from_numpy(b).cuda()
    W = sb.TILE_WIDE
    for k, f in enumerate((2, 1)):
        arr.set_sampling_level(k)
        arr.set_tiles(k, 0, 0)
        S0 = arr.forward(balls).clone()
        ref = oracle.forward(b, wl.sensors.pos, wl.sensors.normal, wl.c, dt_of(wl, f),
                             -(-wl.T // f), threads=threads())
        assert rel_l2(S0.cpu().numpy(), ref) <= TRACE_TOL
        for tile in (32, 2048, 32 | W, 512 | W, 2048 | W):
            arr.set_tiles(k, tile, 0)
            assert torch.equal(arr.forward(balls), S0), (f, tile)
        arr.set_tiles(k, 0, 0)


@pytest.mark.parametrize("sort", [False, True])
def test_adjoint_windows_crossing_the_record_end(sb, sort):
    """A record that ends inside the balls' arrival range: the tiny cloud
    reaches the 20 mm cap at cells ~480-590 of 40 MHz and T = 560, so many
    pairs' windows run past the record's end, where the staged windows are
    padded with zeros. Full and p0-only gradients against the oracle at two
    levels, sorted (staged) and unsorted (longer windows, partly unstaged)."""
    wl = workloads.tiny(n_init=1500, T=560, sort=sort)
    b = wl.init.stack()
    n = b.shape[1]
    arr = make_array(sb, wl, (2, 1), n)
    balls = torch.from_numpy(b).cuda()
    rng = np.random.default_rng(12)
    d = np.linalg.norm(b[:3].T[:, None, :] - wl.sensors.pos[None], axis=2)
    for k, f in enumerate((2, 1)):
        Tk = -(-560 // f)
        h = wl.c * dt_of(wl, f)
        assert np.mean((d + b[3][:, None]) / h > Tk) > 0.05  # the case is real
        arr.set_sampling_level(k)
        G = rng.normal(size=(wl.sensors.M, Tk)).astype(np.float32)
        Gd = torch.from_numpy(G).cuda()
        ref = oracle.adjoint(b, wl.sensors.pos, wl.sensors.normal, wl.c, dt_of(wl, f), Tk,
                             G.astype(np.float64), threads=threads())
        g = arr.adjoint(balls, Gd).cpu().numpy()
        for c in range(5):
            assert rel_l2(g[c], ref[c]) <= GRAD_TOL, (f, c)
        gp = arr.adjoint(balls, Gd, mask=sb.MASK_P0).cpu().numpy()
        assert np.all(gp[:4] == 0)
        assert rel_l2(gp[4], ref[4]) <= GRAD_TOL, f


def test_adjoint_unstaged_windows_read_directly(sb):
    """Windows too long to stage next to staged ones in the same CTA: the
    unsorted tiny cloud (a chunk spans the 4 mm cube) sampled at 400 MHz
    reaches 1400-1930 cells of each sensor per chunk, on both sides of the
    1792 cells a staging buffer holds for one window (1024 in the p0-only
    pass, where none is staged). Unstaged windows are read from the global
    row and take no room in a group, so groups mix them with staged ones.
    Full and p0-only gradients against the oracle at 400 MHz and at 200 MHz,
    where every window of the full pass is staged."""
    import dataclasses

    wl = dataclasses.replace(workloads.tiny(n_init=768, M=32, T=6400), fs_mhz=400.0)
    b = wl.init.stack()
    n = b.shape[1]
    h = wl.c / wl.fs_mhz
    spans = []
    for c0 in range(0, n, 128):  # the reach of each 128-ball chunk, in cells
        ch = b[:, c0:c0 + 128]
        lo, hi = ch[:3].min(axis=1), ch[:3].max(axis=1)
        near = np.linalg.norm(np.maximum(np.maximum(lo - wl.sensors.pos, wl.sensors.pos - hi),
                                         0.0), axis=1)
        far = np.linalg.norm(np.maximum(np.abs(wl.sensors.pos - lo), np.abs(wl.sensors.pos - hi)),
                             axis=1)
        spans.append((far - near + 2.0 * ch[3].max()) / h)
    spans = np.concatenate(spans)
    assert 0.2 < np.mean(spans > 1792) < 0.8  # the case is real
    arr = make_array(sb, wl, (2, 1), n)
    balls = torch.from_numpy(b).cuda()
    rng = np.random.default_rng(21)
    for k, f in enumerate((2, 1)):
        Tk = 6400 // f
        arr.set_sampling_level(k)
        G = rng.normal(size=(wl.sensors.M, Tk)).astype(np.float32)
        Gd = torch.from_numpy(G).cuda()
        ref = oracle.adjoint(b, wl.sensors.pos, wl.sensors.normal, wl.c, dt_of(wl, f), Tk,
                             G.astype(np.float64), threads=threads())
        g = arr.adjoint(balls, Gd).cpu().numpy()
        for c in range(5):
            assert rel_l2(g[c], ref[c]) <= GRAD_TOL, (f, c)
        gp = arr.adjoint(balls, Gd, mask=sb.MASK_P0).cpu().numpy()
        assert np.all(gp[:4] == 0)
        assert rel_l2(gp[4], ref[4]) <= GRAD_TOL, f


def test_adjoint_ragged_live_count(sb):
    """A live count below the capacity: the gradients of the live balls equal
    those of the truncated cloud, and the entries past the live count are
    left as they were (for the full and the p0-only kernels)."""
    wl = workloads.tiny(n_init=1000, M=16, T=600)
    b = wl.init.stack()
    cap = b.shape[1]
    arr = make_array(sb, wl, (1,), cap)
    balls = torch.from_numpy(b).cuda()
    rng = np.random.default_rng(31)
    G = torch.from_numpy(rng.normal(size=(wl.sensors.M, 600)).astype(np.float32)).cuda()
    for mask in (sb.MASK_ALL, sb.MASK_P0):
        for n in (1, 129, 700):
            junk = balls.clone()
            junk[:, n:] = torch.from_numpy(rng.normal(size=(5, cap - n)).astype(np.float32)).cuda()
            sentinel = torch.full((5, cap), 7.0, device="cuda")
            g = arr.adjoint(junk, G, n=n, mask=mask, out=sentinel).cpu().numpy()
            assert np.all(g[:, n:] == 7.0), (mask, n)
            ref = arr.adjoint(balls[:, :n].contiguous(), G, mask=mask).cpu().numpy()
            np.testing.assert_array_equal(g[:, :n], ref, err_msg=f"{mask} {n}")
