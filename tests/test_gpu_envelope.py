"""Envelope mesh, ray-casting initialisation and voxel grid on the GPU against
the FP64 oracle (oracle/envelope.py)."""
import numpy as np
import pytest
import torch

from oracle import envelope as E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    import __graft_entry__ as ge

    ge.build()
    from paper_2601_00551_gb300 import slingbag

    torch.cuda.set_device(0)
    return slingbag


def ellipsoid_sensors(M, axes=(12.0, 15.0, 8.0), seed=11):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(M, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return (v * np.array(axes)).astype(np.float32)


def margin(eq, x):
    """Signed distance to the nearest hull plane (negative inside)."""
    return float(np.max(eq[:, :3] @ x + eq[:, 3]))


def test_hull_matches_qhull(sb):
    from scipy.spatial import ConvexHull

    for M, seed in ((64, 1), (500, 2)):
        P = ellipsoid_sensors(M, seed=seed)
        env = sb.Envelope(P)
        V, T = E.envelope_mesh(P)
        assert env.volume == pytest.approx(E.mesh_volume(V, T), rel=1e-12)
        assert env.volume == pytest.approx(ConvexHull(P.astype(np.float64)).volume, rel=1e-12)
        tri = env.faces()
        assert tri.shape == T.shape
        assert set(np.unique(tri)) == set(np.unique(T))
        # every face is outward: all sensors lie behind it
        P64 = P.astype(np.float64)
        for a, b, c in tri:
            n = np.cross(P64[b] - P64[a], P64[c] - P64[a])
            assert np.max((P64 - P64[a]) @ n) <= 1e-9 * np.linalg.norm(n) * 30
        env.close()


def test_flat_array_is_rejected(sb):
    P = np.random.default_rng(0).normal(size=(30, 3)).astype(np.float32)
    P[:, 2] = 1.5
    with pytest.raises(sb.SlingbagError):
        sb.Envelope(P)


@pytest.mark.parametrize("inset", [0.0, 1.5])
def test_classify_matches_oracle(sb, inset):
    from scipy.spatial import ConvexHull

    P = ellipsoid_sensors(64)
    env = sb.Envelope(P)
    V, T = E.envelope_mesh(P)
    eq = ConvexHull(P.astype(np.float64)).equations
    rng = np.random.default_rng(5)
    X = rng.uniform(-14, 14, size=(1500, 3)).astype(np.float32)
    flags = env.classify(torch.from_numpy(np.ascontiguousarray(X.T)).cuda(), inset).cpu().numpy()
    checked = 0
    for x, f in zip(X.astype(np.float64), flags):
        s = margin(eq, x)
        if abs(s) < 1e-6 or abs(s + inset) < 1e-6:
            continue  # on the surface or the inset surface: either answer is valid
        assert bool(f) == E.in_region(V, T, x, inset)
        checked += 1
    assert checked > 1400 and flags.sum() > 100
    env.close()


def test_sample_matches_oracle(sb):
    P = ellipsoid_sensors(64)
    env = sb.Envelope(P)
    V, T = E.envelope_mesh(P)
    n_want, n_cand, seed, inset = 300, 1500, 12345, 1.0
    out, n_dev = env.sample(n_want, n_cand, seed, inset=inset)
    ref, idx = E.sample_cloud(V, T, n_want, seed, inset, 0, n_cand)
    n = int(n_dev.item())
    assert n == ref.shape[1] == n_want
    np.testing.assert_array_equal(out[:, :n].cpu().numpy(), ref)
    # a shorter candidate range stops early; a later range continues the stream
    out2, n2 = env.sample(200, 200, seed, inset=inset, out=torch.zeros((5, 200)).cuda())
    ref2, _ = E.sample_cloud(V, T, 10 ** 6, seed, inset, 0, 200)
    assert int(n2.item()) == ref2.shape[1]
    np.testing.assert_array_equal(out2[:, :ref2.shape[1]].cpu().numpy(), ref2)
    out3, n3 = env.sample(50, 400, seed, inset=inset, first=700)
    ref3, _ = E.sample_cloud(V, T, 50, seed, inset, 700, 400)
    np.testing.assert_array_equal(out3[:, :int(n3.item())].cpu().numpy(), ref3)
    env.close()


def random_balls(n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(-3, 3, n), rng.uniform(-2, 2.5, n), rng.uniform(-1.5, 1.5, n),
                     rng.uniform(0.02, 0.4, n), rng.uniform(-1, 1, n)]).astype(np.float32)


def test_voxelize_matches_oracle(sb):
    b = random_balls(1200, 3)
    origin, h, dims = (-3.2, -2.1, -1.6), 0.1, (64, 46, 32)
    ref = E.voxelize(b, origin, h, dims)
    B = torch.from_numpy(b).cuda()
    got = sb.voxelize(B, origin, h, dims).cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(got != 0, ref != 0)
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-9 * np.abs(ref).max())
    # live count and explicit values
    n_dev = torch.tensor([700], dtype=torch.int32, device="cuda")
    vals = torch.rand(1200, device="cuda")
    got2 = sb.voxelize(B, origin, h, dims, n_dev=n_dev, values=vals).cpu().numpy()
    ref2 = E.voxelize(b[:, :700], origin, h, dims, values=vals[:700].cpu().numpy())
    np.testing.assert_allclose(got2, ref2, rtol=1e-6, atol=1e-9 * np.abs(ref2).max())


def test_voxelize_is_order_independent(sb):
    b = random_balls(3000, 4)
    perm = np.random.default_rng(0).permutation(3000)
    origin, h, dims = (-3.2, -2.1, -1.6), 0.05, (128, 92, 64)
    scratch = torch.zeros(128 * 92 * 64 + 1, dtype=torch.int64, device="cuda")
    v1 = sb.voxelize(torch.from_numpy(b).cuda(), origin, h, dims, scratch=scratch).clone()
    v2 = sb.voxelize(torch.from_numpy(np.ascontiguousarray(b[:, perm])).cuda(), origin, h, dims,
                     scratch=scratch)
    assert torch.equal(v1, v2)
    assert int(scratch.count_nonzero().item()) == 0  # left zero for the next call


def test_voxelize_exact_on_sphere_boundaries(sb):
    """Balls centred on voxel centres with radii whose squares are sums of
    three squares of voxel steps (R = 0.5, 0.75, 1, 1.25 at h = 0.25): many
    voxel centres lie exactly on a sphere (d^2 = R^2 in every precision),
    some radii are one float step larger. The float screen must hand those
    to the exact test and agree with the oracle's strict <."""
    h = 0.25
    origin, dims = (-4.0, -4.0, -4.0), (32, 32, 32)
    rng = np.random.default_rng(9)
    ijk = rng.integers(6, 26, size=(400, 3))
    c = (np.array(origin) + (ijk + 0.5) * h).astype(np.float32)
    R = rng.choice(np.array([0.5, 0.75, 1.0, 1.25], dtype=np.float32), 400)
    R = np.where(rng.uniform(size=400) < 0.3, np.nextafter(R, np.float32(2)), R).astype(np.float32)
    b = np.stack([c[:, 0], c[:, 1], c[:, 2], R, rng.uniform(0.1, 1.0, 400)]).astype(np.float32)
    ref = E.voxelize(b, origin, h, dims)
    got = sb.voxelize(torch.from_numpy(b).cuda(), origin, h, dims).cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(got != 0, ref != 0)
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-9 * np.abs(ref).max())
