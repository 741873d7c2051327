"""Pins of the Gaussian-profile radiator oracle: the continuous wave at fine
sampling, zero mean, the adjoint identity and finite differences."""
import numpy as np
import pytest

import oracle


def one_ball(x=0.3, y=-0.2, z=0.1, a=0.12, p0=0.8):
    return np.array([[x], [y], [z], [a], [p0]])


SENS = np.array([[0.0, 0.0, 20.0], [12.0, -3.0, 15.0], [-14.0, 5.0, 11.0]])
NRM = -SENS / np.linalg.norm(SENS, axis=1, keepdims=True)


def test_fine_sampling_reaches_the_continuous_wave():
    b = one_ball()
    c, dt, T = 1.5, 0.0005, 40000
    S = oracle.forward_gauss(b, SENS[:1], NRM[:1], c, dt, T)[0]
    d = np.linalg.norm(b[:3, 0] - SENS[0])
    w = max(0.0, float(NRM[0] @ (b[:3, 0] - SENS[0])) / d)
    t = (np.arange(T) + 0.5) * dt
    e = d - c * t
    p = 0.8 * w * e * np.exp(-e * e / (2 * 0.12 ** 2)) / (2 * d)
    assert np.max(np.abs(S - p)) < 1e-4 * np.max(np.abs(p))


def test_zero_mean_and_linearity():
    b = np.hstack([one_ball(), one_ball(0.5, 0.4, -0.3, 0.08, 0.3)])
    c, dt, T = 1.5, 0.025, 2048
    S = oracle.forward_gauss(b, SENS, NRM, c, dt, T)
    assert np.max(np.abs(S.sum(axis=1))) < 1e-12 * np.max(np.abs(S))  # telescoping
    S1 = oracle.forward_gauss(b[:, :1], SENS, NRM, c, dt, T)
    S2 = oracle.forward_gauss(b[:, 1:], SENS, NRM, c, dt, T)
    np.testing.assert_allclose(S, S1 + S2, rtol=1e-13, atol=1e-15)


def test_near_pairs_are_skipped_and_counted():
    b = one_ball(0.0, 0.0, 19.5, a=0.1)  # 0.5 mm from the first sensor < 6 a
    _, inside = oracle.forward_gauss(b, SENS, NRM, 1.5, 0.025, 2048, return_inside=True)
    assert inside == 1


def test_adjoint_identity_for_p0():
    rng = np.random.default_rng(0)
    n = 6
    b = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(-1, 1, n),
                  rng.uniform(0.05, 0.2, n), np.ones(n)])
    c, dt, T = 1.5, 0.025, 2048
    cols = []
    for i in range(n):
        bi = b[:, i:i + 1]
        cols.append(oracle.forward_gauss(bi, SENS, NRM, c, dt, T).reshape(-1))
    A = np.stack(cols, axis=1)
    y = rng.normal(size=(3, T))
    g = oracle.adjoint_gauss(b, SENS, NRM, c, dt, T, y)
    np.testing.assert_allclose(g[4], A.T @ y.reshape(-1), rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("comp", [0, 1, 2, 3])
def test_gradients_match_central_differences(comp):
    rng = np.random.default_rng(1)
    b = np.hstack([one_ball(), one_ball(-0.4, 0.2, 0.6, 0.15, 0.5)])
    c, dt, T = 1.5, 0.025, 2048
    G = rng.normal(size=(3, T))
    g = oracle.adjoint_gauss(b, SENS, NRM, c, dt, T, G)
    for i in range(2):
        hstep = 1e-6
        bp, bm = b.copy(), b.copy()
        bp[comp, i] += hstep
        bm[comp, i] -= hstep
        fd = (np.sum(G * oracle.forward_gauss(bp, SENS, NRM, c, dt, T)) -
              np.sum(G * oracle.forward_gauss(bm, SENS, NRM, c, dt, T))) / (2 * hstep)
        assert g[comp, i] == pytest.approx(fd, rel=1e-6, abs=1e-10)
