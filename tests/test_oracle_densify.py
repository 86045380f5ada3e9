"""Pins of the resampling and densify / prune oracle against facts that do not
come from the oracle itself: the defining triangular system, the covariance of
many draws against a library inverse, closed forms for diagonal factors, and
hand-built cases whose outcome the rules fix."""
import math

import numpy as np
import pytest

from oracle import densify as D

BETA = 1e-4
DC = dict(grad_threshold=2e-4, min_opacity=0.005, size_threshold=0.01, split_factor=1.6)


def _tri_column(rng, scale=1.0):
    p = np.zeros(11)
    p[0:3] = rng.uniform(-1, 1, 3)
    p[3:9] = rng.uniform(-2, 2, 6) * scale
    p[[3, 6, 8]] = rng.uniform(2, 6, 3)
    p[9] = 1.0
    p[10] = 0.5
    return p


def test_sample_solves_the_transposed_factor():
    """w = y - mu satisfies L^T w = z (not L w = z, not L^-1 z)."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        p = _tri_column(rng)
        z = rng.normal(size=3)
        w = D.sample_offset(p, D.COV_TRI, BETA, z)
        L = D.tri_factor(p, BETA)
        np.testing.assert_allclose(L.T @ w, z, rtol=1e-12, atol=1e-12)
        assert not np.allclose(L @ w, z)


def test_sample_covariance_is_the_inverse_precision():
    """The covariance of 100,000 draws matches inv(L L^T) (a library inverse)."""
    rng = np.random.default_rng(1)
    p = _tri_column(rng)
    p[4:6] = [3.0, -2.0]
    p[7] = 1.5
    m = 100000
    z = rng.normal(size=(3, m))
    y = D.sample(p[:, None], D.COV_TRI, BETA, np.zeros(m, np.int64), z)
    L = D.tri_factor(p, BETA)
    sigma = np.linalg.inv(L @ L.T)
    emp = np.cov(y)
    scale = np.sqrt(np.outer(np.diag(sigma), np.diag(sigma)))
    assert np.max(np.abs(emp - sigma) / scale) < 0.02
    np.testing.assert_allclose(y.mean(axis=1), p[0:3], atol=4 * np.sqrt(np.diag(sigma) / m).max())


def test_sample_diagonal_factor_closed_form():
    rng = np.random.default_rng(2)
    p = _tri_column(rng)
    p[[4, 5, 7]] = 0.0
    z = rng.normal(size=3)
    w = D.sample_offset(p, D.COV_TRI, BETA, z)
    np.testing.assert_allclose(w, z / (p[[3, 6, 8]] ** 2 + BETA), rtol=1e-14)


def test_sample_scale_rotation_covariance():
    rng = np.random.default_rng(3)
    p = np.zeros(12)
    p[3:6] = np.log([0.3, 0.05, 0.01])
    p[6:10] = rng.normal(size=4)
    m = 100000
    z = rng.normal(size=(3, m))
    y = D.sample(p[:, None], D.COV_SCALE_ROT, BETA, np.zeros(m, np.int64), z)
    q = p[6:10] / np.linalg.norm(p[6:10])
    R = D.rotation(q)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)
    sigma = R @ np.diag(np.exp(2 * p[3:6])) @ R.T
    emp = np.cov(y)
    scale = np.sqrt(np.outer(np.diag(sigma), np.diag(sigma)))
    assert np.max(np.abs(emp - sigma) / scale) < 0.02


def test_tri_trace_fp32_is_the_trace_of_sigma():
    rng = np.random.default_rng(4)
    for _ in range(20):
        p = _tri_column(rng)
        L = D.tri_factor(p, BETA)
        ref = np.trace(np.linalg.inv(L @ L.T))
        got = float(D.tri_trace32(p.astype(np.float32), np.float32(BETA)))
        assert abs(got - ref) <= 1e-5 * ref


def _cases():
    """Four Gaussians: faded (pruned), quiet (kept), small and busy (cloned),
    large and busy (split)."""
    rng = np.random.default_rng(5)
    P = np.stack([_tri_column(rng) for _ in range(4)], 1)
    P[9, 0] = math.log(0.004 / 0.996)          # opacity 0.004 < 0.005
    P[[3, 6, 8], 2] = 30.0                      # L_kk = 900: trace Sigma ~ 3.7e-6 < 1e-4
    P[[4, 5, 7], 2] = 0.0
    P[[3, 6, 8], 3] = 2.0                       # L_kk = 4: trace Sigma ~ 0.19 > 1e-4
    stats = np.zeros((2, 4))
    stats[:, 0] = [1.0, 1.0]                    # busy but faded
    stats[:, 1] = [1e-5, 2.0]                   # mean 5e-6: quiet
    stats[:, 2] = [3e-3, 2.0]                   # mean 1.5e-3: busy
    stats[:, 3] = [3e-3, 2.0]
    return P, stats


def test_densify_rules_on_handmade_cases():
    P, stats = _cases()
    m = np.arange(44, dtype=np.float64).reshape(11, 4) + 1.0
    v = m * 2
    rng = np.random.default_rng(6)
    z = rng.normal(size=(6, 4))
    out, mo, vo, act = D.densify(P.astype(np.float32), m, v, stats, z, D.COV_TRI, BETA, DC)
    assert list(act) == [0, 1, 2, 3]
    assert out.shape == (11, 5)
    P32 = P.astype(np.float32).astype(np.float64)
    # kept with its moments, then the original and a moment-free clone
    np.testing.assert_array_equal(out[:, 0], P32[:, 1])
    np.testing.assert_array_equal(mo[:, 0], m[:, 1])
    np.testing.assert_array_equal(out[:, 1], P32[:, 2])
    np.testing.assert_array_equal(out[:, 2], P32[:, 2])
    np.testing.assert_array_equal(mo[:, 1], m[:, 2])
    assert not mo[:, 2].any() and not vo[:, 2].any()
    # two children of the split Gaussian: precision phi^2 L L^T, means mu + L^-T z
    L = D.tri_factor(P32[:, 3], BETA)
    for c in range(2):
        ch = out[:, 3 + c]
        Lc = D.tri_factor(ch, BETA)
        np.testing.assert_allclose(Lc @ Lc.T, 1.6 ** 2 * (L @ L.T), rtol=1e-12)
        np.testing.assert_allclose(L.T @ (ch[0:3] - P32[0:3, 3]), z[3 * c:3 * c + 3, 3], rtol=1e-12)
        assert ch[9] == P32[9, 3] and ch[10] == P32[10, 3]
        assert not mo[:, 3 + c].any()


def test_densify_scale_rotation_split_and_prune_all():
    rng = np.random.default_rng(7)
    P = np.zeros((12, 2))
    P[3:6, 0] = np.log([0.05, 0.02, 0.01])      # largest scale 0.05 > 0.01: split
    P[3:6, 1] = np.log([0.005, 0.002, 0.001])   # 0.005: clone
    P[6:10] = rng.normal(size=(4, 2))
    P[10] = 2.0
    stats = np.array([[1.0, 1.0], [1.0, 1.0]])
    z = rng.normal(size=(6, 2))
    out, mo, vo, act = D.densify(P.astype(np.float32), P * 0, P * 0, stats, z, D.COV_SCALE_ROT,
                                 BETA, DC)
    assert list(act) == [3, 2]
    np.testing.assert_allclose(out[3:6, 0], P.astype(np.float32)[3:6, 0] - math.log(1.6), rtol=1e-6)
    P[10] = -10.0                                # every opacity below 0.005
    out, _, _, act = D.densify(P.astype(np.float32), P * 0, P * 0, stats, z, D.COV_SCALE_ROT,
                               BETA, DC)
    assert out.shape == (12, 0) and not act.any()


def test_stats_update_counts_only_seen_gaussians():
    g = np.array([[3.0, 0.0], [4.0, 0.0], [0.0, 0.0]])
    s = D.stats_update(g, np.zeros((2, 2)))
    np.testing.assert_array_equal(s, [[5.0, 0.0], [1.0, 0.0]])
