"""Parity of resampling and the densify / prune step (row f2) with the oracle:
decisions and copies bit-exact (the decisions are taken in FP32 with the same
operation order on both sides), drawn means and children's factors within the
FP32 error of one back substitution."""
import math

import numpy as np
import pytest
import torch

from oracle import densify as D
from paper_2505_05643_gb300 import binding as B
from paper_2505_05643_gb300 import render as R
from paper_2505_05643_gb300 import synth

pytestmark = pytest.mark.gpu


def _params(cov, n, seed, aniso=False):
    rng = np.random.default_rng(seed)
    g = synth.gaussians_anisotropic(rng, n) if aniso else synth.gaussians_scale_rot(rng, n, 0.003, 0.1)
    if cov == B.UG_COV_TRI:
        g = synth.scale_rot_to_tri(g, 1e-4)
    return R.pack_params(g, cov).astype(np.float32)


def _dc_dict(dc):
    return dict(grad_threshold=dc.grad_threshold, min_opacity=dc.min_opacity,
                size_threshold=dc.size_threshold, split_factor=dc.split_factor)


def _check_draws(y32, P, src, z, cov, beta):
    """Drawn points y (FP32) of the Gaussians src against the oracle. TRI: the
    back substitution is backward stable, so the check is its residual,
    |L^T (y - mu) - z| <= 1e-6 (|L^T| |y - mu| + |z|) + |L^T| ulp(y) (a forward
    error bound would need the factor's condition number, up to 1e4 here);
    SCALE_ROT: |y - y_ref| <= 1e-5 |S z| + ulp(y) (R is orthogonal)."""
    y32 = np.asarray(y32, np.float32)
    ulp = np.spacing(np.abs(y32)).astype(np.float64)
    y = y32.astype(np.float64)
    for k in range(y.shape[1]):
        p = P[:, src[k]].astype(np.float64)
        w = y[:, k] - p[0:3]
        if cov == B.UG_COV_TRI:
            LT = D.tri_factor(p, beta).T
            r = np.abs(LT @ w - z[:, k])
            bound = 1e-6 * (np.abs(LT) @ np.abs(w) + np.abs(z[:, k])) + np.abs(LT) @ ulp[:, k]
        else:
            ref = D.sample_offset(p, cov, beta, z[:, k])
            r = np.abs(w - ref)
            bound = 1e-5 * np.abs(np.exp(p[3:6]) * z[:, k]).max() + ulp[:, k]
        assert np.all(r <= bound), (k, r, bound)


@pytest.mark.parametrize("cov", [B.UG_COV_TRI, B.UG_COV_SCALE_ROT])
@pytest.mark.parametrize("aniso", [False, True])
def test_sample_parity(cov, aniso):
    n, m = 20000, 20000
    P = _params(cov, n, 11, aniso)
    rng = np.random.default_rng(12)
    idx = rng.integers(0, n, m).astype(np.int32)
    z = rng.normal(size=(3, m)).astype(np.float32)
    cfg = R.make_config(cov_param=cov)
    y = torch.empty((3, m), device="cuda")
    B.ug_sample(cfg, torch.from_numpy(P).cuda(), n, torch.from_numpy(idx).cuda(), m,
                torch.from_numpy(z).cuda(), y)
    _check_draws(y.cpu().numpy(), P, idx, z.astype(np.float64), cov, cfg.beta)


def test_densify_stats_bit_exact():
    rng = np.random.default_rng(13)
    n = 100003
    g = rng.normal(0, 1e-3, (3, n)).astype(np.float32)
    g[:, rng.random(n) < 0.2] = 0.0
    s0 = rng.random((2, n)).astype(np.float32)
    stats = torch.from_numpy(s0.copy()).cuda()
    B.ug_densify_stats(torch.from_numpy(g).cuda(), n, stats)
    np.testing.assert_array_equal(stats.cpu().numpy(), D.stats_update(g, s0))


def _mixed_case(cov, n, seed):
    """Parameters with every action well represented: a tenth faded, a third
    busy; extents spread across the size threshold."""
    P = _params(cov, n, seed)
    rng = np.random.default_rng(seed + 1)
    row_logit = 9 if cov == B.UG_COV_TRI else 10
    faded = rng.random(n) < 0.1
    P[row_logit, faded] = np.float32(math.log(0.002 / 0.998))
    stats = np.zeros((2, n), np.float32)
    stats[1] = rng.integers(0, 5, n)
    busy = rng.random(n) < 0.35
    stats[0] = np.where(busy, 1e-3, 1e-5).astype(np.float32) * stats[1]
    m = rng.normal(size=P.shape).astype(np.float32)
    v = rng.random(P.shape).astype(np.float32)
    z = rng.normal(size=(6, n)).astype(np.float32)
    return P, m, v, stats, z


def _run_densify(cov, P, m, v, stats, z, cap, dc):
    cfg = R.make_config(cov_param=cov)
    n = P.shape[1]
    rows = P.shape[0]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    po = torch.full((rows, cap), float("nan"), device="cuda")
    mo = torch.full_like(po, float("nan"))
    vo = torch.full_like(po, float("nan"))
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    scratch = torch.empty(B.ug_densify_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    B.ug_densify(cfg, dc, dev(P), dev(m), dev(v), n, dev(stats), dev(z), cap, po, mo, vo, n_out,
                 scratch)
    torch.cuda.synchronize()
    return (po.cpu().numpy().astype(np.float64), mo.cpu().numpy().astype(np.float64),
            vo.cpu().numpy().astype(np.float64), int(n_out.item()), cfg)


@pytest.mark.parametrize("cov", [B.UG_COV_TRI, B.UG_COV_SCALE_ROT])
def test_densify_parity(cov):
    n = 20000
    P, m, v, stats, z = _mixed_case(cov, n, 21)
    dc = B.ug_densify_config_default()
    dc.size_threshold = 0.05  # extents of this scene straddle it
    po, mo, vo, n_out, cfg = _run_densify(cov, P, m, v, stats, z, 2 * n, dc)
    ref_p, ref_m, ref_v, act = D.densify(P, m, v, stats, z.astype(np.float64), cov, cfg.beta,
                                        _dc_dict(dc))
    counts = np.bincount(act, minlength=4)
    assert min(counts) > 500, counts  # every action is exercised
    assert n_out == ref_p.shape[1]
    po, mo, vo = po[:, :n_out], mo[:, :n_out], vo[:, :n_out]
    np.testing.assert_array_equal(mo, ref_m)
    np.testing.assert_array_equal(vo, ref_v)
    # copies bit-exact; children: means within the FP32 error of the draw,
    # factors / log scales within FP32 rounding
    child = np.array([c for a in act for c in ([False] if a == 1 else [False, False] if a == 2
                                               else [True, True] if a == 3 else [])])
    np.testing.assert_array_equal(po[:, ~child], ref_p[:, ~child])
    rows_cov = range(3, 9) if cov == B.UG_COV_TRI else range(3, 10)
    for r in rows_cov:
        np.testing.assert_allclose(po[r, child], ref_p[r, child], rtol=2e-6, atol=1e-7)
    np.testing.assert_array_equal(po[-2:, child], ref_p[-2:, child])
    src = np.repeat(np.arange(n), [0 if a == 0 else 1 if a == 1 else 2 for a in act])
    first = np.concatenate([[True], src[1:] != src[:-1]])  # first of a Gaussian's outputs
    zc = np.where(first[child], 0, 1)                      # child 0 draws z[0:3], child 1 z[3:6]
    zz = np.stack([z[3 * c:3 * c + 3, i] for c, i in zip(zc, src[child])], 1).astype(np.float64)
    _check_draws(po[0:3, child].astype(np.float32), P, src[child], zz, cov, cfg.beta)


def test_densify_capacity_and_empty():
    cov = B.UG_COV_TRI
    n = 5000
    P, m, v, stats, z = _mixed_case(cov, n, 31)
    dc = B.ug_densify_config_default()
    dc.size_threshold = 0.05
    full_p, _, _, n_full, _ = _run_densify(cov, P, m, v, stats, z, 2 * n, dc)
    cap = n_full // 2
    po, _, _, n_out, _ = _run_densify(cov, P, m, v, stats, z, cap, dc)
    assert n_out == n_full  # the count needed is reported
    # the Gaussians whose outputs fit are written as with room for all
    written = ~np.isnan(po[0])
    k = int(np.argmin(written)) if not written.all() else cap
    assert k >= cap - 1
    np.testing.assert_array_equal(po[:, :k], full_p[:, :k])
    # every Gaussian faded: nothing out
    row_logit = 9
    P[row_logit] = -20.0
    _, _, _, n_out, _ = _run_densify(cov, P, m, v, stats, z, 2 * n, dc)
    assert n_out == 0
