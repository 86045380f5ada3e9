"""Backward parity: the CUDA gradient (backward rasterizer + chain rule)
against the oracle's FP64 analytic gradient and FP64 central differences;
the autograd.Function; the MSE loss kernel."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_05643_gb300 import binding as B
from paper_2505_05643_gb300 import render as R
from paper_2505_05643_gb300 import synth

from gpu_helpers import (GRAD_FLOOR, GRAD_RTOL, fp32_inputs, gpu_render, grad_floor_scale,
                         oracle_config)

pytestmark = pytest.mark.gpu


def _grad_rows(grads_t, cov_param, subset=None):
    g = grads_t.cpu().numpy().astype(np.float64)  # (rows, n)
    rows = g.T
    return rows if subset is None else rows[subset]


def _check_grads(gpu, ref, gabs, names, what):
    tol = GRAD_RTOL * np.abs(ref) + GRAD_FLOOR * gabs + 1e-30
    err = np.abs(gpu - ref)
    bad = np.argwhere(err > tol)
    if len(bad):
        k, p = bad[0]
        raise AssertionError(
            f"{what}: {len(bad)} of {err.size} gradient entries out of tolerance; first: "
            f"gaussian row {k} param {names[p]}: gpu {gpu[k, p]:.6e} ref {ref[k, p]:.6e} "
            f"abs-sum {gabs[k, p]:.3e}; worst rel {(err / (np.abs(ref) + 1e-30)).max():.3e}")
    return float((err / tol).max())


def _backward_case(g, pl, cfg, target, subset=None, split=False):
    """GPU gradient with the oracle's dL/dC, C and alpha as inputs (the
    forward's own FP32 error is tested separately; dL/dw = r (c - C) is
    sensitive to C where c is close to C), against the oracle's gradient at
    the same inputs as the GPU receives them (FP32). Returns the compared
    rows, the reference, the floor scale (grad_floor_scale) and the gradient."""
    ocfg = oracle_config(cfg)
    ref = oracle.render(g, pl, ocfg)
    _, gimg = oracle.mse_loss_grad(ref["image"], target)
    im64, al64, gi64 = fp32_inputs(ref["image"], ref["alpha"], gimg)
    r, params, image, alpha = gpu_render(g, pl, cfg)
    gi = torch.from_numpy(gi64.astype(np.float32)).cuda()
    im_t = torch.from_numpy(im64.astype(np.float32)).cuda()
    al_t = torch.from_numpy(al64.astype(np.float32)).cuda()
    if split:  # rows a7 and a8 through their own entry points
        grads = torch.empty_like(params)
        B.ug_render_backward_raster(r.plan, r.ws, im_t, al_t, gi)
        B.ug_preprocess_backward(r.plan, R.gaussians_struct(params, r.cov), r.ws,
                                 R.grads_struct(grads, r.cov))
        assert r.status()["status"] == B.UG_OK
    else:
        grads = r.backward(params, im_t, al_t, gi)
    torch.cuda.synchronize()
    gref, gabs, amb, gpre = oracle.render_grad(g, pl, ocfg, im64, al64, gi64, subset=subset,
                                               with_ambiguity=True, with_pre=True)
    gpu = _grad_rows(grads, cfg.cov_param, subset)
    # a Gaussian with an inclusion decision within rounding of an edge may
    # include or drop that pixel (either is correct): compare the others
    keep = ~amb
    assert keep.mean() > 0.9, keep.mean()
    return gpu[keep], gref[keep], grad_floor_scale(gabs, gpre)[keep], grads


@pytest.mark.parametrize("cov_param", [B.UG_COV_SCALE_ROT, B.UG_COV_TRI])
@pytest.mark.parametrize("cutoff", [B.UG_CUTOFF_BOX, B.UG_CUTOFF_BOX_AND_ELLIPSOID])
def test_grad_small_scene(cov_param, cutoff):
    rng = np.random.default_rng(31)
    g = synth.gaussians_scale_rot(rng, 1500, 0.03, 0.15)
    g["logit"] = rng.uniform(-1, 2, 1500).astype(np.float32)
    if cov_param == B.UG_COV_TRI:
        g = synth.scale_rot_to_tri(g, 1e-4)
    pl = synth.planes_random(rng, [(64, 64), (50, 70)])
    target = rng.uniform(0, 1, pl["total_pixels"])
    cfg = R.make_config(cov_param=cov_param, cutoff=cutoff)
    gpu, gref, gabs, _ = _backward_case(g, pl, cfg, target)
    _check_grads(gpu, gref, gabs, oracle.param_names(cov_param), f"small cov{cov_param} cut{cutoff}")


@pytest.mark.parametrize("cov_param", [B.UG_COV_SCALE_ROT, B.UG_COV_TRI])
def test_grad_split_entry_points(cov_param):
    """ug_render_backward_raster followed by ug_preprocess_backward gives the
    gradient of ug_render_backward."""
    rng = np.random.default_rng(36)
    g = synth.gaussians_scale_rot(rng, 1200, 0.03, 0.15)
    if cov_param == B.UG_COV_TRI:
        g = synth.scale_rot_to_tri(g, 1e-4)
    pl = synth.planes_random(rng, [(64, 64), (45, 61)])
    target = rng.uniform(0, 1, pl["total_pixels"])
    cfg = R.make_config(cov_param=cov_param)
    gpu, gref, gabs, _ = _backward_case(g, pl, cfg, target, split=True)
    _check_grads(gpu, gref, gabs, oracle.param_names(cov_param), f"split cov{cov_param}")


def test_grad_fp64_branch():
    """Triangular front-end with every Gaussian on the FP64 branch."""
    rng = np.random.default_rng(35)
    g = synth.scale_rot_to_tri(synth.gaussians_scale_rot(rng, 1200, 0.03, 0.15), 1e-4)
    pl = synth.planes_random(rng, [(64, 64), (48, 40)])
    target = rng.uniform(0, 1, pl["total_pixels"])
    cfg = R.make_config(cov_param=B.UG_COV_TRI, fp64_ratio=1.0)
    gpu, gref, gabs, _ = _backward_case(g, pl, cfg, target)
    _check_grads(gpu, gref, gabs, oracle.param_names(0), "fp64 branch")


def test_grad_extreme_anisotropy():
    """The first 20,000 Gaussians of the bench workload (axis ratios log-uniform
    to 1e4, triangular front-end) on four of its planes (up to 512^2): every
    gradient entry of 2,000 Gaussians within rel 1e-3 plus the abs-sum floor."""
    g, pl = synth.workload_aniso_1m()
    n = 20000
    g = synth.scale_rot_to_tri({k: np.ascontiguousarray(v[..., :n]) for k, v in g.items()}, 1e-4)
    pl = synth.select_planes(pl, [0, 1, 2, 3])
    rng = np.random.default_rng(37)
    target = rng.uniform(0, 1, pl["total_pixels"])
    sub = np.sort(rng.choice(n, 2000, replace=False))
    cfg = R.make_config(cov_param=B.UG_COV_TRI)
    gpu, gref, gabs, _ = _backward_case(g, pl, cfg, target, subset=sub)
    assert np.count_nonzero(np.abs(gref).sum(1)) > 200  # Gaussians that reach a pixel
    _check_grads(gpu, gref, gabs, oracle.param_names(0), "aniso cut")


def test_grad_needles_thinner_than_2e_minus_20_pixels():
    """Records whose pixel-unit factor r11 exceeds 2^20 (needles a million
    times thinner than a pixel) take the backward's ten-operation pixel loop
    (the nine-operation form needs every t1^2 of the footprint finite). Their
    box decisions sit within rounding of a pixel edge, so the oracle counts them
    as ambiguous; the test checks that the records exist, that every gradient
    entry is finite, and that the other Gaussians match the oracle."""
    rng = np.random.default_rng(41)
    g = synth.gaussians_scale_rot(rng, 600, 0.05, 0.2)
    g["mean"] *= 0.5
    k = 40  # needles: thin along x, on the plane z = 0, centred on pixel columns
    cols = rng.integers(4, 28, k)
    g["mean"][0, :k] = ((cols + 0.5 - 16) / 16).astype(np.float32)
    g["mean"][1, :k] = rng.uniform(-0.5, 0.5, k).astype(np.float32)
    g["mean"][2, :k] = 0.0
    g["log_scale"][:, :k] = np.log(np.array([[1e-9], [0.1], [0.1]], np.float32))
    g["quat"][:, :k] = np.array([[1.0], [0.0], [0.0], [0.0]], np.float32)
    pl = synth._pack_planes(np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]),
                            np.array([[0.0, 1.0, 0.0]]), [(32, 32)])
    target = rng.uniform(0, 1, pl["total_pixels"])
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT, tile=16, variant=5, variant_bwd=5)
    gpu, gref, gabs, grads = _backward_case(g, pl, cfg, target)
    r, _, _, _ = gpu_render(g, pl, cfg)
    dv = r.debug_views()
    assert (dv["rec_a"][:, 2] > 2.0 ** 20).sum() >= k // 2
    assert torch.isfinite(grads).all()
    _check_grads(gpu, gref, gabs, oracle.param_names(1), "needles")


@pytest.mark.parametrize("tile,variant", [(16, v) for v in range(1, 6)] + [(8, 0), (8, 1)])
def test_grad_variants(tile, variant):
    """Every compiled backward variant (footprint height, stages, records per
    stage) against the oracle's gradient, on dense tiles that span several
    stages (items stay queued across stages, so the stage-release rule is
    exercised) and on a sparse plane."""
    rng = np.random.default_rng(32)
    g = synth.gaussians_scale_rot(rng, 4000, 0.05, 0.3)
    pl = synth.planes_random(rng, [(40, 33), (64, 64)], origin_range=0.05)
    target = rng.uniform(0, 1, pl["total_pixels"])
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT, tile=tile, variant=min(variant, 2),
                        variant_bwd=variant)
    gpu, gref, gabs, _ = _backward_case(g, pl, cfg, target)
    _check_grads(gpu, gref, gabs, oracle.param_names(1), f"variant t{tile} v{variant}")


@pytest.mark.parametrize("tile", [16, 8])
def test_grad_binning_footprint_tests_against_own_tests(tile):
    """The 8x8-footprint backward takes its footprint tests from the binning
    (the sorted keys' top byte); the 8x4-footprint variant tests its own. On
    an extreme-anisotropy scene with many culled footprints both give the same
    gradient up to the order of the atomic additions, with or without a
    forward pass between bin/sort and the backward, and the same gradient
    after the scatter forward (which leaves the keys as they are)."""
    rng = np.random.default_rng(37)
    g, pl = synth.workload_aniso_1m()
    g = {k: v[..., :20000] for k, v in g.items()}
    g = synth.scale_rot_to_tri(g, 1e-4)
    pl = synth.planes_random(rng, [(128, 128), (96, 160)])
    cfg = R.make_config(cov_param=B.UG_COV_TRI, tile=tile, variant=0, variant_bwd=0)
    r, params, image, alpha = gpu_render(g, pl, cfg)
    gi = torch.from_numpy(rng.normal(0, 1, pl["total_pixels"]).astype(np.float32)).cuda()
    im_t = torch.from_numpy(image.astype(np.float32)).cuda()
    al_t = torch.from_numpy(alpha.astype(np.float32)).cuda()

    def gradient(variant_bwd):
        r.plan.cfg.variant_bwd = variant_bwd
        grads = torch.empty_like(params)
        B.ug_render_backward_raster(r.plan, r.ws, im_t, al_t, gi)
        B.ug_preprocess_backward(r.plan, R.gaussians_struct(params, r.cov), r.ws,
                                 R.grads_struct(grads, r.cov))
        torch.cuda.synchronize()
        st = r.status()
        assert st["status"] == B.UG_OK
        return grads.cpu().numpy().astype(np.float64), st["evaluated_pairs_bwd"]

    binned, ev1 = gradient(0)
    own, ev2 = gradient(1)
    assert ev1 > 0 and ev2 > 0
    # bin/sort again and run the backward with no forward in between
    B.ug_preprocess(r.plan, R.gaussians_struct(params, r.cov), r.d_planes, r.ws)
    B.ug_bin_sort(r.plan, r.ws)
    no_fwd, ev3 = gradient(0)
    im2, al2 = torch.empty_like(im_t), torch.empty_like(al_t)
    B.ug_render_scatter(r.plan, r.ws, im2, al2)
    after_scatter, ev4 = gradient(0)
    assert ev1 == ev3 == ev4
    scale = np.abs(binned).max(axis=1, keepdims=True) + 1e-30  # per parameter row
    for other in (own, no_fwd, after_scatter):
        err = np.abs(binned - other)
        assert np.all(err <= 1e-5 * scale + 1e-4 * np.abs(other)), (err / scale).max(axis=1)


def test_grad_many_planes_and_dense_tiles():
    """Gradient parity with 80 planes in one launch (planes beyond the
    rasterizers' 64-plane shared table; plane groups of the cull, list and
    gather) and, on a dense plane, tiles spanning several record stages."""
    rng = np.random.default_rng(43)
    g = synth.gaussians_scale_rot(rng, 2500, 0.03, 0.15)
    sizes = [(24 + (k % 5) * 7, 20 + (k % 3) * 9) for k in range(79)] + [(40, 40)]
    pl = synth.planes_random(rng, sizes)
    target = rng.uniform(0, 1, pl["total_pixels"])
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    gpu, gref, gabs, _ = _backward_case(g, pl, cfg, target)
    _check_grads(gpu, gref, gabs, oracle.param_names(1), "80 planes")
    rng = np.random.default_rng(44)
    g = synth.gaussians_scale_rot(rng, 4000, 0.05, 0.3)
    pl = synth.planes_random(rng, [(40, 40), (33, 21)], origin_range=0.05)
    target = rng.uniform(0, 1, pl["total_pixels"])
    gpu, gref, gabs, _ = _backward_case(g, pl, cfg, target)
    _check_grads(gpu, gref, gabs, oracle.param_names(1), "dense tiles")


def test_grad_50k_16_planes_subset_and_fd():
    """50,000 scale/rotation Gaussians, 16 planes of 256x256, MSE against
    targets rendered by the oracle from a separate seed-1 set of 50,000;
    gradients of a random subset of 500 Gaussians against the FP64 oracle
    gradient, and a sample against Richardson-extrapolated FP64 central
    differences at rel 1e-3."""
    g, pl = synth.workload_grad_50k(seed=0)
    g_t, _ = synth.workload_grad_50k(seed=1)
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    ocfg = oracle_config(cfg)
    target = oracle.render(g_t, pl, ocfg)["image"]
    subset = np.random.default_rng(0).choice(50_000, 500, replace=False)
    _, _, amb = oracle.render_grad(g, pl, ocfg, np.zeros(pl["total_pixels"]),
                                   np.ones(pl["total_pixels"]), np.zeros(pl["total_pixels"]),
                                   subset=subset, with_ambiguity=True)
    subset = subset[~amb]
    gpu, gref, gabs, _ = _backward_case(g, pl, cfg, target, subset=subset)
    names = oracle.param_names(1)
    _check_grads(gpu, gref, gabs, names, "grad_50k")
    # Central differences of the FP64 oracle loss on parameters whose pixel sets
    # do not change at theta +- h and theta +- h/2, Richardson-extrapolated:
    # D(h) = (L(theta + h) - L(theta - h)) / 2h = L' + c h^2 + O(h^4), so
    # (4 D(h/2) - D(h)) / 3 = L' + O(h^4). Each parameter's step is scaled to
    # its natural size (the means by the Gaussian's smallest scale), which puts
    # the truncation error far below the GPU's tolerance of rel 1e-3.
    base = oracle.render(g, pl, ocfg)
    covp = oracle.covp_rows(g, 1)
    keys = [("mean", r) for r in range(3)] + [("log_scale", r) for r in range(3)] + \
        [("quat", r) for r in range(4)] + [("logit", None), ("intensity", None)]
    checked = 0

    def loss_at(k, key, row, delta, pix0, w0):
        gg = {kk: vv[..., k:k + 1].astype(np.float64).copy() for kk, vv in g.items()}
        if row is None:
            gg[key][0] += delta
        else:
            gg[key][row, 0] += delta
        pix, w = oracle.contrib(gg["mean"][:, 0], oracle.covp_rows(gg, 1)[0],
                                gg["logit"][0], gg["intensity"][0], pl, ocfg)
        sa = base["sa"].copy()
        sc = base["sc"].copy()
        np.subtract.at(sa, pix0, w0)
        np.subtract.at(sc, pix0, w0 * float(g["intensity"][k]))
        np.add.at(sa, pix, w)
        np.add.at(sc, pix, w * float(gg["intensity"][0]))
        C = (sc + ocfg.alpha_bg * ocfg.c_bg) / (sa + ocfg.alpha_bg)
        return np.mean((C - target) ** 2), np.array_equal(pix, pix0)

    for si in range(12):
        k = int(subset[si])
        pix0, w0 = oracle.contrib(g["mean"][:, k], covp[k], g["logit"][k], g["intensity"][k], pl, ocfg)
        if len(pix0) < 20:
            continue
        smin = float(np.exp(g["log_scale"][:, k].min()))
        for pi, (key, row) in enumerate(keys):
            h = 1e-2 * smin if key == "mean" else 1e-3
            d, same = [], True
            for hh in (h, h / 2):
                lp, s1 = loss_at(k, key, row, hh, pix0, w0)
                lm, s2 = loss_at(k, key, row, -hh, pix0, w0)
                same &= s1 and s2
                d.append((lp - lm) / (2 * hh))
            if not same:
                continue
            fd = (4 * d[1] - d[0]) / 3
            assert abs(fd - gpu[si, pi]) <= 1e-3 * abs(fd) + 1e-4 * gabs[si, pi] + 1e-15, \
                (k, key, row, fd, gpu[si, pi], d)
            checked += 1
    assert checked >= 20


def test_autograd_function_matches_direct_call():
    rng = np.random.default_rng(33)
    g = synth.gaussians_scale_rot(rng, 800, 0.03, 0.15)
    pl = synth.planes_random(rng, [(48, 48)] * 2)
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    r = R.Renderer(800, pl, cfg)
    params = torch.from_numpy(R.pack_params(g, 1)).cuda().requires_grad_(True)
    target = torch.rand(pl["total_pixels"], device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    image = R.UGRender.apply(params, r)
    loss = torch.mean((image - target) ** 2)
    loss.backward()
    image2, alpha2 = r.forward(params.detach())
    gi = 2 * (image2 - target) / image2.numel()
    direct = r.backward(params.detach(), image2, alpha2, gi)
    torch.testing.assert_close(params.grad, direct, rtol=1e-5, atol=1e-9)


def test_mse_loss_kernel():
    rng = np.random.default_rng(34)
    for n in (1, 1000, 3 * 65536 + 7, 4 * 65536, 6688768):  # scalar and float4 paths
        img = rng.uniform(0, 1, n).astype(np.float32)
        tgt = rng.uniform(0, 1, n).astype(np.float32)
        it, tt = torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda()
        grad = torch.empty_like(it)
        loss = torch.empty(B.UG_MSE_LOSS_FLOATS, device="cuda")
        B.ug_mse_loss_grad(it, tt, n, grad, loss)
        L, G = oracle.mse_loss_grad(img, tgt)
        np.testing.assert_allclose(loss[0].item(), L, rtol=1e-6)
        np.testing.assert_allclose(grad.cpu().numpy(), G, rtol=1e-6, atol=1e-12)
        loss2 = torch.empty_like(loss)
        B.ug_mse_loss_grad(it, tt, n, grad, loss2)
        assert loss2[0].item() == loss[0].item()  # deterministic


def test_gaussian_sharded_render_and_gradient_on_one_gpu():
    """The Gaussian decomposition with the library's own entry points: two
    halves of the Gaussians rendered separately, their partial sums S_a =
    alpha - a_bg and S_c = C alpha - a_bg c_bg added, the image formed from the
    sums, and each half's gradient taken with the global image and alpha:
    the same image and gradient as rendering all Gaussians at once (up to FP32
    rounding and the order of the backward's atomic sums)."""
    rng = np.random.default_rng(45)
    g = synth.gaussians_scale_rot(rng, 3000, 0.03, 0.15)
    pl = synth.planes_random(rng, [(64, 64), (48, 40)])
    target = torch.from_numpy(rng.uniform(0, 1, pl["total_pixels"]).astype(np.float32)).cuda()
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    abg, cbg = cfg.alpha_bg, cfg.c_bg
    r_full, p_full, image_f, alpha_f = gpu_render(g, pl, cfg)
    halves = [np.arange(0, 3000, 2), np.arange(1, 3000, 2)]
    parts = []
    for h in halves:
        gh = {k: v[..., h] for k, v in g.items()}
        r, p, im, al = gpu_render(gh, pl, cfg)
        parts.append((r, p, im, al))
    S_a = sum(al - abg for _, _, _, al in parts)
    S_c = sum(im * al - abg * cbg for _, _, im, al in parts)
    alpha = S_a + abg
    image = (S_c + abg * cbg) / alpha
    np.testing.assert_allclose(alpha, alpha_f, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(image, image_f, rtol=1e-5, atol=1e-6)
    im_t = torch.from_numpy(image.astype(np.float32)).cuda()
    al_t = torch.from_numpy(alpha.astype(np.float32)).cuda()
    gi = 2 * (im_t - target) / im_t.numel()
    full = r_full.backward(p_full, im_t, al_t, gi).cpu().numpy()
    sharded = np.zeros_like(full)
    for h, (r, p, _, _) in zip(halves, parts):
        sharded[:, h] = r.backward(p, im_t, al_t, gi).cpu().numpy()
    scale = np.abs(full).max(axis=1, keepdims=True) + 1e-30
    assert np.all(np.abs(sharded - full) <= 1e-5 * scale + 1e-4 * np.abs(full))
