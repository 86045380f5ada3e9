"""The data-plane kernels on one GPU: the MSE part of a plane-split batch
(ug_mse_loss_grad_part), the plane-split training step's local gradients (their
sum over the emulated ranks is the full batch's gradient), and the partial
sums and compositing of the Gaussian split (ug_shard_sums, ug_composite). The
all-reduce between the emulated ranks is a plain sum of their buffers."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_05643_gb300 import binding as B
from paper_2505_05643_gb300 import parallel
from paper_2505_05643_gb300 import render as R
from paper_2505_05643_gb300 import synth
from paper_2505_05643_gb300 import train as T

from gpu_helpers import assert_forward_parity, gpu_render, oracle_config

pytestmark = pytest.mark.gpu


def test_mse_part_sums_to_the_full_loss():
    rng = np.random.default_rng(60)
    n = 300_001
    a = torch.from_numpy(rng.uniform(0, 1, n).astype(np.float32)).cuda()
    b = torch.from_numpy(rng.uniform(0, 1, n).astype(np.float32)).cuda()
    cut = 123_457
    gf = torch.empty_like(a)
    lf = torch.zeros(B.UG_MSE_LOSS_FLOATS, device="cuda")
    B.ug_mse_loss_grad(a, b, n, gf, lf)
    g0, g1 = torch.empty(cut, device="cuda"), torch.empty(n - cut, device="cuda")
    l0 = torch.zeros(B.UG_MSE_LOSS_FLOATS, device="cuda")
    l1 = torch.zeros(B.UG_MSE_LOSS_FLOATS, device="cuda")
    B.ug_mse_loss_grad_part(a[:cut], b[:cut], cut, n, g0, l0)
    B.ug_mse_loss_grad_part(a[cut:], b[cut:], n - cut, n, g1, l1)
    torch.cuda.synchronize()
    d = (a.double() - b.double()).cpu().numpy()
    ref = np.mean(d ** 2)
    assert abs(float(l0[0]) + float(l1[0]) - ref) <= 1e-6 * ref
    # the gradient is elementwise 2 d / n_total: the same bits as the full call
    assert torch.equal(torch.cat([g0, g1]), gf)
    # n_total = n is the full call
    l2 = torch.zeros(B.UG_MSE_LOSS_FLOATS, device="cuda")
    g2 = torch.empty_like(a)
    B.ug_mse_loss_grad_part(a, b, n, n, g2, l2)
    torch.cuda.synchronize()
    assert torch.equal(g2, gf) and float(l2[0]) == float(lf[0])
    with pytest.raises(B.UgError):
        B.ug_mse_loss_grad_part(a, b, n, n - 1, g2, l2)


def test_plane_split_local_gradients_sum_to_the_full_gradient():
    """Two emulated ranks, each with a PlaneSplitStep over its contiguous share
    of the planes and the loss divided by all ranks' pixels: the sum of their
    local gradients (what the all-reduce forms) equals the full batch's
    gradient, and the sum of their loss parts the full loss."""
    rng = np.random.default_rng(61)
    g = synth.gaussians_scale_rot(rng, 4000, 0.03, 0.15)
    sizes = [(64, 64), (48, 40), (56, 56), (40, 72), (64, 48)]
    pl = synth.planes_random(rng, sizes)
    gt = synth.gaussians_scale_rot(np.random.default_rng(62), 3000, 0.03, 0.15)
    target = oracle.render(gt, pl, oracle.Config(cov_param=1))["image"].astype(np.float32)
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    params = torch.from_numpy(R.pack_params(g, B.UG_COV_SCALE_ROT)).cuda()
    # the full batch on one "rank"
    rf = R.Renderer(len(g["logit"]), pl, cfg)
    full = T.TrainStep(rf, params.clone(), torch.from_numpy(target).cuda())
    rf.preprocess(full.params)
    B.ug_preprocess(rf.plan, full.g_struct, rf.d_planes, rf.ws)
    B.ug_bin_sort(rf.plan, rf.ws)
    B.ug_render(rf.plan, rf.ws, full.image, full.alpha)
    B.ug_mse_loss_grad(full.image, full.targets, full.image.numel(), full.grad_image, full.loss)
    B.ug_render_backward(rf.plan, full.g_struct, rf.d_planes, rf.ws, full.image, full.alpha,
                         full.grad_image, full.grad_struct)
    world = 2
    total = pl["total_pixels"]
    grads, losses = [], []
    for rank in range(world):
        sub, idx = parallel.plane_shard(pl, rank, world)
        tsub = np.concatenate([target[pl["offset"][p]:pl["offset"][p] + sizes[p][0] * sizes[p][1]]
                               for p in idx])
        r = R.Renderer(len(g["logit"]), sub, cfg)
        st = parallel.PlaneSplitStep(r, params.clone(), torch.from_numpy(tsub).cuda(), total)
        r.preprocess(st.params)
        st.enqueue_local()
        assert r.status()["status"] == B.UG_OK
        grads.append(st.grads.clone())
        losses.append(float(st.loss[0]))
    torch.cuda.synchronize()
    summed = (grads[0] + grads[1]).cpu().numpy().astype(np.float64)
    ref = full.grads.cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max(axis=1, keepdims=True) + 1e-30
    assert np.all(np.abs(summed - ref) <= 1e-5 * scale + 1e-4 * np.abs(ref))
    assert abs(sum(losses) - float(full.loss[0])) <= 1e-5 * float(full.loss[0])


def test_gaussian_split_partial_sums_and_composite():
    """Three emulated ranks render thirds of the Gaussians; ug_shard_sums gives
    each rank's (S_a, S_c), their sum (the all-reduce) goes through
    ug_composite: the image and alpha match the oracle's full render within
    the forward tolerance."""
    rng = np.random.default_rng(63)
    g = synth.gaussians_scale_rot(rng, 3000, 0.03, 0.15)
    pl = synth.planes_random(rng, [(64, 64), (48, 40)])
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    n_px = pl["total_pixels"]
    world = 3
    total = torch.zeros(2 * n_px, device="cuda")
    for rank in range(world):
        lo, hi = parallel.gaussian_shard(len(g["logit"]), rank, world)
        gs = {k: v[..., lo:hi] for k, v in g.items()}
        r = R.Renderer(hi - lo, pl, cfg)
        p = torch.from_numpy(R.pack_params(gs, cfg.cov_param)).cuda()
        image, alpha = r.forward(p)
        sums = torch.empty(2 * n_px, device="cuda")
        B.ug_shard_sums(image, alpha, n_px, cfg.alpha_bg, cfg.c_bg, sums)
        total += sums
    image, alpha = torch.empty(n_px, device="cuda"), torch.empty(n_px, device="cuda")
    B.ug_composite(total, n_px, cfg.alpha_bg, cfg.c_bg, image, alpha)
    torch.cuda.synchronize()
    ref = oracle.render(g, pl, oracle_config(cfg))
    assert_forward_parity(image.cpu().numpy().astype(np.float64),
                          alpha.cpu().numpy().astype(np.float64), ref, "gaussian split")
    with pytest.raises(B.UgError):
        B.ug_composite(total[1:], n_px - 1, cfg.alpha_bg, cfg.c_bg, image, alpha)  # misaligned


def test_gaussian_split_forward_on_one_rank_is_the_render():
    """With no process group (one rank), gaussian_split_forward's partial sums
    and composite return the plain render up to the rounding of C alpha."""
    rng = np.random.default_rng(64)
    g = synth.gaussians_scale_rot(rng, 2000, 0.03, 0.15)
    pl = synth.planes_random(rng, [(64, 64), (40, 48)])
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    r, p, image_ref, alpha_ref = gpu_render(g, pl, cfg)
    image, alpha = r.new_image(), r.new_image()
    sums = torch.empty(2 * pl["total_pixels"], device="cuda")
    parallel.gaussian_split_forward(r, p, image, alpha, sums)
    torch.cuda.synchronize()
    np.testing.assert_allclose(alpha.cpu().numpy(), alpha_ref, rtol=2e-7, atol=1e-9)
    np.testing.assert_allclose(image.cpu().numpy(), image_ref, rtol=1e-6, atol=1e-9)
