"""Parity at the bench workload's full size, in the launch configuration the
bench times: the 1,000,000-Gaussian extreme-anisotropy scene (axis ratios
log-uniform to 1e4, triangular front-end) on all 64 ragged planes (6,688,768
pixels), tile 16, forward rasterizer variant 5, backward variant 5. Every
pixel of the image and alpha is compared with the FP64 oracle at the stated
tolerance, and every gradient entry of 2,000 sampled Gaussians (the oracle
computes the gradient of any subset of Gaussians on its own)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_05643_gb300 import binding as B
from paper_2505_05643_gb300 import render as R
from paper_2505_05643_gb300 import synth

from gpu_helpers import assert_forward_parity, grad_floor_scale, oracle_config
from test_gpu_backward import _check_grads, _grad_rows

pytestmark = pytest.mark.gpu


def _gpu_backward(r, params, image, alpha, grad_image):
    """The GPU gradient for the given C, alpha and dL/dC, and those inputs as
    the GPU receives them (rounded to FP32, back in FP64): the oracle's
    gradient is evaluated at the same inputs. dL/dw = r (c - C) cancels where
    an intensity c is close to C (every c is 0.5 in the paper's
    initialisation and C is about 0.4998), and the FP32 rounding of C alone
    would then move the FP64 reference by 1e-4 of a per-pair sum."""
    im32, al32, gi32 = (np.asarray(x, np.float32) for x in (image, alpha, grad_image))
    grads = r.backward(params, torch.from_numpy(im32).cuda(), torch.from_numpy(al32).cuda(),
                       torch.from_numpy(gi32).cuda())
    torch.cuda.synchronize()
    return grads, im32.astype(np.float64), al32.astype(np.float64), gi32.astype(np.float64)


def test_full_bench_workload_parity():
    g, pl = synth.workload_aniso_1m()
    g = synth.scale_rot_to_tri(g, 1e-4)
    n = len(g["logit"])
    cfg = R.make_config(cov_param=B.UG_COV_TRI, tile=16, variant=5, variant_bwd=5)
    ocfg = oracle_config(cfg)
    r = R.Renderer(n, pl, cfg)
    assert n == 1_000_000 and r.P == 64 and r.total_pixels == 6_688_768
    params = torch.from_numpy(R.pack_params(g, cfg.cov_param)).cuda()
    image, alpha = r.forward(params)
    torch.cuda.synchronize()
    st = r.status()
    assert st["fp64_records"] > 0.8 * st["records"]  # the extended-precision branch dominates
    ref = oracle.render(g, pl, ocfg)
    assert abs(st["box_pixels"] - ref["pairs"]) <= 1e-3 * ref["pairs"]
    assert_forward_parity(image.cpu().numpy().astype(np.float64),
                          alpha.cpu().numpy().astype(np.float64), ref, "full bench workload")

    # gradient of an MSE loss against random targets, with the oracle's C and
    # alpha as the backward's inputs (its own error is isolated)
    rng = np.random.default_rng(41)
    target = rng.uniform(0, 1, ref["image"].size)
    _, gimg = oracle.mse_loss_grad(ref["image"], target)
    grads, im32, al32, gi32 = _gpu_backward(r, params, ref["image"], ref["alpha"], gimg)
    sub = np.sort(rng.choice(n, 2000, replace=False))
    gref, gabs, amb, gpre = oracle.render_grad(g, pl, ocfg, im32, al32, gi32, subset=sub,
                                               with_ambiguity=True, with_pre=True)
    gpu = _grad_rows(grads, cfg.cov_param, sub)
    keep = ~amb
    assert keep.mean() > 0.9, keep.mean()
    assert np.count_nonzero(np.abs(gref[keep]).sum(1)) > 500  # Gaussians that reach a pixel
    _check_grads(gpu[keep], gref[keep], grad_floor_scale(gabs, gpre)[keep],
                 oracle.param_names(0), "full bench workload")


def _parity(g, pl, cfg, n_sub, seed, what):
    """Forward (every pixel) and gradient (n_sub sampled Gaussians, MSE against
    random targets, the oracle's C and alpha as inputs) against the oracle."""
    ocfg = oracle_config(cfg)
    n = len(g["logit"])
    r = R.Renderer(n, pl, cfg)
    params = torch.from_numpy(R.pack_params(g, cfg.cov_param)).cuda()
    image, alpha = r.forward(params)
    torch.cuda.synchronize()
    ref = oracle.render(g, pl, ocfg)
    assert_forward_parity(image.cpu().numpy().astype(np.float64),
                          alpha.cpu().numpy().astype(np.float64), ref, what)
    rng = np.random.default_rng(seed)
    target = rng.uniform(0, 1, ref["image"].size)
    _, gimg = oracle.mse_loss_grad(ref["image"], target)
    grads, im32, al32, gi32 = _gpu_backward(r, params, ref["image"], ref["alpha"], gimg)
    sub = np.sort(rng.choice(n, n_sub, replace=False))
    gref, gabs, amb, gpre = oracle.render_grad(g, pl, ocfg, im32, al32, gi32, subset=sub,
                                               with_ambiguity=True, with_pre=True)
    gpu = _grad_rows(grads, cfg.cov_param, sub)
    keep = ~amb
    assert keep.mean() > 0.9, keep.mean()
    assert np.count_nonzero(np.abs(gref[keep]).sum(1)) > n_sub // 10
    _check_grads(gpu[keep], gref[keep], grad_floor_scale(gabs, gpre)[keep],
                 oracle.param_names(cfg.cov_param), what)
    return ref


def test_train_200k_full_step_parity():
    """The batched training workload at its full size: 200,000 Gaussians in the
    paper's initialisation, the 32 sweep poses of one step at 256^2."""
    g, poses, _ = synth.workload_train_200k()
    pl = synth.select_planes(poses, list(range(32)))
    cfg = R.make_config(cov_param=B.UG_COV_TRI, tile=16, variant=5, variant_bwd=5)
    ref = _parity(g, pl, cfg, 2000, 43, "train_200k step")
    assert ref["pairs"] > 5e8  # about 340 pairs per pixel


def test_recon_3m_sampled_planes_parity():
    """The reconstruction workload's 3,000,000 Gaussians (paper initialisation)
    on four of its 256^2 training poses and one of the bench's 512^2 novel
    slices (every plane of a step is independent, so four planes sample it)."""
    g, _, train, _ = synth.workload_recon()
    novel = synth.planes_random(np.random.default_rng(7), [(512, 512)] * 512)
    pl = synth.concat_planes(synth.select_planes(train, [0, 1, 2, 3]),
                             synth.select_planes(novel, [0]))
    cfg = R.make_config(cov_param=B.UG_COV_TRI, tile=16, variant=5, variant_bwd=5)
    ref = _parity(g, pl, cfg, 1000, 47, "recon 3M")
    assert ref["pairs"] > 1e9
