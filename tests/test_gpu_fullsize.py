"""Parity at the bench workload's full size, in the launch configuration the
bench times: the 1,000,000-Gaussian extreme-anisotropy scene (axis ratios
log-uniform to 1e4, triangular front-end) on all 64 ragged planes (6,688,768
pixels), tile 16, forward rasterizer variant 5, backward variant 0. Every
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

from gpu_helpers import assert_forward_parity, oracle_config
from test_gpu_backward import _check_grads, _grad_rows

pytestmark = pytest.mark.gpu


def test_full_bench_workload_parity():
    g, pl = synth.workload_aniso_1m()
    g = synth.scale_rot_to_tri(g, 1e-4)
    n = len(g["logit"])
    cfg = R.make_config(cov_param=B.UG_COV_TRI, tile=16, variant=5, variant_bwd=0)
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
    gi = torch.from_numpy(gimg.astype(np.float32)).cuda()
    im_t = torch.from_numpy(ref["image"].astype(np.float32)).cuda()
    al_t = torch.from_numpy(ref["alpha"].astype(np.float32)).cuda()
    grads = r.backward(params, im_t, al_t, gi)
    torch.cuda.synchronize()
    sub = np.sort(rng.choice(n, 2000, replace=False))
    gref, gabs, amb = oracle.render_grad(g, pl, ocfg, ref["image"], ref["alpha"], gimg,
                                         subset=sub, with_ambiguity=True)
    gpu = _grad_rows(grads, cfg.cov_param, sub)
    keep = ~amb
    assert keep.mean() > 0.9, keep.mean()
    assert np.count_nonzero(np.abs(gref[keep]).sum(1)) > 500  # Gaussians that reach a pixel
    _check_grads(gpu[keep], gref[keep], gabs[keep], oracle.param_names(0), "full bench workload")
