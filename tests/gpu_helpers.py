"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle)."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2505_05643_gb300 import binding as B
from paper_2505_05643_gb300 import render as R

# Forward tolerance of the GPU FP32 image: |gpu - oracle| <= ATOL + RTOL |oracle|.
RTOL = 1e-4
ATOL = 1e-6

# Gradient tolerance: |gpu - ref| <= GRAD_RTOL |ref| + GRAD_FLOOR S + GRAD_PRE S_pre.
# S is the oracle's sum of |per-pair term| (the scale of FP32 rounding in a sum
# that cancels): relative 1e-3 as stated for the gradient, and a floor of 1e-4
# of the absolute sum (FP32 sums of 1e3-1e5 terms carry a relative error of the
# absolute sum of about sqrt(n) * 6e-8 <= 2e-5). S_pre is the same sum with |c -
# C| in dL/dw = G (c - C) / alpha replaced by |c| + |C|: the backward forms
# G c / alpha and G C / alpha in FP32 (C itself is the forward's FP32 output),
# so where an intensity c is close to the image value C (every c is 0.5 in the
# paper's initialisation) a per-pair term carries a few FP32 ulps of its size
# before that cancellation: GRAD_PRE = 8 ulps of it.
GRAD_RTOL = 1e-3
GRAD_FLOOR = 1e-4
GRAD_PRE = 8 * 2.0 ** -24


def grad_floor_scale(gabs, gpre):
    """Per entry, the scale S of the GRAD_FLOOR term that also carries the
    GRAD_PRE term: GRAD_FLOOR * S = GRAD_FLOOR * gabs + GRAD_PRE * gpre."""
    return gabs + (GRAD_PRE / GRAD_FLOOR) * gpre


def fp32_inputs(*arrays):
    """Arrays as the GPU receives them (rounded to FP32) and back in FP64: the
    oracle's gradient is evaluated at the same C, alpha and dL/dC."""
    return tuple(np.asarray(np.asarray(a, np.float32), np.float64) for a in arrays)


def oracle_config(cfg: B.ug_config) -> oracle.Config:
    return oracle.Config(chi2=float(np.float32(cfg.chi2)), beta=float(np.float32(cfg.beta)),
                         alpha_bg=float(np.float32(cfg.alpha_bg)), c_bg=float(np.float32(cfg.c_bg)),
                         cutoff=int(cfg.cutoff), cov_param=int(cfg.cov_param))


def gpu_render(g: dict, planes: dict, cfg: B.ug_config, **kw):
    n = len(g["logit"])
    r = R.Renderer(n, planes, cfg, **kw)
    params = torch.from_numpy(R.pack_params(g, cfg.cov_param)).cuda()
    image, alpha = r.forward(params)
    torch.cuda.synchronize()
    return r, params, image.cpu().numpy().astype(np.float64), alpha.cpu().numpy().astype(np.float64)


def forward_bound(ref: dict) -> tuple[np.ndarray, np.ndarray]:
    """Per-pixel allowed |error| of (image, alpha): the stated tolerance plus,
    where the oracle flags ambiguous decisions (total weight A), the largest
    change those decisions can make: A for alpha and A / (alpha - A) for C
    (every intensity lies in [0, 1])."""
    A = ref["amb"]
    img_tol = ATOL + RTOL * np.abs(ref["image"]) + np.where(A > 0, A / np.maximum(ref["alpha"] - A, 1e-30), 0)
    alp_tol = ATOL + RTOL * np.abs(ref["alpha"]) + A
    return img_tol, alp_tol


def assert_forward_parity(image, alpha, ref, what=""):
    img_tol, alp_tol = forward_bound(ref)
    ei = np.abs(image - ref["image"])
    ea = np.abs(alpha - ref["alpha"])
    bad_i = np.flatnonzero(ei > img_tol)
    bad_a = np.flatnonzero(ea > alp_tol)
    msg = (f"{what}: image max err {ei.max():.3e} ({len(bad_i)} px over), "
           f"alpha max err {ea.max():.3e} ({len(bad_a)} px over); first {bad_i[:5]} "
           f"gpu {image[bad_i[:5]]} ref {ref['image'][bad_i[:5]]}")
    assert len(bad_i) == 0 and len(bad_a) == 0, msg
    return float(ei.max()), float(ea.max())
