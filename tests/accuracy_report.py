"""Error of every output of the CUDA path against the FP64 oracle, per
workload: the forward image and alpha (per pixel) and the gradient of every
parameter row (per Gaussian), as max absolute error, max error relative to the
stated tolerance, and the fraction within it. Pixels and Gaussians with an
inclusion decision within rounding of an edge (where either decision is
correct) are counted apart.

Run on a GPU from the repository root:

    python tests/accuracy_report.py [--out REPORT.md]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import oracle  # noqa: E402
from gpu_helpers import (ATOL, GRAD_FLOOR, GRAD_PRE, GRAD_RTOL, RTOL, forward_bound,  # noqa: E402
                         fp32_inputs, gpu_render, grad_floor_scale, oracle_config)
from paper_2505_05643_gb300 import binding as B  # noqa: E402
from paper_2505_05643_gb300 import render as R  # noqa: E402
from paper_2505_05643_gb300 import synth  # noqa: E402



def forward_rows(name, image, alpha, ref):
    """Per output: the worst error against the stated tolerance over the pixels
    whose every inclusion decision is clear (the arithmetic's error), and over
    the pixels with an ambiguous decision against the tolerance widened by the
    ambiguous weight (a flipped decision there moves the value by at most that
    weight, so the ratio stays below 1 by construction)."""
    img_tol, alp_tol = forward_bound(ref)
    amb = ref["amb"] > 0
    rows = []
    for what, got, exp, tol in (("image C", image, ref["image"], img_tol),
                                ("alpha S_a + a_bg", alpha, ref["alpha"], alp_tol)):
        err = np.abs(got - exp)
        ratio = err / tol
        clear = float(ratio[~amb].max()) if (~amb).any() else 0.0
        ambig = float(ratio[amb].max()) if amb.any() else 0.0
        rows.append((name, what, got.size, int(amb.sum()), float(err.max()), clear, ambig,
                     float((err <= tol).mean())))
    return rows


def grad_rows(name, grads_t, cov_param, gref, gabs, amb, subset=None):
    gpu = grads_t.cpu().numpy().astype(np.float64).T
    if subset is not None:
        gpu = gpu[subset]
    keep = ~amb
    rows = []
    for k, pname in enumerate(oracle.param_names(cov_param)):
        a, b, s = gpu[keep, k], gref[keep, k], gabs[keep, k]
        tol = GRAD_RTOL * np.abs(b) + GRAD_FLOOR * s + 1e-30
        err = np.abs(a - b)
        rows.append((name, f"dL/d{pname}", int(keep.sum()), int(amb.sum()), float(err.max()),
                     float((err / tol).max()), None, float((err <= tol).mean())))
    return rows


def case(name, g, pl, cfg, target_seed=7, subset=None):
    ocfg = oracle_config(cfg)
    ref = oracle.render(g, pl, ocfg)
    r, params, image, alpha = gpu_render(g, pl, cfg)
    rows = forward_rows(name, image, alpha, ref)
    tgt = np.random.default_rng(target_seed).uniform(0, 1, pl["total_pixels"])
    _, gimg = oracle.mse_loss_grad(ref["image"], tgt)
    im64, al64, gi64 = fp32_inputs(ref["image"], ref["alpha"], gimg)
    gi = torch.from_numpy(gi64.astype(np.float32)).cuda()
    im_t = torch.from_numpy(im64.astype(np.float32)).cuda()
    al_t = torch.from_numpy(al64.astype(np.float32)).cuda()
    grads = r.backward(params, im_t, al_t, gi)
    torch.cuda.synchronize()
    gref, gabs, amb, gpre = oracle.render_grad(g, pl, ocfg, im64, al64, gi64, subset=subset,
                                               with_ambiguity=True, with_pre=True)
    rows += grad_rows(name, grads, int(cfg.cov_param), gref, grad_floor_scale(gabs, gpre), amb,
                      subset)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    t0 = time.time()
    rows = []
    g, pl = synth.workload_fwd_2k()
    for cov, tag in ((B.UG_COV_SCALE_ROT, "scale/rot"), (B.UG_COV_TRI, "tri")):
        gg = synth.scale_rot_to_tri(g, 1e-4) if cov == B.UG_COV_TRI else g
        rows += case(f"fwd_2k {tag}", gg, pl, R.make_config(cov_param=cov))
    g, pl = synth.workload_grad_50k()
    sub = np.random.default_rng(0).choice(len(g["logit"]), 500, replace=False)
    rows += case("grad_50k scale/rot (500 Gaussians)", g, pl,
                 R.make_config(cov_param=B.UG_COV_SCALE_ROT), subset=sub)
    g, pl = synth.workload_aniso_1m()
    g = synth.scale_rot_to_tri(g, 1e-4)
    sub = np.random.default_rng(0).choice(len(g["logit"]), 2000, replace=False)
    rows += case("aniso_1m tri, all 64 planes (gradients: 2000 Gaussians)", g, pl,
                 R.make_config(cov_param=B.UG_COV_TRI, variant=5, variant_bwd=5), subset=sub)
    g, poses, _ = synth.workload_train_200k()
    sub = np.random.default_rng(0).choice(len(g["logit"]), 2000, replace=False)
    rows += case("train_200k tri, the 32 poses of a step (gradients: 2000 Gaussians)", g,
                 synth.select_planes(poses, list(range(32))),
                 R.make_config(cov_param=B.UG_COV_TRI, variant=5, variant_bwd=5), subset=sub)
    g, _, train, _ = synth.workload_recon()
    novel = synth.planes_random(np.random.default_rng(7), [(512, 512)] * 512)
    pl5 = synth.concat_planes(synth.select_planes(train, [0, 1, 2, 3]),
                              synth.select_planes(novel, [0]))
    sub = np.random.default_rng(0).choice(len(g["logit"]), 1000, replace=False)
    rows += case("recon 3M tri, 4 training poses + a 512^2 novel slice (gradients: 1000 "
                 "Gaussians)", g, pl5,
                 R.make_config(cov_param=B.UG_COV_TRI, variant=5, variant_bwd=5), subset=sub)
    lines = ["| workload | output | n compared | n ambiguous (either decision valid) | max abs err | "
             "max err / tolerance, clear decisions | max err / tolerance, ambiguous pixels | "
             "fraction within tolerance |", "|---|---|---|---|---|---|---|---|"]
    for w, o, n, na, e, et, ea, f in rows:
        amb_col = "—" if ea is None else f"{ea:.3g}"
        lines.append(f"| {w} | {o} | {n} | {na} | {e:.3e} | {et:.3g} | {amb_col} | {f:.5f} |")
    text = "\n".join(lines)
    print(text)
    print(f"({time.time() - t0:.0f} s)")
    if args.out:
        with open(args.out, "w") as f:
            f.write("# Error of every output against the FP64 oracle (GB300)\n\n")
            f.write("Command (GB300, from the repository root, after `python -c \"import "
                    "__graft_entry__ as g; g.build()\"`):\n\n")
            f.write(f"```\npython tests/accuracy_report.py --out {args.out}\n```\n\n")
            f.write(f"Tolerances: image and alpha |err| <= {ATOL:g} + {RTOL:g} |ref| (plus, at "
                    "pixels with an ambiguous edge decision, the weight A those decisions "
                    "involve: a flipped decision there moves the value by at most A, so the "
                    "ambiguous pixels' ratio is below 1 by construction and the clear pixels' "
                    "ratio measures the arithmetic); gradients |err| <= "
                    f"{GRAD_RTOL:g} |ref| + {GRAD_FLOOR:g} sum |per-pair term| + {GRAD_PRE:.3g} "
                    "sum |per-pair term before the cancellation in c - C| (Gaussians with "
                    "an ambiguous decision excluded). The GPU gradient is evaluated with the "
                    "oracle's image and alpha as inputs (rounded to FP32, as the GPU receives them; the "
                    "oracle's gradient at the same inputs), so it isolates the backward's error.\n\n")
            f.write(text + "\n")


if __name__ == "__main__":
    main()
