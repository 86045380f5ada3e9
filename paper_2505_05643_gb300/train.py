"""One training step of the plane rasterizer as a sequence of library calls:

    ug_preprocess -> ug_bin_sort -> ug_render -> ug_mse_loss_grad
        -> ug_render_backward -> ug_adam_step

All state (parameters, gradients, Adam moments, step counter, learning-rate
schedule, targets, loss) lives in device tensors owned here, so the whole
step can be enqueued eagerly or captured once in a CUDA graph and replayed.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B
from . import render as R

# Sec. 4.5: Adam, lr 0.05 for all Gaussian parameters except the means, whose
# lr starts at 1.6e-4 and decays exponentially (to 1.6e-6 over the run here).
LR_DEFAULT = 0.05
LR_MEAN_INIT = 1.6e-4
LR_MEAN_FINAL = 1.6e-6
BETA1, BETA2, EPS = 0.9, 0.999, 1e-15


DSSIM_LAMBDA = 0.2  # weight of the D-SSIM term in Kerbl et al.'s loss


class TrainStep:
    def __init__(self, renderer: R.Renderer, params: torch.Tensor, targets: torch.Tensor,
                 decay_steps: int = 30000, lr: float = LR_DEFAULT, loss: str = "mse",
                 plane_shape: tuple | None = None):
        """loss: "mse" (the bench's loss) or "l1_dssim" ((1 - 0.2) L1 + 0.2 (1 - SSIM),
        Kerbl et al.'s loss; needs every plane of the same plane_shape = (W, H))."""
        self.r = renderer
        self.params = params
        self.targets = targets
        dev = params.device
        if loss not in ("mse", "l1_dssim"):
            raise ValueError(f"unknown loss {loss}")
        self.loss_kind = loss
        if loss == "l1_dssim":
            if plane_shape is None:
                raise ValueError("the L1 + D-SSIM loss needs planes of one shape (W, H)")
            W, H = plane_shape
            self.dssim_shape = (renderer.plan.num_planes, int(W), int(H))
            self.dssim_scratch = torch.empty(B.ug_l1_dssim_scratch_floats(*self.dssim_shape),
                                             dtype=torch.float32, device=dev)
        self.grads = torch.zeros_like(params)
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.image = renderer.new_image()
        self.alpha = renderer.new_image()
        self.grad_image = renderer.new_image()
        self.loss = torch.zeros(B.UG_MSE_LOSS_FLOATS, dtype=torch.float32, device=dev)
        self.step = torch.zeros(1, dtype=torch.int32, device=dev)
        rows = np.zeros(renderer.rows, dtype=[("lr_init", "<f4"), ("lr_final", "<f4"),
                                              ("decay_steps", "<i4"), ("reserved", "<i4")])
        for k in range(renderer.rows):
            if k < 3:
                rows[k] = (LR_MEAN_INIT, LR_MEAN_FINAL, decay_steps, 0)
            else:
                rows[k] = (lr, lr, 0, 0)
        self.lr_rows = torch.from_numpy(rows.view(np.uint8).copy()).to(dev)
        self.g_struct = R.gaussians_struct(params, renderer.cov)
        self.grad_struct = R.grads_struct(self.grads, renderer.cov)
        self.graph = None

    def enqueue(self, stream=None, targets_ready=None):
        """Issue the six calls of one step on `stream` (no host synchronisation).
        targets_ready: an event recorded after the step's targets were written
        (e.g. by a host-to-device copy on another stream); the loss waits for it,
        the preprocess, sort and forward do not."""
        r = self.r
        B.ug_preprocess(r.plan, self.g_struct, r.d_planes, r.ws, stream)
        B.ug_bin_sort(r.plan, r.ws, stream)
        B.ug_render(r.plan, r.ws, self.image, self.alpha, stream)
        if targets_ready is not None:
            (stream or torch.cuda.current_stream()).wait_event(targets_ready)
        if self.loss_kind == "mse":
            B.ug_mse_loss_grad(self.image, self.targets, self.image.numel(), self.grad_image,
                               self.loss, stream)
        else:
            P, W, H = self.dssim_shape
            B.ug_l1_dssim_loss_grad(self.image, self.targets, P, W, H, DSSIM_LAMBDA,
                                    self.dssim_scratch, self.grad_image, self.loss, stream)
        B.ug_render_backward(r.plan, self.g_struct, r.d_planes, r.ws, self.image, self.alpha,
                             self.grad_image, self.grad_struct, stream)
        B.ug_adam_step(self.params, self.grads, self.m, self.v, r.rows, r.n, self.lr_rows,
                       self.step, BETA1, BETA2, EPS, stream)

    def kernels_per_step(self) -> int:
        """Kernels of this library launched by one step (memsets excluded)."""
        # preprocess: planes, cull, scan, list, 2 records, live tiles, scan, emit
        pre = 9
        sort = 4 * int(self.r.plan.sort_passes) + 1  # per pass: hist, 2 scan, scatter; ranges
        # render 1, mse 2, backward: zero, raster, chain, gather = 4, adam 2
        return pre + sort + 1 + 2 + 4 + 2

    def ensure_capacity(self):
        """Run one checked forward so the workspace holds this step's records."""
        self.r.preprocess(self.params, check=True)
        self.g_struct = R.gaussians_struct(self.params, self.r.cov)

    def capture(self, stream: torch.cuda.Stream):
        """Capture one step in a CUDA graph (after a warm-up on `stream`)."""
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=stream):
            self.enqueue(stream)
        return self.graph
