"""Data-parallel training across ranks (one process per GPU).

The plane rasterizer shards two ways, each with one exchange step:

Plane split (the training step's data parallelism). Planes are independent
images: each rank renders its own planes against a replica of the Gaussians.
The mean squared error over all ranks' pixels is the sum of per-rank parts
when every part is divided by the global pixel count
(``ug_mse_loss_grad_part``), and the gradient is linear in dL/dC, so the
per-Gaussian gradient rows of all ranks add up to the full gradient: one
all-reduce (sum) of the [rows][n] gradient buffer before Adam, which then runs
identically on every rank and keeps the replicated parameters equal.

Gaussian split (for Gaussian counts beyond one GPU). Image formation divides
two order-independent sums over Gaussians (Sec. 4.1, Eq. alpha-combine and
Eq. colour-combine), so the per-pixel partial sums (S_a, S_c) of shards of the
Gaussians add up to the full ones: each rank renders its shard over all
planes, ``ug_shard_sums`` turns the result into partial sums, one all-reduce
of two floats per pixel sums them, and ``ug_composite`` forms the global image
and alpha. Each rank's backward over its own shard then needs no exchange.

The collectives are torch.distributed all-reduces on plain device buffers
(NCCL on GPUs, gloo on CPU tensors); every other step is the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

from . import binding as B
from . import render as R
from . import synth
from . import train as T


def split_planes(pixels_per_plane, world: int) -> list[np.ndarray]:
    """Contiguous blocks of plane indices, one per rank, with pixel counts as
    equal as a contiguous split allows (each rank gets at least one plane when
    there are at least `world` planes)."""
    px = np.asarray(pixels_per_plane, dtype=np.int64)
    P = len(px)
    if world < 1:
        raise ValueError("world must be >= 1")
    if P < world:
        raise ValueError(f"{P} planes cannot be split over {world} ranks")
    cum = np.concatenate([[0], np.cumsum(px)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        # first plane of rank r: the boundary closest to r / world of the pixels,
        # leaving at least one plane for every later rank and taking one for this
        k = int(np.argmin(np.abs(cum - total * r / world)))
        k = min(max(k, cuts[-1] + 1), P - (world - r))
        cuts.append(k)
    cuts.append(P)
    return [np.arange(cuts[r], cuts[r + 1]) for r in range(world)]


def plane_shard(planes: dict, rank: int, world: int) -> tuple[dict, np.ndarray]:
    """This rank's planes (re-packed, pixel offsets from 0) and their indices."""
    sizes = planes["size"]
    idx = split_planes(sizes[:, 0].astype(np.int64) * sizes[:, 1], world)[rank]
    return synth.select_planes(planes, idx), idx


def gaussian_shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of this rank's contiguous block of the n Gaussians."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    base, extra = divmod(int(n), world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def allreduce_sum_(t: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum of t over the ranks of `group` (t itself when not
    distributed or with one rank)."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def global_count(n_local: int, device=None, group=None) -> int:
    """Sum of an integer count over the ranks."""
    t = torch.tensor([int(n_local)], dtype=torch.int64, device=device)
    allreduce_sum_(t, group)
    return int(t.item())


class PlaneSplitStep(T.TrainStep):
    """A training step whose planes are this rank's share of a plane-split
    batch: the loss part is divided by the pixels of all ranks, and the
    gradient rows (with the loss value) are summed over the ranks before Adam.

    enqueue() issues the whole step; enqueue_local() the calls up to the
    gradient and enqueue_update() the all-reduce and Adam, so that the local
    part can be captured in a CUDA graph while the collective runs eagerly."""

    def __init__(self, renderer: R.Renderer, params: torch.Tensor, targets: torch.Tensor,
                 total_pixels: int, group=None, **kw):
        super().__init__(renderer, params, targets, **kw)
        if self.loss_kind != "mse":
            raise ValueError("the plane split is written for the MSE loss")
        self.total_pixels = int(total_pixels)
        if self.total_pixels < renderer.total_pixels:
            raise ValueError("total_pixels must count every rank's pixels")
        self.group = group

    def enqueue_local(self, stream=None, targets_ready=None):
        r = self.r
        B.ug_preprocess(r.plan, self.g_struct, r.d_planes, r.ws, stream)
        B.ug_bin_sort(r.plan, r.ws, stream)
        B.ug_render(r.plan, r.ws, self.image, self.alpha, stream)
        if targets_ready is not None:
            (stream or torch.cuda.current_stream()).wait_event(targets_ready)
        B.ug_mse_loss_grad_part(self.image, self.targets, self.image.numel(), self.total_pixels,
                                self.grad_image, self.loss, stream)
        B.ug_render_backward(r.plan, self.g_struct, r.d_planes, r.ws, self.image, self.alpha,
                             self.grad_image, self.grad_struct, stream)

    def enqueue_update(self, stream=None):
        r = self.r
        with torch.cuda.stream(stream or torch.cuda.current_stream()):
            allreduce_sum_(self.grads, self.group)
            allreduce_sum_(self.loss[:1], self.group)
        B.ug_adam_step(self.params, self.grads, self.m, self.v, r.rows, r.n, self.lr_rows,
                       self.step, T.BETA1, T.BETA2, T.EPS, stream)

    def enqueue(self, stream=None, targets_ready=None):
        self.enqueue_local(stream, targets_ready)
        self.enqueue_update(stream)


def gaussian_split_forward(renderer: R.Renderer, params_shard: torch.Tensor, image: torch.Tensor,
                           alpha: torch.Tensor, sums: torch.Tensor, group=None, stream=None):
    """Forward of a Gaussian-sharded render: this rank's shard rendered over
    all planes, its partial (S_a, S_c) summed over the ranks, and the global
    image and alpha composited into `image` and `alpha` (all ranks hold the
    same result). `sums` is a device buffer of 2 x total_pixels floats."""
    n = renderer.total_pixels
    cfg = renderer.cfg
    renderer.forward(params_shard, image, alpha, check=False, stream=stream)
    B.ug_shard_sums(image, alpha, n, cfg.alpha_bg, cfg.c_bg, sums, stream)
    with torch.cuda.stream(stream or torch.cuda.current_stream()):
        allreduce_sum_(sums, group)
    B.ug_composite(sums, n, cfg.alpha_bg, cfg.c_bg, image, alpha, stream)
    return image, alpha
