"""Choice of the tile edge and the rasterizer variants for one workload, by
timing them on the device (the workload's own records and tile lists):

- tile edge: 16 or 8 pixels (binning and sort cost against culling granularity);
- forward variant: lane groups per 8x8 footprint, i.e. pixels per lane (8, 4, 2),
  and for the 16-pixel tile the record pipeline's shape: records per
  shared-memory stage (64, 128, 256) and stages in the ring (2, 3, 4);
- backward variant: footprint height (8 or 4 rows), and for the 16-pixel tile
  stages (3, 4) and records per stage (64, 128, 256).

The forward and backward variants do not interact, so each is timed on its
own, per tile edge, between CUDA events on the launching stream; a tile edge
scores its preprocess + sort time plus its best forward and best backward.
"""
from __future__ import annotations

import torch

from . import binding as B
from . import render as R


def _time(fn, stream, warmup: int, reps: int) -> float:
    """Median milliseconds of fn() enqueued on stream."""
    for _ in range(warmup):
        fn()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ts.sort()
    return ts[len(ts) // 2]


def autotune(n: int, planes: dict, params: torch.Tensor, targets: torch.Tensor, cov_param: int,
             cutoff: int = B.UG_CUTOFF_BOX, tiles=(16, 8), warmup: int = 2, reps: int = 7,
             **cfg_kw):
    """Returns (config, table): the fastest configuration for rendering `params`
    on `planes` with MSE against `targets`, and the measured milliseconds
    {tile: {"pre_sort": t, "fwd": [t per variant], "bwd": [t per variant]}}."""
    stream = torch.cuda.current_stream()
    table, best = {}, None
    for tile in tiles:
        nf, nb = B.ug_num_variants(tile), B.ug_num_variants_bwd(tile)
        if nf == 0:
            continue
        cfg = R.make_config(cov_param=cov_param, cutoff=cutoff, tile=tile, variant=0,
                            variant_bwd=0, **cfg_kw)
        r = R.Renderer(n, planes, cfg)
        r.preprocess(params, check=True)  # sizes the workspace for these records
        g = R.gaussians_struct(params, r.cov)
        image, alpha, gimg = r.new_image(), r.new_image(), r.new_image()
        loss = torch.zeros(B.UG_MSE_LOSS_FLOATS, dtype=torch.float32, device=params.device)

        def pre_sort():
            B.ug_preprocess(r.plan, g, r.d_planes, r.ws, stream)
            B.ug_bin_sort(r.plan, r.ws, stream)

        t_pre = _time(pre_sort, stream, warmup, reps)
        fwd = []
        for v in range(nf):
            r.plan.cfg.variant = v
            fwd.append(_time(lambda: B.ug_render(r.plan, r.ws, image, alpha, stream), stream,
                             warmup, reps))
        r.plan.cfg.variant = min(range(nf), key=lambda v: fwd[v])
        B.ug_render(r.plan, r.ws, image, alpha, stream)
        B.ug_mse_loss_grad(image, targets, image.numel(), gimg, loss, stream)
        bwd = []
        for v in range(nb):
            r.plan.cfg.variant_bwd = v
            bwd.append(_time(lambda: B.ug_render_backward_raster(r.plan, r.ws, image, alpha, gimg,
                                                                  stream), stream, warmup, reps))
        st = r.status()
        if st["status"] != B.UG_OK:
            raise B.UgError(st["status"], f"autotune (tile {tile})")
        total = t_pre + min(fwd) + min(bwd)
        table[tile] = {"pre_sort": t_pre, "fwd": fwd, "bwd": bwd, "total": total}
        if best is None or total < best[0]:
            best = (total, tile, min(range(nf), key=lambda v: fwd[v]),
                    min(range(nb), key=lambda v: bwd[v]))
        del r, image, alpha, gimg
        torch.cuda.empty_cache()
    if best is None:
        raise ValueError("no supported tile size among " + str(tiles))
    _, tile, v, vb = best
    cfg = R.make_config(cov_param=cov_param, cutoff=cutoff, tile=tile, variant=v, variant_bwd=vb,
                        **cfg_kw)
    return cfg, table
