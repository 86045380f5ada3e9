"""Multi-rank host logic on CPU with two gloo ranks (no GPU): the plane
decomposition of the gradient (each rank renders its share of the planes with
the FP64 oracle and the per-rank gradients are summed) equals the gradient of
all planes at once, and the bench's max-over-ranks reductions."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene():
    from paper_2505_05643_gb300 import synth
    rng = np.random.default_rng(41)
    g = synth.gaussians_scale_rot(rng, 300, 0.05, 0.2)
    pl = synth.planes_random(rng, [(24, 24), (20, 28), (16, 16), (24, 18)])
    target = rng.uniform(0, 1, pl["total_pixels"])
    return g, pl, target


def _worker(rank, world, port, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2505_05643_gb300 import synth
        import bench
        g, pl, target = _scene()
        cfg = oracle.Config(cov_param=1)
        n_total = pl["total_pixels"]
        mine = [p for p in range(len(pl["size"])) if p % world == rank]
        sub = synth.select_planes(pl, mine)
        # this rank's pixels of the target, in its planes' order
        offs = pl["offset"]
        sizes = pl["size"]
        tsub = np.concatenate([target[offs[p]:offs[p] + sizes[p, 0] * sizes[p, 1]] for p in mine])
        out = oracle.render(g, sub, cfg)
        gimg = 2.0 * (out["image"] - tsub) / n_total  # dL/dC of the mean over ALL pixels
        gr, _ = oracle.render_grad(g, sub, cfg, out["image"], out["alpha"], gimg)
        t = torch.from_numpy(np.ascontiguousarray(gr))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        mx = bench.max_over_ranks(1.0 + rank)
        ok = bench.all_ok_over_ranks(rank != 1)
        if rank == 0:
            out_q.put((t.numpy(), mx, ok))
    finally:
        dist.destroy_process_group()


def test_plane_sharded_gradient_equals_full_gradient():
    import oracle
    g, pl, target = _scene()
    cfg = oracle.Config(cov_param=1)
    out = oracle.render(g, pl, cfg)
    _, gimg = oracle.mse_loss_grad(out["image"], target)
    full, _ = oracle.render_grad(g, pl, cfg, out["image"], out["alpha"], gimg)
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    summed, mx, ok = q.get()
    assert mx == 2.0 and ok is False
    scale = np.abs(full).max()
    assert np.allclose(summed, full, rtol=1e-10, atol=1e-12 * scale)


def _gauss_worker(rank, world, port, out_q):
    """Gaussian decomposition: each rank renders the planes with its share of
    the Gaussians, the partial sums S_a = sum w and S_c = sum w c are summed
    over the ranks (one all-reduce of two floats per pixel), the image is formed
    from the global sums, and each rank's gradient of its own Gaussians uses
    the global image and alpha (no further exchange)."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        g, pl, target = _scene()
        cfg = oracle.Config(cov_param=1)
        n = len(g["logit"])
        mine = np.arange(rank, n, world)
        gs = {k: v[..., mine] for k, v in g.items()}
        out = oracle.render(gs, pl, cfg)
        s_a = out["alpha"] - cfg.alpha_bg
        s_c = out["image"] * out["alpha"] - cfg.alpha_bg * cfg.c_bg
        t = torch.from_numpy(np.stack([s_a, s_c]))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        S_a, S_c = t[0].numpy(), t[1].numpy()
        alpha = S_a + cfg.alpha_bg
        image = (S_c + cfg.alpha_bg * cfg.c_bg) / alpha
        _, gimg = oracle.mse_loss_grad(image, target)
        gr, _ = oracle.render_grad(gs, pl, cfg, image, alpha, gimg)
        full = np.zeros((n, gr.shape[1]))
        full[mine] = gr
        tg = torch.from_numpy(full)
        dist.all_reduce(tg, op=dist.ReduceOp.SUM)  # only to collect the result on rank 0
        if rank == 0:
            out_q.put((image, alpha, tg.numpy()))
    finally:
        dist.destroy_process_group()


def test_gaussian_sharded_render_and_gradient_equal_full():
    import oracle
    g, pl, target = _scene()
    cfg = oracle.Config(cov_param=1)
    out = oracle.render(g, pl, cfg)
    _, gimg = oracle.mse_loss_grad(out["image"], target)
    full, _ = oracle.render_grad(g, pl, cfg, out["image"], out["alpha"], gimg)
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_gauss_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    image, alpha, grads = q.get()
    np.testing.assert_allclose(image, out["image"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(alpha, out["alpha"], rtol=1e-12, atol=1e-14)
    scale = np.abs(full).max()
    assert np.allclose(grads, full, rtol=1e-10, atol=1e-12 * scale)
