"""Multi-rank host logic on CPU with two gloo ranks (no GPU), through the
package's own data-plane functions (paper_2505_05643_gb300.parallel: the plane
and Gaussian splits, the global pixel count, the all-reduce); the FP64 oracle
stands in for the kernels each rank would launch. The plane decomposition of
the gradient equals the gradient of all planes at once, the Gaussian
decomposition of the render and gradient equals the full ones, and the bench's
max-over-ranks reductions work."""
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
        import bench
        from paper_2505_05643_gb300 import parallel
        g, pl, target = _scene()
        cfg = oracle.Config(cov_param=1)
        sub, mine = parallel.plane_shard(pl, rank, world)
        # this rank's pixels of the target, in its planes' order
        offs = pl["offset"]
        sizes = pl["size"]
        tsub = np.concatenate([target[offs[p]:offs[p] + sizes[p, 0] * sizes[p, 1]] for p in mine])
        n_total = parallel.global_count(sub["total_pixels"])
        assert n_total == pl["total_pixels"]
        out = oracle.render(g, sub, cfg)
        # the loss part of ug_mse_loss_grad_part: dL/dC of the mean over ALL pixels
        gimg = 2.0 * (out["image"] - tsub) / n_total
        loss = np.sum((out["image"] - tsub) ** 2) / n_total
        gr, _ = oracle.render_grad(g, sub, cfg, out["image"], out["alpha"], gimg)
        t = torch.from_numpy(np.ascontiguousarray(gr))
        parallel.allreduce_sum_(t)
        lt = parallel.allreduce_sum_(torch.tensor([loss], dtype=torch.float64))
        mx = bench.max_over_ranks(1.0 + rank)
        ok = bench.all_ok_over_ranks(rank != 1)
        if rank == 0:
            out_q.put((t.numpy(), float(lt[0]), mx, ok))
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
    summed, loss, mx, ok = q.get()
    assert mx == 2.0 and ok is False
    scale = np.abs(full).max()
    assert np.allclose(summed, full, rtol=1e-10, atol=1e-12 * scale)
    assert np.isclose(loss, np.mean((out["image"] - target) ** 2), rtol=1e-12)


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
        from paper_2505_05643_gb300 import parallel
        g, pl, target = _scene()
        cfg = oracle.Config(cov_param=1)
        n = len(g["logit"])
        lo, hi = parallel.gaussian_shard(n, rank, world)
        mine = np.arange(lo, hi)
        gs = {k: v[..., mine] for k, v in g.items()}
        out = oracle.render(gs, pl, cfg)
        # the partial sums of ug_shard_sums, interleaved per pixel
        s_a = out["alpha"] - cfg.alpha_bg
        s_c = out["image"] * out["alpha"] - cfg.alpha_bg * cfg.c_bg
        t = torch.from_numpy(np.ascontiguousarray(np.stack([s_a, s_c], axis=1)))
        parallel.allreduce_sum_(t)
        S_a, S_c = t[:, 0].numpy(), t[:, 1].numpy()
        alpha = S_a + cfg.alpha_bg
        image = (S_c + cfg.alpha_bg * cfg.c_bg) / alpha
        _, gimg = oracle.mse_loss_grad(image, target)
        gr, _ = oracle.render_grad(gs, pl, cfg, image, alpha, gimg)
        full = np.zeros((n, gr.shape[1]))
        full[mine] = gr
        tg = torch.from_numpy(full)
        parallel.allreduce_sum_(tg)  # only to collect the result on rank 0
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


def test_split_planes_contiguous_balanced_and_complete():
    from paper_2505_05643_gb300 import parallel
    rng = np.random.default_rng(5)
    for world in (1, 2, 3, 4, 8):
        for P in (world, world + 1, 17, 64):
            px = rng.choice([128 ** 2, 192 ** 2, 256 ** 2, 384 ** 2, 512 ** 2], size=P)
            parts = parallel.split_planes(px, world)
            assert len(parts) == world
            assert np.array_equal(np.concatenate(parts), np.arange(P))  # contiguous, complete
            assert all(len(p) >= 1 for p in parts)
            loads = np.array([px[p].sum() for p in parts])
            # no rank is more than one plane's pixels above an even share
            assert loads.max() <= px.sum() / world + px.max()
    with pytest.raises(ValueError):
        parallel.split_planes([1, 2], 3)


def test_gaussian_shard_covers_every_gaussian_once():
    from paper_2505_05643_gb300 import parallel
    for n in (1, 7, 100, 1_000_003):
        for world in (1, 2, 3, 8):
            bounds = [parallel.gaussian_shard(n, r, world) for r in range(world)]
            assert bounds[0][0] == 0 and bounds[-1][1] == n
            assert all(bounds[r][1] == bounds[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in bounds]
            assert max(sizes) - min(sizes) <= 1
