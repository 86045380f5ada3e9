"""Benchmark of the GB300 plane rasterizer: one fwd+bwd+Adam training step of
the 1,000,000-Gaussian extreme-anisotropy workload (64 planes per launch,
square sizes drawn from {128, 192, 256, 384, 512}, triangular front-end, box
cut-off), captured in one CUDA graph and replayed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. `value` is useful Gaussian-pixel pairs per second: the
pairs the box cut-off includes (each evaluated in the forward and again in the
backward pass of a step) divided by the step time; `steps_per_s` is the train
step rate. Every step starts from the same state (initial parameters, zero Adam
moments), restored by a device copy inside the step, so the workload does not
drift with the number of steps. `--impl reference` times the FP64 CPU oracle (the only other
implementation of this method) on a bounded sample of the same workload.

Beside `value`: `e2e` (the same graph-captured step replayed through the public
API with the targets and poses copied from pinned host memory and the loss and
status read back every step; the targets double-buffered so that their copy
overlaps the previous step), `roofline` (the backward rasterizer's FP32-pipe fraction, the forward's
beside it, and every phase's time), `cpu_baseline` (the FP64 oracle on the host
cores), `clocks` (SM clock and throttle reasons sampled during the timed
region) and `gpu_launches`. Other modes: `--workload train_200k` (the batched
graph step against one plane per launch), `--workload recon` (reconstruction
run: SSIM over time, novel-slice images per second), `--workload densify`,
`--workload loss`, and `--ablation scatter` (the paper's atomic scatter forward
against the tile gather).
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP32-pipe operations per evaluated (pixel, record) pair, an FMA counting once:
# the essential per-pixel arithmetic of the formulation the rasterizers
# implement, without per-row or per-item set-up and without box masking.
#   forward:  t1 = r11 dx + r12 dy (1, r12 dy per row), e = lw2 - t1^2 - t2^2
#             (2, t2 per row), S_a += w (1), S_c += w c (1), dy (1)      -> 6
#   backward: t1 (1), e (1), g = (r c - r C) w (2), sum r w (1), sum g (1),
#             g t1 (1), sum g t1 (1), sum g t1 dx (1)                      -> 9
# each plus one MUFU.EX2, which runs at a quarter of the FP32 rate and binds
# only below 4 FP32 operations per pixel.
FWD_OPS = 6
BWD_OPS = 9
# DRAM bytes (read + write) of one launch of each rasterizer on this workload,
# from a one-pass ncu capture of the kernel as it stands; None when the kernel has
# changed since the counters were taken.
BWD_TRAFFIC = 551366656  # 473,574,912 read + 77,791,744 written (k_render_bwd, variant 5)
FWD_TRAFFIC = 323985664  # 279,489,792 read + 44,495,872 written (k_render_fwd, variant 5)

METRIC = "Gaussian·pixel evals/s and fwd+bwd train steps/s, 1M Gaussians, 1×GB300"
WORKLOAD = "aniso_1m: 1,000,000 Gaussians, axis ratios log-uniform to 1e4, 64 planes/launch " \
           "sized from {128,192,256,384,512}^2, fwd+bwd+Adam step"


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a per-rank float over all ranks (the step time the bench
    reports for N > 1); x itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    """Sum of a per-rank float over all ranks; x itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def all_ok_over_ranks(ok: bool, device=None) -> bool:
    """True when every rank reports ok."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return bool(ok)
    t = torch.tensor([0 if ok else 1], dtype=torch.int32, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return int(t.item()) == 0


def _clock_sampler(gpu_index: int, path: str):
    fields = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={fields}",
                              "--format=csv,noheader,nounits", "-lms", "50"],
                             stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except Exception:
        return None, None


def _wait_for_samples(path: str, timeout_s: float = 5.0):
    """Block until the sampler has written its first line (nvidia-smi start-up)."""
    t0 = time.time()
    while time.time() - t0 < timeout_s:
        try:
            if os.path.getsize(path) > 0:
                return
        except OSError:
            pass
        time.sleep(0.05)


def _clock_summary(path: str, t_start: datetime.datetime, t_stop: datetime.datetime) -> dict:
    """Median SM clock and active throttle reasons of the samples taken between
    t_start and t_stop (host wall clock, the same clock nvidia-smi stamps)."""
    sm, smax, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                clk, cmax = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            if ts < t_start or ts > t_stop:
                continue
            sm.append(clk)
            smax = max(smax, cmax)
            for name, val in zip(names, parts[6:10]):
                if val.lower().startswith("active") or val == "0x0000000000000001" or val == "1":
                    reasons.add(name)
    except OSError:
        pass
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax or None,
            "reasons": sorted(reasons), "samples": len(sm)}


def _workload(n_override=None):
    """The model (seed 0) and a hidden volume of the same distribution (seed 1)
    whose rendering on the same planes is the training target."""
    from paper_2505_05643_gb300 import synth
    g, pl = synth.workload_aniso_1m(seed=0)
    hidden, _ = synth.workload_aniso_1m(seed=1)
    if n_override:
        g = {k: v[..., :n_override] for k, v in g.items()}
        hidden = {k: v[..., :n_override] for k, v in hidden.items()}
    return synth.scale_rot_to_tri(g, 1e-4), pl, synth.scale_rot_to_tri(hidden, 1e-4)


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(g, pl, sample_planes=(0,), threads=0):
    """FP64 oracle (scatter forward + analytic backward) on a bounded sample
    of planes of the same workload. Returns (pairs/s, seconds, cores, pairs)."""
    import oracle
    from paper_2505_05643_gb300 import synth
    cfg = oracle.Config(cov_param=0)
    idx = np.asarray(sample_planes)
    sub = synth.select_planes(pl, idx)
    tgt = synth.target_images(np.random.default_rng(7), sub["total_pixels"])
    t0 = time.perf_counter()
    out = oracle.render(g, sub, cfg, mode="scatter", threads=threads)
    _, gimg = oracle.mse_loss_grad(out["image"], tgt)
    oracle.render_grad(g, sub, cfg, out["image"], out["alpha"], gimg, threads=threads)
    dt = time.perf_counter() - t0
    cores = threads or oracle.max_threads()
    return out["pairs"] / dt, dt, cores, out["pairs"]


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    g, pl, _ = _workload()
    sizes = pl["size"][:, 0]
    # each step: the oracle's forward + backward over a few of the 64 planes (all
    # 1M Gaussians), different planes each step, so that K steps take about a
    # minute or two on 16 host cores; the oracle has no warm state
    per_step = 4 if args.steps <= 50 else 1
    rates, secs, cores, total_pairs = [], [], 1, 0
    for k in range(args.steps):
        sample = [(per_step * k + j) % len(sizes) for j in range(per_step)]
        rate, dt, cores, pairs = cpu_oracle_rate(g, pl, sample)
        rates.append(rate)
        secs.append(dt)
        total_pairs += pairs
    value = float(total_pairs / np.sum(secs))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{per_step} of the 64 planes per step"},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                         "sample": "FP64 oracle scatter forward + analytic backward on "
                                   f"{per_step} of 64 planes per step (planes rotate), "
                                   "all 1,000,000 Gaussians, "
                                   f"{total_pairs} pairs in {np.sum(secs):.1f} s"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU
def run_ours(args):
    import torch
    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2505_05643_gb300 import binding as B
    from paper_2505_05643_gb300 import render as R
    from paper_2505_05643_gb300 import train as T

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass

    # Plane split (weak scaling): every rank renders its own 64 planes (rank 0
    # the workload's planes, rank r > 0 planes of the same sizes in other
    # random poses) against a replica of the Gaussians; the per-Gaussian
    # gradients are summed over the ranks (one all-reduce) before Adam.
    g, pl, hidden = _workload(args.n)
    if world > 1 and rank > 0:
        from paper_2505_05643_gb300 import synth
        pl = synth.planes_random(np.random.default_rng(1000 + rank),
                                 [tuple(int(x) for x in sz) for sz in pl["size"]])
    cfg = R.make_config(cov_param=B.UG_COV_TRI, cutoff=B.UG_CUTOFF_BOX, tile=args.tile,
                        variant=args.variant, variant_bwd=args.variant_bwd)
    n = len(g["logit"])
    # training data: the hidden volume rendered on the same planes (untimed)
    hid = R.Renderer(len(hidden["logit"]), pl, cfg)
    targets, _ = hid.forward(torch.from_numpy(R.pack_params(hidden, B.UG_COV_TRI)).to(dev))
    targets = targets.clone()
    target = targets.cpu().numpy()
    del hid
    params = torch.from_numpy(R.pack_params(g, B.UG_COV_TRI)).to(dev)
    tuned = None
    if not args.no_autotune:  # tile edge and variants chosen on this workload (untimed)
        from paper_2505_05643_gb300 import tune
        cfg, table = tune.autotune(n, pl, params, targets, B.UG_COV_TRI, B.UG_CUTOFF_BOX)
        tuned = {"tile": int(cfg.tile), "variant": int(cfg.variant),
                 "variant_bwd": int(cfg.variant_bwd),
                 "ms": {str(k): {kk: (round(vv, 4) if isinstance(vv, float) else
                                      [round(x, 4) for x in vv]) for kk, vv in t.items()}
                        for k, t in table.items()}}
        print(f"[bench] autotune: {tuned}", file=sys.stderr)
    renderer = R.Renderer(n, pl, cfg)
    r = renderer
    if world > 1:
        from paper_2505_05643_gb300 import parallel
        total_px = parallel.global_count(renderer.total_pixels, dev)
        step = parallel.PlaneSplitStep(renderer, params, targets, total_px)
    else:
        step = T.TrainStep(renderer, params, targets)
    s = torch.cuda.Stream(device=dev)
    st_dev = torch.zeros(64, dtype=torch.uint8, device=dev)

    # Every step starts from the same state: the initial parameters, zero Adam
    # moments and step counter 0, copied on the device at the start of the step
    # (inside the timed region). Without it the workload would drift with K:
    # at the paper's learning rate the boxes of this scene grow several-fold
    # within a few hundred steps.
    state0 = [t.clone() for t in (step.params, step.m, step.v, step.step)]

    def reset_on(stream):
        with torch.cuda.stream(stream):
            for dst, src in zip((step.params, step.m, step.v, step.step), state0):
                dst.copy_(src, non_blocking=True)

    def restore():
        reset_on(torch.cuda.current_stream())
        torch.cuda.synchronize()

    def read_status():
        B.ug_read_status(r.plan, r.ws, st_dev, s)
        s.synchronize()
        return B.ug_ws_status.from_buffer_copy(st_dev.cpu().numpy().tobytes())

    # sizing run: W + K checked eager steps; grow the workspace until none
    # overflows (a capacity overflow reports the counts it needed)
    st0 = renderer.preprocess(params, check=True)
    need = {"rec": st0["records"], "inst": st0["instances"]}

    def grow():
        rec = int(need["rec"] * 1.25) + 4096
        inst = min(int(need["inst"] * 1.25) + 65536, (1 << 31) - 1)
        renderer._alloc(rec, inst)
        step.g_struct = R.gaussians_struct(params, B.UG_COV_TRI)

    def note(x):
        need["rec"] = max(need["rec"], int(x.records))
        need["inst"] = max(need["inst"], int(x.instances))
        if x.status not in (B.UG_OK, B.UG_ERR_CAPACITY):
            raise RuntimeError(f"device status {x.status}")
        return x.status == B.UG_OK

    for attempt in range(12):
        grow()
        restore()
        ok = True
        with torch.cuda.stream(s):
            for k in range(args.warmup):
                reset_on(s)
                step.enqueue(s)
                if not note(read_status()):
                    ok = False
                    break
        if ok:
            break
    else:
        raise RuntimeError("workspace sizing did not converge")
    print(f"[bench] workspace: {renderer.plan.record_capacity} records, "
          f"{renderer.plan.instance_capacity} instances", file=sys.stderr)

    # ---- timed region: K replays of the captured step after W warm-up replays.
    # The backward's atomics make the trajectory differ slightly from the sizing
    # run's; a capacity overflow in the timed steps resizes and measures again.
    clk_path = os.path.join(tempfile.gettempdir(), f"ug_bench_clocks_{os.getpid()}_{rank}.csv")
    status_log = torch.zeros((args.warmup + args.steps, 64), dtype=torch.uint8, device=dev)
    for attempt in range(3):
        restore()
        s.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            reset_on(s)
            if world > 1:
                step.enqueue_local(s)  # the all-reduce runs eagerly after the replay
            else:
                step.enqueue(s)

        def one(k):
            graph.replay()
            if world > 1:
                step.enqueue_update(s)
            B.ug_read_status(renderer.plan, renderer.ws, status_log[k], s)

        with torch.cuda.stream(s):
            for k in range(args.warmup):
                one(k)
        s.synchronize()
        sampler, fh = _clock_sampler(dev.index or 0, clk_path)
        _wait_for_samples(clk_path)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t_start = datetime.datetime.now()
        # events at the start, at every quarter of the K steps and at the end
        # (recorded between replays on the launching stream): the quarters give
        # the spread of the step time within the one timed region
        cuts = sorted({0, args.steps} | {args.steps * q // 4 for q in range(1, 4)})
        ev = {c: torch.cuda.Event(enable_timing=True) for c in cuts}
        ev[0].record(s)
        with torch.cuda.stream(s):
            for k in range(args.steps):
                one(args.warmup + k)
                if k + 1 in ev:
                    ev[k + 1].record(s)
        torch.cuda.synchronize()
        t_stop = datetime.datetime.now()
        total_ms = ev[0].elapsed_time(ev[args.steps])
        segments = [ev[a].elapsed_time(ev[b]) / (b - a) for a, b in zip(cuts[:-1], cuts[1:])
                    if b > a]
        if sampler is not None:
            time.sleep(0.15)  # let the sampler flush the last interval
            sampler.terminate()
            sampler.wait()
            fh.close()
        sts = [B.ug_ws_status.from_buffer_copy(row.tobytes()) for row in status_log.cpu().numpy()]
        ok = all_ok_over_ranks(all([note(x) for x in sts]), dev)
        if ok:
            break
        print("[bench] capacity overflow in the timed steps: resizing and measuring again",
              file=sys.stderr)
        grow()
    else:
        raise RuntimeError("capacity overflow in the timed steps")
    clocks = _clock_summary(clk_path, t_start, t_stop)
    ms_step = max_over_ranks(total_ms / args.steps, dev)
    timing = {"timed_s": total_ms * 1e-3, "segments_ms_per_step": segments,
              "spread": (max(segments) - min(segments)) / statistics.median(segments)}
    if clocks.get("sm_mhz"):
        # step time in SM clock cycles at the median sampled clock, and the
        # step time that cycle count would take at the maximum clock
        timing["mcycles_per_step"] = ms_step * clocks["sm_mhz"] * 1e-3
        if clocks.get("sm_max_mhz"):
            timing["ms_per_step_at_max_clock"] = ms_step * clocks["sm_mhz"] / clocks["sm_max_mhz"]
    pairs = float(np.mean([x.box_pixels for x in sts[args.warmup:]]))
    value = sum_over_ranks(pairs, dev) / (ms_step * 1e-3)

    # ---- phase timing: the same W + K steps eagerly, CUDA events on the
    # launching stream around each call of the step
    e = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
    for attempt in range(3):
        restore()
        bwd_ms, fwd_ms, chain_ms, pre_ms, eager_st = [], [], [], [], []
        ok = True
        with torch.cuda.stream(s):
            for k in range(args.warmup + args.steps):
                reset_on(s)
                e[0].record(s)
                B.ug_preprocess(r.plan, step.g_struct, r.d_planes, r.ws, s)
                B.ug_bin_sort(r.plan, r.ws, s)
                e[1].record(s)
                B.ug_render(r.plan, r.ws, step.image, step.alpha, s)
                e[2].record(s)
                if world > 1:
                    B.ug_mse_loss_grad_part(step.image, step.targets, step.image.numel(),
                                            step.total_pixels, step.grad_image, step.loss, s)
                else:
                    B.ug_mse_loss_grad(step.image, step.targets, step.image.numel(),
                                       step.grad_image, step.loss, s)
                e[3].record(s)
                B.ug_render_backward_raster(r.plan, r.ws, step.image, step.alpha, step.grad_image,
                                            s)
                e[4].record(s)
                B.ug_preprocess_backward(r.plan, step.g_struct, r.ws, step.grad_struct, s)
                e[5].record(s)
                if world > 1:
                    step.enqueue_update(s)  # all-reduce of the gradients, then Adam
                else:
                    B.ug_adam_step(step.params, step.grads, step.m, step.v, r.rows, r.n,
                                   step.lr_rows, step.step, T.BETA1, T.BETA2, T.EPS, s)
                x = read_status()
                if not note(x):
                    ok = False
                    break
                if k >= args.warmup:
                    eager_st.append(x)
                    pre_ms.append(e[0].elapsed_time(e[1]))
                    fwd_ms.append(e[1].elapsed_time(e[2]))
                    bwd_ms.append(e[3].elapsed_time(e[4]))
                    chain_ms.append(e[4].elapsed_time(e[5]))
        if ok:
            break
        grow()
    else:
        raise RuntimeError("capacity overflow in the phase-timing steps")

    # ---- e2e: the training step as a user runs it, from host buffers: the
    # step's inputs (targets and plane poses) copied from pinned host memory, and
    # its loss and status read back into pinned host memory, every step. The step
    # is captured once per targets buffer (two device buffers: the next step's
    # targets are copied on their own stream while the current step runs) and
    # replayed; the plane poses are copied on the step's stream before each
    # replay. The host runs up to two steps ahead of the device (double-buffered
    # read-back): it reads step k's results after issuing step k + 1, as a
    # training loop that logs its loss would.
    h_targets = torch.from_numpy(target).pin_memory()
    h_planes = torch.from_numpy(r.host_planes.view(np.uint8).copy()).pin_memory()
    h_loss = torch.zeros((2, 1), dtype=torch.float32).pin_memory()
    h_st = torch.zeros((2, 64), dtype=torch.uint8).pin_memory()
    copy_s = torch.cuda.Stream()
    targets_in = [torch.cuda.Event(), torch.cuda.Event()]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    tbuf = [step.targets, torch.empty_like(step.targets)]
    for attempt in range(3):
        restore()
        s.wait_stream(torch.cuda.current_stream())
        graphs = []
        for b in range(2):
            step.targets = tbuf[b]
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                reset_on(s)
                if world > 1:
                    step.enqueue_local(s)  # the all-reduce runs eagerly after the replay
                else:
                    step.enqueue(s)
            graphs.append(g)
        step.targets = tbuf[0]
        e2e_st, e2e_loss = [], []

        def collect(b):
            done[b].synchronize()
            e2e_st.append(B.ug_ws_status.from_buffer_copy(h_st[b].numpy().tobytes()))
            e2e_loss.append(float(h_loss[b, 0]))

        def one(k):
            b = k % 2
            # this buffer was last read by step k - 2
            with torch.cuda.stream(copy_s):
                if k >= 2:
                    copy_s.wait_event(done[b])
                tbuf[b].copy_(h_targets, non_blocking=True)
                targets_in[b].record(copy_s)
            r.d_planes.copy_(h_planes, non_blocking=True)
            s.wait_event(targets_in[b])
            graphs[b].replay()
            if world > 1:
                step.enqueue_update(s)
            h_loss[b].copy_(step.loss[:1], non_blocking=True)
            B.ug_read_status(r.plan, r.ws, h_st[b], s)
            done[b].record(s)

        with torch.cuda.stream(s):
            for k in range(args.warmup):
                one(k)
        s.synchronize()
        e2e_st, e2e_loss = [], []
        t0 = time.perf_counter()
        with torch.cuda.stream(s):
            for k in range(args.steps):
                if k >= 2:
                    collect(k % 2)  # step k - 2's results; its buffers are then free
                one(k)
            for k in range(max(args.steps - 2, 0), args.steps):
                collect(k % 2)
        e2e_s = (time.perf_counter() - t0) / args.steps
        assert all(np.isfinite(e2e_loss))
        if all([note(x) for x in e2e_st]):
            break
        grow()
    else:
        raise RuntimeError("capacity overflow in the end-to-end steps")
    e2e_pairs = float(np.mean([x.box_pixels for x in e2e_st]))
    e2e = {"value": sum_over_ranks(e2e_pairs, dev) / max_over_ranks(e2e_s, dev),
           "unit": "pairs/s",
           "h2d_bytes_per_step": int(h_targets.numel() * 4 + h_planes.numel()),
           "d2h_bytes_per_step": 4 + 64}

    # ---- roofline of the dominant kernel: the backward rasterizer (FP32-pipe
    # bound), timed as the ug_render_backward_raster call (its zeroing of the
    # per-record gradient buffer included).
    # Unit: one evaluated (pixel, record) pair. Algorithmic FP32-pipe operations
    # per evaluated pair (an FMA counts once): forward FWD_OPS, backward BWD_OPS,
    # each plus one MUFU.EX2 (32/clk/SM, not binding at these op counts). Peak
    # from unit counts and clocks: SMs x 128 FP32 lanes x max SM clock (2070 MHz).
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fmax = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    fp32_peak = sms * 128 * fmax
    bwd_s = float(np.mean(bwd_ms)) * 1e-3
    fwd_s = float(np.mean(fwd_ms)) * 1e-3
    evaluated = float(np.mean([x.evaluated_pairs for x in eager_st]))
    evaluated_bwd = float(np.mean([x.evaluated_pairs_bwd for x in eager_st]))
    pairs_eager = float(np.mean([x.box_pixels for x in eager_st]))
    roof = {"bound": "alu", "kernel": "k_render_bwd (ug_render_backward_raster)",
            "achieved": BWD_OPS * evaluated_bwd / bwd_s / 1e12, "peak": fp32_peak / 1e12,
            "unit": "Tops/s (FP32 pipe)", "frac": BWD_OPS * evaluated_bwd / bwd_s / fp32_peak,
            "traffic": BWD_TRAFFIC,
            "units_per_launch": evaluated_bwd, "ops_per_unit": BWD_OPS,
            "peak_note": "derived: SMs x 128 FP32 lanes x max SM clock",
            "fwd": {"kernel": "k_render_fwd (ug_render)", "ms": fwd_s * 1e3,
                    "ops_per_unit": FWD_OPS, "units_per_launch": evaluated,
                    "achieved": FWD_OPS * evaluated / fwd_s / 1e12,
                    "frac": FWD_OPS * evaluated / fwd_s / fp32_peak, "traffic": FWD_TRAFFIC},
            "bwd_ms": bwd_s * 1e3, "box_pairs_per_launch": pairs_eager,
            "evaluated_over_box_pairs": evaluated / pairs_eager,
            "evaluated_bwd_over_box_pairs": evaluated_bwd / pairs_eager,
            # the same launches per useful pair (the box cut-off's pairs,
            # counted exactly), with the same op counts: the rate of the
            # paper's work unit, the pairs the kernels skip as exact FP32 zeros
            # included
            "per_useful_pair": {
                "units_per_launch": pairs_eager,
                "bwd": {"ops_per_unit": BWD_OPS,
                        "achieved": BWD_OPS * pairs_eager / bwd_s / 1e12,
                        "frac": BWD_OPS * pairs_eager / bwd_s / fp32_peak},
                "fwd": {"ops_per_unit": FWD_OPS,
                        "achieved": FWD_OPS * pairs_eager / fwd_s / 1e12,
                        "frac": FWD_OPS * pairs_eager / fwd_s / fp32_peak}},
            "phases_ms": {"preprocess+bin_sort": float(np.mean(pre_ms)),
                          "render": fwd_s * 1e3, "render_backward_raster": bwd_s * 1e3,
                          "preprocess_backward": float(np.mean(chain_ms))}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        sizes = pl["size"][:, 0]
        sample = list(range(min(args.cpu_planes, len(sizes))))
        rate, dt, cores, cp = cpu_oracle_rate(g, pl, sample)
        cpu = {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle scatter forward + analytic backward on planes "
                         f"0..{len(sample) - 1} of 64 ({cp} pairs) with all {n} Gaussians "
                         f"(initial parameters), {dt:.1f} s"}
    launches = step.kernels_per_step() * args.steps
    batching = None
    if rank == 0 and world == 1 and not args.no_train_compare:
        # the batched graph-captured step against one plane per launch on the
        # 200k training workload (its own Gaussians, poses and targets)
        del step, renderer, r, graph
        torch.cuda.empty_cache()
        tc = train_compare(args.compare_steps, 3, int(cfg.tile), int(cfg.variant),
                           int(cfg.variant_bwd))
        acc = tc["accuracy"]
        lm = acc["loss_mean_last"]
        batching = {"workload": tc["config"]["workload"], "steps": tc["steps"],
                    "tile": tc["config"]["tile"], "variant": tc["config"]["variant"],
                    "variant_bwd": tc["config"]["variant_bwd"],
                    "batched_ms_per_step": tc["ms_per_step"],
                    "per_plane_ms_per_step": tc["per_plane"]["ms_per_step"],
                    "factor": tc["speedup"],
                    "first_step_grad_rel_l2_diff": acc["first_step_grad_rel_l2_diff"],
                    "loss_mean_last": lm, "loss_mean_last_steps": acc["loss_mean_last_steps"],
                    "rel_diff_loss_mean_last": abs(lm[0] - lm[1]) / abs(lm[1]),
                    "note": "Adam (eps 1e-15) takes full steps on gradients that are rounding "
                            "noise, so the two trajectories part after a few steps; accuracy "
                            "is compared on the first step's gradient and the late loss level"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "gaussians": n, "planes": len(pl["size"]),
                       "pixels": int(pl["total_pixels"]), "pairs_per_step": pairs,
                       "tile": int(cfg.tile), "variant": int(cfg.variant),
                       "variant_bwd": int(cfg.variant_bwd), "autotune": tuned, "graph": True,
                       "targets": "hidden 1M-Gaussian volume (seed 1) rendered on the same planes",
                       "l2": "working set > L2 (129 MB); no flush",
                       "state": "every step starts from the initial parameters and zero Adam "
                                "moments (device copy inside the timed step)",
                       "parallelism": (f"plane split x{world}: each rank its own 64 planes, "
                                       "one all-reduce of the per-Gaussian gradients per step"
                                       if world > 1 else "single GPU")},
            "steps_per_s": 1e3 / ms_step,
            "gpu_launches": launches,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "timing": timing, "batched_vs_per_plane": batching,
            "fp64_records": int(sts[-1].fp64_records), "records": int(sts[-1].records),
            "instances": int(sts[-1].instances),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------- batching
def run_train_compare(args):
    print(json.dumps(train_compare(args.steps, args.warmup, args.tile, args.variant,
                                   args.variant_bwd)), flush=True)
    return 0


def train_compare(K, W, tile=16, variant=0, variant_bwd=0):
    """Training workload (200,000 Gaussians in the paper's initialisation,
    fitted to a hidden 100,000-Gaussian volume on 32 sweep poses of 256x256 per
    step): the batched step (all 32 planes per launch, the whole step captured
    in one CUDA graph) against the plain form (preprocess, sort, render and
    backward launched plane by plane, gradients summed, then Adam), from the
    same initial state over the same pose schedule. Reports both step times,
    the speed-up and the difference of the two loss trajectories. Both forms
    use the same tile edge and rasterizer variants (in the default bench line,
    the autotuner's choice on the bench workload)."""
    import torch
    from paper_2505_05643_gb300 import binding as B
    from paper_2505_05643_gb300 import render as R
    from paper_2505_05643_gb300 import synth
    from paper_2505_05643_gb300 import train as T
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    g, poses, hidden = synth.workload_train_200k()
    n, P, pool = len(g["logit"]), 32, len(poses["size"])
    npx = int(poses["size"][0, 0] * poses["size"][0, 1])
    windows = [[(P * k + j) % pool for j in range(P)] for k in range(pool // P)]
    cfg = R.make_config(cov_param=B.UG_COV_TRI, tile=tile, variant=variant,
                        variant_bwd=variant_bwd)
    # targets on every pose of the pool (untimed)
    hid = R.Renderer(len(hidden["logit"]), poses, R.make_config(cov_param=B.UG_COV_SCALE_ROT))
    tpool, _ = hid.forward(torch.from_numpy(R.pack_params(hidden, B.UG_COV_SCALE_ROT)).to(dev))
    tpool = tpool.clone().view(pool, npx)
    del hid
    win_planes = [synth.select_planes(poses, w) for w in windows]
    win_struct = [torch.from_numpy(synth.planes_to_struct(wp).view(np.uint8).copy()).to(dev)
                  for wp in win_planes]
    win_idx = [torch.tensor(w, device=dev) for w in windows]
    # one-plane structs (pixel offset 0) for the plane-by-plane form
    one_struct = [[torch.from_numpy(synth.planes_to_struct(synth.select_planes(wp, [p]))
                                    .view(np.uint8).copy()).to(dev) for p in range(P)]
                  for wp in win_planes]
    p0 = torch.from_numpy(R.pack_params(g, B.UG_COV_TRI)).to(dev)
    s = torch.cuda.Stream(device=dev)

    # ---- batched
    rb = R.Renderer(n, win_planes[0], cfg)
    targets = torch.empty(P * npx, dtype=torch.float32, device=dev)
    step = T.TrainStep(rb, p0.clone(), targets)

    def reset(st):
        st.params.copy_(p0)
        st.m.zero_()
        st.v.zero_()
        st.step.zero_()

    def inputs(k, stream):
        w = k % len(windows)
        with torch.cuda.stream(stream):
            rb.d_planes.copy_(win_struct[w], non_blocking=True)
            targets.copy_(tpool.index_select(0, win_idx[w]).view(-1), non_blocking=True)

    # sizing: W + K checked eager steps (the records grow as the Gaussians move),
    # then a 25 % margin for the timed runs' slightly different trajectories
    need = [0, 0]
    for attempt in range(8):
        reset(step)
        ok = True
        for k in range(W + K):
            inputs(k, torch.cuda.current_stream())
            step.enqueue()
            st = rb.status()
            need = [max(need[0], st["records"]), max(need[1], st["instances"])]
            if st["status"] == B.UG_ERR_CAPACITY:
                rb._alloc(int(need[0] * 1.3) + 4096, int(need[1] * 1.3) + 65536)
                step.g_struct = R.gaussians_struct(step.params, rb.cov)
                ok = False
                break
            assert st["status"] == B.UG_OK, st
        if ok:
            break
    rb._alloc(max(int(need[0] * 1.25) + 4096, int(rb.plan.record_capacity)),
              max(int(need[1] * 1.25) + 65536, int(rb.plan.instance_capacity)))
    step.g_struct = R.gaussians_struct(step.params, rb.cov)
    reset(step)
    torch.cuda.synchronize()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        step.enqueue(s)
    loss_b = torch.zeros(K, device=dev)
    grad_b0 = torch.zeros_like(step.grads)

    def batched_run(record):
        reset(step)
        torch.cuda.synchronize()
        for k in range(K):
            inputs(k, s)
            with torch.cuda.stream(s):
                graph.replay()
                if record:
                    loss_b[k].copy_(step.loss[0])
                    if k == 0:
                        grad_b0.copy_(step.grads)

    with torch.cuda.stream(s):
        for k in range(W):
            inputs(k, s)
            graph.replay()
    s.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    batched_run(False)  # warm
    s.synchronize()
    reset(step)
    torch.cuda.synchronize()
    e0.record(s)
    batched_run(True)
    e1.record(s)
    s.synchronize()
    ms_b = e0.elapsed_time(e1) / K
    params_b = step.params.clone()
    st = rb.status(s)
    assert st["status"] == B.UG_OK, st

    # ---- per plane
    rps = [R.Renderer(n, synth.select_planes(win_planes[0], [p]), cfg) for p in range(P)]
    params = p0.clone()
    grads = torch.zeros_like(params)
    gpl = torch.zeros_like(params)
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    stp = torch.zeros(1, dtype=torch.int32, device=dev)
    image, alpha, gimg = (torch.empty(P * npx, device=dev) for _ in range(3))
    loss = torch.zeros(B.UG_MSE_LOSS_FLOATS, device=dev)
    lr_rows = step.lr_rows
    gs = R.gaussians_struct(params, B.UG_COV_TRI)
    gps = R.grads_struct(gpl, B.UG_COV_TRI)

    def plain_step(k, stream, check):
        w = k % len(windows)
        for p, rp in enumerate(rps):
            rp.d_planes.copy_(one_struct[w][p], non_blocking=True)
            if check:
                rp.preprocess(params, check=True)
            else:
                B.ug_preprocess(rp.plan, gs, rp.d_planes, rp.ws, stream)
            B.ug_bin_sort(rp.plan, rp.ws, stream)
            B.ug_render(rp.plan, rp.ws, image[p * npx:(p + 1) * npx], alpha[p * npx:(p + 1) * npx],
                        stream)
        targets.copy_(tpool.index_select(0, win_idx[w]).view(-1), non_blocking=True)
        B.ug_mse_loss_grad(image, targets, P * npx, gimg, loss, stream)
        for p, rp in enumerate(rps):
            B.ug_render_backward(rp.plan, gs, rp.d_planes, rp.ws, image[p * npx:(p + 1) * npx],
                                 alpha[p * npx:(p + 1) * npx], gimg[p * npx:(p + 1) * npx], gps,
                                 stream)
            if p == 0:
                grads.copy_(gpl)
            else:
                grads.add_(gpl)
        B.ug_adam_step(params, grads, m, v, rb.rows, n, lr_rows, stp, T.BETA1, T.BETA2, T.EPS,
                       stream)

    def plain_reset():
        params.copy_(p0)
        m.zero_()
        v.zero_()
        stp.zero_()

    plain_reset()
    for k in range(W + K):  # sizing (checked) and warm-up
        plain_step(k, torch.cuda.current_stream(), True)
    for rp in rps:  # margin for the timed run's slightly different trajectory
        rp._alloc(int(rp.plan.record_capacity * 1.25) + 1024,
                  int(rp.plan.instance_capacity * 1.25) + 4096)
    gs = R.gaussians_struct(params, B.UG_COV_TRI)
    plain_reset()
    torch.cuda.synchronize()
    loss_p = torch.zeros(K, device=dev)
    grad_p0 = torch.zeros_like(grads)
    with torch.cuda.stream(s):
        e0.record(s)
        for k in range(K):
            plain_step(k, s, False)
            loss_p[k].copy_(loss[0])
            if k == 0:
                grad_p0.copy_(grads)
        e1.record(s)
    s.synchronize()
    ms_p = e0.elapsed_time(e1) / K
    for rp in rps:
        st = rp.status(s)
        assert st["status"] == B.UG_OK, st
    lb, lp = loss_b.cpu().numpy(), loss_p.cpu().numpy()
    rel = np.abs(lb - lp) / np.abs(lp)
    # the first step starts both forms from the same parameters: their
    # gradients agree up to FP32 summation order
    gb0, gp0 = grad_b0.double(), grad_p0.double()
    grad_rel = float((gb0 - gp0).norm() / gp0.norm())
    tail = max(1, min(20, K // 4))  # whole cycles of the 5 pose windows when K >= 100
    dparam = float((params_b - params).abs().max())
    moved = float((params_b - p0).abs().max())
    line = {
        "metric": "train steps/s, 200k Gaussians, 32 planes of 256x256: batched graph vs "
                  "one plane per launch",
        "value": 1e3 / ms_b, "unit": "steps/s", "n_gpus": 1, "steps": K, "warmup": W,
        "ms_per_step": ms_b, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "train_200k: 200,000 Gaussians (paper init), hidden 100,000-"
                               "Gaussian volume (seed 2), 160 sweep poses, 32 per step",
                   "tile": int(cfg.tile), "variant": int(cfg.variant),
                   "variant_bwd": int(cfg.variant_bwd)},
        "per_plane": {"ms_per_step": ms_p, "steps_per_s": 1e3 / ms_p,
                      "form": "eager: per plane preprocess, sort, render; one MSE; per plane "
                              "backward with the gradients summed; Adam"},
        "speedup": ms_p / ms_b,
        # both forms sum the same terms in different orders (and the backward's
        # atomics in no fixed order), so their trajectories part slowly; Adam
        # (normalised steps) lets the rounding differences grow over the run
        "accuracy": {"first_step_grad_rel_l2_diff": grad_rel,
                     "loss_mean_last": [float(lb[-tail:].mean()), float(lp[-tail:].mean())],
                     "loss_mean_last_steps": tail,
                     "loss_first": [float(lb[0]), float(lp[0])],
                     "loss_last": [float(lb[-1]), float(lp[-1])],
                     "max_rel_loss_diff": float(np.max(rel)),
                     "max_rel_loss_diff_first_20": float(np.max(rel[:20])),
                     "rel_loss_diff_at": {str(k): float(rel[k]) for k in (0, 9, 49, 99, 199)
                                          if k < len(rel)},
                     "max_param_diff": dparam, "max_param_change": moved},
    }
    return line


# ---------------------------------------------------------------- reconstruction
def run_recon(args):
    """Reconstruction run: Gaussians in the paper's initialisation fitted to a
    hidden synthetic volume with MSE (or L1 + D-SSIM) and Adam (the paper's
    learning rates, the means' rate decaying over the run), each step on 32
    poses drawn from a pool of training poses; SSIM and PSNR (the evaluator
    kernel) on the evaluation poses and on up to 128 training poses every
    --recon-eval steps; the training time to reach SSIM thresholds, without
    and with the densify / prune step (--recon-densify); then forward-only
    novel-slice rendering of 512x512 planes, images per second.
    --recon-poses random: random training and held-out poses (256x256);
    slices: the paper's ideal setting (Sec. 5.1), training on linearly spaced
    axial slices and evaluating on linearly spaced axial, coronal and sagittal
    slices (160 of each, 160x160)."""
    import torch
    from paper_2505_05643_gb300 import binding as B
    from paper_2505_05643_gb300 import render as R
    from paper_2505_05643_gb300 import synth
    from paper_2505_05643_gb300 import train as T
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n, steps, every = args.recon_n, args.recon_steps, args.recon_eval
    slices = args.recon_poses == "slices"
    size = args.recon_size or (160 if slices else 256)
    pool_n, held_n = (160, 160) if slices else (320, 128)
    g, hidden, tr, te = synth.workload_recon(n=n, hidden_n=args.recon_hidden, size=size,
                                             train_pool=pool_n, held_out=held_n,
                                             poses=args.recon_poses)
    P = 32
    npx = size * size
    cfg = R.make_config(cov_param=B.UG_COV_TRI)
    cfg_h = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    hp = torch.from_numpy(R.pack_params(hidden, B.UG_COV_SCALE_ROT)).to(dev)

    def render_targets(planes, chunk=32):
        outs = []
        for c0 in range(0, len(planes["size"]), chunk):
            sub = synth.select_planes(planes, list(range(c0, min(c0 + chunk, len(planes["size"])))))
            img, _ = R.Renderer(len(hidden["logit"]), sub, cfg_h).forward(hp)
            outs.append(img.clone())
        torch.cuda.empty_cache()
        return torch.cat(outs).view(-1, npx)

    t_train = render_targets(tr)   # (pool, npx)
    t_test = render_targets(te)    # (evaluation poses, npx)
    pool = len(tr["size"])
    rng = np.random.default_rng(6)
    win_struct = {}

    def pose_struct(idx):
        key = tuple(idx)
        if key not in win_struct:
            win_struct[key] = torch.from_numpy(
                synth.planes_to_struct(synth.select_planes(tr, list(idx))).view(np.uint8).copy()).to(dev)
        return win_struct[key]

    p_init = torch.from_numpy(R.pack_params(g, B.UG_COV_TRI)).to(dev)
    scratch = torch.empty(B.ug_ssim_scratch_floats(32, size, size), device=dev)
    ss, ps = torch.empty(32, device=dev), torch.empty(32, device=dev)
    train_idx = np.linspace(0, pool - 1, min(128, pool)).round().astype(np.int64)
    train_eval_planes = synth.select_planes(tr, list(train_idx))
    train_eval_tgt = t_train.index_select(0, torch.from_numpy(train_idx).to(dev))

    def eval_set(planes, tgt, nn):
        m = len(planes["size"])
        return [(R.Renderer(nn, synth.select_planes(planes, list(range(c0, min(c0 + 32, m)))), cfg),
                 tgt[c0:min(c0 + 32, m)].reshape(-1)) for c0 in range(0, m, 32)]

    def evaluate(es, params):
        vals_s, vals_p = [], []
        for rr, tt in es:
            img, _ = rr.forward(params)
            m = len(rr.host_planes)
            B.ug_ssim(img, tt, m, size, size, scratch, ss[:m], ps[:m])
            vals_s.append(ss[:m].cpu().numpy().copy())
            vals_p.append(ps[:m].cpu().numpy().copy())
        return np.concatenate(vals_s), np.concatenate(vals_p)

    def train(densify):
        """One training run from the initial Gaussians; with densify, the
        densify / prune step (ug_densify_stats every step, ug_densify every
        --densify-every steps in [--densify-every, steps / 2], up to
        --densify-max times the initial count), Adam moments carried."""
        params = p_init.clone()
        nn = n
        r = R.Renderer(nn, synth.select_planes(tr, list(range(P))), cfg)
        targets = torch.empty(P * npx, device=dev)
        step = T.TrainStep(r, params, targets, decay_steps=steps, loss=args.recon_loss,
                           plane_shape=(size, size))
        sets = {}

        def record(k, train_s, loss=None):
            if nn not in sets:  # evaluation renderers for this Gaussian count
                sets.clear()
                torch.cuda.empty_cache()
                sets[nn] = (eval_set(te, t_test, nn), eval_set(train_eval_planes, train_eval_tgt, nn))
            sv, pv = evaluate(sets[nn][0], params)
            st, _ = evaluate(sets[nn][1], params)
            h = {"step": k, "train_s": train_s, "ssim": float(sv.mean()), "psnr": float(pv.mean()),
                 "train_ssim": float(st.mean()), "gaussians": nn}
            if slices:  # axial, coronal, sagittal means
                h["ssim_axes"] = [float(x.mean()) for x in np.split(sv, 3)]
            if loss is not None:
                h["loss"] = loss
            return h

        history = [record(0, 0.0)]
        train_ms = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        rng = np.random.default_rng(6)
        order = rng.permutation(pool)
        dcfg = B.ug_densify_config_default()
        stats = torch.zeros((2, nn), device=dev) if densify else None
        zgen = torch.Generator(device=dev)
        zgen.manual_seed(8)
        dlog = []
        for k in range(steps):
            o = (k * P) % pool
            if k > 0 and o < P:  # a new epoch: a new order of the training poses
                order = rng.permutation(pool)
            idx = np.sort(order[o:o + P]) if o + P <= pool else np.sort(order[:P])
            r.d_planes.copy_(pose_struct(idx))
            targets.copy_(t_train.index_select(0, torch.from_numpy(idx).to(dev)).view(-1))
            e0.record()
            r.preprocess(params, check=True)  # grows the workspace when the records outgrow it
            step.g_struct = R.gaussians_struct(params, B.UG_COV_TRI)
            B.ug_bin_sort(r.plan, r.ws)
            B.ug_render(r.plan, r.ws, step.image, step.alpha)
            if args.recon_loss == "mse":
                B.ug_mse_loss_grad(step.image, targets, step.image.numel(), step.grad_image,
                                   step.loss)
            else:
                B.ug_l1_dssim_loss_grad(step.image, targets, *step.dssim_shape, T.DSSIM_LAMBDA,
                                        step.dssim_scratch, step.grad_image, step.loss)
            B.ug_render_backward(r.plan, step.g_struct, r.d_planes, r.ws, step.image, step.alpha,
                                 step.grad_image, step.grad_struct)
            if densify:
                B.ug_densify_stats(step.grads, nn, stats)  # the mean rows come first
            B.ug_adam_step(params, step.grads, step.m, step.v, r.rows, nn, step.lr_rows, step.step,
                           T.BETA1, T.BETA2, T.EPS)
            if densify and (k + 1) % args.densify_every == 0 and k + 1 <= steps // 2 \
                    and nn < args.densify_max * n:
                if dcfg.grad_threshold == B.ug_densify_config_default().grad_threshold:
                    # the threshold, fixed at the first interval: the level of
                    # the top 2 % of the counted Gaussians' mean |dL/dmu|
                    st_h = stats.cpu().numpy()
                    cnt = st_h[1] > 0
                    mean = st_h[0][cnt] / st_h[1][cnt]
                    dcfg.grad_threshold = float(np.quantile(mean, 0.98)) if mean.size else 1.0
                cap = 2 * nn
                po = torch.empty((r.rows, cap), device=dev)
                mo, vo = torch.empty_like(po), torch.empty_like(po)
                n_out = torch.zeros(1, dtype=torch.int64, device=dev)
                z = torch.randn((6, nn), device=dev, generator=zgen)
                scr = torch.empty(B.ug_densify_scratch_bytes(nn), dtype=torch.uint8, device=dev)
                B.ug_densify(cfg, dcfg, params, step.m, step.v, nn, stats, z, cap, po, mo, vo,
                             n_out, scr)
                new_n = int(n_out.item())
                assert 0 < new_n <= cap
                params = po[:, :new_n].contiguous()
                m_new, v_new = mo[:, :new_n].contiguous(), vo[:, :new_n].contiguous()
                stp = step.step.clone()
                del po, mo, vo, scr, z, step, r
                torch.cuda.empty_cache()
                dlog.append({"step": k + 1, "before": nn, "after": new_n})
                nn = new_n
                r = R.Renderer(nn, synth.select_planes(tr, list(range(P))), cfg)
                step = T.TrainStep(r, params, targets, decay_steps=steps, loss=args.recon_loss,
                                   plane_shape=(size, size))
                step.m.copy_(m_new)
                step.v.copy_(v_new)
                step.step.copy_(stp)
                stats = torch.zeros((2, nn), device=dev)
            e1.record()
            e1.synchronize()
            train_ms += e0.elapsed_time(e1)
            stt = r.status()
            assert stt["status"] == B.UG_OK, stt
            if (k + 1) % every == 0 or k + 1 == steps:
                history.append(record(k + 1, train_ms / 1e3, float(step.loss[0])))
                hh = history[-1]
                print(f"[recon{' densify' if densify else ''}] step {k + 1} train "
                      f"{hh['train_s']:.2f} s ssim {hh['ssim']:.4f} (train poses "
                      f"{hh['train_ssim']:.4f}) psnr {hh['psnr']:.2f} gaussians {nn}",
                      file=sys.stderr)
        sets.clear()
        return history, params, train_ms, nn, dlog, dcfg.grad_threshold

    def time_to(history, th, key="ssim"):
        for h in history:
            if h[key] >= th:
                return h["train_s"]
        return None

    runs = {}
    modes = {"off": [False], "on": [True], "both": [False, True]}[args.recon_densify]
    for densify in modes:
        history, params_run, train_ms, n_final, dlog, thr = train(densify)
        runs["densify" if densify else "plain"] = {
            "train_s": train_ms / 1e3, "ms_per_step": train_ms / steps,
            "gaussians_final": n_final,
            "time_to_ssim": {str(th): time_to(history, th) for th in (0.8, 0.9, 0.95, 0.99)},
            "time_to_train_ssim": {str(th): time_to(history, th, "train_ssim")
                                   for th in (0.9, 0.95, 0.99)},
            "final": history[-1], "history": history,
            **({"densify_steps": dlog, "grad_threshold": thr,
                "densify_every": args.densify_every, "densify_max": args.densify_max}
               if densify else {})}
        if not densify or "plain" not in runs:
            params = params_run  # the novel-slice rendering below uses the plain run's model
        else:
            del params_run
        torch.cuda.empty_cache()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = int(params.shape[1])

    # novel-slice rendering: 512 random poses of 512x512, 32 per launch (fewer
    # when a launch would hold more than 2^31 tile instances)
    novel = synth.planes_random(np.random.default_rng(7), [(512, 512)] * 512)
    per = 32
    while True:
        try:
            nr = R.Renderer(n, synth.select_planes(novel, list(range(per))), cfg)
            chunks = [torch.from_numpy(synth.planes_to_struct(synth.select_planes(
                novel, list(range(c0, c0 + per)))).view(np.uint8).copy()).to(dev)
                for c0 in range(0, 512, per)]
            for c in chunks:  # sizing pass
                nr.d_planes.copy_(c)
                nr.forward(params)
            break
        except B.UgError as err:
            if err.status != B.UG_ERR_CAPACITY or per == 1:
                raise
            per //= 2
            nr = None
            torch.cuda.empty_cache()
    img, al = nr.new_image(), nr.new_image()
    torch.cuda.synchronize()
    e0.record()
    for c in chunks:
        nr.d_planes.copy_(c, non_blocking=True)
        B.ug_preprocess(nr.plan, R.gaussians_struct(params, B.UG_COV_TRI), nr.d_planes, nr.ws)
        B.ug_bin_sort(nr.plan, nr.ws)
        B.ug_render(nr.plan, nr.ws, img, al)
    e1.record()
    e1.synchronize()
    novel_s = e0.elapsed_time(e1) / 1e3
    assert nr.status()["status"] == B.UG_OK
    line = {
        "metric": "reconstruction: training time to held-out SSIM, and novel-slice images/s",
        "value": 512 / novel_s, "unit": "images/s (512x512 novel slices)",
        "n_gpus": 1, "dtype": "f32", "data": "synthetic",
        "novel_planes_per_launch": per,
        "config": {"workload": f"recon: {n} Gaussians (paper init) fitted to a hidden "
                               f"{args.recon_hidden}-Gaussian volume (seed 3), {steps} steps of 32 "
                               f"poses from a pool of {pool} at {size}x{size}, "
                               + (f"evaluated on {held_n} linearly spaced axial, coronal and "
                                  f"sagittal slices each (training: {pool} axial slices)"
                                  if slices else f"{len(te['size'])} held-out poses (seed 4)"),
                   "poses": args.recon_poses, "loss": args.recon_loss},
        "runs": runs,
        "novel_slice_model": "plain" if "plain" in runs else "densify",
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- ablation
def run_scatter_ablation(args):
    """Forward of the bench workload two ways from the same records: the tile
    gather (bin + sort + ug_render) against the paper's phase-2 atomic scatter
    (ug_render_scatter, no binning); times, speed-up and image difference."""
    import torch
    from paper_2505_05643_gb300 import binding as B
    from paper_2505_05643_gb300 import render as R
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    g, pl, _ = _workload(args.n)
    cfg = R.make_config(cov_param=B.UG_COV_TRI, cutoff=B.UG_CUTOFF_BOX, tile=args.tile,
                        variant=args.variant, variant_bwd=args.variant_bwd)
    n = len(g["logit"])
    r = R.Renderer(n, pl, cfg)
    params = torch.from_numpy(R.pack_params(g, B.UG_COV_TRI)).to(dev)
    st = r.preprocess(params, check=True)
    s = torch.cuda.current_stream()
    im_g, al_g, im_s, al_s = (r.new_image() for _ in range(4))

    def gather():
        B.ug_bin_sort(r.plan, r.ws, s)
        B.ug_render(r.plan, r.ws, im_g, al_g, s)

    def scatter():
        B.ug_render_scatter(r.plan, r.ws, im_s, al_s, s)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(args.steps):
            fn()
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) / args.steps

    ms_g, ms_s = timed(gather), timed(scatter)
    st2 = r.status()
    assert st2["status"] == B.UG_OK, st2
    d = (im_g - im_s).abs()
    line = {
        "metric": "forward of the bench workload: tile gather vs the paper's atomic scatter",
        "value": float(st["box_pixels"]) / (ms_g * 1e-3), "unit": "pairs/s",
        "ms_gather_bin_sort_render": ms_g, "ms_scatter": ms_s, "speedup": ms_s / ms_g,
        "box_pairs": int(st["box_pixels"]), "records": int(st["records"]),
        "max_abs_image_diff": float(d.max()),
        "max_rel_image_diff": float((d / im_g.abs().clamp_min(1e-6)).max()),
        "steps": args.steps, "warmup": args.warmup,
        "config": {"workload": WORKLOAD, "gaussians": n, "tile": int(cfg.tile),
                   "variant": int(cfg.variant)},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- densify (row f2)
def run_densify(args):
    """Resampling and the densify / prune step on the bench workload's 1M
    Gaussians (triangular front-end): synthetic densify statistics (a third of
    the Gaussians above the gradient threshold, a tenth below the opacity
    floor), standard normal draws from a seeded generator. Times ug_densify (the
    whole step: decision, output scan, emit) and ug_sample (1M draws) with CUDA
    events; both are memory-bound, so each reports its algorithmic bytes per
    call against the measured HBM copy bandwidth."""
    import torch

    from paper_2505_05643_gb300 import binding as B
    from paper_2505_05643_gb300 import render as R
    from paper_2505_05643_gb300 import synth

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    g, _ = synth.workload_aniso_1m()
    if args.n:
        g = {k: v[..., :args.n] for k, v in g.items()}
    g = synth.scale_rot_to_tri(g, 1e-4)
    cov = B.UG_COV_TRI
    P = torch.from_numpy(R.pack_params(g, cov)).cuda()
    rows, n = P.shape
    rng = np.random.default_rng(5)
    faded = torch.from_numpy(rng.random(n) < 0.1).cuda()
    P[9][faded] = float(np.log(0.002 / 0.998))
    cnt = torch.from_numpy(rng.integers(0, 5, n).astype(np.float32)).cuda()
    busy = torch.from_numpy(rng.random(n) < 0.35).cuda()
    stats = torch.stack([torch.where(busy, 1e-3, 1e-5) * cnt, cnt]).contiguous()
    m = torch.from_numpy(rng.normal(size=(rows, n)).astype(np.float32)).cuda()
    v = torch.from_numpy(rng.random((rows, n)).astype(np.float32)).cuda()
    z = torch.from_numpy(rng.normal(size=(6, n)).astype(np.float32)).cuda()
    cap = 2 * n
    po = torch.empty((rows, cap), device="cuda")
    mo, vo = torch.empty_like(po), torch.empty_like(po)
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    scratch = torch.empty(B.ug_densify_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    cfg = R.make_config(cov_param=cov)
    dc = B.ug_densify_config_default()
    idx = torch.arange(n, dtype=torch.int32, device="cuda")
    y = torch.empty((3, n), device="cuda")

    def timed(fn, reps):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    reps = max(1, args.steps)
    ms_d = timed(lambda: B.ug_densify(cfg, dc, P, m, v, n, stats, z, cap, po, mo, vo, n_out,
                                      scratch), reps)
    ms_s = timed(lambda: B.ug_sample(cfg, P, n, idx, n, z, y), reps)
    n_o = int(n_out.item())
    # algorithmic bytes (a lower bound: the draws read for the split Gaussians
    # are not counted): densify reads params, moments and stats and writes the
    # outputs (params and moments); ug_sample reads an index, the mean and
    # factor rows (9 floats) and three draws, and writes three floats per draw
    bytes_d = n * (3 * rows * 4 + 8) + n_o * 3 * rows * 4
    bytes_s = n * (4 + 9 * 4 + 12 + 12)
    line = {
        "metric": "densify / prune step and resampling, 1M Gaussians (TRI)",
        "value": n / (ms_d * 1e-3), "unit": "Gaussians/s (densify step)", "n_gpus": 1,
        "steps": reps, "warmup": max(3, args.warmup), "higher_is_better": True, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "aniso_1m parameters, TRI; a third busy, a tenth faded",
                   "n": n, "n_out": n_o},
        "densify_ms": ms_d, "sample_ms": ms_s, "samples_per_s": n / (ms_s * 1e-3),
        "roofline": {"bound": "hbm", "unit": "GB/s", "peak": hbm,
                     "densify": {"achieved": bytes_d / (ms_d * 1e-3) / 1e9,
                                 "frac": bytes_d / (ms_d * 1e-3) / 1e9 / hbm,
                                 "bytes_per_call": bytes_d},
                     "sample": {"achieved": bytes_s / (ms_s * 1e-3) / 1e9,
                                "frac": bytes_s / (ms_s * 1e-3) / 1e9 / hbm,
                                "bytes_per_call": bytes_s}},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- L1 + D-SSIM loss (row f4)
def run_loss(args):
    """The fused L1 + D-SSIM loss and its gradient on a training step's images
    (32 planes of 256 x 256, synthetic image and target), timed with CUDA events
    against the MSE kernel on the same images; both are memory-bound, so the
    line reports the algorithmic bytes per call against the measured HBM copy
    bandwidth (D-SSIM: images read, five window maps and three gradient maps
    written and read, gradient written)."""
    import torch

    from paper_2505_05643_gb300 import binding as B

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    P, W, H = 32, 256, 256
    gen = torch.Generator(device="cuda").manual_seed(3)
    x = torch.rand(P * H * W, device="cuda", generator=gen)
    t = (x + 0.1 * torch.randn(P * H * W, device="cuda", generator=gen)).clamp(0, 1)
    scratch = torch.empty(B.ug_l1_dssim_scratch_floats(P, W, H), device="cuda")
    grad = torch.empty_like(x)
    loss = torch.empty(1, device="cuda")
    mse_loss = torch.empty(B.UG_MSE_LOSS_FLOATS, device="cuda")

    def timed(fn, reps):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    reps = max(1, args.steps)
    ms_d = timed(lambda: B.ug_l1_dssim_loss_grad(x, t, P, W, H, 0.2, scratch, grad, loss), reps)
    ms_m = timed(lambda: B.ug_mse_loss_grad(x, t, x.numel(), grad, mse_loss), reps)
    n = P * W * H
    Wv, Hv = W - 10, H - 10
    bytes_d = 4 * (2 * n + 2 * 5 * P * H * Wv + 2 * 3 * P * Hv * Wv + 2 * 3 * P * Hv * W + 2 * n + n)
    bytes_m = 12 * n
    line = {
        "metric": "L1 + D-SSIM loss and gradient, 32 planes of 256x256",
        "value": n / (ms_d * 1e-3), "unit": "pixels/s", "n_gpus": 1, "steps": reps,
        "warmup": max(3, args.warmup), "higher_is_better": True, "dtype": "f32",
        "data": "synthetic", "config": {"workload": "32 planes of 256x256, lambda 0.2"},
        "l1_dssim_ms": ms_d, "mse_ms": ms_m, "loss": float(loss.item()),
        "roofline": {"bound": "hbm", "unit": "GB/s", "peak": hbm,
                     "l1_dssim": {"achieved": bytes_d / (ms_d * 1e-3) / 1e9,
                                  "frac": bytes_d / (ms_d * 1e-3) / 1e9 / hbm,
                                  "bytes_per_call": bytes_d},
                     "mse": {"achieved": bytes_m / (ms_m * 1e-3) / 1e9,
                             "frac": bytes_m / (ms_m * 1e-3) / 1e9 / hbm,
                             "bytes_per_call": bytes_m}},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--variant", type=int, default=0, help="forward rasterizer variant")
    ap.add_argument("--variant-bwd", type=int, default=0, help="backward rasterizer variant")
    ap.add_argument("--cpu-planes", type=int, default=64, help="planes in the CPU oracle sample")
    ap.add_argument("--n", type=int, default=None, help="use the first n Gaussians (testing)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-train-compare", action="store_true",
                    help="skip the batched vs one-plane-per-launch comparison (train_200k)")
    ap.add_argument("--compare-steps", type=int, default=200,
                    help="steps of the batched vs one-plane-per-launch comparison")
    ap.add_argument("--workload", default="aniso_1m",
                    choices=["aniso_1m", "train_200k", "recon", "densify", "loss"],
                    help="train_200k: batched graph step against one plane per launch; "
                         "recon: reconstruction run with SSIM on held-out poses; "
                         "densify: the densify / prune step and resampling; "
                         "loss: the L1 + D-SSIM loss and gradient")
    ap.add_argument("--recon-n", type=int, default=3_000_000)
    ap.add_argument("--recon-hidden", type=int, default=1_000_000)
    ap.add_argument("--recon-steps", type=int, default=2000)
    ap.add_argument("--recon-eval", type=int, default=100)
    ap.add_argument("--recon-loss", default="mse", choices=["mse", "l1_dssim"],
                    help="training loss of the reconstruction run")
    ap.add_argument("--recon-poses", default="random", choices=["random", "slices"],
                    help="random: random training and held-out poses; slices: linearly spaced "
                         "axial training slices, axial/coronal/sagittal evaluation slices")
    ap.add_argument("--recon-densify", default="both", choices=["off", "on", "both"],
                    help="reconstruction run without and/or with the densify / prune step")
    ap.add_argument("--densify-every", type=int, default=100,
                    help="steps between densify / prune steps (up to half the run)")
    ap.add_argument("--densify-max", type=float, default=2.0,
                    help="no densify step once the count exceeds this times the initial one")
    ap.add_argument("--recon-size", type=int, default=None,
                    help="plane edge in pixels (default 256 random, 160 slices)")
    ap.add_argument("--ablation", default=None, choices=["scatter"],
                    help="scatter: the forward as the paper's atomic scatter vs the tile gather")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use --tile/--variant/--variant-bwd instead of the autotuner's choice")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "train_200k":
        return run_train_compare(args)
    if args.workload == "recon":
        return run_recon(args)
    if args.workload == "densify":
        return run_densify(args)
    if args.workload == "loss":
        return run_loss(args)
    if args.ablation == "scatter":
        return run_scatter_ablation(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
