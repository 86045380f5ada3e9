"""Adam parity: the fused CUDA Adam step against the FP64 oracle (which is
pinned to torch.optim.Adam), with per-row learning rates and the exponential
decay schedule, including the device-side step counter."""
import numpy as np
import pytest
import torch

from oracle import adam as OA
from paper_2505_05643_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _rows_tensor(specs):
    arr = np.zeros(len(specs), dtype=[("lr_init", "<f4"), ("lr_final", "<f4"),
                                      ("decay_steps", "<i4"), ("reserved", "<i4")])
    for k, (a, b, d) in enumerate(specs):
        arr[k] = (a, b, d, 0)
    return torch.from_numpy(arr.view(np.uint8).copy()).cuda(), arr


@pytest.mark.parametrize("n", [1, 7, 4096, 100_003])
def test_adam_matches_oracle(n):
    rng = np.random.default_rng(n)
    rows = 5
    specs = [(1.6e-4, 1.6e-6, 30), (1.6e-4, 1.6e-6, 30), (0.05, 0.05, 0), (0.05, 0.05, 0),
             (0.01, 0.001, 5)]
    d_rows, arr = _rows_tensor(specs)
    p0 = rng.standard_normal((rows, n)).astype(np.float32)
    p = torch.from_numpy(p0.copy()).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    b1, b2, eps = np.float32(0.9), np.float32(0.999), np.float32(1e-15)
    pr, mr, vr = p0.astype(np.float64), np.zeros((rows, n)), np.zeros((rows, n))
    for t in range(1, 9):
        g = (rng.standard_normal((rows, n)) * 10.0 ** rng.uniform(-5, 1, (rows, 1))).astype(np.float32)
        g[:, ::3] = 0.0
        B.ug_adam_step(p, torch.from_numpy(g).cuda(), m, v, rows, n, d_rows, step,
                       float(b1), float(b2), float(eps))
        lrs = np.array([OA.decayed_lr(a, b, d, t) for a, b, d in specs])[:, None]
        pr, mr, vr = OA.adam_step(pr, g.astype(np.float64), mr, vr, lrs, t, float(b1), float(b2),
                                  float(eps))
        got = p.cpu().numpy().astype(np.float64)
        # FP32 state: one rounding of p per step (6e-8 |p|) and an update of
        # size <= lr computed to a few FP32 ulps
        tol = 1.2e-7 * t * np.abs(pr) + 1e-5 * lrs * t
        assert np.all(np.abs(got - pr) <= tol), (t, np.abs(got - pr).max())
    assert step.item() == 8


def test_adam_graph_capture_advances_step():
    n, rows = 1024, 2
    d_rows, _ = _rows_tensor([(0.05, 0.05, 0), (1e-3, 1e-5, 10)])
    p = torch.zeros(rows, n, device="cuda")
    g = torch.ones(rows, n, device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        B.ug_adam_step(p, g, m, v, rows, n, d_rows, step, 0.9, 0.999, 1e-15, stream=s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        B.ug_adam_step(p, g, m, v, rows, n, d_rows, step, 0.9, 0.999, 1e-15, stream=s)
    for _ in range(4):
        graph.replay()
    torch.cuda.synchronize()
    assert step.item() == 5  # 1 eager call + 4 replays (capture does not execute)
