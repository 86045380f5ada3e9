"""Pin of the FP64 Adam oracle against the library optimiser torch.optim.Adam."""
import numpy as np
import torch

from oracle import adam


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(0)
    p0 = rng.standard_normal((5, 64))
    lrs = np.array([0.05, 0.05, 1.6e-4, 0.01, 0.05])
    p_t = [torch.tensor(p0[r].copy(), requires_grad=True) for r in range(5)]
    opt = torch.optim.Adam([{"params": [p_t[r]], "lr": float(lrs[r])} for r in range(5)],
                           betas=(0.9, 0.999), eps=1e-15)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for t in range(1, 8):
        g = rng.standard_normal((5, 64)) * (10.0 ** rng.uniform(-6, 1, (5, 1)))
        g[0, :5] = 0.0  # zero gradients stay finite with a tiny eps
        for r in range(5):
            p_t[r].grad = torch.tensor(g[r])
        opt.step()
        p, m, v = adam.adam_step(p, g, m, v, lrs[:, None], t, 0.9, 0.999, 1e-15)
        ref = np.stack([x.detach().numpy() for x in p_t])
        np.testing.assert_allclose(p, ref, rtol=1e-14, atol=1e-15)


def test_decayed_lr_endpoints_and_geometric_midpoint():
    assert adam.decayed_lr(1.6e-4, 1.6e-6, 1000, 0) == 1.6e-4
    assert abs(adam.decayed_lr(1.6e-4, 1.6e-6, 1000, 1000) - 1.6e-6) < 1e-18
    assert abs(adam.decayed_lr(1.6e-4, 1.6e-6, 1000, 500) - 1.6e-5) < 1e-17
    assert abs(adam.decayed_lr(1.6e-4, 1.6e-6, 1000, 5000) - 1.6e-6) < 1e-18
    assert adam.decayed_lr(0.05, 0.05, 1000, 300) == 0.05
