"""Adam in FP64 NumPy (test infrastructure).

The paper trains with Adam (Sec. 4.5: learning rate 0.05 for all Gaussian
parameters, means from 0.00016 with exponential decay). This is the textbook
update with bias correction, written out step by step:

    m <- b1 m + (1 - b1) g
    v <- b2 v + (1 - b2) g^2
    p <- p - (lr / (1 - b1^t)) * m / (sqrt(v) / sqrt(1 - b2^t) + eps)

and the exponential decay of a learning rate from lr_init to lr_final over
``decay_steps`` steps (held at lr_final afterwards):

    lr(t) = lr_init * (lr_final / lr_init) ** min(t / decay_steps, 1)
"""
from __future__ import annotations

import numpy as np


def decayed_lr(lr_init: float, lr_final: float, decay_steps: int, t: int) -> float:
    if decay_steps <= 0 or lr_init == lr_final:
        return float(lr_init)
    frac = min(float(t) / float(decay_steps), 1.0)
    return float(lr_init * (lr_final / lr_init) ** frac)


def adam_step(p, g, m, v, lr, t: int, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-15):
    """One Adam step at step number t (1-based) in FP64. ``lr`` is a scalar or
    an array broadcastable to p. Returns new (p, m, v)."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g
    bc1 = 1.0 - b1 ** t
    bc2 = 1.0 - b2 ** t
    denom = np.sqrt(v) / np.sqrt(bc2) + eps
    p = p - (np.asarray(lr, np.float64) / bc1) * m / denom
    return p, m, v
