"""Host model (NumPy FP32, no GPU) of the backward rasterizer's nine-operation
pixel loop, which takes the per-row sum of g t1^2 from the weight's exponent
n = t1^2 + c (c = t2^2 - lw2 >= 0 for the row) as sum g n - c sum g, against
the ten-operation form that squares t1. The difference must stay within the
rounding the kernel's comment states (below 2^-19 c of the row's sum of |g|:
eight terms of size about c g, each rounded a few times), rows outside the box
(c a large finite number) must give exactly zero, never a NaN, and so must
columns whose t1 is huge (the far sentinel column)."""
import numpy as np

F = np.float32
BIG_N = F(2.0 ** 100)


def row_sums(t1, c, p):
    """Both forms for one row of 8 pixels: t1 (8,), row constant c, pixel
    factors p (8,) (g = w p). Returns (direct, fast, sum |g|), FP32 throughout."""
    n = (t1 * t1 + c).astype(F)  # the exponent the weight needs (one FMA in the kernel)
    w = np.exp2(-n.astype(np.float64)).astype(F)  # stand-in for ex2.approx
    g = (w * p).astype(F)
    direct = F(0)
    fast_gn = F(0)
    s1 = F(0)
    for k in range(8):
        gu = F(g[k] * t1[k])
        direct = F(direct + F(gu * t1[k]))
        fast_gn = F(fast_gn + F(g[k] * n[k]))
        s1 = F(s1 + g[k])
    fast = F(fast_gn - F(c * s1))
    return float(direct), float(fast), float(np.abs(g).sum())


def test_fast_form_within_its_rounding():
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(20000):
        c = F(rng.uniform(0, 150))
        t1 = (rng.standard_normal(8) * rng.uniform(0.1, 4)).astype(F)
        p = rng.uniform(-1, 1, 8).astype(F)
        d, f, sg = row_sums(t1, c, p)
        bound = 2.0 ** -22 * float(c) * sg + 2.0 ** -20 * (abs(d) + sg * 128)
        assert abs(d - f) <= bound + 1e-30, (d, f, bound)
        worst = max(worst, abs(d - f) / (float(c) * sg + 1e-30))
    assert worst < 2.0 ** -19


def test_zero_weights_give_zero_not_nan():
    # a row outside the box: c is the large finite exponent, every weight 0
    t1 = np.linspace(-3, 3, 8).astype(F)
    d, f, _ = row_sums(t1, BIG_N, np.ones(8, F))
    assert d == 0.0 and f == 0.0
    # far sentinel columns: t1 = r11 * 2^40 with r11 <= 2^20, so t1^2 stays finite
    r11 = F(2.0 ** 20)
    t1 = np.full(8, r11 * F(2.0 ** 40), F)
    d, f, _ = row_sums(t1, F(3.0), np.ones(8, F))
    assert np.isfinite(f) and f == 0.0 and d == 0.0
