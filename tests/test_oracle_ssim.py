"""Pins of the SSIM/PSNR oracle: the definition's own special cases and a
second formulation (separable correlation with SciPy) of the same sums."""
import numpy as np
import pytest

from oracle import ssim as S


def test_window_is_normalised_gaussian():
    w = S.window()
    assert w.shape == (11, 11) and abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w, w.T) and w[5, 5] == w.max()
    # ratio of neighbouring taps of the 1-D Gaussian: exp(-(2k+1)/(2 sigma^2))
    g = w[5] / w[5].sum()
    assert np.isclose(g[6] / g[5], np.exp(-1.0 / (2 * 1.5 ** 2)), rtol=1e-13)


def test_identical_images_give_one():
    x = np.random.default_rng(0).uniform(0, 1, (40, 37))
    assert abs(S.ssim(x, x) - 1.0) < 1e-13


def test_constant_images_closed_form():
    """Two constant images a, b: variances and covariance vanish, so SSIM =
    (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 0.3, 0.7
    got = S.ssim(np.full((20, 30), a), np.full((20, 30), b))
    assert abs(got - (2 * a * b + S.C1) / (a * a + b * b + S.C1)) < 1e-13


def test_negated_structure():
    """y = 2m - x (mirror about the window mean m of a zero-mean pattern):
    equal means and variances, covariance -sigma^2, so the structure term is
    (C2 - 2 s^2) / (2 s^2 + C2)."""
    rng = np.random.default_rng(1)
    x = 0.5 + 0.1 * rng.standard_normal((30, 30))
    y = 1.0 - x
    m = S.ssim_map(x, y)
    # direct per-window check at one position against the formula
    w = S.window()
    px, py = x[3:14, 4:15], y[3:14, 4:15]
    mx, my = (w * px).sum(), (w * py).sum()
    sx = (w * px * px).sum() - mx * mx
    sxy = (w * px * py).sum() - mx * my
    assert abs(sxy + sx) < 1e-12  # covariance is minus the variance
    exp = ((2 * mx * my + S.C1) * (2 * sxy + S.C2)) / ((mx * mx + my * my + S.C1) * (2 * sx + S.C2))
    assert abs(m[3, 4] - exp) < 1e-12


def test_separable_formulation_agrees():
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(2)
    x, y = rng.uniform(0, 1, (33, 41)), rng.uniform(0, 1, (33, 41))
    r = np.arange(11) - 5.0
    g = np.exp(-r * r / (2 * 1.5 ** 2))
    g /= g.sum()

    def filt(a):  # separable 'valid' correlation: rows then columns
        t = scipy_signal.correlate(a, g[None, :], mode="valid")
        return scipy_signal.correlate(t, g[:, None], mode="valid")

    mx, my = filt(x), filt(y)
    sxx, syy, sxy = filt(x * x) - mx * mx, filt(y * y) - my * my, filt(x * y) - mx * my
    ref = ((2 * mx * my + S.C1) * (2 * sxy + S.C2)) / ((mx * mx + my * my + S.C1) * (sxx + syy + S.C2))
    assert np.allclose(S.ssim_map(x, y), ref, rtol=1e-12, atol=1e-13)


def test_psnr_closed_form():
    x = np.zeros((10, 10))
    y = np.full((10, 10), 0.1)
    assert abs(S.psnr(x, y) - 20.0) < 1e-12  # MSE 0.01 -> 20 dB


def test_ssim_grad_central_differences():
    """The analytic gradient of the mean SSIM against central differences of
    ssim() itself on a 16 x 14 image (interior, edge and corner pixels)."""
    from oracle import ssim as S
    rng = np.random.default_rng(50)
    x = rng.uniform(0, 1, (14, 16))
    y = np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1)
    g = S.ssim_grad(x, y)
    h = 1e-6
    for (i, j) in [(0, 0), (0, 7), (5, 5), (13, 15), (7, 12), (10, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[i, j] += h
        xm[i, j] -= h
        fd = (S.ssim(xp, y) - S.ssim(xm, y)) / (2 * h)
        assert abs(fd - g[i, j]) <= 1e-7 + 1e-5 * abs(fd), (i, j, fd, g[i, j])


def test_ssim_grad_vanishes_at_equality():
    """SSIM is at its maximum 1 where the images are equal: zero gradient."""
    from oracle import ssim as S
    rng = np.random.default_rng(51)
    x = rng.uniform(0, 1, (20, 23))
    assert np.abs(S.ssim_grad(x, x)).max() < 1e-12


def test_l1_dssim_loss_central_differences():
    from oracle import ssim as S
    rng = np.random.default_rng(52)
    P, W, H = 2, 13, 12
    x = rng.uniform(0, 1, P * H * W)
    t = rng.uniform(0, 1, P * H * W)
    L, g = S.l1_dssim_loss_grad(x, t, P, W, H, 0.2)
    # L1 part alone at lam = 0: sign / n
    L0, g0 = S.l1_dssim_loss_grad(x, t, P, W, H, 0.0)
    np.testing.assert_allclose(g0, np.sign(x - t) / x.size)
    assert abs(L0 - np.abs(x - t).mean()) < 1e-15
    h = 1e-6
    for k in [0, 5, 100, 200, 311]:
        xp, xm = x.copy(), x.copy()
        xp[k] += h
        xm[k] -= h
        fd = (S.l1_dssim_loss_grad(xp, t, P, W, H, 0.2)[0]
              - S.l1_dssim_loss_grad(xm, t, P, W, H, 0.2)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-8 + 1e-5 * abs(fd), (k, fd, g[k])
