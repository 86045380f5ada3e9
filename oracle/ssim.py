"""SSIM and PSNR of rendered slices in FP64 NumPy (test infrastructure; only
tests, the smoke check and the bench's CPU legs use it).

The paper evaluates reconstructions with SSIM (Wang et al., 2004) and PSNR
(Sec. 5). Its window parameters are not printed; this follows the original
definition: an 11 x 11 Gaussian window with sigma 1.5 (normalised to sum 1),
C1 = (0.01 L)^2 and C2 = (0.03 L)^2 with data range L = 1, evaluated at every
position where the window lies inside the image ("valid" positions), and the
mean over those positions:

    mu_x = sum w x,  sigma_x^2 = sum w x^2 - mu_x^2,  sigma_xy = sum w x y - mu_x mu_y
    SSIM = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2))

PSNR = 10 log10(L^2 / MSE) over the whole image.
"""
from __future__ import annotations

import numpy as np

WIN = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def window() -> np.ndarray:
    """The normalised 11 x 11 Gaussian window (outer product of the 1-D one)."""
    r = np.arange(WIN) - (WIN - 1) / 2.0
    g = np.exp(-(r * r) / (2.0 * SIGMA * SIGMA))
    g /= g.sum()
    return np.outer(g, g)


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """SSIM at every valid window position of two H x W images (FP64)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = window()
    from numpy.lib.stride_tricks import sliding_window_view
    px = sliding_window_view(x, (WIN, WIN))  # (H-10, W-10, 11, 11)
    py = sliding_window_view(y, (WIN, WIN))
    mx = np.einsum("ijab,ab->ij", px, w)
    my = np.einsum("ijab,ab->ij", py, w)
    sxx = np.einsum("ijab,ab->ij", px * px, w) - mx * mx
    syy = np.einsum("ijab,ab->ij", py * py, w) - my * my
    sxy = np.einsum("ijab,ab->ij", px * py, w) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def ssim(x: np.ndarray, y: np.ndarray) -> float:
    return float(ssim_map(x, y).mean())


def psnr(x: np.ndarray, y: np.ndarray) -> float:
    """PSNR in dB; +inf for identical images."""
    d = np.asarray(x, np.float64) - np.asarray(y, np.float64)
    mse = float(np.mean(d * d))
    return float("inf") if mse == 0.0 else float(10.0 * np.log10(1.0 / mse))


def ssim_planes(image: np.ndarray, target: np.ndarray, P: int, W: int, H: int):
    """Per-plane SSIM and PSNR of P planes of W x H pixels stored one after the
    other (row-major)."""
    a = np.asarray(image, np.float64).reshape(P, H, W)
    b = np.asarray(target, np.float64).reshape(P, H, W)
    return (np.array([ssim(a[p], b[p]) for p in range(P)]),
            np.array([psnr(a[p], b[p]) for p in range(P)]))


def ssim_grad(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """d(mean SSIM)/dx of one H x W image (FP64), from the chain rule over every
    valid window position p: with A1 = 2 mu_x mu_y + C1, A2 = 2 s_xy + C2,
    B1 = mu_x^2 + mu_y^2 + C1, B2 = s_x^2 + s_y^2 + C2 and S = A1 A2 / (B1 B2),
      dS/dmu_x = 2 A2 (mu_y B1 - A1 mu_x) / (B1^2 B2),  dS/ds_x^2 = -S / B2,
      dS/ds_xy = 2 A1 / (B1 B2);
    pixel q of the window at p enters mu_x with weight w(q - p), s_x^2 with
    w(q - p)(2 x_q - 2 mu_x) and s_xy with w(q - p)(y_q - mu_y), so
      dS(p)/dx_q = w(q - p) (a(p) + b(p) x_q + c(p) y_q),
      a = dS/dmu_x - 2 mu_x dS/ds_x^2 - mu_y dS/ds_xy,  b = 2 dS/ds_x^2,  c = dS/ds_xy,
    summed over the positions whose window holds q and divided by their count."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = window()
    from numpy.lib.stride_tricks import sliding_window_view
    px = sliding_window_view(x, (WIN, WIN))
    py = sliding_window_view(y, (WIN, WIN))
    mx = np.einsum("ijab,ab->ij", px, w)
    my = np.einsum("ijab,ab->ij", py, w)
    vx = np.einsum("ijab,ab->ij", px * px, w) - mx * mx
    vy = np.einsum("ijab,ab->ij", py * py, w) - my * my
    cxy = np.einsum("ijab,ab->ij", px * py, w) - mx * my
    A1, A2 = 2 * mx * my + C1, 2 * cxy + C2
    B1, B2 = mx * mx + my * my + C1, vx + vy + C2
    S = A1 * A2 / (B1 * B2)
    d_mx = 2 * A2 * (my * B1 - A1 * mx) / (B1 * B1 * B2)
    d_vx = -S / B2
    d_cxy = 2 * A1 / (B1 * B2)
    a = d_mx - 2 * mx * d_vx - my * d_cxy
    b = 2 * d_vx
    c = d_cxy
    Hv, Wv = S.shape
    ga, gb, gc = (np.zeros_like(x) for _ in range(3))
    for i in range(WIN):
        for j in range(WIN):
            ga[i:i + Hv, j:j + Wv] += w[i, j] * a
            gb[i:i + Hv, j:j + Wv] += w[i, j] * b
            gc[i:i + Hv, j:j + Wv] += w[i, j] * c
    return (ga + x * gb + y * gc) / S.size


def l1_dssim_loss_grad(image: np.ndarray, target: np.ndarray, P: int, W: int, H: int,
                       lam: float = 0.2):
    """The training loss Kerbl et al. use, which the paper takes over (Sec. 4.5):
    L = (1 - lam) mean|x - y| + lam (1 - SSIM), SSIM the mean over the P planes
    of each plane's mean SSIM; returns (L, dL/dx) in FP64. The L1 term's
    derivative at x = y is taken as 0."""
    x = np.asarray(image, np.float64).reshape(P, H, W)
    t = np.asarray(target, np.float64).reshape(P, H, W)
    n = x.size
    s = np.array([ssim(x[p], t[p]) for p in range(P)])
    L = (1 - lam) * np.abs(x - t).mean() + lam * (1 - s.mean())
    g = (1 - lam) * np.sign(x - t) / n
    for p in range(P):
        g[p] -= lam / P * ssim_grad(x[p], t[p])
    return float(L), g.reshape(-1)
