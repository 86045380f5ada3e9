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
