"""The SSIM/PSNR evaluator kernel against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import ssim as S
from paper_2505_05643_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _gpu(image, target, P, W, H):
    scratch = torch.empty(B.ug_ssim_scratch_floats(P, W, H), dtype=torch.float32, device="cuda")
    ss = torch.empty(P, dtype=torch.float32, device="cuda")
    ps = torch.empty(P, dtype=torch.float32, device="cuda")
    B.ug_ssim(torch.from_numpy(image.astype(np.float32)).cuda(),
              torch.from_numpy(target.astype(np.float32)).cuda(), P, W, H, scratch, ss, ps)
    torch.cuda.synchronize()
    return ss.cpu().numpy().astype(np.float64), ps.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("W,H", [(64, 50), (11, 11), (300, 17)])
def test_ssim_psnr_parity(W, H):
    rng = np.random.default_rng(W * 1000 + H)
    P = 3
    base = rng.uniform(0, 1, (P, H, W))
    noisy = np.clip(base + 0.05 * rng.standard_normal((P, H, W)), 0, 1)
    img = base.astype(np.float32).astype(np.float64)
    tgt = noisy.astype(np.float32).astype(np.float64)
    gs, gp = _gpu(img.ravel(), tgt.ravel(), P, W, H)
    rs, rp = S.ssim_planes(img.ravel(), tgt.ravel(), P, W, H)
    assert np.max(np.abs(gs - rs)) < 2e-5, (gs, rs)
    assert np.max(np.abs(gp - rp)) < 1e-3, (gp, rp)


def test_ssim_of_identical_and_smooth_images():
    """Identical images give 1; smooth images (small variances, where the
    variance terms cancel the most) stay within the tolerance."""
    P, W, H = 2, 96, 96
    yy, xx = np.mgrid[0:H, 0:W] / 96.0
    a = 0.5 + 0.01 * np.sin(6 * xx) * np.cos(5 * yy)
    img = np.stack([a, a]).astype(np.float32).astype(np.float64)
    tgt = np.stack([a, a + 0.002 * np.cos(7 * yy)]).astype(np.float32).astype(np.float64)
    gs, _ = _gpu(img.ravel(), tgt.ravel(), P, W, H)
    rs, _ = S.ssim_planes(img.ravel(), tgt.ravel(), P, W, H)
    assert abs(gs[0] - 1.0) < 1e-6
    assert np.max(np.abs(gs - rs)) < 2e-5, (gs, rs)


def test_ssim_rejects_small_images():
    assert B.ug_ssim_scratch_floats(1, 10, 40) == 0
    scratch = torch.empty(16, dtype=torch.float32, device="cuda")
    x = torch.zeros(10 * 40, dtype=torch.float32, device="cuda")
    out = torch.empty(1, dtype=torch.float32, device="cuda")
    with pytest.raises(B.UgError):
        B.ug_ssim(x, x, 1, 10, 40, scratch, out)


@pytest.mark.parametrize("lam", [0.2, 1.0, 0.0])
def test_l1_dssim_loss_grad_parity(lam):
    """The fused L1 + D-SSIM loss and its gradient against the FP64 oracle on
    three ragged-sized planes (images with structure, targets perturbed)."""
    from oracle import ssim as S
    rng = np.random.default_rng(60)
    P, W, H = 3, 70, 45
    x = rng.uniform(0, 1, (P, H, W))
    x = (x + np.roll(x, 1, 2) + np.roll(x, 1, 1)) / 3  # some spatial correlation
    t = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1)
    x, t = x.astype(np.float32).reshape(-1), t.astype(np.float32).reshape(-1)
    L, g = S.l1_dssim_loss_grad(x, t, P, W, H, lam)
    xt, tt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    scratch = torch.empty(B.ug_l1_dssim_scratch_floats(P, W, H), device="cuda")
    grad = torch.empty_like(xt)
    loss = torch.empty(1, device="cuda")
    B.ug_l1_dssim_loss_grad(xt, tt, P, W, H, lam, scratch, grad, loss)
    torch.cuda.synchronize()
    assert abs(loss.item() - L) <= 1e-5 * abs(L) + 1e-7
    gg = grad.cpu().numpy().astype(np.float64)
    err = np.abs(gg - g)
    # FP32 window sums and SSIM terms: 1e-4 of the largest SSIM-part gradient
    ssim_part = np.abs(g - (1 - lam) * np.sign(x.astype(np.float64) - t) / x.size).max()
    assert np.all(err <= 1e-4 * ssim_part + 1e-9), (err.max(), ssim_part)
    grad2 = torch.empty_like(grad)
    B.ug_l1_dssim_loss_grad(xt, tt, P, W, H, lam, scratch, grad2, loss)
    assert torch.equal(grad, grad2)  # deterministic
