"""Pins of the oracle's analytic FP64 gradient: central finite differences of
the oracle's own forward (FP64), and torch float64 autograd of an independent
probe-frame formulation on tiny inputs. No GPU needed."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle
from paper_2505_05643_gb300 import synth


def _scene(cov_param, n=200, seed=0, sizes=((32, 32), (24, 40))):
    rng = np.random.default_rng(seed)
    g = synth.gaussians_scale_rot(rng, n, 0.05, 0.2)
    g["mean"] *= 0.5
    g["intensity"] = rng.uniform(0, 1, n).astype(np.float32)
    g["logit"] = rng.uniform(-1, 2, n).astype(np.float32)
    if cov_param == 0:
        g = synth.scale_rot_to_tri(g, 1e-4)
    pl = synth.planes_random(rng, list(sizes), origin_range=0.2)
    target = rng.uniform(0, 1, pl["total_pixels"])
    g = {k: v.astype(np.float64) for k, v in g.items()}
    return g, pl, target


def _loss(g, pl, cfg, target):
    out = oracle.render(g, pl, cfg)
    return oracle.mse_loss_grad(out["image"], target)[0], out


def _param_view(g, cov_param):
    """(key, row) pairs in oracle parameter order."""
    keys = [("mean", r) for r in range(3)]
    keys += [("tri", r) for r in range(6)] if cov_param == 0 else \
        [("log_scale", r) for r in range(3)] + [("quat", r) for r in range(4)]
    keys += [("logit", None), ("intensity", None)]
    return keys


@pytest.mark.parametrize("cov_param,cutoff", [(1, 0), (0, 0), (1, 1)])
def test_grad_matches_central_differences(cov_param, cutoff):
    g, pl, target = _scene(cov_param, seed=1 + cov_param)
    cfg = oracle.Config(cov_param=cov_param, cutoff=cutoff)
    L0, out = _loss(g, pl, cfg, target)
    _, gimg = oracle.mse_loss_grad(out["image"], target)
    rng = np.random.default_rng(0)
    sub = rng.choice(len(g["logit"]), 12, replace=False)
    grads, gabs = oracle.render_grad(g, pl, cfg, out["image"], out["alpha"], gimg, subset=sub)
    h = 1e-6
    checked = 0
    covk = "tri" if cov_param == 0 else None
    for si, k in enumerate(sub):
        base_pix, _ = oracle.contrib(g["mean"][:, k], oracle.covp_rows(g, cov_param)[k],
                                     g["logit"][k], g["intensity"][k], pl, cfg)
        if len(base_pix) == 0:
            continue
        for pi, (key, row) in enumerate(_param_view(g, cov_param)):
            vals = []
            same = True
            for sgn in (+1, -1):
                g2 = {kk: vv.copy() for kk, vv in g.items()}
                if row is None:
                    g2[key][k] += sgn * h
                else:
                    g2[key][row, k] += sgn * h
                pix, _ = oracle.contrib(g2["mean"][:, k], oracle.covp_rows(g2, cov_param)[k],
                                        g2["logit"][k], g2["intensity"][k], pl, cfg)
                same &= np.array_equal(pix, base_pix)
                vals.append(_loss(g2, pl, cfg, target)[0])
            if not same:  # an inclusion decision moved: FD is not a derivative here
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            an = grads[si, pi]
            # truncation O(h^2) plus the rounding of two FP64 losses divided by 2h
            tol = 1e-5 * abs(an) + 1e-7 * gabs[si, pi] + 8 * 2.2e-16 * max(abs(v) for v in vals) / h
            assert abs(fd - an) <= tol, (k, key, row, fd, an)
            checked += 1
    assert checked > 60


def _torch_dense(gt, pl, cfg, mask_src):
    """Probe-frame formulation of Eq. mahalanobis-3d in torch float64:
    Sigma3D = W Sigma W^T with Sigma = (L L^T)^-1 or R diag(s^2) R^T,
    q = (x_|0 - mu3D)^T Sigma3D^-1 (x_|0 - mu3D); the inclusion mask comes
    from the oracle's geometry (a constant of the derivative)."""
    images = []
    n = gt["logit"].shape[0]
    for p in range(len(pl["size"])):
        u = torch.tensor(pl["u"][p], dtype=torch.float64)
        v = torch.tensor(pl["v"][p], dtype=torch.float64)
        o = torch.tensor(pl["origin"][p], dtype=torch.float64)
        Wr = torch.stack([u, v, torch.linalg.cross(u, v)])
        W, H = (int(s) for s in pl["size"][p])
        x1 = (torch.arange(W, dtype=torch.float64) + 0.5 - W / 2) * float(pl["pitch"][p, 0])
        x2 = (torch.arange(H, dtype=torch.float64) + 0.5 - H / 2) * float(pl["pitch"][p, 1])
        X2, X1 = torch.meshgrid(x2, x1, indexing="ij")
        X = torch.stack([X1.reshape(-1), X2.reshape(-1), torch.zeros(W * H, dtype=torch.float64)])
        sa = torch.zeros(W * H, dtype=torch.float64)
        sc = torch.zeros(W * H, dtype=torch.float64)
        for k in range(n):
            if cfg.cov_param == 0:
                t = gt["tri"][:, k]
                L = torch.zeros(3, 3, dtype=torch.float64)
                L = L.index_put((torch.tensor([0, 1, 2, 1, 2, 2]), torch.tensor([0, 0, 0, 1, 1, 2])),
                                torch.stack([t[0] ** 2 + cfg.beta, t[1], t[2], t[3] ** 2 + cfg.beta,
                                             t[4], t[5] ** 2 + cfg.beta]))
                S = torch.linalg.inv(L @ L.T)
            else:
                q = gt["quat"][:, k]
                q = q / torch.linalg.norm(q)
                w_, x_, y_, z_ = q
                R = torch.stack([
                    torch.stack([1 - 2 * (y_ * y_ + z_ * z_), 2 * (x_ * y_ - w_ * z_), 2 * (x_ * z_ + w_ * y_)]),
                    torch.stack([2 * (x_ * y_ + w_ * z_), 1 - 2 * (x_ * x_ + z_ * z_), 2 * (y_ * z_ - w_ * x_)]),
                    torch.stack([2 * (x_ * z_ - w_ * y_), 2 * (y_ * z_ + w_ * x_), 1 - 2 * (x_ * x_ + y_ * y_)])])
                S = R @ torch.diag(torch.exp(2 * gt["log_scale"][:, k])) @ R.T
            m = Wr @ (gt["mean"][:, k] - o)
            S3 = Wr @ S @ Wr.T
            d = X - m[:, None]
            qq = torch.einsum("in,ij,jn->n", d, torch.linalg.inv(S3), d)
            w = torch.sigmoid(gt["logit"][k]) * torch.exp(-0.5 * qq)
            msk = torch.tensor(mask_src[p][k])
            sa = sa + torch.where(msk, w, torch.zeros_like(w))
            sc = sc + torch.where(msk, w * gt["intensity"][k], torch.zeros_like(w))
        images.append((sc + cfg.alpha_bg * cfg.c_bg) / (sa + cfg.alpha_bg))
    return torch.cat(images)


@pytest.mark.parametrize("cov_param", [0, 1])
def test_grad_matches_torch_autograd(cov_param):
    g, pl, target = _scene(cov_param, n=6, seed=7, sizes=((8, 8), (8, 8)))
    for p in range(2):  # exactly orthonormal axes so both frames agree to rounding
        R = Rotation.random(random_state=70 + p).as_matrix()
        pl["u"] = pl["u"].astype(np.float64)
        pl["v"] = pl["v"].astype(np.float64)
        pl["u"][p], pl["v"][p] = R[:, 0], R[:, 1]
    pl["origin"] = pl["origin"].astype(np.float64) * 0.2
    cfg = oracle.Config(cov_param=cov_param)
    out = oracle.render(g, pl, cfg)
    assert out["pairs"] > 30
    # inclusion masks per (plane, gaussian, pixel) from the oracle's own per-Gaussian contributions
    masks = []
    for p in range(2):
        masks.append([])
    covp = oracle.covp_rows(g, cov_param)
    for k in range(6):
        pix, _ = oracle.contrib(g["mean"][:, k], covp[k], g["logit"][k], g["intensity"][k], pl, cfg)
        for p in range(2):
            W, H = pl["size"][p]
            m = np.zeros(W * H, bool)
            loc = pix[(pix >= pl["offset"][p]) & (pix < pl["offset"][p] + W * H)] - pl["offset"][p]
            m[loc] = True
            masks[p].append(m)
    gt = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in g.items()}
    img = _torch_dense(gt, pl, cfg, masks)
    np.testing.assert_allclose(img.detach().numpy(), out["image"], rtol=1e-12, atol=1e-14)
    tt = torch.tensor(target)
    loss = torch.mean((img - tt) ** 2)
    loss.backward()
    _, gimg = oracle.mse_loss_grad(out["image"], target)
    grads, _ = oracle.render_grad(g, pl, cfg, out["image"], out["alpha"], gimg)
    ref = []
    for key, row in _param_view(g, cov_param):
        gr = gt[key].grad.numpy()
        ref.append(gr[row] if row is not None else gr)
    ref = np.stack(ref, axis=1)
    np.testing.assert_allclose(grads, ref, rtol=1e-8, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("cov_param", [0, 1])
def test_pre_cancellation_sums(cov_param):
    """The absolute sums before the cancellation in c - C: the gradient and the
    plain absolute sums are unchanged by asking for them; they bound the plain
    sums from above (|c - C| <= |c| + |C|) and equal them for the intensity row
    (dL/dc has no c - C); with every intensity equal to the image value they
    stay positive while the plain sums of the rows through dL/dw vanish."""
    g, pl, target = _scene(cov_param, seed=5)
    cfg = oracle.Config(cov_param=cov_param)
    _, out = _loss(g, pl, cfg, target)
    _, gimg = oracle.mse_loss_grad(out["image"], target)
    sub = np.arange(0, len(g["logit"]), 7)
    grads, gabs = oracle.render_grad(g, pl, cfg, out["image"], out["alpha"], gimg, subset=sub)
    grads2, gabs2, gpre = oracle.render_grad(g, pl, cfg, out["image"], out["alpha"], gimg,
                                             subset=sub, with_pre=True)
    assert np.array_equal(grads, grads2) and np.array_equal(gabs, gabs2)
    assert np.all(gpre >= gabs * (1 - 1e-12))
    np.testing.assert_array_equal(gpre[:, -1], gabs[:, -1])
    # c = C everywhere: an image of constant value with every intensity equal to it
    flat = np.full_like(out["image"], 0.25)
    g2 = dict(g)
    g2["intensity"] = np.full_like(g["intensity"], 0.25)
    _, gabs3, gpre3 = oracle.render_grad(g2, pl, cfg, flat, out["alpha"], gimg, subset=sub,
                                         with_pre=True)
    reach = gabs3[:, -1] > 0  # Gaussians that reach a pixel
    assert reach.any()
    assert np.all(gabs3[reach, :-1] == 0)
    assert np.all(gpre3[reach, :3].sum(1) > 0)
