"""Pins of the FP64 oracle against facts that do not come from the oracle:
printed values, closed forms of Gaussian conditioning, brute force, library
routines and invariances. No GPU needed."""
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.stats import chi2 as chi2_dist

import oracle
from paper_2505_05643_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def one_gauss(mean, log_s, quat_wxyz, logit=1.0, c=0.8):
    return dict(mean=np.asarray(mean, np.float64).reshape(3, 1),
                log_scale=np.asarray(log_s, np.float64).reshape(3, 1),
                quat=np.asarray(quat_wxyz, np.float64).reshape(4, 1),
                logit=np.array([logit]), intensity=np.array([c]))


def plane_dict(origin, u, v, W, H, pitch):
    return dict(origin=np.asarray(origin, np.float64).reshape(1, 3),
                u=np.asarray(u, np.float64).reshape(1, 3), v=np.asarray(v, np.float64).reshape(1, 3),
                pitch=np.array([[pitch, pitch]]), size=np.array([[W, H]]),
                offset=np.array([0]), total_pixels=W * H)


def scipy_cov(log_s, quat_wxyz):
    """Covariance R diag(s^2) R^T with R from scipy (library quaternion code)."""
    w, x, y, z = quat_wxyz
    R = Rotation.from_quat([x, y, z, w]).as_matrix()
    return R @ np.diag(np.exp(2 * np.asarray(log_s))) @ R.T


def pixel_centres(W, H, pitch):
    j = np.arange(W)
    i = np.arange(H)
    x1 = (j + 0.5 - W / 2) * pitch
    x2 = (i + 0.5 - H / 2) * pitch
    X1, X2 = np.meshgrid(x1, x2)  # [i, j]
    return X1.ravel(), X2.ravel()


# ------------------------------------------------------------------ printed values
def test_worked_example_initial_variance():
    cfg = oracle.Config(cov_param=0, beta=1e-4)
    for l, printed in _read_golden("init_variance.txt"):
        _, cov = oracle.covariance(np.full((1, 6), float(l)), cfg)
        assert round(cov[0, 0, 0], 4) == float(printed)


def test_printed_constants():
    rows = {r[0]: float(r[1]) for r in _read_golden("constants.txt")}
    assert abs(rows["chi2_3dof_p95"] - chi2_dist.ppf(0.95, 3)) < 1e-3
    assert oracle.CHI2_95_PRINTED == rows["chi2_3dof_p95"]
    assert round(1.0 / (1.0 + np.exp(-1.0)), 3) == rows["alpha_init"]


# ------------------------------------------------------------------ covariance
def test_precision_matches_library_forms():
    rng = np.random.default_rng(3)
    g = synth.gaussians_scale_rot(rng, 50)
    cfg = oracle.Config(cov_param=1)
    prec, cov = oracle.covariance(oracle.covp_rows(g, 1), cfg)
    for k in range(50):
        S = scipy_cov(g["log_scale"][:, k].astype(np.float64), g["quat"][:, k].astype(np.float64))
        np.testing.assert_allclose(cov[k], S, rtol=1e-9, atol=1e-15)
        np.testing.assert_allclose(prec[k] @ S, np.eye(3), atol=1e-8)
    # triangular: Sigma^-1 = L L^T with the activated diagonal (numpy matmul + inv)
    t = rng.uniform(-2, 2, (20, 6))
    cfg0 = oracle.Config(cov_param=0, beta=1e-3)
    prec, cov = oracle.covariance(t, cfg0)
    for k in range(20):
        L = np.array([[t[k, 0] ** 2 + 1e-3, 0, 0], [t[k, 1], t[k, 3] ** 2 + 1e-3, 0],
                      [t[k, 2], t[k, 4], t[k, 5] ** 2 + 1e-3]])
        np.testing.assert_allclose(prec[k], L @ L.T, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(cov[k], np.linalg.inv(L @ L.T), rtol=1e-8)


def test_scale_rot_to_tri_round_trip():
    rng = np.random.default_rng(4)
    g = synth.gaussians_scale_rot(rng, 30)
    t = synth.scale_rot_to_tri(g, beta=1e-4)
    p1, _ = oracle.covariance(oracle.covp_rows(g, 1), oracle.Config(cov_param=1))
    p0, _ = oracle.covariance(oracle.covp_rows(t, 0), oracle.Config(cov_param=0, beta=1e-4))
    np.testing.assert_allclose(p0, p1, rtol=2e-6, atol=1e-4 * np.abs(p1).max())


# ------------------------------------------------------------------ closed forms
def test_K1_plane_through_mean_restricted_precision():
    """Plane through the mean: w(x) = alpha exp(-1/2 x^T P12 x), P12 the
    in-plane block of the probe-frame precision (Gaussian restriction)."""
    rng = np.random.default_rng(5)
    for trial in range(5):
        mu = rng.uniform(-0.3, 0.3, 3)
        ls = np.log(rng.uniform(0.05, 0.15, 3))
        q = rng.standard_normal(4)
        g = one_gauss(mu, ls, q)
        R = Rotation.random(random_state=trial).as_matrix()
        u, v = R[:, 0], R[:, 1]
        W = H = 31
        pitch = 0.02
        pl = plane_dict(mu, u, v, W, H, pitch)
        cfg = oracle.Config(cov_param=1, chi2=1e6)  # box covers the whole image
        out = oracle.render(g, pl, cfg, mode="dense")
        Pi = np.linalg.inv(scipy_cov(ls, q))
        B = np.stack([u, v], axis=1)
        P12 = B.T @ Pi @ B
        X1, X2 = pixel_centres(W, H, pitch)
        d = np.stack([X1, X2])
        w = (1 / (1 + np.exp(-1.0))) * np.exp(-0.5 * np.einsum("in,ij,jn->n", d, P12, d))
        np.testing.assert_allclose(out["sa"], w, rtol=1e-10, atol=1e-300)


def test_K2_isotropic_at_plane_distance():
    """Isotropic sigma at plane distance d: peak scaled by exp(-d^2 / 2 sigma^2);
    the whole image is alpha exp(-(d^2 + r^2) / 2 sigma^2)."""
    sigma, dist = 0.1, 0.07
    R = Rotation.random(random_state=11).as_matrix()
    u, v, nrm = R[:, 0], R[:, 1], R[:, 2]
    o = np.array([0.1, -0.2, 0.05])
    foot = o + 0.03 * u - 0.05 * v
    mu = foot + dist * nrm
    g = one_gauss(mu, np.log([sigma] * 3), [0.3, 0.1, -0.5, 0.7])
    W = H = 40
    pitch = 0.015
    pl = plane_dict(o, u, v, W, H, pitch)
    cfg = oracle.Config(cov_param=1)
    out = oracle.render(g, pl, cfg, mode="dense")
    X1, X2 = pixel_centres(W, H, pitch)
    r2 = (X1 - 0.03) ** 2 + (X2 + 0.05) ** 2
    alpha = 1 / (1 + np.exp(-1.0))
    w_ref = alpha * np.exp(-(dist ** 2 + r2) / (2 * sigma ** 2))
    inside = out["sa"] > 0
    # box half-extent in-plane for an isotropic Gaussian is sqrt(chi2) sigma
    h = np.sqrt(7.815) * sigma
    box = (np.abs(X1 - 0.03) <= h) & (np.abs(X2 + 0.05) <= h)
    assert np.array_equal(inside, box)
    np.testing.assert_allclose(out["sa"][inside], w_ref[inside], rtol=1e-11)
    # single Gaussian: C = w c / (w + a_bg)
    np.testing.assert_allclose(out["image"][inside], w_ref[inside] * 0.8 / (w_ref[inside] + 1e-3),
                               rtol=1e-11)


def test_K3_off_plane_gaussian_conditioning():
    """General off-plane Gaussian: q(x) = m3^2/S33 + (x - x*)^T P12 (x - x*),
    x* = m12 - m3 S12,3 / S33 (textbook conditioning of a Gaussian)."""
    rng = np.random.default_rng(8)
    for trial in range(6):
        ls = np.log(rng.uniform(0.03, 0.2, 3))
        q = rng.standard_normal(4)
        R = Rotation.random(random_state=100 + trial).as_matrix()
        u, v, nrm = R[:, 0], R[:, 1], R[:, 2]
        o = rng.uniform(-0.2, 0.2, 3)
        mu = o + rng.uniform(-0.1, 0.1) * u + rng.uniform(-0.1, 0.1) * v + rng.uniform(-0.08, 0.08) * nrm
        g = one_gauss(mu, ls, q)
        W, H, pitch = 24, 20, 0.02
        pl = plane_dict(o, u, v, W, H, pitch)
        cfg = oracle.Config(cov_param=1, chi2=1e6)
        out = oracle.render(g, pl, cfg, mode="dense")
        S = scipy_cov(ls, q)
        Wr = np.stack([u, v, nrm])
        m = Wr @ (mu - o)
        S3 = Wr @ S @ Wr.T
        P12 = np.linalg.inv(S3)[:2, :2]
        xs = m[:2] - m[2] * S3[:2, 2] / S3[2, 2]
        q0 = m[2] ** 2 / S3[2, 2]
        X1, X2 = pixel_centres(W, H, pitch)
        d = np.stack([X1 - xs[0], X2 - xs[1]])
        qq = q0 + np.einsum("in,ij,jn->n", d, P12, d)
        w = (1 / (1 + np.exp(-1.0))) * np.exp(-0.5 * qq)
        np.testing.assert_allclose(out["sa"], w, rtol=1e-9, atol=1e-300)


def test_K4_box_is_the_ellipsoid_aabb():
    """Half-extents equal the max coordinate over the chi2 ellipsoid surface,
    found by brute-force sampling and by the exact extreme points."""
    rng = np.random.default_rng(9)
    g = synth.gaussians_scale_rot(rng, 12, 0.02, 0.2)
    pl = synth.planes_random(rng, [(16, 16)])
    R = Rotation.random(random_state=9).as_matrix()  # exactly orthonormal FP64 axes
    pl["u"], pl["v"] = R[:, 0][None], R[:, 1][None]
    cfg = oracle.Config(cov_param=1)
    geo = oracle.geometry(g, pl, cfg)
    Wr = np.stack([R[:, 0], R[:, 1], np.cross(R[:, 0], R[:, 1])])
    z = rng.standard_normal((3, 200000))
    z /= np.linalg.norm(z, axis=0)
    for k in range(12):
        S = scipy_cov(g["log_scale"][:, k].astype(np.float64), g["quat"][:, k].astype(np.float64))
        S3 = Wr @ S @ Wr.T
        C = np.linalg.cholesky(S3)
        pts = np.sqrt(7.815) * (C @ z)  # q = chi2 on the surface
        hmax = np.abs(pts).max(axis=1)
        h = geo["h"][0, k]
        assert np.all(hmax <= h * (1 + 1e-12))
        np.testing.assert_allclose(hmax, h, rtol=2e-3)
        for a in range(3):
            e = np.zeros(3)
            e[a] = 1
            xa = np.sqrt(7.815) * S3 @ e / np.sqrt(S3[a, a])
            assert abs(xa @ np.linalg.solve(S3, xa) - 7.815) < 1e-9
            np.testing.assert_allclose(abs(xa[a]), h[a], rtol=1e-10)


@pytest.mark.parametrize("cov_param", [0, 1])
def test_box_is_the_ellipsoid_bound_for_fp32_frames_and_needles(cov_param):
    """The box half-extent is the largest probe coordinate r_k . (X - mu) over
    the chi2 ellipsoid, sqrt(chi2 r_k^T Sigma r_k) (Sec. 4.3, Eq. boundary),
    also when the frame rows are FP32 (orthonormal only to about 1e-7) and
    the Gaussians are needles and discs with axis ratios up to 1e4: the
    oracle's half-extents against the definition evaluated with 50 digits
    from the same inputs (Sigma from the factor, u and v as given, n = u x v).
    The cofactor form of W Sigma^-1 W^T, exact only for an orthonormal frame,
    is off by up to per cent here."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(19)
    g = synth.gaussians_anisotropic(rng, 40)  # axis ratios log-uniform to 1e4
    if cov_param == 0:
        g = synth.scale_rot_to_tri(g, 1e-4)
    pl = synth.planes_random(rng, [(64, 64)] * 3)  # FP32 axes
    cfg = oracle.Config(cov_param=cov_param)
    geo = oracle.geometry(g, pl, cfg)
    chi2 = mp.mpf(cfg.chi2)
    worst = 0.0
    for k in range(40):
        if cov_param == 0:
            t = [mp.mpf(float(x)) for x in g["tri"][:, k]]
            b = mp.mpf(cfg.beta)
            L = mp.matrix([[t[0] ** 2 + b, 0, 0], [t[1], t[3] ** 2 + b, 0],
                           [t[2], t[4], t[5] ** 2 + b]])
            Li = L ** -1
            S = Li.T * Li
        else:
            q = [mp.mpf(float(x)) for x in g["quat"][:, k]]
            nq = mp.sqrt(sum(x * x for x in q))
            w, x, y, z = (c / nq for c in q)
            R = mp.matrix([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                           [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                           [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
            D = mp.diag([mp.exp(2 * mp.mpf(float(s))) for s in g["log_scale"][:, k]])
            S = R * D * R.T
        for p in range(3):
            u = [mp.mpf(float(c)) for c in pl["u"][p]]
            v = [mp.mpf(float(c)) for c in pl["v"][p]]
            n = [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]
            for a, r in enumerate((u, v, n)):
                rv = mp.matrix(r)
                h = mp.sqrt(chi2 * (rv.T * S * rv)[0])
                rel = abs(geo["h"][p, k, a] - float(h)) / float(h)
                worst = max(worst, rel)
    assert worst < 1e-12, worst


def test_phase1_reject_rule():
    """A Gaussian is kept on a plane iff |m3| <= h3 (Sec. 4.4, item 1)."""
    rng = np.random.default_rng(10)
    g = synth.gaussians_scale_rot(rng, 3000)
    pl = synth.planes_random(rng, [(32, 32)] * 3)
    cfg = oracle.Config(cov_param=1)
    geo = oracle.geometry(g, pl, cfg)
    m3 = geo["m"][..., 2]
    h3 = geo["h"][..., 2]
    assert np.array_equal(geo["visible"], np.abs(m3) <= h3)
    assert 0.01 < geo["visible"].mean() < 0.5


# ------------------------------------------------------------------ brute force
def _second_formulation(g, pl, cfg):
    """Eq. mahalanobis-3d taken literally in the probe frame: mu3D = W mu,
    Sigma3D = W Sigma W^T (library inverse), x_|0 = (x1, x2, 0), textbook AABB
    half-extents sqrt(chi2 Sigma3D_kk); every pixel x every Gaussian."""
    n = g["logit"].shape[0]
    out_sa = []
    out_sc = []
    for p in range(len(pl["size"])):
        u = pl["u"][p].astype(np.float64)
        v = pl["v"][p].astype(np.float64)
        o = pl["origin"][p].astype(np.float64)
        Wr = np.stack([u, v, np.cross(u, v)])
        W, H = pl["size"][p]
        X1 = ((np.arange(W) + 0.5 - W / 2) * float(pl["pitch"][p, 0]))[None, :].repeat(H, 0).ravel()
        X2 = ((np.arange(H) + 0.5 - H / 2) * float(pl["pitch"][p, 1]))[:, None].repeat(W, 1).ravel()
        sa = np.zeros(W * H)
        sc = np.zeros(W * H)
        for k in range(n):
            if cfg.cov_param == 1:
                S = scipy_cov(g["log_scale"][:, k].astype(np.float64), g["quat"][:, k].astype(np.float64))
            else:
                t = g["tri"][:, k].astype(np.float64)
                L = np.array([[t[0] ** 2 + cfg.beta, 0, 0], [t[1], t[3] ** 2 + cfg.beta, 0],
                              [t[2], t[4], t[5] ** 2 + cfg.beta]])
                S = np.linalg.inv(L @ L.T)
            m = Wr @ (g["mean"][:, k].astype(np.float64) - o)
            S3 = Wr @ S @ Wr.T
            h = np.sqrt(cfg.chi2 * np.diag(S3))
            if m[2] - h[2] > 0 or m[2] + h[2] < 0:
                continue
            d = np.stack([X1 - m[0], X2 - m[1], np.full_like(X1, -m[2])])
            qq = np.einsum("in,ij,jn->n", d, np.linalg.inv(S3), d)
            inside = (np.abs(X1 - m[0]) <= h[0]) & (np.abs(X2 - m[1]) <= h[1])
            if cfg.cutoff == 1:
                inside &= qq <= cfg.chi2
            w = 1 / (1 + np.exp(-float(g["logit"][k]))) * np.exp(-0.5 * qq)
            sa += np.where(inside, w, 0.0)
            sc += np.where(inside, w * float(g["intensity"][k]), 0.0)
        out_sa.append(sa)
        out_sc.append(sc)
    return np.concatenate(out_sa), np.concatenate(out_sc)


@pytest.mark.parametrize("cov_param,cutoff", [(1, 0), (0, 0), (1, 1), (0, 1)])
def test_K9_brute_force_second_formulation(cov_param, cutoff):
    rng = np.random.default_rng(20 + cov_param + 2 * cutoff)
    g = synth.gaussians_scale_rot(rng, 8, 0.1, 0.5)
    g["mean"] *= 0.3
    if cov_param == 0:
        g = synth.scale_rot_to_tri(g, 1e-4)
    pl = synth.planes_random(rng, [(8, 8), (8, 8)], origin_range=0.1)
    for p in range(2):  # exactly orthonormal FP64 axes: both frames then agree to rounding
        R = Rotation.random(random_state=40 + p).as_matrix()
        pl["u"] = pl["u"].astype(np.float64)
        pl["v"] = pl["v"].astype(np.float64)
        pl["u"][p], pl["v"][p] = R[:, 0], R[:, 1]
    cfg = oracle.Config(cov_param=cov_param, cutoff=cutoff)
    out = oracle.render(g, pl, cfg, mode="dense")
    sa, sc = _second_formulation(g, pl, cfg)
    assert out["amb"].max() == 0
    assert (sa > 0).sum() > 20
    np.testing.assert_allclose(out["sa"], sa, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(out["sc"], sc, rtol=1e-12, atol=1e-300)


def test_dense_equals_scatter_bitwise():
    g, pl = synth.workload_fwd_2k()
    cfg = oracle.Config(cov_param=1)
    d = oracle.render(g, pl, cfg, mode="dense")
    s = oracle.render(g, pl, cfg, mode="scatter")
    assert d["pairs"] == s["pairs"]
    for k in ("image", "alpha", "sa", "sc", "amb"):
        assert np.array_equal(d[k], s[k]), k


# ------------------------------------------------------------------ invariances
def _rigid(g, pl, Q, t):
    """Move scene and planes together by x -> Q x + t."""
    g2 = {k: np.array(v, copy=True) for k, v in g.items()}
    g2["mean"] = (Q @ g["mean"].astype(np.float64) + t[:, None])
    rq = Rotation.from_matrix(Q)
    qs = g["quat"].astype(np.float64)
    r = rq * Rotation.from_quat(np.stack([qs[1], qs[2], qs[3], qs[0]], axis=1))
    xyzw = r.as_quat()
    g2["quat"] = np.stack([xyzw[:, 3], xyzw[:, 0], xyzw[:, 1], xyzw[:, 2]])
    pl2 = dict(pl)
    pl2["origin"] = (Q @ pl["origin"].astype(np.float64).T).T + t
    pl2["u"] = (Q @ pl["u"].astype(np.float64).T).T
    pl2["v"] = (Q @ pl["v"].astype(np.float64).T).T
    return g2, pl2


@pytest.mark.parametrize("cutoff", [0, 1])
def test_K7_joint_rigid_motion(cutoff):
    g, pl = synth.workload_fwd_2k()
    g = {k: v.astype(np.float64) for k, v in g.items()}
    pl = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) and v.dtype == np.float32 else v)
          for k, v in pl.items()}
    cfg = oracle.Config(cov_param=1, cutoff=cutoff)
    a = oracle.render(g, pl, cfg)
    Q = Rotation.random(random_state=7).as_matrix()
    g2, pl2 = _rigid(g, pl, Q, np.array([0.3, -0.2, 0.1]))
    b = oracle.render(g2, pl2, cfg)
    ok = (a["amb"] == 0) & (b["amb"] == 0)
    assert ok.mean() > 0.99
    np.testing.assert_allclose(a["image"][ok], b["image"][ok], rtol=1e-10, atol=1e-12)


def test_K7_permutation_and_convexity():
    g, pl = synth.workload_fwd_2k()
    cfg = oracle.Config(cov_param=1)
    a = oracle.render(g, pl, cfg)
    perm = np.random.default_rng(1).permutation(2000)
    g2 = {k: v[..., perm] for k, v in g.items()}
    b = oracle.render(g2, pl, cfg)
    np.testing.assert_allclose(a["image"], b["image"], rtol=1e-12, atol=1e-15)
    assert a["pairs"] == b["pairs"]
    # C is a convex combination of the c_i and c_bg
    assert a["image"].min() >= 0.0 and a["image"].max() <= g["intensity"].max() + 1e-12


def test_K7_quarter_turn_in_plane():
    """Box mode: turning the probe axes by 90 degrees (u, v) -> (v, -u) on a
    square grid rotates the image; the box maps onto itself."""
    g, pl = synth.workload_fwd_2k()
    cfg = oracle.Config(cov_param=1)
    a = oracle.render(g, pl, cfg)
    pl2 = dict(pl)
    pl2["u"] = pl["v"].copy()
    pl2["v"] = -pl["u"].copy()
    b = oracle.render(g, pl2, cfg)
    W = 64
    for p in range(4):
        A = a["image"][p * W * W:(p + 1) * W * W].reshape(W, W)
        B = b["image"][p * W * W:(p + 1) * W * W].reshape(W, W)
        # new[i', j'] = old[j', W - 1 - i']
        np.testing.assert_allclose(B, A[:, ::-1].T, rtol=1e-10, atol=1e-13)


def test_K7_ellipsoid_mode_in_plane_rotation():
    """Ellipsoid mode is exactly in-plane rotation invariant: the value at a
    world point does not depend on how the probe axes turn about n."""
    rng = np.random.default_rng(12)
    g = synth.gaussians_scale_rot(rng, 400, 0.05, 0.2)
    g["mean"] *= 0.3
    g = {k: v.astype(np.float64) for k, v in g.items()}
    cfg = oracle.Config(cov_param=1, cutoff=1)
    R = Rotation.random(random_state=3).as_matrix()
    u, v = R[:, 0], R[:, 1]
    pts = rng.uniform(-0.2, 0.2, (20, 2))
    for x1, x2 in pts:
        o = x1 * u + x2 * v
        vals = []
        for th in (0.0, 0.4, 1.3, 2.9):
            ur = np.cos(th) * u + np.sin(th) * v
            vr = -np.sin(th) * u + np.cos(th) * v
            out = oracle.render(g, plane_dict(o, ur, vr, 1, 1, 0.01), cfg, mode="dense")
            vals.append(out["image"][0])
        np.testing.assert_allclose(vals, vals[0], rtol=1e-10, atol=1e-14)
