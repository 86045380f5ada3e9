"""The oracle's ambiguity margins bound the rounding of the CUDA path's FP32
inclusion decisions.

The oracle reports a pair as ambiguous (either decision correct) when its
inclusion margin is within amb * pitch + amb_abs of an in-plane box edge, or
within amb * h3 + amb_abs of the plane test (amb = 1e-5, amb_abs = 2e-6 world
units; Sec. 4.3 Eq. boundary and Sec. 4.4's two tests). Here the kernel's FP32
decision quantities are reproduced operation by operation in NumPy float32
(the probe-frame mean m = R (mu - o), the half-extents h = sqrt(chi2 |F^-1 r|^2)
with F^-1 by forward substitution, and the pixel-unit box edges (m1 -+ h1) /
pitch + W/2 - 1/2), for the Gaussians the kernel sends down its FP32 geometry,
and compared with FP64. The extended-precision branch takes the same FP32
decisions from its inverse factor computed in double words and rounded once
(emulated by the FP64 inverse rounded to FP32), also checked here. Every error must stay well inside the margin, and the
absolute term must be needed: the relative one alone is too small."""
import numpy as np

import oracle
from paper_2505_05643_gb300 import synth

f32 = np.float32
AMB = oracle.Config().amb
AMB_ABS = oracle.Config().amb_abs
CHI2 = f32(7.815)
BETA = f32(1e-4)


def fma(a, b, c):
    """FP32 fused multiply-add (the float64 product of two floats is exact;
    the sum is rounded once to float64, then to float32)."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(f32)


def dot3(a, b):
    return fma(a[2], b[2], fma(a[1], b[1], (a[0] * b[0]).astype(f32)))


def _fp64_inverse(tri):
    t = tri.astype(np.float64)
    b = float(BETA)
    L = np.zeros((t.shape[1], 3, 3))
    L[:, 0, 0], L[:, 1, 1], L[:, 2, 2] = t[0] ** 2 + b, t[3] ** 2 + b, t[5] ** 2 + b
    L[:, 1, 0], L[:, 2, 0], L[:, 2, 1] = t[1], t[2], t[4]
    return np.linalg.inv(L)


def kernel_decisions(tri, mu, pl_o, pl_u, pl_v, pu, W, extended=False):
    """FP32 decision quantities as the record kernel computes them for the
    triangular front-end: the plane test margin h3 - |m3| and the first and
    last pixel-unit box edge along u. extended: the inverse factor of the
    extended-precision branch (accurate, rounded once to FP32) instead of the
    FP32 forward substitution."""
    if extended:
        Li = _fp64_inverse(tri).astype(f32)
        i00, i11, i22 = Li[:, 0, 0], Li[:, 1, 1], Li[:, 2, 2]
        i10, i20, i21 = Li[:, 1, 0], Li[:, 2, 0], Li[:, 2, 1]
    else:
        t = [tri[k].astype(f32) for k in range(6)]
        F00, F11, F22 = fma(t[0], t[0], BETA), fma(t[3], t[3], BETA), fma(t[5], t[5], BETA)
        F10, F20, F21 = t[1], t[2], t[4]
        i00, i11, i22 = ((f32(1) / F00).astype(f32), (f32(1) / F11).astype(f32),
                         (f32(1) / F22).astype(f32))
        i10 = -((F10 * i00).astype(f32) * i11).astype(f32)
        i21 = -((F21 * i11).astype(f32) * i22).astype(f32)
        i20 = -(fma(F21, i10, (F20 * i00).astype(f32)) * i22).astype(f32)
    u, v, o = pl_u.astype(f32), pl_v.astype(f32), pl_o.astype(f32)
    n = np.stack([fma(u[1], v[2], -(u[2] * v[1]).astype(f32)),
                  fma(u[2], v[0], -(u[0] * v[2]).astype(f32)),
                  fma(u[0], v[1], -(u[1] * v[0]).astype(f32))])
    d = [(mu[k].astype(f32)[None, :] - o[k][:, None]).astype(f32) for k in range(3)]

    def fi_apply(r):
        z0 = (i00 * r[0]).astype(f32)
        z1 = fma(i11, r[1], (i10 * r[0]).astype(f32))
        z2 = fma(i22, r[2], fma(i21, r[1], (i20 * r[0]).astype(f32)))
        return [z0, z1, z2]

    def extent(r):
        z = fi_apply([r[k][:, None] for k in range(3)])
        return np.sqrt((CHI2 * dot3(z, z)).astype(f32)).astype(f32)

    m3 = dot3([n[k][:, None] for k in range(3)], d)
    m1 = dot3([u[k][:, None] for k in range(3)], d)
    h3, h1 = extent(n), extent(u)
    inv = (f32(1) / pu.astype(f32)).astype(f32)[:, None]
    shift = (f32(0.5) * W.astype(f32) - f32(0.5)).astype(f32)[:, None]
    lo = fma((m1 - h1).astype(f32), inv, shift)
    hi = fma((m1 + h1).astype(f32), inv, shift)
    return (h3 - np.abs(m3)).astype(np.float64), lo.astype(np.float64), hi.astype(np.float64)


def exact_decisions(tri, mu, pl_o, pl_u, pl_v, pu, W):
    """The same quantities in FP64 from the same FP32 inputs (the oracle's
    definition: n = u x v, h_k^2 = chi2 r_k^T Sigma r_k)."""
    t = tri.astype(np.float64)
    b = float(BETA)
    L = np.zeros((t.shape[1], 3, 3))
    L[:, 0, 0], L[:, 1, 1], L[:, 2, 2] = t[0] ** 2 + b, t[3] ** 2 + b, t[5] ** 2 + b
    L[:, 1, 0], L[:, 2, 0], L[:, 2, 1] = t[1], t[2], t[4]
    Li = np.linalg.inv(L)
    u, v, o = pl_u.astype(np.float64), pl_v.astype(np.float64), pl_o.astype(np.float64)
    n = np.cross(u.T, v.T).T
    d = mu.astype(np.float64)[None, :, :] - o.T[:, :, None]  # (P, 3, n)
    m3 = np.einsum("kp,pkn->pn", n, d)
    m1 = np.einsum("kp,pkn->pn", u, d)

    def extent(r):  # (3, P) -> (P, n)
        z = np.einsum("nij,jp->pni", Li, r)
        return np.sqrt(float(CHI2) * (z * z).sum(-1))

    h3, h1 = extent(n), extent(u)
    shift = 0.5 * W.astype(np.float64)[:, None] - 0.5
    p = pu.astype(np.float64)[:, None]
    return h3 - np.abs(m3), (m1 - h1) / p + shift, (m1 + h1) / p + shift, h3


def _check(g_tri, mu, planes, select, extended=False):
    o, u, v = planes["origin"].T, planes["u"].T, planes["v"].T
    pu = planes["pitch"][:, 0].astype(np.float64)
    W = planes["size"][:, 0]
    k_pl, k_lo, k_hi = kernel_decisions(g_tri, mu, o, u, v, pu, W, extended)
    e_pl, e_lo, e_hi, h3 = exact_decisions(g_tri, mu, o, u, v, pu, W)
    sel = np.broadcast_to(select[None, :], k_pl.shape)
    plane_err = np.abs(k_pl - e_pl)[sel]
    plane_tol = (AMB * h3 + AMB_ABS)[sel]
    # in-plane edges in world units, against amb * pitch + amb_abs
    p = pu[:, None]
    edge_err = np.maximum(np.abs(k_lo - e_lo), np.abs(k_hi - e_hi)) * p
    edge_tol = np.broadcast_to(AMB * p + AMB_ABS, edge_err.shape)
    return (plane_err / plane_tol).max(), (edge_err[sel] / edge_tol[sel]).max(), \
        plane_err.max(), edge_err[sel].max(), (edge_err[sel] / (AMB * p + 0 * edge_err)[sel]).max()


def _fp32_branch(g_tri, mu, planes, ratio=1e3, reach=20.0):
    """Which Gaussians the cull sends down the FP32 geometry (axis-ratio
    proxy ||L||_F ||L^-1||_F and ||L||_F (|mu| + max |o|))."""
    t = g_tri.astype(np.float64)
    b = float(BETA)
    L = np.zeros((t.shape[1], 3, 3))
    L[:, 0, 0], L[:, 1, 1], L[:, 2, 2] = t[0] ** 2 + b, t[3] ** 2 + b, t[5] ** 2 + b
    L[:, 1, 0], L[:, 2, 0], L[:, 2, 1] = t[1], t[2], t[4]
    fro = np.linalg.norm(L, axis=(1, 2))
    prox = fro * np.linalg.norm(np.linalg.inv(L), axis=(1, 2))
    size = fro * (np.linalg.norm(mu, axis=0) + np.linalg.norm(planes["origin"], axis=1).max())
    return (prox <= ratio) & (size <= reach)


def _planes(rng):
    return synth.planes_random(rng, [(s, s) for s in (64, 128, 256, 384, 512, 96, 200, 512)])


def test_margins_cover_fp32_decisions_of_ordinary_gaussians():
    """Scale/rotation draws with scales 0.01-0.1 (the fwd_2k and grad_50k
    distributions), all on the FP32 geometry (as with fp32_reach = inf)."""
    rng = np.random.default_rng(71)
    g = synth.scale_rot_to_tri(synth.gaussians_scale_rot(rng, 100_000, 0.01, 0.1), float(BETA))
    pl = _planes(rng)
    sel = _fp32_branch(g["tri"], g["mean"], pl, reach=np.inf)
    assert sel.mean() > 0.99
    r_pl, r_edge, abs_pl, abs_edge, rel_only = _check(g["tri"], g["mean"], pl, sel)
    assert r_pl < 0.5 and r_edge < 0.5, (r_pl, r_edge)
    # the errors are ulps of the scene's coordinates, not of the pixel: the
    # relative term alone (1e-5 of a pixel) would not cover them
    assert rel_only > 1.0, rel_only
    assert abs_edge < AMB_ABS and abs_pl < AMB_ABS


def test_margins_cover_fp32_decisions_of_paper_init_and_default_criterion():
    """The paper's initialisation (L_ij ~ U[4, 5)) and the bench workload's
    anisotropic draws, on whatever the default criterion leaves to FP32."""
    rng = np.random.default_rng(72)
    g1 = synth.gaussians_paper_init(rng, 50_000)
    g2 = synth.scale_rot_to_tri(synth.gaussians_anisotropic(rng, 50_000), float(BETA))
    pl = _planes(rng)
    for g in (g1, g2):
        sel = _fp32_branch(g["tri"], g["mean"], pl)
        if sel.sum() == 0:
            continue
        r_pl, r_edge, *_ = _check(g["tri"], g["mean"], pl, sel)
        assert r_pl < 0.5 and r_edge < 0.5, (r_pl, r_edge)


def test_margins_cover_fp32_decisions_of_the_extended_branch():
    """The bench workload's extreme anisotropy (axis ratios to 1e4): the
    Gaussians the default criterion sends down the extended-precision branch
    take their decisions in FP32 from the accurately computed inverse factor,
    rounded once; every error stays well inside the margins."""
    rng = np.random.default_rng(74)
    g = synth.scale_rot_to_tri(synth.gaussians_anisotropic(rng, 100_000), float(BETA))
    pl = _planes(rng)
    sel = ~_fp32_branch(g["tri"], g["mean"], pl)
    assert sel.mean() > 0.9
    r_pl, r_edge, abs_pl, abs_edge, _ = _check(g["tri"], g["mean"], pl, sel, extended=True)
    assert r_pl < 0.5 and r_edge < 0.5, (r_pl, r_edge)
    assert abs_edge < AMB_ABS and abs_pl < AMB_ABS
    # the FP32 forward substitution would not do for these (its error grows
    # with the factor's condition)
    r_pl32, r_edge32, *_ = _check(g["tri"], g["mean"], pl, sel, extended=False)
    assert max(r_pl32, r_edge32) > max(r_pl, r_edge)


def test_emulation_detects_a_planted_error():
    """The check has teeth: an edge moved by one FP32 ulp of the plane
    coordinates more than the kernel's own rounding (a mean rounded a second
    time) stays inside, but one moved by 2e-6 world units does not."""
    rng = np.random.default_rng(73)
    g = synth.scale_rot_to_tri(synth.gaussians_scale_rot(rng, 2000, 0.01, 0.1), float(BETA))
    pl = _planes(rng)
    o, u, v = pl["origin"].T, pl["u"].T, pl["v"].T
    pu = pl["pitch"][:, 0].astype(np.float64)
    W = pl["size"][:, 0]
    _, k_lo, _ = kernel_decisions(g["tri"], g["mean"], o, u, v, pu, W)
    _, e_lo, _, _ = exact_decisions(g["tri"], g["mean"], o, u, v, pu, W)
    shifted = k_lo + 2 * AMB_ABS / pu[:, None]
    assert (np.abs(shifted - e_lo) * pu[:, None] > AMB * pu[:, None] + AMB_ABS).any()
