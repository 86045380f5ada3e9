"""Forward parity: the CUDA rasterizer against the FP64 oracle, element by
element, on seeded workloads that span several tiles with ragged tails, and
on the edge cases of the method."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_05643_gb300 import binding as B
from paper_2505_05643_gb300 import render as R
from paper_2505_05643_gb300 import synth

from gpu_helpers import assert_forward_parity, gpu_render, oracle_config

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cov_param", [B.UG_COV_SCALE_ROT, B.UG_COV_TRI])
@pytest.mark.parametrize("cutoff", [B.UG_CUTOFF_BOX, B.UG_CUTOFF_BOX_AND_ELLIPSOID])
def test_fwd_2k_parity(cov_param, cutoff):
    """2,000 Gaussians, 4 random planes of 64x64 (seed 0), both front-ends and cut-offs."""
    g, pl = synth.workload_fwd_2k()
    if cov_param == B.UG_COV_TRI:
        g = synth.scale_rot_to_tri(g, 1e-4)
    cfg = R.make_config(cov_param=cov_param, cutoff=cutoff)
    r, _, image, alpha = gpu_render(g, pl, cfg)
    ref = oracle.render(g, pl, oracle_config(cfg))
    assert ref["pairs"] > (40000 if cutoff == B.UG_CUTOFF_BOX else 15000)
    assert_forward_parity(image, alpha, ref, "fwd_2k")
    st = r.status()
    assert st["status"] == 0 and st["records"] > 500


@pytest.mark.parametrize("fp64_ratio,fp32_reach", [(1e3, float("inf")), (1.0, 20.0)])
def test_fwd_2k_fp64_branch(fp64_ratio, fp32_reach):
    """The triangular front-end with every Gaussian on the FP32 geometry
    (fp32_reach = inf; axis ratios here are below 1e3) and with every Gaussian
    on the extended-precision branch (fp64_ratio = 1) gives the same parity."""
    g, pl = synth.workload_fwd_2k()
    g = synth.scale_rot_to_tri(g, 1e-4)
    cfg = R.make_config(cov_param=B.UG_COV_TRI, fp64_ratio=fp64_ratio, fp32_reach=fp32_reach)
    r, _, image, alpha = gpu_render(g, pl, cfg)
    ref = oracle.render(g, pl, oracle_config(cfg))
    assert_forward_parity(image, alpha, ref, f"fp64_ratio {fp64_ratio} fp32_reach {fp32_reach}")
    st = r.status()
    if fp64_ratio == 1.0:  # every visible record (records also counts rejected candidates)
        assert st["fp64_records"] > 0.8 * st["records"] and st["fp64_records"] > 500
    else:
        assert st["fp64_records"] == 0


def _aniso_cut(n=20000, planes=(0, 1, 2, 3)):
    """The first n Gaussians of the bench workload (axis ratios log-uniform to
    1e4, triangular front-end) and some of its planes (sizes from {128, 192,
    256, 384, 512}^2)."""
    g, pl = synth.workload_aniso_1m()
    g = {k: np.ascontiguousarray(v[..., :n]) for k, v in g.items()}
    return synth.scale_rot_to_tri(g, 1e-4), synth.select_planes(pl, list(planes))


def test_fwd_extreme_anisotropy_parity():
    """Axis ratios up to 1e4 (needles and discs far thinner than a pixel) on
    planes up to 512^2: every pixel within the stated tolerance (Sec. 4.2's
    stable parameterisation at the bench workload's anisotropy)."""
    g, pl = _aniso_cut()
    assert int(pl["size"].max()) >= 384
    cfg = R.make_config(cov_param=B.UG_COV_TRI)
    r, _, image, alpha = gpu_render(g, pl, cfg)
    ref = oracle.render(g, pl, oracle_config(cfg))
    assert_forward_parity(image, alpha, ref, "aniso cut")
    st = r.status()
    assert st["fp64_records"] > 0.8 * st["records"]  # records also counts rejected candidates
    assert abs(st["box_pixels"] - ref["pairs"]) <= 1e-3 * ref["pairs"]


def test_fwd_extreme_anisotropy_random_planes():
    """The same shapes on random planes with a ratio of 1e4 everywhere."""
    rng = np.random.default_rng(3)
    g = synth.scale_rot_to_tri(synth.gaussians_anisotropic(rng, 20000), 1e-4)
    pl = synth.planes_random(rng, [(128, 128), (256, 256), (512, 512)])
    cfg = R.make_config(cov_param=B.UG_COV_TRI)
    r, _, image, alpha = gpu_render(g, pl, cfg)
    ref = oracle.render(g, pl, oracle_config(cfg))
    assert_forward_parity(image, alpha, ref, "aniso random planes")


def test_more_planes_than_shared_memory_table():
    """80 planes in one launch (the rasterizers keep 64 planes' tile data in
    shared memory and look the rest up in global memory; the cull stages planes
    64 at a time; the list and gather kernels walk planes 32 at a time)."""
    rng = np.random.default_rng(41)
    g = synth.gaussians_scale_rot(rng, 3000, 0.03, 0.15)
    sizes = [(24 + (k % 5) * 7, 20 + (k % 3) * 9) for k in range(80)]
    pl = synth.planes_random(rng, sizes)
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    r, _, image, alpha = gpu_render(g, pl, cfg)
    ref = oracle.render(g, pl, oracle_config(cfg))
    assert ref["pairs"] > 20000
    assert_forward_parity(image, alpha, ref, "80 planes")
    assert r.status()["status"] == 0


def test_dense_tiles_span_many_stages():
    """5,000 Gaussians on one 40x40 plane: most tiles hold several hundred
    records, so a tile spans several 128-record stages of the rasterizers'
    record pipeline and the backward's item queue wraps many times."""
    rng = np.random.default_rng(42)
    g = synth.gaussians_scale_rot(rng, 5000, 0.05, 0.3)
    pl = synth.planes_random(rng, [(40, 40)], origin_range=0.05)
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    r, _, image, alpha = gpu_render(g, pl, cfg)
    ref = oracle.render(g, pl, oracle_config(cfg))
    st = r.status()
    assert st["instances"] / 9 > 400  # 9 tiles of 16x16
    assert_forward_parity(image, alpha, ref, "dense tiles")


@pytest.mark.parametrize("tile,variant", [(16, v) for v in range(6)] + [(8, v) for v in range(3)])
def test_ragged_planes_all_variants(tile, variant):
    """Planes whose sizes are not multiples of the tile (ragged tails), several
    sizes in one launch, every compiled rasterizer variant."""
    rng = np.random.default_rng(5)
    g = synth.gaussians_scale_rot(rng, 3000, 0.02, 0.15)
    pl = synth.planes_random(rng, [(70, 45), (33, 97), (128, 16), (1, 1), (17, 3)])
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT, tile=tile, variant=variant, variant_bwd=0)
    _, _, image, alpha = gpu_render(g, pl, cfg)
    ref = oracle.render(g, pl, oracle_config(cfg))
    assert_forward_parity(image, alpha, ref, f"ragged t{tile} v{variant}")


def test_fwd_paper_init_triangular():
    """The paper's initialisation (Sec. 4.5): l_ij in [4, 5), c = 0.5, alpha = 0.731."""
    rng = np.random.default_rng(11)
    g = synth.gaussians_paper_init(rng, 4000)
    pl = synth.planes_random(rng, [(96, 96), (64, 80)])
    cfg = R.make_config(cov_param=B.UG_COV_TRI)
    _, _, image, alpha = gpu_render(g, pl, cfg)
    ref = oracle.render(g, pl, oracle_config(cfg))
    assert ref["pairs"] / len(ref["image"]) > 5
    assert_forward_parity(image, alpha, ref, "paper init")


def test_empty_and_degenerate_inputs():
    """No Gaussian at all, a Gaussian set that misses every plane, a 1x1 plane."""
    rng = np.random.default_rng(2)
    pl = synth.planes_random(rng, [(20, 20), (1, 1)])
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT, c_bg=0.25)
    # n = 0: background only
    g0 = {k: v[..., :0] for k, v in synth.gaussians_scale_rot(rng, 1).items()}
    r = R.Renderer(0, pl, cfg)
    image, alpha = r.forward(torch.zeros((12, 0), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    np.testing.assert_allclose(image.cpu().numpy(), 0.25, rtol=1e-6)
    np.testing.assert_allclose(alpha.cpu().numpy(), 1e-3, rtol=1e-6)
    # Gaussians far outside every plane's box
    g = synth.gaussians_scale_rot(rng, 64)
    g["mean"][:] = 50.0
    _, _, image, alpha = gpu_render(g, pl, cfg)
    np.testing.assert_allclose(image, 0.25, rtol=1e-6)
    assert oracle.render(g, pl, oracle_config(cfg))["pairs"] == 0


def test_single_gaussian_closed_form():
    """One isotropic Gaussian at plane distance d: C = w c / (w + a_bg),
    w = alpha exp(-(d^2 + r^2) / 2 sigma^2) inside the box (pin K2 on the GPU)."""
    sigma, dist = 0.1, 0.05
    pl = synth.planes_random(np.random.default_rng(4), [(64, 64)], origin_range=0.0)
    u, v = pl["u"][0].astype(np.float64), pl["v"][0].astype(np.float64)
    nrm = np.cross(u, v)
    mu = 0.1 * u - 0.05 * v + dist * nrm
    g = dict(mean=mu.reshape(3, 1).astype(np.float32),
             log_scale=np.full((3, 1), np.log(sigma), np.float32),
             quat=np.array([[1.0], [0.0], [0.0], [0.0]], np.float32),
             logit=np.array([1.0], np.float32), intensity=np.array([0.7], np.float32))
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    _, _, image, alpha = gpu_render(g, pl, cfg)
    p = 2.0 / 64
    x1 = (np.arange(64) + 0.5 - 32) * p
    X1, X2 = np.meshgrid(x1, x1)
    r2 = (X1 - 0.1) ** 2 + (X2 + 0.05) ** 2
    w = (1 / (1 + np.e ** -1)) * np.exp(-(dist ** 2 + r2) / (2 * sigma ** 2))
    h = np.sqrt(7.815) * sigma
    inside = ((np.abs(X1 - 0.1) <= h) & (np.abs(X2 + 0.05) <= h)).ravel()
    expect = np.where(inside, w.ravel() * 0.7 / (w.ravel() + 1e-3), 0.0)
    np.testing.assert_allclose(image, expect, rtol=2e-4, atol=1e-6)


def test_plane_change_between_calls():
    """Poses updated in device memory (same sizes) are picked up."""
    rng = np.random.default_rng(8)
    g = synth.gaussians_scale_rot(rng, 2000)
    pl_a = synth.planes_random(rng, [(48, 48)] * 3)
    pl_b = synth.planes_random(rng, [(48, 48)] * 3)
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    r = R.Renderer(2000, pl_a, cfg)
    params = torch.from_numpy(R.pack_params(g, cfg.cov_param)).cuda()
    r.forward(params)
    r.set_planes(pl_b)
    image, alpha = r.forward(params)
    ref = oracle.render(g, pl_b, oracle_config(cfg))
    assert_forward_parity(image.cpu().numpy().astype(np.float64),
                          alpha.cpu().numpy().astype(np.float64), ref, "replanned")


def test_invalid_plane_in_device_memory_sets_status():
    rng = np.random.default_rng(9)
    g = synth.gaussians_scale_rot(rng, 100)
    pl = synth.planes_random(rng, [(16, 16)])
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    r = R.Renderer(100, pl, cfg)
    bad = synth.planes_to_struct(pl)
    bad["u"][0] = [2.0, 0.0, 0.0]
    r.d_planes.copy_(torch.from_numpy(bad.view(np.uint8).copy()))
    params = torch.from_numpy(R.pack_params(g, cfg.cov_param)).cuda()
    with pytest.raises(B.UgError) as e:
        r.forward(params)
    assert e.value.status == B.UG_ERR_INVALID_PLANE


def test_bounded_waits_run_out_and_report():
    """The rasterizers' waits are bounded: with the test hook set, no stage is
    ever issued, every consumer wait runs out (about a second), the launch ends
    with UG_ERR_TIMEOUT in the status (detail 1: forward, 2: backward), and the
    context stays usable: clearing the hook gives the same image as before."""
    import time
    g, pl = synth.workload_fwd_2k()
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    r, params, image0, _ = gpu_render(g, pl, cfg)
    im = torch.empty(pl["total_pixels"], device="cuda")
    al = torch.empty_like(im)
    B.ug_debug_stall_pipeline(r.plan, r.ws, True)
    t0 = time.time()
    B.ug_render(r.plan, r.ws, im, al)
    torch.cuda.synchronize()
    assert time.time() - t0 < 30.0
    st = r.status()
    assert st["status"] == B.UG_ERR_TIMEOUT and st["detail"] == 1, st
    # the backward's consumers (status cleared by hand: it keeps the first failure)
    r.ws[:4].zero_()
    B.ug_render_backward_raster(r.plan, r.ws, im, al, torch.zeros_like(im))
    torch.cuda.synchronize()
    st = r.status()
    assert st["status"] == B.UG_ERR_TIMEOUT and st["detail"] == 2, st
    B.ug_debug_stall_pipeline(r.plan, r.ws, False)
    image1, _ = r.forward(params)
    torch.cuda.synchronize()
    assert r.status()["status"] == B.UG_OK
    assert np.array_equal(image1.cpu().numpy().astype(np.float64), image0)


def test_capacity_overflow_is_reported_and_recovered():
    g, pl = synth.workload_fwd_2k()
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    r = R.Renderer(2000, pl, cfg, record_capacity=16, instance_capacity=32)
    params = torch.from_numpy(R.pack_params(g, cfg.cov_param)).cuda()
    B.ug_preprocess(r.plan, R.gaussians_struct(params, cfg.cov_param), r.d_planes, r.ws)
    st = r.status()
    assert st["status"] == B.UG_ERR_CAPACITY and st["records"] > 16
    image, alpha = r.forward(params)  # grows and retries
    ref = oracle.render(g, pl, oracle_config(cfg))
    assert_forward_parity(image.cpu().numpy().astype(np.float64),
                          alpha.cpu().numpy().astype(np.float64), ref, "regrown")


def test_forward_is_deterministic():
    g, pl = synth.workload_fwd_2k()
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT)
    r = R.Renderer(2000, pl, cfg)
    params = torch.from_numpy(R.pack_params(g, cfg.cov_param)).cuda()
    a, _ = r.forward(params)
    b, _ = r.forward(params)
    assert torch.equal(a, b)


@pytest.mark.parametrize("cutoff", [B.UG_CUTOFF_BOX, B.UG_CUTOFF_BOX_AND_ELLIPSOID])
def test_scatter_ablation_parity(cutoff):
    """The paper's phase-2 atomic scatter (kept as an ablation) against the
    oracle, and against the tile gather to FP32 rounding of the sums."""
    rng = np.random.default_rng(61)
    g = synth.gaussians_scale_rot(rng, 3000, 0.02, 0.15)
    pl = synth.planes_random(rng, [(70, 45), (64, 64), (33, 97)])
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT, cutoff=cutoff)
    r, params, image, alpha = gpu_render(g, pl, cfg)
    im2, al2 = r.new_image(), r.new_image()
    B.ug_render_scatter(r.plan, r.ws, im2, al2)
    assert r.status()["status"] == B.UG_OK
    im2 = im2.cpu().numpy().astype(np.float64)
    al2 = al2.cpu().numpy().astype(np.float64)
    ref = oracle.render(g, pl, oracle_config(cfg))
    assert_forward_parity(im2, al2, ref, "scatter")
    assert np.allclose(im2, image, rtol=2e-5, atol=1e-7)
    assert np.allclose(al2, alpha, rtol=2e-5, atol=1e-7)
