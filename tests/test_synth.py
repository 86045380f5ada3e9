"""Sanity of the seeded input generators (distributions and layout)."""
import numpy as np

from paper_2505_05643_gb300 import synth


def test_planes_are_orthonormal_and_packed():
    rng = np.random.default_rng(0)
    pl = synth.planes_random(rng, [(64, 32), (16, 16), (128, 128)])
    u = pl["u"].astype(np.float64)
    v = pl["v"].astype(np.float64)
    assert np.abs(np.linalg.norm(u, axis=1) - 1).max() < 1e-6
    assert np.abs(np.linalg.norm(v, axis=1) - 1).max() < 1e-6
    assert np.abs((u * v).sum(1)).max() < 1e-6
    assert list(pl["offset"]) == [0, 64 * 32, 64 * 32 + 256]
    assert pl["total_pixels"] == 64 * 32 + 256 + 128 * 128
    s = synth.planes_to_struct(pl)
    assert s.dtype.itemsize == 64 and s["width"][0] == 64 and s["height"][0] == 32
    np.testing.assert_allclose(s["pitch_u"], 2.0 / pl["size"][:, 0])


def test_sweep_pool_is_smooth():
    pool = synth.planes_sweep_pool(np.random.default_rng(2), pool=160)
    o = pool["origin"].astype(np.float64)
    step = np.linalg.norm(np.diff(o, axis=0), axis=1)
    np.testing.assert_allclose(step, step[0], rtol=1e-5)
    assert abs(np.linalg.norm(o[-1] - o[0]) - 1.8) < 1e-5
    n = np.cross(pool["u"], pool["v"])
    # jitter is at most 5 degrees about each in-plane axis
    cosang = np.abs((n * n[0]).sum(1))
    assert cosang.min() > np.cos(np.deg2rad(15))


def test_anisotropic_ratios():
    g = synth.gaussians_anisotropic(np.random.default_rng(1), 20000)
    s = np.exp(g["log_scale"].astype(np.float64))
    ratio = s.max(0) / s.min(0)
    assert ratio.max() > 5e3 and ratio.max() <= 1e4 * 1.001
    assert 0.0099 < s.max(0).min() and s.max(0).max() < 0.1001


def test_workloads_deterministic():
    a, pa = synth.workload_fwd_2k()
    b, pb = synth.workload_fwd_2k()
    for k in a:
        assert np.array_equal(a[k], b[k])
    assert pa["total_pixels"] == 4 * 64 * 64
    g = synth.gaussians_paper_init(np.random.default_rng(0), 100)
    assert g["tri"].min() >= 4.0 and g["tri"].max() < 5.0
    assert np.all(g["intensity"] == 0.5)


def test_slice_sets_cover_the_cube():
    """Linearly spaced slices: one per equal layer along the axis, each spanning
    the cube's cross-section; the three orientations are mutually orthogonal."""
    ax = synth.planes_slices(160, 160, axis=2)
    z = ax["origin"][:, 2].astype(np.float64)
    np.testing.assert_allclose(np.diff(z), 2.0 / 160, rtol=1e-5)
    assert abs(z[0] + 1 - 1 / 160) < 1e-6 and abs(z[-1] - 1 + 1 / 160) < 1e-6
    np.testing.assert_allclose(ax["pitch"], 2.0 / 160)
    three = synth.concat_planes(*(synth.planes_slices(4, 8, axis=a) for a in (2, 1, 0)))
    n = np.cross(three["u"].astype(np.float64), three["v"].astype(np.float64))
    np.testing.assert_allclose(np.abs(n[[0, 4, 8]]), np.eye(3)[[2, 1, 0]])
    assert list(three["offset"]) == [64 * k for k in range(12)]
    np.testing.assert_allclose(three["pitch"], 0.25)
    g, _, tr, te = synth.workload_recon(n=10, hidden_n=10, train_pool=16, held_out=8, size=32,
                                        poses="slices")
    assert len(tr["size"]) == 16 and len(te["size"]) == 24
