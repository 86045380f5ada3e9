"""The C-ABI library builds, loads and exports every symbol include/ug.h
declares; host-side argument checks (no GPU work). No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2505_05643_gb300 import binding as B
from paper_2505_05643_gb300 import build_lib, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ug.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(ug_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return B.load()


def test_header_declares_the_hot_path(lib):
    names = declared_functions()
    for f in ("ug_preprocess", "ug_bin_sort", "ug_render", "ug_render_backward", "ug_adam_step"):
        assert f in names
    assert set(names) == set(B.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def declared_arity():
    src = open(os.path.join(ROOT, "include", "ug.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(ug_\w+)\s*\(([^)]*)\)\s*;", src):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_declares_every_signature(lib):
    """Every entry point has ctypes argument types with the header's arity
    (undeclared, ctypes would pass 64-bit pointers as 32-bit ints)."""
    arity = declared_arity()
    assert set(arity) == set(B.EXPORTS)
    for name, k in arity.items():
        assert getattr(lib, name).argtypes is not None, name
        assert len(getattr(lib, name).argtypes) == k, name


def test_versions_and_strings(lib):
    assert B.ug_version() >= 100
    assert B.status_string(B.UG_ERR_CAPACITY).startswith("record or instance")
    assert B.ug_num_variants(16) >= 1 and B.ug_num_variants(8) >= 1 and B.ug_num_variants(12) == 0
    assert B.ug_num_variants_bwd(16) >= 2 and B.ug_num_variants_bwd(8) >= 2
    assert B.ug_num_variants_bwd(12) == 0


def _planes(sizes=((64, 64), (70, 45))):
    return synth.planes_to_struct(synth.planes_random(np.random.default_rng(0), list(sizes)))


def test_plan_layout(lib):
    cfg = B.ug_config_default()
    pl = _planes()
    plan = B.ug_plan_init(cfg, 1000, pl, 5000, 20000)
    assert plan.total_tiles == 16 + 5 * 3
    assert plan.total_pixels == 64 * 64 + 70 * 45
    assert plan.key_bits == 5 and plan.sort_passes == 1
    assert plan.chunks == 32
    allo = list(plan.off)
    n_sec = max(i for i, o in enumerate(allo) if o) + 1  # sections in use; the rest are 0
    assert n_sec >= 24 and all(o == 0 for o in allo[n_sec:])
    offs = allo[:n_sec]
    assert all(o % 256 == 0 for o in offs) and offs == sorted(offs)
    assert plan.workspace_bytes >= offs[-1]
    cfg.tile = 8
    plan8 = B.ug_plan_init(cfg, 1000, pl, 5000, 20000)
    assert plan8.total_tiles == 64 + 9 * 6


def test_plan_rejects_bad_arguments(lib):
    cfg = B.ug_config_default()
    pl = _planes()
    bad = pl.copy()
    bad["u"][0] = [1.0, 0.1, 0.0]  # not unit
    with pytest.raises(B.UgError) as e:
        B.ug_plan_init(cfg, 10, bad, 10, 10)
    assert e.value.status == B.UG_ERR_INVALID_ARGUMENT
    overlap = pl.copy()
    overlap["pixel_offset"][1] = 100  # overlaps plane 0
    with pytest.raises(B.UgError):
        B.ug_plan_init(cfg, 10, overlap, 10, 10)
    with pytest.raises(B.UgError):
        B.ug_plan_init(cfg, 10, pl, 10, 1 << 31)
    c2 = B.ug_config_default()
    c2.tile = 12
    with pytest.raises(B.UgError) as e:
        B.ug_plan_init(c2, 10, pl, 10, 10)
    assert e.value.status == B.UG_ERR_NOT_SUPPORTED
    c3 = B.ug_config_default()
    c3.beta = 0.0
    with pytest.raises(B.UgError):
        B.ug_plan_init(c3, 10, pl, 10, 10)


def test_calls_reject_null_and_small_workspace(lib):
    cfg = B.ug_config_default()
    plan = B.ug_plan_init(cfg, 10, _planes(), 10, 10)
    g = B.ug_gaussians()
    # NULL workspace -> synchronous error, nothing launched
    st = lib.ug_preprocess(ctypes.byref(plan), ctypes.byref(g), None, None, 0, None)
    assert st == B.UG_ERR_INVALID_ARGUMENT
    st = lib.ug_bin_sort(ctypes.byref(plan), ctypes.c_void_p(256), 16, None)
    assert st == B.UG_ERR_WORKSPACE_TOO_SMALL
    st = lib.ug_mse_loss_grad(None, None, 10, None, None, None)
    assert st == B.UG_ERR_INVALID_ARGUMENT
    st = lib.ug_adam_step(None, None, None, None, 1, 10, None, None, 0.9, 0.999, 1e-15, None)
    assert st == B.UG_ERR_INVALID_ARGUMENT


def test_loss_and_evaluator_calls_check_their_arguments(lib):
    """SSIM, L1 + D-SSIM: sizes below the 11 x 11 window, a weight outside
    [0, 1], missing pointers and short scratch are refused before any launch."""
    nz = ctypes.c_void_p(256)  # never dereferenced: every call below returns first
    assert lib.ug_ssim_scratch_floats(0, 16, 16) == 0
    assert lib.ug_ssim_scratch_floats(1, 10, 40) == 0
    assert lib.ug_ssim_scratch_floats(1, 11, 11) > 0
    assert lib.ug_l1_dssim_scratch_floats(1, 40, 10) == 0
    need = lib.ug_l1_dssim_scratch_floats(2, 32, 24)
    assert need >= 2 * 32 * 24
    ok = [nz, nz, 2, 32, 24, ctypes.c_float(0.2), nz, need, nz, nz, None]
    for i, bad in ((0, None), (1, None), (6, None), (8, None), (9, None)):
        args = list(ok)
        args[i] = bad
        assert lib.ug_l1_dssim_loss_grad(*args) == B.UG_ERR_INVALID_ARGUMENT
    for lam in (-0.1, 1.5, float("nan")):
        args = list(ok)
        args[5] = ctypes.c_float(lam)
        assert lib.ug_l1_dssim_loss_grad(*args) == B.UG_ERR_INVALID_ARGUMENT
    args = list(ok)
    args[3] = 10
    assert lib.ug_l1_dssim_loss_grad(*args) == B.UG_ERR_INVALID_ARGUMENT
    args = list(ok)
    args[7] = need - 1
    assert lib.ug_l1_dssim_loss_grad(*args) == B.UG_ERR_WORKSPACE_TOO_SMALL
    s_need = lib.ug_ssim_scratch_floats(2, 32, 24)
    assert lib.ug_ssim(nz, nz, 2, 32, 24, nz, s_need, None, None, None) == B.UG_ERR_INVALID_ARGUMENT
    assert lib.ug_ssim(nz, nz, 2, 32, 24, nz, s_need - 1, nz, nz, None) == \
        B.UG_ERR_WORKSPACE_TOO_SMALL


def test_densify_and_sample_calls_check_their_arguments(lib):
    """Resampling and densify / prune: bad parametrisation or beta, negative or
    out-of-range counts, missing pointers, thresholds outside their domain and
    short scratch are refused before any launch; the defaults are the
    documented ones."""
    nz = ctypes.c_void_p(256)
    dc = B.ug_densify_config()
    assert lib.ug_densify_config_default(None) == B.UG_ERR_INVALID_ARGUMENT
    assert lib.ug_densify_config_default(ctypes.byref(dc)) == B.UG_OK
    assert (dc.min_opacity, dc.split_factor) == (np.float32(0.005), np.float32(1.6))
    cfg = B.ug_config_default()
    bad_cov = B.ug_config_default()
    bad_cov.cov_param = 7
    bad_beta = B.ug_config_default()
    bad_beta.beta = 0.0
    for c in (bad_cov, bad_beta):
        assert lib.ug_sample(ctypes.byref(c), nz, 10, nz, 4, nz, nz, None) == \
            B.UG_ERR_INVALID_ARGUMENT
    assert lib.ug_sample(ctypes.byref(cfg), nz, 10, nz, -1, nz, nz, None) == \
        B.UG_ERR_INVALID_ARGUMENT
    assert lib.ug_sample(ctypes.byref(cfg), nz, 10, None, 4, nz, nz, None) == \
        B.UG_ERR_INVALID_ARGUMENT
    assert lib.ug_densify_stats(nz, 0, nz, None) == B.UG_ERR_INVALID_ARGUMENT
    assert lib.ug_densify_stats(None, 5, nz, None) == B.UG_ERR_INVALID_ARGUMENT
    assert lib.ug_densify_scratch_bytes(0) == 0
    n = 1000
    need = lib.ug_densify_scratch_bytes(n)
    assert need >= 8 * n

    def densify(c=cfg, d=dc, n_=n, cap=2 * n, scratch=nz, sbytes=need, params=nz):
        return lib.ug_densify(ctypes.byref(c), ctypes.byref(d), params, nz, nz, n_, nz, nz, cap,
                              nz, nz, nz, nz, scratch, sbytes, None)

    assert densify(n_=0) == B.UG_ERR_INVALID_ARGUMENT
    assert densify(n_=1 << 31) == B.UG_ERR_INVALID_ARGUMENT
    assert densify(cap=0) == B.UG_ERR_INVALID_ARGUMENT
    assert densify(c=bad_cov) == B.UG_ERR_INVALID_ARGUMENT
    assert densify(params=None) == B.UG_ERR_INVALID_ARGUMENT
    assert densify(scratch=None) == B.UG_ERR_INVALID_ARGUMENT
    for field, value in (("min_opacity", 0.0), ("min_opacity", 1.0), ("split_factor", 1.0),
                         ("size_threshold", 0.0), ("grad_threshold", float("nan"))):
        d = B.ug_densify_config()
        lib.ug_densify_config_default(ctypes.byref(d))
        setattr(d, field, value)
        assert densify(d=d) == B.UG_ERR_INVALID_ARGUMENT, field
    assert densify(sbytes=need - 1) == B.UG_ERR_WORKSPACE_TOO_SMALL
