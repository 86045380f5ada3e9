"""ctypes binding of libug (include/ug.h): the same entry points, names and
argument order, with torch tensors in place of raw device pointers.

This module only marshals arguments; every step of the rasterizer runs in
the CUDA library. If the library cannot be loaded, every call raises: there
is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build_lib

UG_OK = 0
UG_ERR_INVALID_ARGUMENT = 1
UG_ERR_WORKSPACE_TOO_SMALL = 2
UG_ERR_CAPACITY = 3
UG_ERR_CUDA = 4
UG_ERR_TIMEOUT = 5
UG_ERR_NOT_SUPPORTED = 6
UG_ERR_INVALID_PLANE = 7
UG_ERR_INTERNAL = 8

UG_COV_TRI = 0
UG_COV_SCALE_ROT = 1
UG_CUTOFF_BOX = 0
UG_CUTOFF_BOX_AND_ELLIPSOID = 1
UG_MSE_LOSS_FLOATS = 1025

# Every exported symbol declared in include/ug.h.
EXPORTS = (
    "ug_version", "ug_status_string", "ug_num_variants", "ug_num_variants_bwd",
    "ug_config_default", "ug_plan_init",
    "ug_preprocess", "ug_bin_sort", "ug_render", "ug_mse_loss_grad", "ug_render_backward",
    "ug_adam_step", "ug_read_status", "ug_debug_views", "ug_mse_loss_grad_static",
    "ug_mse_loss_grad_part", "ug_shard_sums", "ug_composite",
    "ug_debug_stall_pipeline",
    "ug_render_backward_raster", "ug_preprocess_backward", "ug_render_scatter",
    "ug_ssim_scratch_floats", "ug_ssim",
    "ug_densify_config_default", "ug_sample", "ug_densify_stats", "ug_densify_scratch_bytes",
    "ug_densify", "ug_l1_dssim_scratch_floats", "ug_l1_dssim_loss_grad",
)
UG_MSE_STATIC_MAX_N = 1 << 30


class UgError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class ug_config(ctypes.Structure):
    _fields_ = [("chi2", ctypes.c_float), ("beta", ctypes.c_float),
                ("alpha_bg", ctypes.c_float), ("c_bg", ctypes.c_float),
                ("cutoff", ctypes.c_int32), ("cov_param", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("fp64_ratio", ctypes.c_float), ("variant_bwd", ctypes.c_int32),
                ("fp32_reach", ctypes.c_float), ("reserved", ctypes.c_int32)]


class ug_densify_config(ctypes.Structure):
    _fields_ = [("grad_threshold", ctypes.c_float), ("min_opacity", ctypes.c_float),
                ("size_threshold", ctypes.c_float), ("split_factor", ctypes.c_float),
                ("reserved", ctypes.c_int32 * 4)]


class ug_plan(ctypes.Structure):
    _fields_ = [("cfg", ug_config), ("n", ctypes.c_int64), ("num_planes", ctypes.c_int32),
                ("total_tiles", ctypes.c_int32), ("total_pixels", ctypes.c_int64),
                ("record_capacity", ctypes.c_int64), ("instance_capacity", ctypes.c_int64),
                ("key_bits", ctypes.c_int32), ("sort_passes", ctypes.c_int32),
                ("chunks", ctypes.c_int64), ("workspace_bytes", ctypes.c_size_t),
                ("off", ctypes.c_size_t * 32)]


class ug_gaussians(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in
                ("mean", "tri", "log_scale", "quat", "opacity_logit", "intensity")]


class ug_gaussian_grads(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in
                ("mean", "tri", "log_scale", "quat", "opacity_logit", "intensity")]


class ug_ws_status(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("detail", ctypes.c_int32),
                ("records", ctypes.c_int64), ("instances", ctypes.c_int64),
                ("fp64_records", ctypes.c_int64), ("box_pixels", ctypes.c_int64),
                ("evaluated_pairs", ctypes.c_int64), ("evaluated_pairs_bwd", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 1)]


class ug_adam_row(ctypes.Structure):
    _fields_ = [("lr_init", ctypes.c_float), ("lr_final", ctypes.c_float),
                ("decay_steps", ctypes.c_int32), ("reserved", ctypes.c_int32)]


assert ctypes.sizeof(ug_config) == 48
assert ctypes.sizeof(ug_ws_status) == 64
assert ctypes.sizeof(ug_adam_row) == 16

_lib = None


def library_path() -> str:
    return build_lib.LIB


def load(build_if_missing: bool = True):
    """Load libug.so (building it first if it is missing and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = build_lib.LIB
    if not os.path.exists(path) or not build_lib.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"libug.so not built at {path}")
        build_lib.build()
    lib = ctypes.CDLL(path)
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    P = ctypes.POINTER
    lib.ug_version.restype = i32
    lib.ug_version.argtypes = []
    lib.ug_status_string.restype = ctypes.c_char_p
    lib.ug_status_string.argtypes = [ctypes.c_int]
    lib.ug_num_variants.restype = i32
    lib.ug_num_variants.argtypes = [i32]
    lib.ug_num_variants_bwd.restype = i32
    lib.ug_num_variants_bwd.argtypes = [i32]
    lib.ug_config_default.argtypes = [P(ug_config)]
    lib.ug_plan_init.argtypes = [P(ug_config), i64, vp, i32, i64, i64, P(ug_plan)]
    lib.ug_preprocess.argtypes = [P(ug_plan), P(ug_gaussians), vp, vp, ctypes.c_size_t, vp]
    lib.ug_bin_sort.argtypes = [P(ug_plan), vp, ctypes.c_size_t, vp]
    lib.ug_render.argtypes = [P(ug_plan), vp, ctypes.c_size_t, vp, vp, vp]
    lib.ug_mse_loss_grad.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.ug_mse_loss_grad_static.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.ug_mse_loss_grad_part.argtypes = [vp, vp, i64, i64, vp, vp, vp]
    lib.ug_shard_sums.argtypes = [vp, vp, i64, f32, f32, vp, vp]
    lib.ug_composite.argtypes = [vp, i64, f32, f32, vp, vp, vp]
    lib.ug_render_backward.argtypes = [P(ug_plan), P(ug_gaussians), vp, vp, ctypes.c_size_t, vp,
                                       vp, vp, P(ug_gaussian_grads), vp]
    lib.ug_ssim_scratch_floats.argtypes = [i32, i32, i32]
    lib.ug_ssim.argtypes = [vp, vp, i32, i32, i32, vp, ctypes.c_size_t, vp, vp, vp]
    lib.ug_render_scatter.argtypes = [P(ug_plan), vp, ctypes.c_size_t, vp, vp, vp]
    lib.ug_render_backward_raster.argtypes = [P(ug_plan), vp, ctypes.c_size_t, vp, vp, vp, vp]
    lib.ug_preprocess_backward.argtypes = [P(ug_plan), P(ug_gaussians), vp, ctypes.c_size_t,
                                           P(ug_gaussian_grads), vp]
    lib.ug_adam_step.argtypes = [vp, vp, vp, vp, i32, i64, vp, vp, f32, f32, f32, vp]
    lib.ug_read_status.argtypes = [P(ug_plan), vp, ctypes.c_size_t, vp, vp]
    lib.ug_debug_stall_pipeline.argtypes = [P(ug_plan), vp, ctypes.c_size_t, i32, vp]
    lib.ug_l1_dssim_scratch_floats.argtypes = [i32, i32, i32]
    lib.ug_l1_dssim_loss_grad.argtypes = [vp, vp, i32, i32, i32, f32, vp, ctypes.c_size_t, vp, vp,
                                          vp]
    lib.ug_densify_config_default.argtypes = [P(ug_densify_config)]
    lib.ug_sample.argtypes = [P(ug_config), vp, i64, vp, i64, vp, vp, vp]
    lib.ug_densify_stats.argtypes = [vp, i64, vp, vp]
    lib.ug_densify_scratch_bytes.argtypes = [i64]
    lib.ug_densify.argtypes = [P(ug_config), P(ug_densify_config), vp, vp, vp, i64, vp, vp, i64,
                               vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
    lib.ug_debug_views.argtypes = [P(ug_plan), vp, ctypes.c_size_t, P(vp), P(vp), P(vp), P(vp),
                                   P(vp), P(vp), P(vp), P(vp)]
    for name in EXPORTS:
        fn = getattr(lib, name)
        # an undeclared signature would pass Python ints as 32-bit C ints
        if fn.argtypes is None:
            raise RuntimeError(f"binding declares no argument types for {name}")
        if name not in ("ug_version", "ug_status_string", "ug_num_variants",
                        "ug_ssim_scratch_floats", "ug_densify_scratch_bytes",
                        "ug_l1_dssim_scratch_floats"):
            fn.restype = ctypes.c_int
    lib.ug_ssim_scratch_floats.restype = ctypes.c_size_t
    lib.ug_densify_scratch_bytes.restype = ctypes.c_size_t
    lib.ug_l1_dssim_scratch_floats.restype = ctypes.c_size_t
    _lib = lib
    return lib


def status_string(status: int) -> str:
    try:
        return load().ug_status_string(int(status)).decode()
    except Exception:  # pragma: no cover
        return f"status {status}"


def _check(status: int, what: str):
    if status != UG_OK:
        raise UgError(status, what)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ entry points
def ug_version() -> int:
    return int(load().ug_version())


def ug_num_variants(tile: int) -> int:
    return int(load().ug_num_variants(tile))


def ug_num_variants_bwd(tile: int) -> int:
    return int(load().ug_num_variants_bwd(tile))


def ug_config_default() -> ug_config:
    cfg = ug_config()
    _check(load().ug_config_default(ctypes.byref(cfg)), "ug_config_default")
    return cfg


def ug_plan_init(cfg: ug_config, n: int, host_planes: np.ndarray, record_capacity: int,
                 instance_capacity: int) -> ug_plan:
    host_planes = np.ascontiguousarray(host_planes)
    plan = ug_plan()
    st = load().ug_plan_init(ctypes.byref(cfg), int(n), host_planes.ctypes.data, len(host_planes),
                             int(record_capacity), int(instance_capacity), ctypes.byref(plan))
    _check(st, "ug_plan_init")
    return plan


def ug_preprocess(plan: ug_plan, gaussians: ug_gaussians, d_planes, ws, stream=None):
    _check(load().ug_preprocess(ctypes.byref(plan), ctypes.byref(gaussians), _ptr(d_planes),
                                _ptr(ws), ws.numel(), _stream(stream)), "ug_preprocess")


def ug_bin_sort(plan: ug_plan, ws, stream=None):
    _check(load().ug_bin_sort(ctypes.byref(plan), _ptr(ws), ws.numel(), _stream(stream)),
           "ug_bin_sort")


def ug_render(plan: ug_plan, ws, image, alpha, stream=None):
    _check(load().ug_render(ctypes.byref(plan), _ptr(ws), ws.numel(), _ptr(image), _ptr(alpha),
                            _stream(stream)), "ug_render")


def ug_mse_loss_grad(image, target, n: int, grad_image, loss, stream=None):
    _check(load().ug_mse_loss_grad(_ptr(image), _ptr(target), int(n), _ptr(grad_image),
                                   _ptr(loss), _stream(stream)), "ug_mse_loss_grad")


def ug_mse_loss_grad_part(image, target, n: int, n_total: int, grad_image, loss, stream=None):
    """MSE part of a larger image set: sums divided by n_total instead of n."""
    _check(load().ug_mse_loss_grad_part(_ptr(image), _ptr(target), int(n), int(n_total),
                                        _ptr(grad_image), _ptr(loss), _stream(stream)),
           "ug_mse_loss_grad_part")


def ug_shard_sums(image, alpha, n: int, alpha_bg: float, c_bg: float, sums, stream=None):
    """Partial sums (S_a, S_c) per pixel of a Gaussian shard's render."""
    _check(load().ug_shard_sums(_ptr(image), _ptr(alpha), int(n), float(alpha_bg), float(c_bg),
                                _ptr(sums), _stream(stream)), "ug_shard_sums")


def ug_composite(sums, n: int, alpha_bg: float, c_bg: float, image, alpha, stream=None):
    """Image and alpha from the summed (S_a, S_c) of all shards."""
    _check(load().ug_composite(_ptr(sums), int(n), float(alpha_bg), float(c_bg), _ptr(image),
                               _ptr(alpha), _stream(stream)), "ug_composite")


def ug_mse_loss_grad_static(image, target, n: int, grad_image, loss, stream=None):
    """MSE loss and gradient with the partial sums in the library's own static
    device array: `loss` is one device float; nothing is allocated."""
    _check(load().ug_mse_loss_grad_static(_ptr(image), _ptr(target), int(n), _ptr(grad_image),
                                          _ptr(loss), _stream(stream)), "ug_mse_loss_grad_static")


def ug_render_backward(plan: ug_plan, gaussians: ug_gaussians, d_planes, ws, image, alpha,
                       grad_image, grads: ug_gaussian_grads, stream=None):
    _check(load().ug_render_backward(ctypes.byref(plan), ctypes.byref(gaussians), _ptr(d_planes),
                                     _ptr(ws), ws.numel(), _ptr(image), _ptr(alpha),
                                     _ptr(grad_image), ctypes.byref(grads), _stream(stream)),
           "ug_render_backward")


def ug_ssim_scratch_floats(P: int, W: int, H: int) -> int:
    return int(load().ug_ssim_scratch_floats(int(P), int(W), int(H)))


def ug_ssim(image, target, P: int, W: int, H: int, scratch, ssim=None, psnr=None, stream=None):
    """Per-image mean SSIM and PSNR of P images of W x H pixels (device tensors)."""
    _check(load().ug_ssim(_ptr(image), _ptr(target), int(P), int(W), int(H), _ptr(scratch),
                          scratch.numel(), _ptr(ssim), _ptr(psnr), _stream(stream)), "ug_ssim")


def ug_render_scatter(plan: ug_plan, ws, image, alpha, stream=None):
    _check(load().ug_render_scatter(ctypes.byref(plan), _ptr(ws), ws.numel(), _ptr(image),
                                    _ptr(alpha), _stream(stream)), "ug_render_scatter")


def ug_render_backward_raster(plan: ug_plan, ws, image, alpha, grad_image, stream=None):
    _check(load().ug_render_backward_raster(ctypes.byref(plan), _ptr(ws), ws.numel(), _ptr(image),
                                            _ptr(alpha), _ptr(grad_image), _stream(stream)),
           "ug_render_backward_raster")


def ug_preprocess_backward(plan: ug_plan, gaussians: ug_gaussians, ws,
                           grads: ug_gaussian_grads, stream=None):
    _check(load().ug_preprocess_backward(ctypes.byref(plan), ctypes.byref(gaussians), _ptr(ws),
                                         ws.numel(), ctypes.byref(grads), _stream(stream)),
           "ug_preprocess_backward")


def ug_adam_step(param, grad, exp_avg, exp_avg_sq, rows: int, n: int, d_rows, d_step,
                 beta1: float, beta2: float, eps: float, stream=None):
    _check(load().ug_adam_step(_ptr(param), _ptr(grad), _ptr(exp_avg), _ptr(exp_avg_sq),
                               int(rows), int(n), _ptr(d_rows), _ptr(d_step), float(beta1),
                               float(beta2), float(eps), _stream(stream)), "ug_adam_step")


def ug_l1_dssim_scratch_floats(P: int, W: int, H: int) -> int:
    return int(load().ug_l1_dssim_scratch_floats(int(P), int(W), int(H)))


def ug_l1_dssim_loss_grad(image, target, P: int, W: int, H: int, lam: float, scratch, grad, loss,
                          stream=None):
    """L = (1 - lam) mean|x - y| + lam (1 - SSIM) into loss[0], dL/dx into grad."""
    _check(load().ug_l1_dssim_loss_grad(_ptr(image), _ptr(target), int(P), int(W), int(H),
                                        float(lam), _ptr(scratch), scratch.numel(), _ptr(grad),
                                        _ptr(loss), _stream(stream)), "ug_l1_dssim_loss_grad")


def ug_densify_config_default() -> ug_densify_config:
    dc = ug_densify_config()
    _check(load().ug_densify_config_default(ctypes.byref(dc)), "ug_densify_config_default")
    return dc


def ug_sample(cfg: ug_config, params, n: int, idx, m: int, z, y, stream=None):
    """y[3][m] = mu + L^-T z (or mu + R S z) for the Gaussians idx[m] of params[rows][n]."""
    _check(load().ug_sample(ctypes.byref(cfg), _ptr(params), int(n), _ptr(idx), int(m), _ptr(z),
                            _ptr(y), _stream(stream)), "ug_sample")


def ug_densify_stats(grad_mean, n: int, stats, stream=None):
    _check(load().ug_densify_stats(_ptr(grad_mean), int(n), _ptr(stats), _stream(stream)),
           "ug_densify_stats")


def ug_densify_scratch_bytes(n: int) -> int:
    return int(load().ug_densify_scratch_bytes(int(n)))


def ug_densify(cfg: ug_config, dc: ug_densify_config, params, exp_avg, exp_avg_sq, n: int, stats,
               z, capacity: int, params_out, exp_avg_out, exp_avg_sq_out, n_out, scratch,
               stream=None):
    _check(load().ug_densify(ctypes.byref(cfg), ctypes.byref(dc), _ptr(params), _ptr(exp_avg),
                             _ptr(exp_avg_sq), int(n), _ptr(stats), _ptr(z), int(capacity),
                             _ptr(params_out), _ptr(exp_avg_out), _ptr(exp_avg_sq_out),
                             _ptr(n_out), _ptr(scratch), scratch.numel() * scratch.element_size(),
                             _stream(stream)), "ug_densify")


def ug_read_status(plan: ug_plan, ws, out, stream=None):
    """Copy the workspace status into `out` (a 64-byte pinned host or device tensor)."""
    _check(load().ug_read_status(ctypes.byref(plan), _ptr(ws), ws.numel(), out.data_ptr(),
                                 _stream(stream)), "ug_read_status")


def ug_debug_stall_pipeline(plan: ug_plan, ws, on: bool, stream=None):
    """Test hook: with on, the rasterizers' producers issue nothing, so their
    consumers' bounded waits run out (UG_ERR_TIMEOUT in the status)."""
    _check(load().ug_debug_stall_pipeline(ctypes.byref(plan), _ptr(ws), ws.numel(), int(bool(on)),
                                          _stream(stream)), "ug_debug_stall_pipeline")


def ug_debug_views(plan: ug_plan, ws):
    ptrs = [ctypes.c_void_p() for _ in range(8)]
    _check(load().ug_debug_views(ctypes.byref(plan), _ptr(ws), ws.numel(),
                                 *[ctypes.byref(p) for p in ptrs]), "ug_debug_views")
    return [p.value for p in ptrs]
