"""FP64 CPU oracle of the UltraGauss plane rasterizer (test infrastructure).

Only tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg use
this package. It shares no code with the CUDA path: the arithmetic is in
``ug_oracle.c`` (plain C, FP64, OpenMP over pixels or Gaussians) and
``adam.py`` (NumPy FP64); this module only marshals arrays.

Functions and what they follow (section / equation of the paper):

* :func:`render`      Eq. alpha-combine, Eq. colour-combine, Eq. us-render,
                      Eq. mahalanobis-3d, Eq. ellipsoid / Eq. boundary cut-off
                      with the two-phase rule of Sec. 4.4; dense (every pixel x
                      every Gaussian) or scatter (same numbers, fewer pairs).
* :func:`render_grad` analytic FP64 gradient of the same formulas (Sec. 4.5).
* :func:`geometry`    probe-frame means, box half-extents, phase-1 flags and
                      exact pixel boxes (Sec. 4.3 - 3.4).
* :func:`covariance`  Eq. tri-param (triangular precision) or the
                      scale/rotation form quoted in Sec. 4.2.
* :func:`contrib`     the included pairs of one Gaussian (for finite
                      differences).
* :mod:`oracle.adam`  Adam (Sec. 4.5 uses Adam; textbook update).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ug_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

CHI2_95_PRINTED = 7.815  # Sec. 4.3: chi^2 for 3 DoF at p = 95 %, as printed


@dataclass
class Config:
    """Cut-off and image-formation constants: chi2 = 7.815 as printed (Sec. 4.3);
    beta, alpha_bg and c_bg are not printed in the paper and take the values
    1e-4, 1e-3 and 0; cutoff 0 is the paper's box, 1 adds the ellipsoid."""
    chi2: float = CHI2_95_PRINTED
    beta: float = 1e-4
    alpha_bg: float = 1e-3
    c_bg: float = 0.0
    cutoff: int = 0      # 0: box (paper), 1: box and ellipsoid
    cov_param: int = 0   # 0: triangular, 1: scale + quaternion
    amb: float = 1e-5      # relative ambiguity margin for FP32 decisions
    amb_abs: float = 2e-6  # absolute margin (world units): FP32 rounding of m and h


class _CConfig(ctypes.Structure):
    _fields_ = [
        ("chi2", ctypes.c_double), ("beta", ctypes.c_double),
        ("alpha_bg", ctypes.c_double), ("c_bg", ctypes.c_double),
        ("amb", ctypes.c_double), ("amb_abs", ctypes.c_double), ("cutoff", ctypes.c_int32),
        ("cov_param", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        lib.or_render.restype = i64
        lib.or_render.argtypes = [i64, P, P, P, P, i32, P, P, P, i32, P, P, P, P, P, i32]
        lib.or_geometry.restype = None
        lib.or_geometry.argtypes = [i64, P, P, P, P, i32, P, P, P, P, P, P, P, P]
        lib.or_render_grad.restype = None
        lib.or_render_grad.argtypes = [i64, P, P, P, P, i32, P, P, P, P, P, P, P, i64, P, P, P, P,
                                       i32]
        lib.or_contrib.restype = i64
        lib.or_contrib.argtypes = [P, P, ctypes.c_double, ctypes.c_double, i32, P, P, P, P, P, i64]
        lib.or_covariance.restype = None
        lib.or_covariance.argtypes = [i64, P, P, P, P]
        lib.or_max_threads.restype = i32
        _lib_handle = lib
    return _lib_handle


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cfg(cfg: Config) -> _CConfig:
    return _CConfig(cfg.chi2, cfg.beta, cfg.alpha_bg, cfg.c_bg, cfg.amb, cfg.amb_abs, cfg.cutoff,
                    cfg.cov_param)


def max_threads() -> int:
    return int(_lib().or_max_threads())


def covp_rows(g: dict, cov_param: int) -> np.ndarray:
    """Covariance parameters as an (n, 6|7) float64 array in oracle order."""
    if cov_param == 0:
        return np.ascontiguousarray(np.asarray(g["tri"], np.float64).T)
    return np.ascontiguousarray(
        np.concatenate([np.asarray(g["log_scale"], np.float64), np.asarray(g["quat"], np.float64)]).T)


def _gauss(g: dict, cov_param: int):
    mean = np.ascontiguousarray(np.asarray(g["mean"], np.float64).T)
    covp = covp_rows(g, cov_param)
    logit = np.ascontiguousarray(np.asarray(g["logit"], np.float64))
    inten = np.ascontiguousarray(np.asarray(g["intensity"], np.float64))
    return mean, covp, logit, inten


def _planes(planes: dict):
    P = len(planes["size"])
    pl = np.zeros((P, 11), np.float64)
    pl[:, 0:3] = planes["origin"]
    pl[:, 3:6] = planes["u"]
    pl[:, 6:9] = planes["v"]
    pl[:, 9:11] = planes["pitch"]
    sz = np.zeros((P, 3), np.int64)
    sz[:, 0:2] = planes["size"]
    sz[:, 2] = planes["offset"]
    total = int((sz[:, 0] * sz[:, 1]).sum()) if P else 0
    total = max(total, int((sz[:, 2] + sz[:, 0] * sz[:, 1]).max()) if P else 0)
    return P, np.ascontiguousarray(pl), np.ascontiguousarray(sz), total


def render(g: dict, planes: dict, cfg: Config, mode: str = "scatter", threads: int = 0) -> dict:
    """Render all planes. Returns image, alpha (= sum w + a_bg), sa, sc, amb
    (FP64 per pixel) and the number of included pairs."""
    mean, covp, logit, inten = _gauss(g, cfg.cov_param)
    P, pl, sz, total = _planes(planes)
    out = {k: np.zeros(total, np.float64) for k in ("image", "alpha", "sa", "sc", "amb")}
    pairs = _lib().or_render(len(logit), _ptr(mean), _ptr(covp), _ptr(logit), _ptr(inten), P,
                             _ptr(pl), _ptr(sz), ctypes.byref(_cfg(cfg)),
                             0 if mode == "dense" else 1, _ptr(out["image"]), _ptr(out["alpha"]),
                             _ptr(out["sa"]), _ptr(out["sc"]), _ptr(out["amb"]), threads)
    out["pairs"] = int(pairs)
    return out


def geometry(g: dict, planes: dict, cfg: Config) -> dict:
    """Per (plane, Gaussian): visible, amb_plane, m (3), h (3), box (j0, j1,
    i0, i1; empty when j0 > j1 or i0 > i1). Arrays shaped (P, n, ...)."""
    mean, covp, logit, inten = _gauss(g, cfg.cov_param)
    P, pl, sz, _ = _planes(planes)
    n = len(logit)
    vis = np.zeros(P * n, np.int32)
    amb = np.zeros(P * n, np.int32)
    m = np.zeros(P * n * 3, np.float64)
    h = np.zeros(P * n * 3, np.float64)
    box = np.zeros(P * n * 4, np.int64)
    _lib().or_geometry(n, _ptr(mean), _ptr(covp), _ptr(logit), _ptr(inten), P, _ptr(pl), _ptr(sz),
                       ctypes.byref(_cfg(cfg)), _ptr(vis), _ptr(amb), _ptr(m), _ptr(h), _ptr(box))
    return dict(visible=vis.reshape(P, n).astype(bool), amb_plane=amb.reshape(P, n).astype(bool),
                m=m.reshape(P, n, 3), h=h.reshape(P, n, 3), box=box.reshape(P, n, 4))


def render_grad(g: dict, planes: dict, cfg: Config, image, alpha, grad_image, subset=None,
                threads: int = 0, with_ambiguity: bool = False, with_pre: bool = False):
    """Analytic FP64 gradient. Returns (grads, grads_abs), each (k, nparam)
    with nparam = 3 + (6|7) + 2 in the order mean, covp, logit, intensity;
    grads_abs is the sum of |per-pair term|. with_ambiguity=True also returns a
    (k,) bool array: the Gaussian has an inclusion decision within the
    ambiguity margin. with_pre=True also returns (last) the same sums with
    |c - C| in dL/dw = G (c - C) / alpha replaced by |c| + |C|: the size of the
    per-pair terms before the cancellation in c - C."""
    mean, covp, logit, inten = _gauss(g, cfg.cov_param)
    P, pl, sz, _ = _planes(planes)
    nc = 6 if cfg.cov_param == 0 else 7
    npar = 3 + nc + 2
    image = np.ascontiguousarray(image, np.float64)
    alpha = np.ascontiguousarray(alpha, np.float64)
    grad_image = np.ascontiguousarray(grad_image, np.float64)
    if subset is None:
        k = len(logit)
        sub_ptr, nsub = None, 0
    else:
        subset = np.ascontiguousarray(subset, np.int64)
        k = len(subset)
        sub_ptr, nsub = _ptr(subset), k
    grads = np.zeros((k, npar), np.float64)
    gabs = np.zeros((k, npar), np.float64)
    gpre = np.zeros((k, npar), np.float64) if with_pre else None
    amb = np.zeros(k, np.int32)
    _lib().or_render_grad(len(logit), _ptr(mean), _ptr(covp), _ptr(logit), _ptr(inten), P,
                          _ptr(pl), _ptr(sz), ctypes.byref(_cfg(cfg)), _ptr(image), _ptr(alpha),
                          _ptr(grad_image), sub_ptr, nsub, _ptr(grads), _ptr(gabs),
                          _ptr(gpre) if with_pre else None, _ptr(amb), threads)
    out = (grads, gabs) + ((amb.astype(bool),) if with_ambiguity else ())
    return out + ((gpre,) if with_pre else ())


def contrib(mean3, covp_row, logit: float, intensity: float, planes: dict, cfg: Config):
    """(pixel indices, weights) of the included pairs of one Gaussian."""
    P, pl, sz, _ = _planes(planes)
    mean3 = np.ascontiguousarray(mean3, np.float64)
    covp_row = np.ascontiguousarray(covp_row, np.float64)
    cap = 1 << 16
    while True:
        pix = np.zeros(cap, np.int64)
        w = np.zeros(cap, np.float64)
        cnt = _lib().or_contrib(_ptr(mean3), _ptr(covp_row), float(logit), float(intensity), P,
                                _ptr(pl), _ptr(sz), ctypes.byref(_cfg(cfg)), _ptr(pix), _ptr(w), cap)
        if cnt <= cap:
            return pix[:cnt], w[:cnt]
        cap = int(cnt)


def covariance(covp: np.ndarray, cfg: Config):
    """World-frame (precision, covariance) of each Gaussian, (n, 3, 3) each.
    ``covp`` is (n, 6|7) in oracle order (see :func:`covp_rows`)."""
    covp = np.ascontiguousarray(covp, np.float64)
    n = covp.shape[0]
    prec = np.zeros((n, 9))
    cov = np.zeros((n, 9))
    _lib().or_covariance(n, _ptr(covp), ctypes.byref(_cfg(cfg)), _ptr(prec), _ptr(cov))
    return prec.reshape(n, 3, 3), cov.reshape(n, 3, 3)


def mse_loss_grad(image, target):
    """L = mean((C - T)^2) and dL/dC = 2 (C - T) / n_px (FP64)."""
    image = np.asarray(image, np.float64)
    target = np.asarray(target, np.float64)
    d = image - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def param_names(cov_param: int):
    cov = ["l11", "l21", "l31", "l22", "l32", "l33"] if cov_param == 0 else \
        ["log_s0", "log_s1", "log_s2", "qw", "qx", "qy", "qz"]
    return ["mu0", "mu1", "mu2"] + cov + ["logit", "intensity"]


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
