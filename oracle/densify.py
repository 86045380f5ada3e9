"""Resampling and the densify / prune step in NumPy (test infrastructure; only
tests, the smoke check and the bench's CPU legs use it).

Sampling (Sec. 4.2): with the triangular precision factor, Sigma^-1 = L L^T,
L = [[l11^2 + beta, 0, 0], [l21, l22^2 + beta, 0], [l31, l32, l33^2 + beta]],
a draw of N(mu, Sigma) is y = mu + L^-T z with z standard normal: Sigma =
L^-T L^-1, so Cov(L^-T z) = Sigma. Here w = L^-T z is the solution of the
upper-triangular system L^T w = z, by back substitution in FP64. For the
scale/rotation front-end Sigma = R S^2 R^T and y = mu + R S z.

Densify / prune (Sec. 4.5 takes the heuristics over from Kerbl et al. without
stating them; the reading is the library's, see ug_densify in ug.h): per
Gaussian, in input order,
  - prune  when sigmoid(logit) < min_opacity (decided as logit < logit(min_opacity));
  - else with mean |dL/dmu| = stats[0] / stats[1] (0 if stats[1] = 0) above the
    gradient threshold: clone (itself and an identical copy) when the extent is
    at most the size threshold, split into two children otherwise;
  - else keep.
The extent is sqrt(trace Sigma) for TRI (decided as trace Sigma > size^2) and
the largest scale for SCALE_ROT (decided on the log scales). These decisions
turn floating point into an integer, so they are taken in the kernel's FP32
with the kernel's operation order (every operation correctly rounded, none
fused); the children's parameters are FP64: means y = mu + L^-T z (two draws
from the parent), covariance Sigma / phi^2, i.e. L' = phi L (l'_kk =
sign(l_kk) sqrt(phi (l_kk^2 + beta) - beta), l'_jk = phi l_jk) or log s' =
log s - log phi; opacity and intensity copied. Kept Gaussians keep their Adam
moments, clones and children start from zero.

Parameters are [rows][n] arrays in the packed row order: mean 3, then tri 6
(l11 l21 l31 l22 l32 l33) or log_scale 3 + quat 4, then logit, intensity.
"""
from __future__ import annotations

import math

import numpy as np

COV_TRI, COV_SCALE_ROT = 0, 1


def tri_factor(p: np.ndarray, beta: float) -> np.ndarray:
    """L (3 x 3, FP64) of one Gaussian's parameter column p."""
    l11, l21, l31, l22, l32, l33 = (float(p[k]) for k in range(3, 9))
    return np.array([[l11 * l11 + beta, 0.0, 0.0],
                     [l21, l22 * l22 + beta, 0.0],
                     [l31, l32, l33 * l33 + beta]])


def back_substitute(U: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Solution w of U w = z for upper-triangular U, last row first."""
    w = np.zeros(3)
    for i in (2, 1, 0):
        w[i] = (z[i] - sum(U[i, j] * w[j] for j in range(i + 1, 3))) / U[i, i]
    return w


def rotation(q: np.ndarray) -> np.ndarray:
    w, x, y, z = (np.asarray(q, np.float64) / np.linalg.norm(np.asarray(q, np.float64)))
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def sample_offset(p: np.ndarray, cov: int, beta: float, z: np.ndarray) -> np.ndarray:
    """L^-T z (TRI) or R S z (SCALE_ROT) for one parameter column, FP64."""
    if cov == COV_TRI:
        return back_substitute(tri_factor(p, beta).T, np.asarray(z, np.float64))
    s = np.exp(np.asarray(p[3:6], np.float64))
    return rotation(p[6:10]) @ (s * np.asarray(z, np.float64))


def sample(params: np.ndarray, cov: int, beta: float, idx: np.ndarray, z: np.ndarray) -> np.ndarray:
    """y[3][m] for the Gaussians idx[m]; z is [3][m]."""
    P = np.asarray(params, np.float64)
    y = np.zeros((3, len(idx)))
    for k, i in enumerate(np.asarray(idx)):
        y[:, k] = P[0:3, i] + sample_offset(P[:, i], cov, beta, z[:, k])
    return y


def stats_update(grad_mean: np.ndarray, stats: np.ndarray) -> np.ndarray:
    """One step of the densify statistics, in the kernel's FP32 operation order."""
    g = np.asarray(grad_mean, np.float32)
    s = (g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]
    out = np.array(stats, np.float32, copy=True)
    hit = s > np.float32(0)
    out[0, hit] = out[0, hit] + np.sqrt(s[hit])
    out[1, hit] = out[1, hit] + np.float32(1)
    return out


def tri_trace32(p32: np.ndarray, beta32: np.float32) -> np.float32:
    """trace Sigma = ||L^-1||_F^2 in FP32, the kernel's operation order."""
    f = np.float32
    l11, l21, l31, l22, l32, l33 = (f(p32[k]) for k in range(3, 9))
    i00 = f(1) / (l11 * l11 + beta32)
    i11 = f(1) / (l22 * l22 + beta32)
    i22 = f(1) / (l33 * l33 + beta32)
    i10 = -((l21 * i00) * i11)
    i21 = -((l32 * i11) * i22)
    i20 = -((l31 * i00 + l32 * i10) * i22)
    t = i00 * i00
    for v in (i10, i11, i20, i21, i22):
        t = t + v * v
    return f(t)


def thresholds(dc: dict) -> dict:
    """The FP32 decision thresholds of a densify configuration."""
    p, sz, phi = float(dc["min_opacity"]), float(dc["size_threshold"]), float(dc["split_factor"])
    return dict(logit_min=np.float32(math.log(p / (1.0 - p))),
                grad=np.float32(dc["grad_threshold"]),
                size2=np.float32(sz * sz), log_size=np.float32(math.log(sz)),
                phi=phi, log_phi=math.log(phi))


def actions(params32: np.ndarray, cov: int, beta: float, stats32: np.ndarray, dc: dict) -> np.ndarray:
    """Per Gaussian: 0 prune, 1 keep, 2 clone, 3 split (FP32 decisions)."""
    t = thresholds(dc)
    P = np.asarray(params32, np.float32)
    S = np.asarray(stats32, np.float32)
    n = P.shape[1]
    row_logit = 9 if cov == COV_TRI else 10
    b32 = np.float32(beta)
    act = np.zeros(n, np.int64)
    for i in range(n):
        if P[row_logit, i] < t["logit_min"]:
            continue
        cnt = S[1, i]
        avg = S[0, i] / cnt if cnt > np.float32(0) else np.float32(0)
        if not (avg > t["grad"]):
            act[i] = 1
            continue
        if cov == COV_TRI:
            large = tri_trace32(P[:, i], b32) > t["size2"]
        else:
            large = max(P[3, i], P[4, i], P[5, i]) > t["log_size"]
        act[i] = 3 if large else 2
    return act


def densify(params: np.ndarray, exp_avg: np.ndarray, exp_avg_sq: np.ndarray, stats: np.ndarray,
            z: np.ndarray, cov: int, beta: float, dc: dict):
    """One densify / prune step. params, moments: [rows][n] (FP32 inputs); stats
    [2][n]; z [6][n]. Returns (params_out, exp_avg_out, exp_avg_sq_out) as FP64
    [rows][n_out] arrays and the per-Gaussian actions."""
    act = actions(params, cov, beta, stats, dc)
    t = thresholds(dc)
    P = np.asarray(params, np.float64)
    M = np.asarray(exp_avg, np.float64)
    V = np.asarray(exp_avg_sq, np.float64)
    rows = P.shape[0]
    cols_p, cols_m, cols_v = [], [], []
    zero = np.zeros(rows)
    for i in range(P.shape[1]):
        a = act[i]
        if a in (1, 2):
            cols_p.append(P[:, i])
            cols_m.append(M[:, i])
            cols_v.append(V[:, i])
        if a == 2:
            cols_p.append(P[:, i].copy())
            cols_m.append(zero)
            cols_v.append(zero)
        if a == 3:
            for c in range(2):
                child = P[:, i].copy()
                child[0:3] = P[0:3, i] + sample_offset(P[:, i], cov, beta, z[3 * c:3 * c + 3, i])
                if cov == COV_TRI:
                    for d in (3, 6, 8):
                        l = P[d, i]
                        lp = math.sqrt(max(t["phi"] * (l * l + beta) - beta, 0.0))
                        child[d] = -lp if l < 0 else lp
                    for d in (4, 5, 7):
                        child[d] = t["phi"] * P[d, i]
                else:
                    child[3:6] = P[3:6, i] - t["log_phi"]
                cols_p.append(child)
                cols_m.append(zero)
                cols_v.append(zero)
    if not cols_p:
        e = np.zeros((rows, 0))
        return e, e.copy(), e.copy(), act
    return (np.stack(cols_p, 1), np.stack(cols_m, 1), np.stack(cols_v, 1), act)
