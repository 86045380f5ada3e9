"""Seeded synthetic inputs: Gaussian sets and probe-plane poses.

This module only draws random numbers and packs arrays. It holds none of the
rasterizer's arithmetic, and it is the one module that both the FP64 oracle
side (tests, CPU baseline) and the CUDA side (binding, bench) use.

The paper's datasets (fetal-brain volumes of 160^3 voxels at 0.6 mm, and
freehand sweeps of 160x160 frames; Sec. 5.1) are not available, so every
input here is synthetic: the cube [-1, 1]^3 stands in for the imaged volume
and each probe plane spans 2 x 2 units; the Gaussians' means start uniform over the
imaged volume, as in the paper's initialisation (Sec. 4.5).

Gaussian parameters are returned in "row" layout (one row per scalar
parameter, n columns), float32, which is the structure-of-arrays layout the
device library reads:

  mean        (3, n)
  tri         (6, n)  l11, l21, l31, l22, l32, l33 of the triangular factor
  log_scale   (3, n)  scale/rotation front-end
  quat        (4, n)  w, x, y, z (not necessarily unit)
  logit       (n,)    opacity logit, alpha = sigmoid(logit)
  intensity   (n,)    scalar ultrasound intensity c_i

Planes are returned as a dict of arrays (origin, u, v, pitch, size, offset).
"""
from __future__ import annotations

import numpy as np

# Field order of one plane record in the C ABI (ug_plane, 64 bytes).
PLANE_DTYPE = np.dtype(
    [
        ("origin", "<f4", (3,)),
        ("u", "<f4", (3,)),
        ("v", "<f4", (3,)),
        ("pitch_u", "<f4"),
        ("pitch_v", "<f4"),
        ("width", "<i4"),
        ("height", "<i4"),
        ("reserved", "<i4"),
        ("pixel_offset", "<i8"),
    ],
    align=True,
)
assert PLANE_DTYPE.itemsize == 64


def random_unit_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotations: a normalised standard-normal 4-vector, (4, n) float64."""
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    return q


def rotation_columns(q: np.ndarray) -> np.ndarray:
    """Rotation matrices of unit quaternions (w, x, y, z), shape (n, 3, 3), float64.

    Used only to orient random probe planes (their u, v axes are the first two
    columns); the Gaussians' own rotations stay quaternions.
    """
    w, x, y, z = q
    R = np.empty((q.shape[1], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def gaussians_scale_rot(rng: np.random.Generator, n: int, scale_lo: float = 0.01,
                        scale_hi: float = 0.1, logit: float = 1.0) -> dict:
    """Scale/rotation Gaussians: means U[-1,1]^3, per-axis scales log-uniform
    in [scale_lo, scale_hi], uniform random unit quaternions, intensities U[0,1].

    Draw order: mean, scale, rotation, intensity. The opacity logit is fixed
    (sigmoid(1) = 0.731 is the paper's initial opacity, Sec. 4.5).
    """
    mean = rng.uniform(-1.0, 1.0, (3, n))
    log_scale = rng.uniform(np.log(scale_lo), np.log(scale_hi), (3, n))
    quat = random_unit_quaternions(rng, n)
    intensity = rng.uniform(0.0, 1.0, n)
    return dict(
        mean=mean.astype(np.float32),
        log_scale=log_scale.astype(np.float32),
        quat=quat.astype(np.float32),
        logit=np.full(n, logit, np.float32),
        intensity=intensity.astype(np.float32),
    )


def gaussians_anisotropic(rng: np.random.Generator, n: int, smax_lo: float = 0.01,
                          smax_hi: float = 0.1, ratio_max: float = 1e4) -> dict:
    """Extreme-anisotropy Gaussians: the largest axis s_max is log-uniform in
    [smax_lo, smax_hi]; each of the other two axes is s_max / r with an
    independent r log-uniform in [1, ratio_max]. Axis order is shuffled.

    Draw order: mean, scale (s_max, r1, r2, axis permutation), rotation,
    intensity.
    """
    mean = rng.uniform(-1.0, 1.0, (3, n))
    log_smax = rng.uniform(np.log(smax_lo), np.log(smax_hi), n)
    log_r = rng.uniform(0.0, np.log(ratio_max), (2, n))
    ls = np.stack([log_smax, log_smax - log_r[0], log_smax - log_r[1]])
    perm = np.argsort(rng.uniform(size=(3, n)), axis=0)
    ls = np.take_along_axis(ls, perm, axis=0)
    quat = random_unit_quaternions(rng, n)
    intensity = rng.uniform(0.0, 1.0, n)
    return dict(
        mean=mean.astype(np.float32),
        log_scale=ls.astype(np.float32),
        quat=quat.astype(np.float32),
        logit=np.ones(n, np.float32),
        intensity=intensity.astype(np.float32),
    )


def gaussians_paper_init(rng: np.random.Generator, n: int) -> dict:
    """The paper's initialisation (Sec. 4.5): means uniform in the volume,
    c_i = 0.5, opacity 0.731 (logit 1), and the six triangular parameters
    uniform in [4, 5)."""
    mean = rng.uniform(-1.0, 1.0, (3, n))
    tri = rng.uniform(4.0, 5.0, (6, n))
    return dict(
        mean=mean.astype(np.float32),
        tri=tri.astype(np.float32),
        logit=np.ones(n, np.float32),
        intensity=np.full(n, 0.5, np.float32),
    )


def scale_rot_to_tri(g: dict, beta: float) -> dict:
    """Re-express scale/rotation draws in the triangular precision
    parametrisation: the lower Cholesky factor of R diag(s^-2) R^T (numpy's
    library Cholesky in float64), with the diagonal stored as
    sqrt(L_kk - beta). This is input preparation for tests and benches that
    want the triangular front-end with a known distribution of shapes."""
    q = g["quat"].astype(np.float64)
    q = q / np.linalg.norm(q, axis=0, keepdims=True)
    R = rotation_columns(q)
    inv_s2 = np.exp(-2.0 * g["log_scale"].astype(np.float64)).T  # (n, 3)
    prec = np.einsum("nij,nj,nkj->nik", R, inv_s2, R)
    L = np.linalg.cholesky(prec)
    diag = np.sqrt(np.maximum(np.stack([L[:, 0, 0], L[:, 1, 1], L[:, 2, 2]]) - beta, 0.0))
    tri = np.stack([diag[0], L[:, 1, 0], L[:, 2, 0], diag[1], L[:, 2, 1], diag[2]])
    out = {k: v for k, v in g.items() if k not in ("log_scale", "quat")}
    out["tri"] = tri.astype(np.float32)
    return out


def _pack_planes(origin, u, v, sizes, extent=2.0) -> dict:
    P = len(sizes)
    size = np.asarray(sizes, np.int64).reshape(P, 2)  # (width, height)
    pitch = np.stack([extent / size[:, 0], extent / size[:, 1]], axis=1)
    npx = size[:, 0] * size[:, 1]
    offset = np.concatenate([[0], np.cumsum(npx)[:-1]]).astype(np.int64)
    return dict(
        origin=np.asarray(origin, np.float32).reshape(P, 3),
        u=np.asarray(u, np.float32).reshape(P, 3),
        v=np.asarray(v, np.float32).reshape(P, 3),
        pitch=pitch.astype(np.float32),
        size=size,
        offset=offset,
        total_pixels=int(npx.sum()),
    )


def planes_random(rng: np.random.Generator, sizes, origin_range: float = 0.5,
                  extent: float = 2.0) -> dict:
    """Planes with origins uniform in [-origin_range, origin_range]^3 and
    uniformly random orientations; each spans extent x extent units.
    ``sizes`` is a list of (width, height) pixel counts."""
    P = len(sizes)
    origin = rng.uniform(-origin_range, origin_range, (P, 3))
    R = rotation_columns(random_unit_quaternions(rng, P))
    return _pack_planes(origin, R[:, :, 0], R[:, :, 1], sizes, extent)


def _axis_rotation(axis: np.ndarray, angle: float) -> np.ndarray:
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * (K @ K)


def planes_sweep_pool(rng: np.random.Generator, pool: int = 160, size=(256, 256),
                      travel: float = 0.9, jitter_deg: float = 5.0,
                      extent: float = 2.0) -> dict:
    """A smooth sweep of probe poses through the volume: origins move at
    constant velocity along a random unit direction d from -travel*d to
    +travel*d; the base frame has normal d; every pose is then turned by
    independent angles U(-jitter, +jitter) about its own u and v axes
    (a stand-in for the paper's 160-slice sweeps with +-5 degree jitter,
    Sec. 5.2)."""
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    a = np.array([1.0, 0.0, 0.0]) if abs(d[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u0 = np.cross(a, d)
    u0 /= np.linalg.norm(u0)
    v0 = np.cross(d, u0)
    origins, us, vs = [], [], []
    jit = np.deg2rad(jitter_deg)
    for k in range(pool):
        t = -travel + 2.0 * travel * k / max(pool - 1, 1)
        Ru = _axis_rotation(u0, rng.uniform(-jit, jit))
        Rv = _axis_rotation(v0, rng.uniform(-jit, jit))
        Rj = Rv @ Ru
        origins.append(t * d)
        us.append(Rj @ u0)
        vs.append(Rj @ v0)
    return _pack_planes(np.array(origins), np.array(us), np.array(vs), [size] * pool, extent)


def planes_slices(count: int, size: int, axis: int = 2, extent: float = 2.0) -> dict:
    """count linearly spaced slices through the cube [-1, 1]^3 normal to the
    given axis (2 axial, 1 coronal, 0 sagittal), at the centres of count equal
    layers, each spanning the cube's cross-section with size x size pixels (a
    stand-in for the paper's evaluation on linearly spaced axial, coronal and
    sagittal cross-sections of a 160^3 volume, Sec. 5.1)."""
    e = np.eye(3)
    u, v = {2: (e[0], e[1]), 1: (e[0], e[2]), 0: (e[1], e[2])}[axis]
    t = -1.0 + (np.arange(count) + 0.5) * 2.0 / count
    origin = np.zeros((count, 3))
    origin[:, axis] = t
    return _pack_planes(origin, np.tile(u, (count, 1)), np.tile(v, (count, 1)),
                        [(size, size)] * count, extent)


def concat_planes(*sets) -> dict:
    """Several plane sets as one (re-packed with fresh pixel offsets)."""
    return _pack_planes(np.concatenate([s["origin"] for s in sets]),
                        np.concatenate([s["u"] for s in sets]),
                        np.concatenate([s["v"] for s in sets]),
                        [tuple(x) for s in sets for x in s["size"]], extent=1.0) | {
                            "pitch": np.concatenate([s["pitch"] for s in sets])}


def select_planes(planes: dict, idx) -> dict:
    """Sub-batch of planes (re-packed with fresh pixel offsets)."""
    idx = np.asarray(idx)
    return _pack_planes(planes["origin"][idx], planes["u"][idx], planes["v"][idx],
                        [tuple(s) for s in planes["size"][idx]],
                        extent=1.0) | {"pitch": planes["pitch"][idx].copy()}


def planes_to_struct(planes: dict) -> np.ndarray:
    """Pack a plane dict into the C ABI's ug_plane array layout."""
    P = len(planes["size"])
    arr = np.zeros(P, PLANE_DTYPE)
    arr["origin"] = planes["origin"]
    arr["u"] = planes["u"]
    arr["v"] = planes["v"]
    arr["pitch_u"] = planes["pitch"][:, 0]
    arr["pitch_v"] = planes["pitch"][:, 1]
    arr["width"] = planes["size"][:, 0]
    arr["height"] = planes["size"][:, 1]
    arr["pixel_offset"] = planes["offset"]
    return arr


def target_images(rng: np.random.Generator, total_pixels: int) -> np.ndarray:
    """Uniform random target intensities in [0, 1] (float32)."""
    return rng.uniform(0.0, 1.0, total_pixels).astype(np.float32)


# ---------------------------------------------------------------- workloads
# Named workloads. Each returns (gaussians, planes, cov_param) from its own
# seeded default_rng stream.

RAGGED_SIZES = (128, 192, 256, 384, 512)


def workload_fwd_2k(seed: int = 0):
    """2,000 scale/rotation Gaussians, 4 random planes of 64x64 (seed 0)."""
    rng = np.random.default_rng(seed)
    g = gaussians_scale_rot(rng, 2000)
    planes = planes_random(rng, [(64, 64)] * 4)
    return g, planes


def workload_grad_50k(seed: int = 0, n: int = 50_000, P: int = 16, size: int = 256):
    """50,000 scale/rotation Gaussians, 16 random planes of 256x256."""
    rng = np.random.default_rng(seed)
    g = gaussians_scale_rot(rng, n)
    planes = planes_random(rng, [(size, size)] * P)
    return g, planes


def workload_aniso_1m(seed: int = 0, n: int = 1_000_000, P: int = 64):
    """1,000,000 extreme-anisotropy Gaussians; 64 planes whose square sizes are
    drawn uniformly from {128, 192, 256, 384, 512}."""
    rng = np.random.default_rng(seed)
    g = gaussians_anisotropic(rng, n)
    sizes = rng.choice(np.array(RAGGED_SIZES), size=P)
    planes = planes_random(rng, [(int(s), int(s)) for s in sizes])
    return g, planes


def workload_train_200k(seed: int = 0, n: int = 200_000, hidden_n: int = 100_000,
                        pool: int = 160, size: int = 256):
    """Training workload: 200,000 Gaussians in the paper's initialisation
    (Sec. 4.5), a hidden 100,000-Gaussian target volume drawn with seed 2 from
    the fwd_2k distributions, and a pool of 160 sweep poses of size x size
    pixels; a training step takes 32 consecutive poses of the pool (cyclic).
    Returns (gaussians, pose pool, hidden gaussians)."""
    rng = np.random.default_rng(seed)
    g = gaussians_paper_init(rng, n)
    poses = planes_sweep_pool(rng, pool, (size, size))
    hidden = gaussians_scale_rot(np.random.default_rng(2), hidden_n)
    return g, poses, hidden


def workload_recon(seed: int = 0, n: int = 3_000_000, hidden_n: int = 1_000_000,
                   train_pool: int = 320, held_out: int = 128, size: int = 256,
                   poses: str = "random"):
    """Reconstruction workload: n Gaussians in the paper's initialisation, a
    hidden target volume of hidden_n Gaussians drawn with seed 3 from the
    fwd_2k distributions, and size x size poses.

    poses "random": a pool of train_pool random training poses (seed 5) and
    held_out random evaluation poses (seed 4). poses "slices" (the paper's
    ideal setting, Sec. 5.1): train_pool linearly spaced axial slices for
    training, and held_out linearly spaced slices along each of the three axes
    (axial, coronal, sagittal) for evaluation.
    Returns (gaussians, hidden gaussians, training poses, evaluation poses)."""
    g = gaussians_paper_init(np.random.default_rng(seed), n)
    hidden = gaussians_scale_rot(np.random.default_rng(3), hidden_n)
    if poses == "slices":
        train = planes_slices(train_pool, size, axis=2)
        test = concat_planes(*(planes_slices(held_out, size, axis=a) for a in (2, 1, 0)))
        return g, hidden, train, test
    train = planes_random(np.random.default_rng(5), [(size, size)] * train_pool)
    test = planes_random(np.random.default_rng(4), [(size, size)] * held_out)
    return g, hidden, train, test
