"""Seeded synthetic scenes and cameras for the five rendering workloads.

This module only draws inputs: Gaussian parameters (structure of arrays,
float32) and pinhole cameras.  It holds none of the rendering arithmetic, so
both the CPU oracle and the CUDA path can consume exactly the same arrays.
Every array is produced by numpy's PCG64 generator from a fixed seed, so the
x86 development host and the aarch64 GPU host see identical bytes.

Scene layout (all float32, C-contiguous):
  mean          [3][N]    world position (metres)
  log_scale     [3][N]    per-axis log standard deviation
  quat          [4][N]    rotation (w, x, y, z), not necessarily unit length
  opacity_logit [N]       opacity = sigmoid(logit)
  sh            [16][3][N] real spherical-harmonics coefficients, degree 3,
                           coefficient index l*l + l + m, then colour channel

Camera layout: dict with width, height, fx, fy, cx, cy (pixel centres at
integer coordinates, cx = (W-1)/2), viewmat [3][4] row-major world->camera
(+x right, +y down, +z forward), campos [3], near.

The paper evaluates on Tanks&Temples, DeepBlending, Mip-NeRF360, Mill-19 and
UrbanScene3D scenes (Sec. 4.1, Table I); none of those datasets or trained
models are available, so these generators stand in for them, borrowing the
paper's resolutions (Table I, and the 2x(3660x3200) VR target of Sec. 1).
"""
from __future__ import annotations

import math

import numpy as np

SH_COEFFS = 16
NEAR = 0.2

# Default workload seeds: scene 1000+c, poses 2000+c, calibration poses 3000+c.
SCENE_SEED = 1000
POSE_SEED = 2000
CALIB_SEED = 3000


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotations as normalised 4-D normals, shape [4][n]."""
    q = rng.standard_normal((4, n), dtype=np.float32)
    nrm = np.sqrt((q.astype(np.float64) ** 2).sum(0))
    nrm[nrm == 0] = 1.0
    return (q / nrm).astype(np.float32)


def _quat_to_mat(q: np.ndarray) -> np.ndarray:
    """Rotation matrix of one unit quaternion (w, x, y, z); used to orient clusters."""
    w, x, y, z = [float(v) for v in q]
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def _sh(rng: np.random.Generator, n: int, dc_mean=0.5, dc_std=0.2, rest_std=0.1) -> np.ndarray:
    sh = np.empty((SH_COEFFS, 3, n), dtype=np.float32)
    sh[0] = rng.normal(dc_mean, dc_std, size=(3, n)).astype(np.float32)
    sh[1:] = (rng.standard_normal((SH_COEFFS - 1, 3, n), dtype=np.float32) * np.float32(rest_std))
    return sh


def scene_uniform_cube(n: int, seed: int) -> dict:
    """16K-style scene: means U[-1,1]^3, log-scale N(-3.5,0.5), opacity logit N(0,1.5)."""
    rng = _rng(seed)
    mean = rng.uniform(-1.0, 1.0, size=(3, n)).astype(np.float32)
    log_scale = rng.normal(-3.5, 0.5, size=(3, n)).astype(np.float32)
    quat = _unit_quats(rng, n)
    logit = rng.normal(0.0, 1.5, size=n).astype(np.float32)
    sh = _sh(rng, n)
    return dict(mean=mean, log_scale=log_scale, quat=quat, opacity_logit=logit, sh=sh)


def scene_clusters(n: int, seed: int, n_clusters: int = 64) -> dict:
    """Surface-like scene: n_clusters flat disks in [-1,1]^3.

    Each cluster is a randomly oriented ellipsoidal slab with in-plane
    semi-axes 0.35*U(0.5,1.5) and 0.02 along its normal.  Gaussians take the
    cluster's frame as rotation, log-scales N(-4.5,0.8) per axis with the
    normal axis a further ln 3 smaller, and opacity logit N(0,2).
    """
    rng = _rng(seed)
    centers = rng.uniform(-1.0, 1.0, size=(n_clusters, 3))
    cq = _unit_quats(rng, n_clusters).astype(np.float64)
    axes = np.stack([0.35 * rng.uniform(0.5, 1.5, n_clusters),
                     0.35 * rng.uniform(0.5, 1.5, n_clusters),
                     np.full(n_clusters, 0.02)], 1)
    counts = [len(a) for a in np.array_split(np.arange(n), n_clusters)]
    mean = np.empty((3, n), dtype=np.float32)
    quat = np.empty((4, n), dtype=np.float32)
    off = 0
    for c in range(n_clusters):
        k = counts[c]
        d = rng.standard_normal((3, k))
        d /= np.linalg.norm(d, axis=0, keepdims=True)
        r = rng.uniform(0.0, 1.0, k) ** (1.0 / 3.0)
        local = d * r * axes[c][:, None]
        R = _quat_to_mat(cq[:, c])
        mean[:, off:off + k] = (R @ local + centers[c][:, None]).astype(np.float32)
        quat[:, off:off + k] = cq[:, c][:, None].astype(np.float32)
        off += k
    log_scale = rng.normal(-4.5, 0.8, size=(3, n)).astype(np.float32)
    log_scale[2] -= np.float32(math.log(3.0))
    logit = rng.normal(0.0, 2.0, size=n).astype(np.float32)
    sh = _sh(rng, n)
    return dict(mean=mean, log_scale=log_scale, quat=quat, opacity_logit=logit, sh=sh)


def scene_city(n: int, seed: int) -> dict:
    """City-scale scene on a 1 km x 1 km ground plane (z up, metres).

    85% of the Gaussians sit on buildings and streets: 60% on facade and roof
    sheets of box buildings, 25% in near-ground street strips along a street
    grid; 15% lie on a sky hemisphere of radius 1.5 km.  Log-scales are
    N(-2.5,1.2) per axis (heavy-tailed log-normal), rotations uniform, opacity
    logit N(0.5,2).
    """
    rng = _rng(seed)
    n_bld = int(round(0.60 * n))
    n_street = int(round(0.25 * n))
    n_sky = n - n_bld - n_street
    mean = np.empty((3, n), dtype=np.float32)

    # Buildings: boxes on a 40 m block grid, kept off the streets.
    n_b = 600
    bx = rng.integers(-12, 12, n_b) * 40.0 + 20.0
    by = rng.integers(-12, 12, n_b) * 40.0 + 20.0
    hw = rng.uniform(5.0, 14.0, n_b)
    hd = rng.uniform(5.0, 14.0, n_b)
    ht = rng.uniform(5.0, 60.0, n_b)
    which = rng.integers(0, n_b, n_bld)
    face = rng.integers(0, 5, n_bld)          # 0..3 walls, 4 roof
    s = rng.uniform(-1.0, 1.0, n_bld)
    h = rng.uniform(0.0, 1.0, n_bld)
    X = bx[which].copy()
    Y = by[which].copy()
    Z = ht[which] * h
    w, d = hw[which], hd[which]
    m0, m1, m2, m3, m4 = (face == 0), (face == 1), (face == 2), (face == 3), (face == 4)
    X[m0] += w[m0]; Y[m0] += s[m0] * d[m0]
    X[m1] -= w[m1]; Y[m1] += s[m1] * d[m1]
    Y[m2] += d[m2]; X[m2] += s[m2] * w[m2]
    Y[m3] -= d[m3]; X[m3] += s[m3] * w[m3]
    X[m4] += s[m4] * w[m4]; Y[m4] += rng.uniform(-1.0, 1.0, int(m4.sum())) * d[m4]
    Z[m4] = ht[which][m4]
    mean[0, :n_bld] = X
    mean[1, :n_bld] = Y
    mean[2, :n_bld] = Z

    # Streets: strips of width 12 m along x = 40k and y = 40k, z in [0, 0.5].
    along = rng.uniform(-500.0, 500.0, n_street)
    lane = rng.integers(-12, 13, n_street) * 40.0 + rng.uniform(-6.0, 6.0, n_street)
    dirx = rng.integers(0, 2, n_street).astype(bool)
    mean[0, n_bld:n_bld + n_street] = np.where(dirx, along, lane)
    mean[1, n_bld:n_bld + n_street] = np.where(dirx, lane, along)
    mean[2, n_bld:n_bld + n_street] = rng.uniform(0.0, 0.5, n_street)

    # Sky: upper hemisphere of radius 1.5 km.
    v = rng.standard_normal((3, n_sky))
    v /= np.linalg.norm(v, axis=0, keepdims=True)
    v[2] = np.abs(v[2])
    mean[:, n_bld + n_street:] = (v * 1500.0).astype(np.float32)

    log_scale = rng.normal(-2.5, 1.2, size=(3, n)).astype(np.float32)
    quat = _unit_quats(rng, n)
    logit = rng.normal(0.5, 2.0, size=n).astype(np.float32)
    sh = _sh(rng, n)
    return dict(mean=mean, log_scale=log_scale, quat=quat, opacity_logit=logit, sh=sh)


def look_at(campos, target, width: int, height: int, fov_x_deg: float,
            up=(0.0, 0.0, 1.0), near: float = NEAR) -> dict:
    """Pinhole camera at `campos` looking at `target` (+x right, +y down, +z forward)."""
    c = np.asarray(campos, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - c
    f /= np.linalg.norm(f)
    upv = np.asarray(up, dtype=np.float64)
    if abs(np.dot(f, upv)) > 0.999:
        upv = np.array([0.0, 1.0, 0.0])
    r = np.cross(f, upv)
    r /= np.linalg.norm(r)
    dn = np.cross(f, r)
    R = np.stack([r, dn, f], 0)
    t = -R @ c
    fx = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    view = np.concatenate([R, t[:, None]], 1).astype(np.float32)
    return dict(width=int(width), height=int(height), fx=float(np.float32(fx)),
                fy=float(np.float32(fx)), cx=float(np.float32((width - 1) * 0.5)),
                cy=float(np.float32((height - 1) * 0.5)), viewmat=view,
                campos=c.astype(np.float32), near=float(near))


def _sphere_dirs(rng, k):
    v = rng.standard_normal((k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def cams_sphere(k: int, seed: int, dist: float, width: int, height: int, fov_x=60.0) -> list:
    rng = _rng(seed)
    return [look_at(dist * d, (0, 0, 0), width, height, fov_x) for d in _sphere_dirs(rng, k)]


def cams_orbit(k: int, dist: float, elev_deg: float, width: int, height: int, fov_x=60.0,
               az0_deg: float = 0.0) -> list:
    cams = []
    for i in range(k):
        az = math.radians(az0_deg + 360.0 * i / k)
        el = math.radians(elev_deg)
        p = dist * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        cams.append(look_at(p, (0, 0, 0), width, height, fov_x))
    return cams


def cams_orbit_random(k: int, seed: int, dist: float, width: int, height: int, fov_x=60.0) -> list:
    rng = _rng(seed)
    cams = []
    for _ in range(k):
        az = rng.uniform(0.0, 2 * math.pi)
        el = math.radians(rng.uniform(5.0, 30.0))
        p = dist * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        cams.append(look_at(p, (0, 0, 0), width, height, fov_x))
    return cams


def cams_city(k_street: int, k_aerial: int, seed: int, width: int, height: int, fov_x=60.0) -> list:
    """Street-level poses at 1.7 m on a street line, and oblique aerial poses at 150-300 m."""
    rng = _rng(seed)
    cams = []
    for _ in range(k_street):
        lane = rng.integers(-10, 11) * 40.0
        along = rng.uniform(-300.0, 300.0)
        if rng.integers(0, 2):
            p = np.array([along, lane, 1.7])
        else:
            p = np.array([lane, along, 1.7])
        yaw = rng.uniform(0.0, 2 * math.pi)
        tgt = p + np.array([math.cos(yaw), math.sin(yaw), -0.05])
        cams.append(look_at(p, tgt, width, height, fov_x))
    for _ in range(k_aerial):
        alt = rng.uniform(150.0, 300.0)
        ang = rng.uniform(0.0, 2 * math.pi)
        p = np.array([250.0 * math.cos(ang), 250.0 * math.sin(ang), alt])
        tgt = np.array([rng.uniform(-100.0, 100.0), rng.uniform(-100.0, 100.0), 0.0])
        cams.append(look_at(p, tgt, width, height, fov_x))
    return cams


def cams_stereo_path(pairs: int, seed: int, width: int, height: int, fov_x=90.0, iod=0.064) -> list:
    """Eye pairs along a street-level path; each eye is offset +-iod/2 along camera right."""
    rng = _rng(seed)
    lane = rng.integers(-10, 11) * 40.0
    start = rng.uniform(-300.0, 200.0)
    cams = []
    for i in range(pairs):
        p = np.array([start + 2.0 * i, lane + 0.5 * math.sin(0.3 * i), 1.7])
        yaw = 0.15 * math.sin(0.5 * i)
        fwd = np.array([math.cos(yaw), math.sin(yaw), -0.03])
        c0 = look_at(p, p + fwd, width, height, fov_x)
        right = c0["viewmat"][0, :3].astype(np.float64)
        for sgn in (-1.0, 1.0):
            pe = p + sgn * 0.5 * iod * right
            cams.append(look_at(pe, pe + fwd, width, height, fov_x))
    return cams


def perturb_scene(scene: dict, seed: int, mean_std=0.01, logit_std=0.1) -> dict:
    """Copy of `scene` with means + N(0, mean_std) and opacity logits + N(0, logit_std)."""
    rng = _rng(seed)
    out = {k: v.copy() for k, v in scene.items()}
    out["mean"] += rng.normal(0.0, mean_std, size=out["mean"].shape).astype(np.float32)
    out["opacity_logit"] += rng.normal(0.0, logit_std, size=out["opacity_logit"].shape).astype(np.float32)
    return out


def fd_subscene(seed: int = 4005, n: int = 64) -> tuple:
    """64 cluster-like Gaussians in front of a 64x64 camera at distance 1.2.

    Opacity logits follow the cluster scene, N(0,2); log-scales are
    N(-3.0,0.3) so that each footprint spans a few pixels.
    """
    rng = _rng(seed)
    mean = rng.uniform(-0.25, 0.25, size=(3, n)).astype(np.float32)
    log_scale = rng.normal(-3.0, 0.3, size=(3, n)).astype(np.float32)
    quat = _unit_quats(rng, n)
    logit = rng.normal(0.0, 2.0, size=n).astype(np.float32)
    sh = _sh(rng, n)
    cam = look_at((0.0, -1.2, 0.3), (0.0, 0.0, 0.0), 64, 64, 60.0)
    return dict(mean=mean, log_scale=log_scale, quat=quat, opacity_logit=logit, sh=sh), cam


# Named workloads (sizes from the benchmark definitions).
WORKLOADS = {
    "c1_cube16k_256": dict(n=16384, width=256, height=256),
    "c2_clusters1m_1080p": dict(n=1048576, width=1920, height=1080),
    "c3_city8m_4608x3456": dict(n=8388608, width=4608, height=3456),
    "c4_city4m_vr16x3660x3200": dict(n=4194304, width=3660, height=3200),
    "c5_clusters1m_1080p_fwdbwd": dict(n=1048576, width=1920, height=1080),
}


def workload(name: str, n: int | None = None, width: int | None = None,
             height: int | None = None, views: int | None = None) -> tuple:
    """(scene, cameras, calibration_cameras) for a named workload.

    `n`, `width`, `height`, `views` may shrink a workload for tests; the
    distribution and camera recipe stay those of the named workload.
    """
    w = WORKLOADS[name]
    n = w["n"] if n is None else n
    W = w["width"] if width is None else width
    H = w["height"] if height is None else height
    if name.startswith("c1"):
        scene = scene_uniform_cube(n, SCENE_SEED + 1)
        cams = cams_sphere(1 if views is None else views, POSE_SEED + 1, 4.0, W, H)
        calib = cams_sphere(16, CALIB_SEED + 1, 4.0, W, H)
    elif name.startswith("c2") or name.startswith("c5"):
        scene = scene_clusters(n, SCENE_SEED + 2)
        cams = cams_orbit(10 if views is None else views, 4.0, 15.0, W, H)
        calib = cams_orbit_random(16, CALIB_SEED + 2, 4.0, W, H)
    elif name.startswith("c3"):
        scene = scene_city(n, SCENE_SEED + 3)
        cams = cams_city(4, 4, POSE_SEED + 3, W, H)
        if views is not None:
            cams = cams[:views]
        calib = cams_city(8, 8, CALIB_SEED + 3, W, H)
    elif name.startswith("c4"):
        scene = scene_city(n, SCENE_SEED + 4)
        pairs = 8 if views is None else max(1, views // 2)
        cams = cams_stereo_path(pairs, POSE_SEED + 4, W, H)
        calib = cams_city(8, 8, CALIB_SEED + 4, W, H, fov_x=90.0)
    else:
        raise KeyError(name)
    return scene, cams, calib
