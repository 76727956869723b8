"""Seeded synthetic point-cloud pairs with the shapes of the paper's workloads.

This module is the single source of inputs for both the GPU path and the
FP64 oracle.  It holds none of the registration method's arithmetic: it only
samples surfaces, casts sensor rays against simple primitives and applies a
known rigid motion, so that every test and benchmark works on seeded,
reproducible data.

The paper evaluates on the Stanford Bunny, the Stanford Lounge Kinect stream
and a Velodyne VLP-16 sequence (Sec. 5, Sec. 6).  None of those datasets is
available here; the generators below stand in for them:

* ``corner_pair``     small object-scale pair (3 orthogonal unit squares and a
                      sphere), the synthetic analogue of the Bunny experiment
                      of Sec. 5 (random rotation, translation per axis).
* ``lidar_pair``      two consecutive spinning-LiDAR sweeps of an urban
                      scene (ground, boxes, poles), analogue of Sec. 6 VLP-16.
* ``lidar_sequence``  a drive of many such sweeps with known poses (frame-to-
                      frame odometry).
* ``depth_pair``      a back-projected pinhole depth image of a room,
                      analogue of the Lounge structured-light frames (Sec. 6).
* ``batched_pairs``   hundreds of uneven plane/sphere/box pairs.
* ``so3_pairs``       pairs under rotations uniform over SO(3) (pose-proposal
                      test data).
* ``so3_scene_set``   scenes sampled twice, each with several SO(3)-uniform
                      poses of its second sample (pose-proposal training
                      data; the rotated clouds are made by ``apply``).
* ``mlp_init``        seeded initial weights of the proposal network.

Convention: a pair holds ``src`` (cloud Z2) and ``tgt`` (cloud Z1, the model
the tree is built on) as float64 (N, 3) arrays and the ground-truth rigid
motion ``T_gt`` (4x4) with ``tgt ~ R_gt @ src + t_gt`` (Eq. 1 maps the source
into the model frame).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "make_rng", "axis_angle_matrix", "random_rotation", "uniform_rotation",
    "rigid", "apply", "to_float4", "corner_scene", "corner_pair",
    "lidar_pair", "lidar_sequence", "depth_pair", "primitive_scene", "primitive_pair",
    "batched_pairs", "so3_pairs", "so3_scene_set", "mlp_init", "blob_cloud",
]


# --------------------------------------------------------------------------
# random motions
# --------------------------------------------------------------------------
def make_rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def axis_angle_matrix(axis, angle) -> np.ndarray:
    """Rotation matrix of ``angle`` radians about unit ``axis``."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + np.sin(angle) * K + (1.0 - np.cos(angle)) * (K @ K)


def random_rotation(rng, max_deg: float) -> np.ndarray:
    """Axis uniform on the sphere, angle uniform in [0, max_deg]."""
    axis = rng.normal(size=3)
    angle = np.deg2rad(rng.uniform(0.0, max_deg))
    return axis_angle_matrix(axis, angle)


def euler_xyz_rotation(rng, max_deg: float) -> np.ndarray:
    """Each axis angle uniform in [-max_deg, max_deg] (Sec. 5 protocol)."""
    ax, ay, az = np.deg2rad(rng.uniform(-max_deg, max_deg, size=3))
    return (axis_angle_matrix([0, 0, 1], az) @ axis_angle_matrix([0, 1, 0], ay)
            @ axis_angle_matrix([1, 0, 0], ax))


def uniform_rotation(rng) -> np.ndarray:
    """Rotation uniform over SO(3) (unit quaternion with Gaussian entries)."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def rigid(R, t) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def apply(T, P) -> np.ndarray:
    return P @ T[:3, :3].T + T[:3, 3]


def to_float4(P) -> np.ndarray:
    """(N, 3) -> contiguous (N, 4) float32 with a zero pad lane (16 B/point)."""
    P = np.asarray(P)
    out = np.zeros((P.shape[0], 4), dtype=np.float32)
    out[:, :3] = P
    return out


# --------------------------------------------------------------------------
# surface sampling helpers
# --------------------------------------------------------------------------
def _sample_rects(rng, rects, n):
    """rects: list of (origin, u, v) parallelograms; area-weighted uniform."""
    areas = np.array([np.linalg.norm(np.cross(u, v)) for _, u, v in rects])
    idx = rng.choice(len(rects), size=n, p=areas / areas.sum())
    o = np.array([r[0] for r in rects])[idx]
    u = np.array([r[1] for r in rects])[idx]
    v = np.array([r[2] for r in rects])[idx]
    a = rng.uniform(size=(n, 1))
    b = rng.uniform(size=(n, 1))
    return o + a * u + b * v


def _sample_sphere(rng, center, radius, n):
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.asarray(center) + radius * d


def _box_rects(lo, hi):
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    ex = np.array([hi[0] - lo[0], 0, 0])
    ey = np.array([0, hi[1] - lo[1], 0])
    ez = np.array([0, 0, hi[2] - lo[2]])
    return [
        (lo, ex, ey), (lo + ez, ex, ey),
        (lo, ex, ez), (lo + ey, ex, ez),
        (lo, ey, ez), (lo + ex, ey, ez),
    ]


# --------------------------------------------------------------------------
# small object-scale scene: 3 orthogonal unit squares + a sphere
# --------------------------------------------------------------------------
def corner_scene(rng, n: int, noise: float = 0.005) -> np.ndarray:
    """Three unit squares on the xy, yz and xz planes meeting at the origin and
    a sphere of radius 0.3 centred at (0.5, 0.5, 0.5); area-weighted uniform
    samples with isotropic N(0, noise^2) jitter."""
    rects = [
        (np.zeros(3), np.array([1.0, 0, 0]), np.array([0, 1.0, 0])),
        (np.zeros(3), np.array([0, 1.0, 0]), np.array([0, 0, 1.0])),
        (np.zeros(3), np.array([1.0, 0, 0]), np.array([0, 0, 1.0])),
    ]
    r = 0.3
    a_sph = 4 * np.pi * r * r
    a_rect = 3.0
    n_sph = rng.binomial(n, a_sph / (a_sph + a_rect))
    P = np.concatenate([
        _sample_rects(rng, rects, n - n_sph),
        _sample_sphere(rng, [0.5, 0.5, 0.5], r, n_sph),
    ])
    P = P[rng.permutation(n)]
    return P + rng.normal(scale=noise, size=P.shape)


def corner_pair(seed: int, n: int = 10000, max_deg: float = 30.0,
                max_t: float = 0.1, noise: float = 0.005) -> dict:
    """Source: ``n`` scene samples.  Target: an independent resample moved by a
    seeded rotation (uniform axis, angle <= max_deg) and translation
    (uniform per axis in [-max_t, max_t])."""
    rng = make_rng(seed)
    src = corner_scene(rng, n, noise)
    R = random_rotation(rng, max_deg)
    t = rng.uniform(-max_t, max_t, size=3)
    T = rigid(R, t)
    tgt = apply(T, corner_scene(rng, n, noise))
    return {"src": src, "tgt": tgt, "T_gt": T, "name": "corner", "seed": seed}


# --------------------------------------------------------------------------
# 64-beam spinning LiDAR in an urban scene
# --------------------------------------------------------------------------
def _urban_scene(rng):
    """Ground z=0, 20 axis-aligned boxes (sides 5-20 m) along both sides of a
    straight street on the x axis, 30 vertical poles (r 0.1-0.3 m, h 3-8 m)."""
    boxes = []
    while len(boxes) < 20:
        sx, sy, sz = rng.uniform(5.0, 20.0, size=3)
        cx = rng.uniform(-60.0, 60.0)
        side = 1.0 if rng.uniform() < 0.5 else -1.0
        gap = rng.uniform(6.0, 25.0)
        cy = side * (gap + sy / 2)
        lo = np.array([cx - sx / 2, cy - sy / 2, 0.0])
        hi = np.array([cx + sx / 2, cy + sy / 2, sz])
        boxes.append((lo, hi))
    poles = []
    while len(poles) < 30:
        px = rng.uniform(-60.0, 60.0)
        py = (1.0 if rng.uniform() < 0.5 else -1.0) * rng.uniform(3.0, 6.0)
        poles.append((px, py, rng.uniform(0.1, 0.3), rng.uniform(3.0, 8.0)))
    return {"boxes": np.array(boxes), "poles": np.array(poles)}


def _cast_urban(scene, origin, dirs, max_range):
    """Nearest hit distance along unit ``dirs`` from ``origin`` (inf = miss)."""
    n = dirs.shape[0]
    best = np.full(n, np.inf)
    # ground plane z = 0
    dz = dirs[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        tg = -origin[2] / dz
    tg = np.where((dz < 0) & (tg > 0), tg, np.inf)
    best = np.minimum(best, tg)
    inv = np.where(np.abs(dirs) > 1e-12, 1.0 / np.where(dirs == 0, 1, dirs), 1e12)
    for lo, hi in scene["boxes"]:
        t1 = (lo - origin) * inv
        t2 = (hi - origin) * inv
        tmin = np.max(np.minimum(t1, t2), axis=1)
        tmax = np.min(np.maximum(t1, t2), axis=1)
        hit = (tmax >= tmin) & (tmin > 0)
        best = np.where(hit & (tmin < best), tmin, best)
    for px, py, r, h in scene["poles"]:
        ox, oy = origin[0] - px, origin[1] - py
        a = dirs[:, 0] ** 2 + dirs[:, 1] ** 2
        b = 2 * (ox * dirs[:, 0] + oy * dirs[:, 1])
        c = ox * ox + oy * oy - r * r
        disc = b * b - 4 * a * c
        ok = (disc >= 0) & (a > 1e-12)
        sq = np.sqrt(np.where(ok, disc, 0.0))
        tc = np.where(ok, (-b - sq) / (2 * np.where(a > 1e-12, a, 1.0)), np.inf)
        z = origin[2] + tc * dirs[:, 2]
        hit = ok & (tc > 0) & (z >= 0) & (z <= h)
        best = np.where(hit & (tc < best), tc, best)
    best[best > max_range] = np.inf
    return best


def _lidar_sweep(rng, scene, center, yaw, beams=64, az_step_deg=0.2,
                 fov_deg=15.0, max_range=100.0, range_noise=0.02):
    el = np.deg2rad(np.linspace(-fov_deg, fov_deg, beams))
    az = np.deg2rad(np.arange(0.0, 360.0, az_step_deg))
    E, A = np.meshgrid(el, az, indexing="ij")  # beam-major scan order
    d_sensor = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A),
                         np.sin(E)], axis=-1).reshape(-1, 3)
    Rz = axis_angle_matrix([0, 0, 1], yaw)
    d_world = d_sensor @ Rz.T
    rng_t = _cast_urban(scene, np.asarray(center, float), d_world, max_range)
    keep = np.isfinite(rng_t)
    r = rng_t[keep] + rng.normal(scale=range_noise, size=keep.sum())
    return d_sensor[keep] * r[:, None]  # sensor frame


def lidar_pair(seed: int, forward: float = 1.0, max_yaw_deg: float = 2.0,
               height: float = 1.8) -> dict:
    """Two sweeps of a 64-beam LiDAR (elevation +-15 deg, 0.2 deg azimuth step,
    1800 x 64 rays, 100 m range, N(0, 0.02^2) m range noise).  The second
    sweep is taken after ``forward`` metres of motion along x and a yaw of at
    most ``max_yaw_deg``.  Points are in each sensor's own frame."""
    rng = make_rng(seed)
    scene = _urban_scene(rng)
    yaw = np.deg2rad(rng.uniform(-max_yaw_deg, max_yaw_deg))
    c1 = np.array([0.0, 0.0, height])
    c2 = np.array([forward, 0.0, height])
    tgt = _lidar_sweep(rng, scene, c1, 0.0)
    src = _lidar_sweep(rng, scene, c2, yaw)
    T = rigid(axis_angle_matrix([0, 0, 1], yaw), c2 - c1)
    return {"src": src, "tgt": tgt, "T_gt": T, "name": "lidar", "seed": seed}


def lidar_sequence(seed: int, frames: int = 20, forward: float = 1.0, max_yaw_deg: float = 2.0,
                   height: float = 1.8, start_x: float = -10.0) -> dict:
    """``frames`` sweeps of the 64-beam LiDAR of ``lidar_pair`` along a drive
    through one urban scene: the sensor advances ``forward`` metres along its
    heading per frame and turns by a yaw drawn in +-max_yaw_deg plus a pull
    back towards the street axis.  ``frames`` holds each sweep in its own
    sensor frame, ``W`` the sensor-to-world pose of every frame and ``T_rel``
    the motion T_rel[k] = W[k-1]^-1 W[k] that maps frame k into frame k-1
    (T_rel[0] = I)."""
    rng = make_rng(seed)
    scene = _urban_scene(rng)
    W = np.empty((frames, 4, 4))
    pts = []
    c = np.array([start_x, 0.0, height])
    psi = 0.0
    for k in range(frames):
        if k:
            c = c + forward * np.array([np.cos(psi), np.sin(psi), 0.0])
            psi = psi - 0.3 * psi - 0.02 * c[1] + np.deg2rad(rng.uniform(-max_yaw_deg, max_yaw_deg))
        W[k] = rigid(axis_angle_matrix([0, 0, 1], psi), c)
        pts.append(_lidar_sweep(rng, scene, c, psi))
    T_rel = np.empty_like(W)
    T_rel[0] = np.eye(4)
    for k in range(1, frames):
        T_rel[k] = np.linalg.inv(W[k - 1]) @ W[k]
    return {"frames": pts, "W": W, "T_rel": T_rel, "name": "lidar_sequence", "seed": seed}


# --------------------------------------------------------------------------
# structured-light depth image of a room
# --------------------------------------------------------------------------
def _room_scene(rng):
    boxes, spheres = [], []
    for _ in range(10):
        if rng.uniform() < 0.5:
            s = rng.uniform(0.2, 0.8, size=3)
            c = np.array([rng.uniform(-2.2, 2.2), rng.uniform(-1.3, 1.5 - s[1] / 2),
                          rng.uniform(1.5, 4.5)])
            boxes.append((c - s / 2, c + s / 2))
        else:
            r = rng.uniform(0.1, 0.4)
            spheres.append((rng.uniform(-2.2, 2.2), rng.uniform(-1.2, 1.2),
                            rng.uniform(1.5, 4.5), r))
    return {"room_lo": np.array([-3.0, -1.5, -1.0]),
            "room_hi": np.array([3.0, 1.5, 5.0]),
            "boxes": boxes, "spheres": spheres}


def _cast_room(scene, origin, dirs):
    inv = 1.0 / np.where(np.abs(dirs) > 1e-12, dirs, 1e-12)
    # inside the room: exit distance of the room box
    t1 = (scene["room_lo"] - origin) * inv
    t2 = (scene["room_hi"] - origin) * inv
    best = np.min(np.maximum(t1, t2), axis=1)
    for lo, hi in scene["boxes"]:
        a = (lo - origin) * inv
        b = (hi - origin) * inv
        tmin = np.max(np.minimum(a, b), axis=1)
        tmax = np.min(np.maximum(a, b), axis=1)
        hit = (tmax >= tmin) & (tmin > 0)
        best = np.where(hit & (tmin < best), tmin, best)
    for cx, cy, cz, r in scene["spheres"]:
        oc = origin - np.array([cx, cy, cz])
        b = dirs @ oc
        c = oc @ oc - r * r
        disc = b * b - c
        ok = disc >= 0
        tc = np.where(ok, -b - np.sqrt(np.where(ok, disc, 0)), np.inf)
        hit = ok & (tc > 0)
        best = np.where(hit & (tc < best), tc, best)
    return best


def _depth_frame(rng, scene, R_wc, c_w, W=640, H=480, f=525.0,
                 hole_frac=0.10):
    u, v = np.meshgrid(np.arange(W, dtype=np.float64),
                       np.arange(H, dtype=np.float64))
    x = (u.ravel() - (W - 1) / 2) / f
    y = (v.ravel() - (H - 1) / 2) / f
    rays_c = np.stack([x, y, np.ones_like(x)], axis=1)  # z = 1 in camera frame
    d_w = rays_c @ R_wc.T
    norm = np.linalg.norm(d_w, axis=1)
    t = _cast_room(scene, c_w, d_w / norm[:, None]) / norm  # depth along z
    z = t + rng.normal(size=t.shape) * (0.0012 * t * t)
    keep = rng.uniform(size=z.shape) >= hole_frac
    return rays_c[keep] * z[keep, None]


def depth_pair(seed: int, max_deg: float = 10.0, max_t: float = 0.2) -> dict:
    """640x480 pinhole depth image (fx = fy = 525) of a 6 x 3 x 6 m room with
    10 random boxes and spheres, back-projected to points; depth noise
    N(0, (0.0012 z^2)^2), 10 % of pixels dropped.  The second camera is moved
    by at most ``max_deg`` rotation and ``max_t`` m translation."""
    rng = make_rng(seed)
    scene = _room_scene(rng)
    R1, c1 = np.eye(3), np.array([0.0, 0.0, -0.5])
    dR = random_rotation(rng, max_deg)
    dt = rng.normal(size=3)
    dt *= rng.uniform(0, max_t) / np.linalg.norm(dt)
    R2, c2 = dR @ R1, c1 + dt
    tgt = _depth_frame(rng, scene, R1, c1)
    src = _depth_frame(rng, scene, R2, c2)
    # p_w = R2 p_c2 + c2 = R1 p_c1 + c1  =>  p_c1 = R1^T R2 p_c2 + R1^T (c2 - c1)
    T = rigid(R1.T @ R2, R1.T @ (c2 - c1))
    return {"src": src, "tgt": tgt, "T_gt": T, "name": "depth", "seed": seed}


# --------------------------------------------------------------------------
# random plane / sphere / box scenes (batched form)
# --------------------------------------------------------------------------
def primitive_scene(rng):
    rects, spheres = [], []
    for _ in range(rng.integers(1, 4)):  # planes
        o = rng.uniform(-1, 1, size=3)
        u = rng.normal(size=3)
        v = rng.normal(size=3)
        u *= rng.uniform(0.5, 2.0) / np.linalg.norm(u)
        v -= (v @ u) / (u @ u) * u
        v *= rng.uniform(0.5, 2.0) / np.linalg.norm(v)
        rects.append((o, u, v))
    for _ in range(rng.integers(1, 4)):  # boxes
        lo = rng.uniform(-1, 1, size=3)
        rects.extend(_box_rects(lo, lo + rng.uniform(0.2, 1.0, size=3)))
    for _ in range(rng.integers(0, 3)):
        spheres.append((rng.uniform(-1, 1, size=3), rng.uniform(0.1, 0.5)))
    return rects, spheres


def _sample_primitives(rng, scene, n, noise):
    rects, spheres = scene
    a_r = sum(np.linalg.norm(np.cross(u, v)) for _, u, v in rects)
    a_s = [4 * np.pi * r * r for _, r in spheres]
    w = np.array([a_r] + a_s)
    cnt = rng.multinomial(n, w / w.sum())
    parts = [_sample_rects(rng, rects, cnt[0])]
    for (c, r), k in zip(spheres, cnt[1:]):
        parts.append(_sample_sphere(rng, c, r, k))
    P = np.concatenate(parts)[rng.permutation(n)]
    return P + rng.normal(scale=noise, size=P.shape)


def primitive_pair(seed: int, n: int, max_deg: float = 30.0,
                   max_t: float = 0.1, noise: float = 0.005) -> dict:
    rng = make_rng(seed)
    scene = primitive_scene(rng)
    src = _sample_primitives(rng, scene, n, noise)
    T = rigid(random_rotation(rng, max_deg), rng.uniform(-max_t, max_t, 3))
    tgt = apply(T, _sample_primitives(rng, scene, n, noise))
    return {"src": src, "tgt": tgt, "T_gt": T, "name": "primitive", "seed": seed}


def batched_pairs(seed: int, count: int = 256, n_lo: int = 2000,
                  n_hi: int = 200000, max_deg: float = 30.0):
    """``count`` independent pairs, sizes log-uniform in [n_lo, n_hi], tree
    depth 3 or 4 per pair (drawn uniformly)."""
    rng = make_rng(seed)
    sizes = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=count)).astype(np.int64)
    depths = rng.integers(3, 5, size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    out = []
    for i in range(count):
        p = primitive_pair(int(seeds[i]), int(sizes[i]), max_deg=max_deg)
        p["depth"] = int(depths[i])
        out.append(p)
    return out


def so3_pairs(seed: int, count: int, n: int):
    """Pairs whose rotation is uniform over SO(3) (any angle up to 180 deg)."""
    rng = make_rng(seed)
    out = []
    for _ in range(count):
        s = int(rng.integers(0, 2**31 - 1))
        r2 = make_rng(s)
        scene = primitive_scene(r2)
        src = _sample_primitives(r2, scene, n, 0.005)
        T = rigid(uniform_rotation(r2), r2.uniform(-0.1, 0.1, 3))
        tgt = apply(T, _sample_primitives(r2, scene, n, 0.005))
        out.append({"src": src, "tgt": tgt, "T_gt": T, "name": "so3", "seed": s})
    return out


def so3_scene_set(seed: int, n_scenes: int, per_scene: int, n: int, max_t: float = 0.1):
    """``n_scenes`` plane/box/sphere scenes, each sampled twice (``src`` and
    ``tgt_base``, float32 (n, 3)), and ``per_scene`` poses per scene with
    rotations uniform over SO(3): pair (i, j) is src[i] against
    apply(T[i, j], tgt_base[i])."""
    rng = make_rng(seed)
    src, base = [], []
    T = np.empty((n_scenes, per_scene, 4, 4))
    for i in range(n_scenes):
        r2 = make_rng(int(rng.integers(0, 2**31 - 1)))
        scene = primitive_scene(r2)
        src.append(_sample_primitives(r2, scene, n, 0.005).astype(np.float32))
        base.append(_sample_primitives(r2, scene, n, 0.005).astype(np.float32))
        for j in range(per_scene):
            T[i, j] = rigid(uniform_rotation(r2), r2.uniform(-max_t, max_t, 3))
    return {"src": src, "tgt_base": base, "T": T}


# layout of the proposal network's flat parameter vector (FP32):
# W1 (256 x 1280), b1 (256), W2 (256 x 256), b2 (256), W3 (9 x 256), b3 (9)
MLP_SHAPES = ((256, 1280), (256,), (256, 256), (256,), (9, 256), (9,))


def mlp_init(seed: int) -> np.ndarray:
    """Flat FP32 parameters: weights uniform in +-sqrt(6 / fan_in) (He
    uniform), biases zero."""
    rng = make_rng(seed)
    parts = []
    for shape in MLP_SHAPES:
        if len(shape) == 2:
            b = np.sqrt(6.0 / shape[1])
            parts.append(rng.uniform(-b, b, size=shape).reshape(-1))
        else:
            parts.append(np.zeros(shape[0]))
    return np.concatenate(parts).astype(np.float32)


# --------------------------------------------------------------------------
# well-separated anisotropic blobs (closed-form checks)
# --------------------------------------------------------------------------
def blob_cloud(seed: int, n_per: int, centers, covs):
    """Samples of len(centers) Gaussian blobs; returns points and true labels."""
    rng = make_rng(seed)
    pts, lab = [], []
    for k, (c, S) in enumerate(zip(centers, covs)):
        L = np.linalg.cholesky(np.asarray(S, float))
        pts.append(np.asarray(c, float) + rng.normal(size=(n_per, 3)) @ L.T)
        lab.append(np.full(n_per, k))
    P = np.concatenate(pts)
    y = np.concatenate(lab)
    perm = rng.permutation(P.shape[0])
    return P[perm], y[perm]
