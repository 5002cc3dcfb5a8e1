"""Seeded synthetic point-cloud pairs shaped like the paper's workloads.

The paper registers KITTI stereo clouds (3k-15k FAST-selected points, depth
<= 55 m, RGB + 19-class semantic distributions; Sec. V-B) and TUM RGB-D
clouds (640x480 depth maps; Sec. V-C).  Those datasets are not available, so
every workload here is synthetic, drawn from numpy's PCG64 with a fixed seed.

This module is shared by the FP64 oracle's tests and by the CUDA path's tests
and benchmark.  It holds only input generation: ray casting, sampling, noise
and feature synthesis.  It contains none of the registration arithmetic (no
kernel, no inner product, no se(3) exponential): the ground-truth rigid
motions are built from unit quaternions.

Every generator returns a ``Pair``:
  X, Z        float32 (N,3) / (M,3) xyz
  FX, FZ      float32 (N,D) / (M,D) features, blocks concatenated
  blocks      list of (kind, dim, scale, sigma); kind "se" is the squared-
              exponential feature kernel of Eq. (newscalar), "dot" the plain
              inner product of Eq. (scalar) / Eq. (tensor_product)
  T_true      float64 (4,4) rigid motion that maps Z's frame into X's frame
              (y = R z + t), i.e. the transform a registration should return
  params      dict of lengthscale schedule, cutoff and iteration limit
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 20121203
N_CLASSES = 19


@dataclasses.dataclass
class Pair:
    X: np.ndarray
    Z: np.ndarray
    FX: np.ndarray
    FZ: np.ndarray
    blocks: list
    T_true: np.ndarray
    params: dict
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def m(self) -> int:
        return int(self.Z.shape[0])


# ---------------------------------------------------------------------------
# rigid motions (quaternion based; used only to place synthetic data)
# ---------------------------------------------------------------------------

def quat_rotation(axis, angle_rad) -> np.ndarray:
    """3x3 rotation matrix of the unit quaternion (cos a/2, sin a/2 * axis)."""
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    qw = math.cos(angle_rad / 2.0)
    qx, qy, qz = axis * math.sin(angle_rad / 2.0)
    return np.array([
        [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
        [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
        [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)],
    ])


def rigid(R, t) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def random_motion(rng, max_angle_deg, max_trans, exact=False) -> np.ndarray:
    """Random rigid motion: a random unit axis and a translation direction.

    ``exact``: the angle and translation norm are exactly the maxima (the
    single-pair cube workload), otherwise uniform in [0, max].
    """
    axis = rng.normal(size=3)
    tdir = rng.normal(size=3)
    tdir /= np.linalg.norm(tdir)
    ang = max_angle_deg if exact else rng.uniform(0.0, max_angle_deg)
    tn = max_trans if exact else rng.uniform(0.0, max_trans)
    return rigid(quat_rotation(axis, math.radians(ang)), tn * tdir)


def apply(T, P) -> np.ndarray:
    P = np.asarray(P, dtype=np.float64)
    return P @ T[:3, :3].T + T[:3, 3]


def inverse(T) -> np.ndarray:
    R = T[:3, :3]
    return rigid(R.T, -R.T @ T[:3, 3])


# ---------------------------------------------------------------------------
# feature synthesis
# ---------------------------------------------------------------------------

_COLOR_DIRS = np.array([[0.8, 0.6, 0.0], [0.0, 0.6, 0.8], [0.6, 0.0, 0.8]])
_COLOR_PHASE = np.array([0.3, 1.7, 4.1])


def smooth_rgb(P_world, wavelength=2.0, base=None) -> np.ndarray:
    """RGB in [0,1]: 1/2 + 1/2 sin(2 pi (p . a_c)/lambda + phi_c) per channel.

    ``base`` (optional (n,3)) modulates the texture by a per-primitive colour.
    The colour is a function of the world position, so one surface point gets
    the same colour in both views.
    """
    P = np.asarray(P_world, dtype=np.float64)
    a = _COLOR_DIRS / np.linalg.norm(_COLOR_DIRS, axis=1, keepdims=True)
    rgb = 0.5 + 0.5 * np.sin(2.0 * math.pi * (P @ a.T) / wavelength + _COLOR_PHASE)
    if base is not None:
        rgb = np.clip(base * (0.6 + 0.4 * rgb), 0.0, 1.0)
    return rgb


def label_distribution(rng, true_class) -> np.ndarray:
    """19-class softmax of N(0, 2^2) logits with +4 on the true class."""
    true_class = np.asarray(true_class)
    logits = rng.normal(0.0, 2.0, size=(true_class.shape[0], N_CLASSES))
    logits[np.arange(true_class.shape[0]), true_class] += 4.0
    logits -= logits.max(axis=1, keepdims=True)
    e = np.exp(logits)
    return e / e.sum(axis=1, keepdims=True)


def bf16_round(a) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32).reshape(a.shape)


def bf16_bits(a) -> np.ndarray:
    """Bit patterns (uint16) of bf16_round(a)."""
    return (bf16_round(a).view(np.uint32) >> 16).astype(np.uint16)


# ---------------------------------------------------------------------------
# surface sampling
# ---------------------------------------------------------------------------

def sample_box_faces(rng, n, size, center=(0.0, 0.0, 0.0)):
    """n points uniform on the 6 faces of an axis-aligned box; face chosen
    with probability proportional to its area.  Returns (points, face_id)."""
    sx, sy, sz = (float(s) for s in size)
    areas = np.array([sy * sz, sy * sz, sx * sz, sx * sz, sx * sy, sx * sy])
    face = rng.choice(6, size=n, p=areas / areas.sum())
    u = rng.uniform(-0.5, 0.5, size=n)
    v = rng.uniform(-0.5, 0.5, size=n)
    P = np.empty((n, 3))
    half = np.array([sx, sy, sz]) / 2.0
    for f in range(6):
        idx = face == f
        ax = f // 2
        sign = 1.0 if f % 2 == 0 else -1.0
        o1, o2 = [a for a in range(3) if a != ax]
        P[idx, ax] = sign * half[ax]
        P[idx, o1] = u[idx] * 2 * half[o1]
        P[idx, o2] = v[idx] * 2 * half[o2]
    return P + np.asarray(center), face


# ---------------------------------------------------------------------------
# workload 1: dense single pair on a 4 m cube
# ---------------------------------------------------------------------------

def cube_pair(n=2000, seed=SEED_BASE + 1, noise=0.005, angle_deg=5.0, trans=0.1) -> Pair:
    """N=M points uniform on the faces of a 4 m cube plus N(0, noise^2) per
    axis, smooth RGB; Z = T_gt X with the same points and features
    (rotation ``angle_deg`` about a random axis, translation ``trans`` m).
    Dense (no cutoff), lengthscale 0.1 m, colour scale 0.2, 50 iterations."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P, _ = sample_box_faces(rng, n, (4.0, 4.0, 4.0))
    P = P + rng.normal(0.0, noise, size=P.shape)
    rgb = smooth_rgb(P)
    T_gt = random_motion(rng, angle_deg, trans, exact=True)
    Zp = apply(T_gt, P)
    X = P.astype(np.float32)
    Z = Zp.astype(np.float32)
    F = rgb.astype(np.float32)
    return Pair(X=X, Z=Z, FX=F.copy(), FZ=F.copy(),
                blocks=[("se", 3, 0.2, 1.0)],
                T_true=inverse(T_gt),
                params=dict(ell=0.1, ell_min=0.1, cutoff_mult=0.0, max_iters=50, anneal=False),
                name="cube-dense-2k")


# ---------------------------------------------------------------------------
# workload 2: stereo-like street scene
# ---------------------------------------------------------------------------

def _street_world(rng, n_boxes=20):
    boxes = []
    for _ in range(n_boxes):
        size = rng.uniform(1.0, 4.0, size=3)
        cx = rng.uniform(-7.0 + size[0] / 2, 7.0 - size[0] / 2)
        cz = rng.uniform(3.0, 40.0)
        lo = np.array([cx - size[0] / 2, 0.0, cz - size[2] / 2])
        hi = np.array([cx + size[0] / 2, size[1], cz + size[2] / 2])
        boxes.append((lo, hi, int(rng.integers(2, N_CLASSES))))
    base = rng.uniform(0.2, 1.0, size=(N_CLASSES, 3))
    return boxes, base


def _raycast_street(origin, dirs, boxes, wall_x=8.0, wall_h=12.0):
    """Nearest hit of rays origin + s*dir against ground (y=0), walls
    (x = +-wall_x, 0<=y<=wall_h) and the axis-aligned boxes.
    Returns (s, class id); s = inf for a miss."""
    n = dirs.shape[0]
    best = np.full(n, np.inf)
    cls = np.full(n, -1, dtype=np.int64)
    with np.errstate(divide="ignore", invalid="ignore"):
        # ground plane y = 0
        s = -origin[1] / dirs[:, 1]
        ok = (s > 1e-6) & (s < best)
        best[ok], cls[ok] = s[ok], 0
        # walls x = +-wall_x
        for wx in (-wall_x, wall_x):
            s = (wx - origin[0]) / dirs[:, 0]
            y = origin[1] + s * dirs[:, 1]
            ok = (s > 1e-6) & (s < best) & (y >= 0.0) & (y <= wall_h)
            best[ok], cls[ok] = s[ok], 1
        # boxes (slab test)
        for lo, hi, c in boxes:
            t0 = (lo - origin) / dirs
            t1 = (hi - origin) / dirs
            tmin = np.nanmax(np.minimum(t0, t1), axis=1)
            tmax = np.nanmin(np.maximum(t0, t1), axis=1)
            ok = (tmax >= tmin) & (tmin > 1e-6) & (tmin < best)
            best[ok], cls[ok] = tmin[ok], c
    return best, cls


def _stereo_view(rng, C_world_from_cam, boxes, base, n, depth_range=(1.0, 40.0),
                 hfov_deg=90.0, aspect=1241.0 / 376.0, noise_k=0.002, batch=65536):
    """Ray-cast random pixels of a pinhole camera (horizontal FOV 90 deg,
    KITTI aspect ratio), keep hits with depth in range until n points,
    perturb along the ray by N(0, (noise_k d^2)^2).  Returns points in the
    camera frame, world points, class ids."""
    tan_h = math.tan(math.radians(hfov_deg) / 2.0)
    tan_v = tan_h / aspect
    Rw = C_world_from_cam[:3, :3]
    o = C_world_from_cam[:3, 3]
    pts_c, pts_w, cls_all = [], [], []
    got = 0
    while got < n:
        u = rng.uniform(-tan_h, tan_h, size=batch)
        v = rng.uniform(-tan_v, tan_v, size=batch)
        d_cam = np.stack([u, v, np.ones(batch)], axis=1)
        d_world = d_cam @ Rw.T
        s, cls = _raycast_street(o, d_world, boxes)
        depth = s  # z component of s * d_cam, since d_cam.z == 1
        keep = np.isfinite(s) & (depth >= depth_range[0]) & (depth <= depth_range[1])
        s, cls, d_cam, d_world = s[keep], cls[keep], d_cam[keep], d_world[keep]
        depth = s
        s_noisy = s + rng.normal(0.0, 1.0, size=s.shape) * noise_k * depth ** 2
        Pw_true = o + s[:, None] * d_world
        Pc = s_noisy[:, None] * d_cam
        pts_c.append(Pc)
        pts_w.append(Pw_true)
        cls_all.append(cls)
        got += Pc.shape[0]
    Pc = np.concatenate(pts_c)[:n]
    Pw = np.concatenate(pts_w)[:n]
    cl = np.concatenate(cls_all)[:n]
    rgb = smooth_rgb(Pw, base=base[cl])
    return Pc, rgb, cl


def street_pair(n=20000, seed=SEED_BASE + 2, max_angle_deg=10.0, max_trans=0.5) -> Pair:
    """Stereo-like pair: ground plane, 2 walls at x = +-8 m, 20 random boxes
    (1-4 m, depth 3-40 m); a camera 1.6 m above the ground looking along +z;
    random pixel rays, hits at depth 1-40 m, noise along the ray
    sigma = 0.002 d^2.  X and Z are independent ray casts from two camera
    poses that differ by a random motion (rotation <= 10 deg, translation
    <= 0.5 m).  Features: RGB (se, scale 0.2) + 19-class labels (dot).
    Lengthscale 0.3 -> 0.05 m annealed, cutoff 3 lengthscales, <= 100 iters."""
    rng = np.random.Generator(np.random.PCG64(seed))
    boxes, base = _street_world(rng)
    C_X = rigid(np.eye(3), np.array([0.0, 1.6, 0.0]))
    D = random_motion(rng, max_angle_deg, max_trans)
    C_Z = C_X @ D
    X, rgbX, clX = _stereo_view(rng, C_X, boxes, base, n)
    Z, rgbZ, clZ = _stereo_view(rng, C_Z, boxes, base, n)
    FX = np.concatenate([rgbX, label_distribution(rng, clX)], axis=1).astype(np.float32)
    FZ = np.concatenate([rgbZ, label_distribution(rng, clZ)], axis=1).astype(np.float32)
    return Pair(X=X.astype(np.float32), Z=Z.astype(np.float32), FX=FX, FZ=FZ,
                blocks=[("se", 3, 0.2, 1.0), ("dot", N_CLASSES, 1.0, 1.0)],
                T_true=inverse(C_X) @ C_Z,
                params=dict(ell=0.3, ell_min=0.05, cutoff_mult=3.0, max_iters=100, anneal=True),
                name="street-20k")


def street_sequence(n_frames=6, n=10000, seed=SEED_BASE + 6, step=0.8, max_yaw_deg=2.0):
    """Odometry sequence in the street world: a camera 1.6 m above the ground
    drives forward along +z about ``step`` m per frame (10 Hz at ~8 m/s, as a
    KITTI sequence) with a random yaw of at most ``max_yaw_deg`` per frame and
    small pitch/roll/height jitter; every frame is an independent ray cast of
    ``n`` points with RGB + 19-class labels, as in street_pair.  Returns
    (frames, C): frames a list of (xyz float32 (n, 3), features float32
    (n, 22)) in each camera's frame, C the world-from-camera poses; the true
    relative motion of frame k+1 into frame k is inverse(C[k]) @ C[k+1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    boxes, base = _street_world(rng)
    C = [rigid(np.eye(3), np.array([0.0, 1.6, 0.0]))]
    for _ in range(n_frames - 1):
        yaw = math.radians(rng.uniform(-max_yaw_deg, max_yaw_deg))
        jit = quat_rotation(rng.normal(size=3), math.radians(rng.uniform(0.0, 0.3)))
        R = quat_rotation([0.0, 1.0, 0.0], yaw) @ jit
        t = np.array([rng.normal(0.0, 0.02), rng.normal(0.0, 0.01), step * rng.uniform(0.9, 1.1)])
        C.append(C[-1] @ rigid(R, t))
    frames = []
    for Ck in C:
        P, rgb, cl = _stereo_view(rng, Ck, boxes, base, n)
        F = np.concatenate([rgb, label_distribution(rng, cl)], axis=1).astype(np.float32)
        frames.append((P.astype(np.float32), F))
    return frames, C


# ---------------------------------------------------------------------------
# workload 3: RGB-D-like room
# ---------------------------------------------------------------------------

def _room_depth(C_world_from_cam, boxes, room_lo, room_hi, W=640, H=480, fx=525.0, fy=525.0,
                cx=319.5, cy=239.5, step=4):
    us = np.arange(0, W, step)
    vs = np.arange(0, H, step)
    uu, vv = np.meshgrid(us, vs)
    d_cam = np.stack([(uu.ravel() - cx) / fx, (vv.ravel() - cy) / fy, np.ones(uu.size)], axis=1)
    Rw = C_world_from_cam[:3, :3]
    o = C_world_from_cam[:3, 3]
    d_w = d_cam @ Rw.T
    best = np.full(d_w.shape[0], np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        # inside of the room box: the exit distance of the ray
        t0 = (room_lo - o) / d_w
        t1 = (room_hi - o) / d_w
        tmax = np.nanmin(np.maximum(t0, t1), axis=1)
        best = np.minimum(best, np.where(tmax > 0, tmax, np.inf))
        for lo, hi in boxes:
            t0 = (lo - o) / d_w
            t1 = (hi - o) / d_w
            tmin = np.nanmax(np.minimum(t0, t1), axis=1)
            tm = np.nanmin(np.maximum(t0, t1), axis=1)
            ok = (tm >= tmin) & (tmin > 1e-6) & (tmin < best)
            best[ok] = tmin[ok]
    return d_cam, best


def room_pair(seed=SEED_BASE + 3, max_angle_deg=5.0, max_trans=0.1, outlier_frac=0.1) -> Pair:
    """RGB-D-like pair: a 6 x 5 x 3 m room (6 planes) with 10 random boxes,
    640x480 pinhole depth (fx=fy=525, cx=319.5, cy=239.5), depth 0.5-5 m,
    noise sigma = 0.01 d, every 4th pixel in u and v (19,200 points), 10 % of
    the points replaced by uniform samples in the room, smooth RGB; a second
    view displaced by a random motion."""
    rng = np.random.Generator(np.random.PCG64(seed))
    room_lo = np.array([-3.0, 0.0, -2.5])
    room_hi = np.array([3.0, 3.0, 2.5])
    boxes = []
    for _ in range(10):
        size = rng.uniform(0.3, 1.2, size=3)
        c = rng.uniform(room_lo + size / 2, room_hi - size / 2)
        c[1] = size[1] / 2
        boxes.append((c - size / 2, c + size / 2))
    # camera in the room, looking along +z and slightly down; y is up in the
    # world, image v grows downward, so flip y
    flip = np.diag([1.0, -1.0, 1.0])
    C_X = rigid(quat_rotation([1, 0, 0], math.radians(-10.0)) @ flip, np.array([0.0, 1.5, -2.0]))
    D = random_motion(rng, max_angle_deg, max_trans)
    C_Z = C_X @ D
    views = []
    for C in (C_X, C_Z):
        d_cam, s = _room_depth(C, boxes, room_lo, room_hi)
        depth = np.clip(s, 0.5, 5.0)
        noisy = depth + rng.normal(0.0, 1.0, size=depth.shape) * 0.01 * depth
        Pc = noisy[:, None] * d_cam
        Pw = apply(C, depth[:, None] * d_cam)
        n_out = int(round(outlier_frac * Pc.shape[0]))
        idx = rng.choice(Pc.shape[0], size=n_out, replace=False)
        Pw_out = rng.uniform(room_lo, room_hi, size=(n_out, 3))
        Pw[idx] = Pw_out
        Pc[idx] = apply(inverse(C), Pw_out)
        views.append((Pc, smooth_rgb(Pw, wavelength=1.0)))
    (X, FX), (Z, FZ) = views
    return Pair(X=X.astype(np.float32), Z=Z.astype(np.float32),
                FX=FX.astype(np.float32), FZ=FZ.astype(np.float32),
                blocks=[("se", 3, 0.2, 1.0)],
                T_true=inverse(C_X) @ C_Z,
                params=dict(ell=0.1, ell_min=0.1, cutoff_mult=3.0, max_iters=50, anneal=False),
                name="room-19k")


# ---------------------------------------------------------------------------
# workload 4: batch of uneven cube pairs (labels + RGB, bf16 storage)
# ---------------------------------------------------------------------------

def batch_pairs(n_pairs=64, seed=SEED_BASE + 4, n_range=(5000, 60000), max_angle_deg=8.0,
                max_trans=0.4) -> list:
    """n_pairs cube pairs; each cloud's size uniform in n_range; X and Z are
    independent samples of the cube; Z is displaced by its own random motion
    (rotation <= 8 deg, translation <= 0.4 m).  RGB + 19-class labels (true
    class = face id), rounded to bf16.  Lengthscale 0.1, colour scale 0.2,
    cutoff 3 lengthscales."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pairs = []
    for k in range(n_pairs):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        m = int(rng.integers(n_range[0], n_range[1] + 1))
        Px, fx_ = sample_box_faces(rng, n, (4.0, 4.0, 4.0))
        Pz, fz_ = sample_box_faces(rng, m, (4.0, 4.0, 4.0))
        Px += rng.normal(0.0, 0.005, size=Px.shape)
        Pz += rng.normal(0.0, 0.005, size=Pz.shape)
        D = random_motion(rng, max_angle_deg, max_trans)
        FX = np.concatenate([smooth_rgb(Px), label_distribution(rng, fx_)], axis=1)
        FZ = np.concatenate([smooth_rgb(Pz), label_distribution(rng, fz_)], axis=1)
        pairs.append(Pair(X=Px.astype(np.float32), Z=apply(D, Pz).astype(np.float32),
                          FX=bf16_round(FX), FZ=bf16_round(FZ),
                          blocks=[("se", 3, 0.2, 1.0), ("dot", N_CLASSES, 1.0, 1.0)],
                          T_true=inverse(D),
                          params=dict(ell=0.1, ell_min=0.1, cutoff_mult=3.0, max_iters=50,
                                      anneal=False, feat_dtype="bf16"),
                          name=f"batch-{k}"))
    return pairs


# ---------------------------------------------------------------------------
# workload 5: large semantic pair on an 80 m deep box
# ---------------------------------------------------------------------------

def large_pair(n=200000, seed=SEED_BASE + 5, angle_deg=5.0, trans=0.1) -> Pair:
    """200,000 points per cloud on the faces of a 20 m wide x 10 m high x
    80 m deep box (noise 0.005 m); X and Z independent samples, Z displaced
    by a rotation of ``angle_deg`` about a random axis and ``trans`` m; RGB +
    19-class labels (true class = face id).  Lengthscale 0.5 -> 0.05 m,
    cutoff 3 lengthscales, <= 200 iterations."""
    rng = np.random.Generator(np.random.PCG64(seed))
    size = (20.0, 10.0, 80.0)
    center = (0.0, 5.0, 40.0)
    Px, fx_ = sample_box_faces(rng, n, size, center)
    Pz, fz_ = sample_box_faces(rng, n, size, center)
    Px += rng.normal(0.0, 0.005, size=Px.shape)
    Pz += rng.normal(0.0, 0.005, size=Pz.shape)
    D = random_motion(rng, angle_deg, trans, exact=True)
    FX = np.concatenate([smooth_rgb(Px), label_distribution(rng, fx_)], axis=1)
    FZ = np.concatenate([smooth_rgb(Pz), label_distribution(rng, fz_)], axis=1)
    return Pair(X=Px.astype(np.float32), Z=apply(D, Pz).astype(np.float32),
                FX=FX.astype(np.float32), FZ=FZ.astype(np.float32),
                blocks=[("se", 3, 0.2, 1.0), ("dot", N_CLASSES, 1.0, 1.0)],
                T_true=inverse(D),
                params=dict(ell=0.5, ell_min=0.05, cutoff_mult=3.0, max_iters=200, anneal=True),
                name="box80-200k")


def random_cloud(rng, n, d_feat=0, extent=1.0, dtype=np.float32):
    """Small uniform cloud with uniform [0,1] features (parity edge cases)."""
    P = rng.uniform(-extent, extent, size=(n, 3)).astype(dtype)
    F = rng.uniform(0.0, 1.0, size=(n, d_feat)).astype(dtype)
    return P, F


WORKLOADS = {
    "cube-dense-2k": cube_pair,
    "street-20k": street_pair,
    "room-19k": room_pair,
    "box80-200k": large_pair,
}
