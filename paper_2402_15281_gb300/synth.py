"""Seeded synthetic inputs: robot, motions, point clouds and initial weights.

This module only draws inputs.  It holds none of the collision-checking
arithmetic (no kinematics, no distances, no network evaluation), so that the
CPU oracle and the CUDA path can both be fed from it without sharing any of
the method's code.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA
2014; finaliser constants as published by Vigna).  Value ``i`` of stream
``(seed, stream)`` is ``fin(base(seed, stream) + (i + 1) * GAMMA)`` taken
modulo 2**64, and a uniform double is its top 53 bits times 2**-53.  The
definition is platform independent, so every machine draws the same inputs.

The workloads follow the paper's setting: a 6-DOF arm, linear joint-space
motions with start and goal drawn within the joint limits (Sec. IV-C), and
an environment given as a point cloud (Sec. IV-B).  The paper's KUKA
geometry, scenes and datasets are not available, so the robot is a seeded
arm of 7 capsules and the clouds are synthetic stand-ins with the shapes of
the paper's workloads (uniform cube, depth-camera view of a bin).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_STREAM_MUL = 0xD1B54A32D192ED03
_U64 = np.uint64


def _fin(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = z ^ (z >> _U64(30))
    z = z * _U64(_M1)
    z = z ^ (z >> _U64(27))
    z = z * _U64(_M2)
    return z ^ (z >> _U64(31))


def _base(seed: int, stream: int) -> np.uint64:
    key = ((seed * GAMMA) ^ (stream * _STREAM_MUL)) & 0xFFFFFFFFFFFFFFFF
    return _fin(np.array([key], dtype=np.uint64))[0]


class Rng:
    """Counter-based SplitMix64 stream.  ``take(n)`` advances the counter."""

    def __init__(self, seed: int, stream: int):
        self.seed, self.stream = int(seed), int(stream)
        self._b = _base(self.seed, self.stream)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        i = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _fin(self._b + i * _U64(GAMMA))

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> _U64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        """Box-Muller on pairs of uniforms; u1 is kept away from zero."""
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        u1 = np.maximum(u1, 2.0 ** -53)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# Purpose codes of the streams (one stream per purpose and seed).
S_ROBOT, S_MOTION, S_CLOUD, S_WEIGHTS, S_SCENE, S_PATH, S_BOX, S_BOX_MOTION = 1, 2, 3, 4, 5, 6, 7, 8

DOF = 6
N_CAPS = 7
DEG = math.pi / 180.0


@dataclass
class Robot:
    """Serial 6R arm in standard Denavit-Hartenberg form plus 7 capsule radii.

    ``dh[j] = (d, a, alpha, theta_offset)`` for joint j.  Capsule j < 6 joins
    the origins of frames j and j+1; capsule 6 runs from the origin of frame 6
    along its z axis for ``tool_len`` metres.
    """
    dh: np.ndarray            # (6, 4) float64
    radius: np.ndarray        # (7,) float64
    tool_len: float
    qmin: np.ndarray          # (6,) float64, rad
    qmax: np.ndarray          # (6,) float64, rad
    seed: int = 1


def make_robot(seed: int = 1) -> Robot:
    """Seeded arm: alpha = (-pi/2, 0, -pi/2, pi/2, -pi/2, 0), theta offsets 0,
    d1, a1, a2, a3, d4, d6 drawn from fixed ranges, other lengths 0, radii in
    [0.04, 0.08] m sorted from base to tool, limits +-170 deg on every joint."""
    r = Rng(seed, S_ROBOT)
    u = r.uniform(6)
    d1 = 0.30 + 0.15 * u[0]
    a1 = 0.02 + 0.04 * u[1]
    a2 = 0.35 + 0.15 * u[2]
    a3 = 0.02 + 0.04 * u[3]
    d4 = 0.35 + 0.15 * u[4]
    d6 = 0.06 + 0.04 * u[5]
    half = math.pi / 2
    dh = np.array([
        [d1, a1, -half, 0.0],
        [0.0, a2, 0.0, 0.0],
        [0.0, a3, -half, 0.0],
        [d4, 0.0, half, 0.0],
        [0.0, 0.0, -half, 0.0],
        [d6, 0.0, 0.0, 0.0],
    ], dtype=np.float64)
    radius = np.sort(r.uniform(N_CAPS, 0.04, 0.08))[::-1].copy()
    lim = 170.0 * DEG
    return Robot(dh=dh, radius=radius, tool_len=0.10,
                 qmin=np.full(DOF, -lim), qmax=np.full(DOF, lim), seed=seed)


def uniform_motions(robot: Robot, n: int, seed: int = 0, max_step_deg: float | None = None):
    """q0, q1 uniform within the joint limits (Sec. IV-C).  With
    ``max_step_deg`` the goal is q0 plus a uniform offset of at most that many
    degrees per joint, clipped to the limits (short motions, so that both
    verdicts occur)."""
    r = Rng(seed, S_MOTION)
    q0 = robot.qmin + (robot.qmax - robot.qmin) * r.uniform(n * DOF).reshape(n, DOF)
    if max_step_deg is None:
        q1 = robot.qmin + (robot.qmax - robot.qmin) * r.uniform(n * DOF).reshape(n, DOF)
    else:
        off = r.uniform(n * DOF, -max_step_deg * DEG, max_step_deg * DEG).reshape(n, DOF)
        q1 = np.clip(q0 + off, robot.qmin, robot.qmax)
    return q0, q1


def _as_points4(xyz: np.ndarray) -> np.ndarray:
    """(P, 3) -> (P, 4) float32 with w = 0 (16-byte records)."""
    out = np.zeros((xyz.shape[0], 4), dtype=np.float32)
    out[:, :3] = xyz.astype(np.float32)
    return out


def cube_cloud(n: int, seed: int = 0, lo=(-0.75, -0.75, 0.0), hi=(0.75, 0.75, 1.5)) -> np.ndarray:
    """n points uniform in a 1.5 m cube standing on the robot's base plane."""
    r = Rng(seed, S_CLOUD)
    u = r.uniform(n * 3).reshape(n, 3)
    lo = np.asarray(lo)
    hi = np.asarray(hi)
    return _as_points4(lo + (hi - lo) * u)


# --------------------------------------------------------------------------
# Bin-picking scene: a depth camera looking into a bin with 30 objects.
# --------------------------------------------------------------------------

BIN_CENTER = np.array([0.60, 0.0, 0.15])
BIN_SIZE = np.array([0.60, 0.40, 0.30])     # inner x, y, z extent, floor at z = 0
CAMERA = np.array([0.60, 0.0, 1.40])
FOV_X, FOV_Y = 60.0 * DEG, 45.0 * DEG


@dataclass
class BinScene:
    boxes: list = field(default_factory=list)      # (center, R, half extents)
    cylinders: list = field(default_factory=list)  # (center, R, radius, half height)


def _random_rotation(u: np.ndarray) -> np.ndarray:
    """Uniform rotation from three uniforms (Shoemake's quaternion method)."""
    u1, u2, u3 = u
    a, b = math.sqrt(1 - u1), math.sqrt(u1)
    w, x, y, z = (a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2),
                  b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3))
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def make_bin_scene(seed: int = 0, n_objects: int = 30) -> BinScene:
    r = Rng(seed, S_SCENE)
    sc = BinScene()
    lo = BIN_CENTER - BIN_SIZE / 2
    for _ in range(n_objects):
        u = r.uniform(10)
        c = np.array([lo[0] + 0.05 + (BIN_SIZE[0] - 0.10) * u[0],
                      lo[1] + 0.05 + (BIN_SIZE[1] - 0.10) * u[1],
                      0.03 + 0.17 * u[2]])
        R = _random_rotation(u[3:6])
        if u[6] < 0.5:
            half = 0.5 * (0.03 + 0.07 * u[7:10])
            sc.boxes.append((c, R, half))
        else:
            rad = 0.02 + 0.03 * u[7]
            hh = 0.5 * (0.03 + 0.07 * u[8])
            sc.cylinders.append((c, R, rad, hh))
    return sc


def _hit_rect(o, d, axis, value, lo2, hi2, other):
    """Ray hit with the rectangle {p[axis] = value, lo2 <= p[other] <= hi2}."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (value - o[axis]) / d[:, axis]
    p = o[None, :] + t[:, None] * d
    ok = (t > 0) & np.all((p[:, other] >= lo2) & (p[:, other] <= hi2), axis=1)
    return np.where(ok, t, np.inf)


def _hit_box(o, d, c, R, half):
    ol = (o - c) @ R            # ray origin in the box frame
    dl = d @ R
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (-half[None, :] - ol[None, :]) / dl
        t2 = (half[None, :] - ol[None, :]) / dl
    tn = np.fmax.reduce(np.minimum(t1, t2), axis=1)
    tf = np.fmin.reduce(np.maximum(t1, t2), axis=1)
    ok = (tn <= tf) & (tn > 0)
    return np.where(ok, tn, np.inf)


def _hit_cylinder(o, d, c, R, rad, hh):
    ol = (o - c) @ R
    dl = d @ R
    best = np.full(d.shape[0], np.inf)
    A = dl[:, 0] ** 2 + dl[:, 1] ** 2
    B = 2 * (ol[0] * dl[:, 0] + ol[1] * dl[:, 1])
    C = ol[0] ** 2 + ol[1] ** 2 - rad * rad
    disc = B * B - 4 * A * C
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (-B - np.sqrt(np.maximum(disc, 0))) / (2 * A)
    z = ol[2] + t * dl[:, 2]
    ok = (disc >= 0) & (A > 0) & (t > 0) & (np.abs(z) <= hh)
    best = np.where(ok, t, best)
    for s in (-hh, hh):
        with np.errstate(divide="ignore", invalid="ignore"):
            tc = (s - ol[2]) / dl[:, 2]
        px = ol[0] + tc * dl[:, 0]
        py = ol[1] + tc * dl[:, 1]
        okc = (tc > 0) & (px * px + py * py <= rad * rad)
        best = np.where(okc & (tc < best), tc, best)
    return best


def bin_cloud(n: int, seed: int = 0, noise: float = 0.002, scene: BinScene | None = None) -> np.ndarray:
    """Depth-camera-like cloud of exactly n hits: a pinhole camera above the bin
    looks straight down (60 x 45 deg field of view); rays at uniform image
    coordinates hit the bin's floor and four walls (with Gaussian range noise
    of ``noise`` metres) or one of the objects (no noise).  Rays that hit
    nothing are dropped and more are cast until n hits are found.  Only the
    part of the image that can see the bin is sampled (every ray outside it
    misses), which leaves the distribution of the hits unchanged."""
    sc = scene if scene is not None else make_bin_scene(seed)
    r = Rng(seed, S_CLOUD)
    lo = BIN_CENTER - BIN_SIZE / 2
    hi = BIN_CENTER + BIN_SIZE / 2
    got = []
    total = 0
    # image window that contains the bin seen from the camera (margin included)
    ux = min(1.0, 1.1 * (BIN_SIZE[0] / 2) / (CAMERA[2] - hi[2]) / math.tan(FOV_X / 2))
    uy = min(1.0, 1.1 * (BIN_SIZE[1] / 2) / (CAMERA[2] - hi[2]) / math.tan(FOV_Y / 2))
    batch = max(2 * n, 4096)
    while total < n:
        u = r.uniform(2 * batch, -1.0, 1.0).reshape(batch, 2) * np.array([ux, uy])
        d = np.stack([u[:, 0] * math.tan(FOV_X / 2), u[:, 1] * math.tan(FOV_Y / 2),
                      -np.ones(batch)], axis=1)
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        o = CAMERA
        planes = [
            _hit_rect(o, d, 2, lo[2], np.array([lo[0], lo[1]]), np.array([hi[0], hi[1]]), [0, 1]),
            _hit_rect(o, d, 0, lo[0], np.array([lo[1], lo[2]]), np.array([hi[1], hi[2]]), [1, 2]),
            _hit_rect(o, d, 0, hi[0], np.array([lo[1], lo[2]]), np.array([hi[1], hi[2]]), [1, 2]),
            _hit_rect(o, d, 1, lo[1], np.array([lo[0], lo[2]]), np.array([hi[0], hi[2]]), [0, 2]),
            _hit_rect(o, d, 1, hi[1], np.array([lo[0], lo[2]]), np.array([hi[0], hi[2]]), [0, 2]),
        ]
        t_wall = np.min(np.stack(planes), axis=0)
        objs = [_hit_box(o, d, *b) for b in sc.boxes] + [_hit_cylinder(o, d, *cy) for cy in sc.cylinders]
        t_obj = np.min(np.stack(objs), axis=0) if objs else np.full(batch, np.inf)
        t = np.minimum(t_wall, t_obj)
        hit = np.isfinite(t)
        eps = r.normal(batch) * noise
        t_noisy = np.where(t_wall <= t_obj, t + eps, t)
        p = o[None, :] + t_noisy[:, None] * d
        got.append(p[hit])
        total += int(hit.sum())
    return _as_points4(np.concatenate(got)[:n])


# Joint configurations for the bin workloads, found offline for the seeded arm
# (seed 1): a pose with the tool above the bin, and a box of joint offsets
# whose goals put the tool down into the bin.  They are plain constants here.
Q_ABOVE_BIN_DEG = np.array([0.0, -71.0, 0.0, 0.0, 68.0, 0.0])
Q_GRASP_DEG = np.array([0.0, -45.0, 22.0, 0.0, 22.0, 0.0])
Q_GRASP_SPREAD_DEG = np.array([14.0, 12.0, 12.0, 30.0, 20.0, 90.0])


def bin_motions(robot: Robot, n: int, seed: int = 0):
    """Grasp motions of the bin workload: q0 is the above-bin pose plus
    U(+-5 deg) per joint, q1 a grasp pose drawn uniformly from a joint box
    reaching into the bin (the paper's into-bin motions, Sec. V-C)."""
    r = Rng(seed, S_MOTION)
    q0 = (Q_ABOVE_BIN_DEG[None, :] + r.uniform(n * DOF, -5.0, 5.0).reshape(n, DOF)) * DEG
    off = r.uniform(n * DOF, -1.0, 1.0).reshape(n, DOF) * Q_GRASP_SPREAD_DEG[None, :]
    q1 = (Q_GRASP_DEG[None, :] + off) * DEG
    return np.clip(q0, robot.qmin, robot.qmax), np.clip(q1, robot.qmin, robot.qmax)


def bin_paths(robot: Robot, n: int, seed: int = 0):
    """Three-segment paths q_start -> q_inVia -> q_outVia -> q_end (the names of
    Sec. V-C): start and end near the above-bin pose, the two vias in the grasp
    box.  Returns (n, 4, 6) joint configurations."""
    r = Rng(seed, S_PATH)
    q = np.empty((n, 4, DOF))
    q[:, 0] = Q_ABOVE_BIN_DEG + r.uniform(n * DOF, -5.0, 5.0).reshape(n, DOF)
    q[:, 1] = Q_GRASP_DEG + r.uniform(n * DOF, -1.0, 1.0).reshape(n, DOF) * Q_GRASP_SPREAD_DEG
    q[:, 2] = q[:, 1] + r.uniform(n * DOF, -8.0, 8.0).reshape(n, DOF)
    q[:, 3] = Q_ABOVE_BIN_DEG + r.uniform(n * DOF, -5.0, 5.0).reshape(n, DOF)
    q *= DEG
    return np.clip(q, robot.qmin, robot.qmax)


S_GRASP = 9


def bin_grasp_paths(robot: Robot, n: int, seed: int = 0):
    """The two-segment motions of Sec. V-C for n grasp candidates: into the
    bin preStart -> preVia -> grasp, out of it grasp -> postVia -> postEnd.
    preStart and postEnd are the above-bin pose plus U(+-5 deg) per joint
    (drawn separately), the grasp is drawn from the grasp box, each via is
    the grasp plus U(+-8 deg) per joint (close to the object).  Returns
    (into (n, 3, 6), out (n, 3, 6)) waypoints."""
    r = Rng(seed, S_GRASP)
    above = lambda: Q_ABOVE_BIN_DEG + r.uniform(n * DOF, -5.0, 5.0).reshape(n, DOF)
    start = above()
    grasp = Q_GRASP_DEG + r.uniform(n * DOF, -1.0, 1.0).reshape(n, DOF) * Q_GRASP_SPREAD_DEG
    pre_via = grasp + r.uniform(n * DOF, -8.0, 8.0).reshape(n, DOF)
    post_via = grasp + r.uniform(n * DOF, -8.0, 8.0).reshape(n, DOF)
    end = above()
    into = np.stack([start, pre_via, grasp], axis=1) * DEG
    out = np.stack([grasp, post_via, end], axis=1) * DEG
    return np.clip(into, robot.qmin, robot.qmax), np.clip(out, robot.qmin, robot.qmax)


# --------------------------------------------------------------------------
# Box world (Sec. V-B)
# --------------------------------------------------------------------------

BOX_LO = np.array([-1.0, -1.0, 0.0])
BOX_HI = np.array([1.0, 1.0, 1.5])


def _quat_to_matrix(w, x, y, z):
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def box_world(seed: int, n_boxes: int = 50, density_per_cm2: float = 0.1):
    """A box-world scene as in Sec. V-B: n_boxes boxes with a uniformly random
    orientation (unit quaternion from three uniforms, Shoemake's method),
    centres uniform in [-1, 1]^2 x [0, 1.5] m, side lengths uniform in
    [1, 10] cm; the cloud samples the box surfaces at density_per_cm2 points
    per cm^2 (round(area * density) points per box, on faces chosen in
    proportion to their area, uniform on the face).
    Returns (points (P, 4) float32, centres (n, 3), rotations (n, 3, 3),
    sides (n, 3))."""
    r = Rng(seed, S_BOX)
    centres = BOX_LO + (BOX_HI - BOX_LO) * r.uniform(3 * n_boxes).reshape(n_boxes, 3)
    u = r.uniform(3 * n_boxes).reshape(n_boxes, 3)
    sides = r.uniform(3 * n_boxes, 0.01, 0.10).reshape(n_boxes, 3)
    rots = np.empty((n_boxes, 3, 3))
    pts = []
    for b in range(n_boxes):
        u1, u2, u3 = u[b]
        x, y = np.sqrt(1 - u1) * np.sin(2 * np.pi * u2), np.sqrt(1 - u1) * np.cos(2 * np.pi * u2)
        z, w = np.sqrt(u1) * np.sin(2 * np.pi * u3), np.sqrt(u1) * np.cos(2 * np.pi * u3)
        rots[b] = _quat_to_matrix(w, x, y, z)
        a, bb, c = sides[b]
        face_area = np.array([bb * c, bb * c, a * c, a * c, a * bb, a * bb])
        n = int(round(face_area.sum() * 1e4 * density_per_cm2))
        if n == 0:
            continue
        cum = np.cumsum(face_area) / face_area.sum()
        f = np.minimum(np.searchsorted(cum, r.uniform(n), side="right"), 5)
        s = r.uniform(2 * n, -0.5, 0.5).reshape(n, 2)
        local = np.empty((n, 3))
        axis, sign = f // 2, np.where(f % 2 == 0, 0.5, -0.5)
        half = np.array([a, bb, c])
        for k in range(n):
            other = [i for i in range(3) if i != axis[k]]
            local[k, axis[k]] = sign[k] * half[axis[k]]
            local[k, other[0]] = s[k, 0] * half[other[0]]
            local[k, other[1]] = s[k, 1] * half[other[1]]
        pts.append(local @ rots[b].T + centres[b])
    xyz = np.concatenate(pts) if pts else np.zeros((0, 3))
    return _as_points4(xyz), centres, rots, sides


def box_world_motions(robot: Robot, n_goals: int, seed: int):
    """One start configuration and n_goals goals, all uniform within the joint
    limits (Sec. V-B): q0 (n_goals, 6) repeats the start, q1 the goals."""
    r = Rng(seed, S_BOX_MOTION)
    start = robot.qmin + (robot.qmax - robot.qmin) * r.uniform(DOF)
    goals = robot.qmin + (robot.qmax - robot.qmin) * r.uniform(n_goals * DOF).reshape(n_goals, DOF)
    return np.repeat(start[None], n_goals, axis=0), goals


# --------------------------------------------------------------------------
# Named workloads: the bin-picking shapes of Sec. V-C, drawn the same way by
# the tests, the benchmark and the script that stores the oracle's verdicts.
# --------------------------------------------------------------------------

def bin_picking_workload(seed: int = 0, n_motions: int = 64, n_points: int = 200_000):
    """n_motions grasp motions (bin_motions) against one n_points bin cloud
    (bin_cloud) of the same seed, arm of seed 1.  Returns (robot, points (P, 4)
    float32, q0, q1)."""
    robot = make_robot(1)
    pts = bin_cloud(n_points, seed=seed)
    q0, q1 = bin_motions(robot, n_motions, seed=seed)
    return robot, pts, q0, q1


def uneven_batch_workload(n_scenes: int = 32, per_scene: int = 16, lo: int = 10_000, hi: int = 500_000):
    """n_scenes bin scenes whose cloud sizes are log-uniform in [lo, hi]
    (scene s: bin_cloud of seed 200 + s), per_scene grasp motions each
    (bin_motions of seed 300 + s), motions grouped by scene.  Returns (robot,
    sizes (S,), clouds (list of (P_s, 4)), q0, q1, motion_scene (M,) int32)."""
    robot = make_robot(1)
    sizes = np.round(np.exp(Rng(3, 77).uniform(n_scenes, np.log(lo), np.log(hi)))).astype(np.int64)
    clouds = [bin_cloud(int(n), seed=200 + s) for s, n in enumerate(sizes)]
    q0s, q1s = [], []
    for s in range(n_scenes):
        a, b = bin_motions(robot, per_scene, seed=300 + s)
        q0s.append(a)
        q1s.append(b)
    scene = np.repeat(np.arange(n_scenes, dtype=np.int32), per_scene)
    return robot, sizes, clouds, np.concatenate(q0s), np.concatenate(q1s), scene


def three_segment_path_workload(n_paths: int = 128, n_points: int = 300_000, seed: int = 4):
    """n_paths three-segment paths (bin_paths) against one bin cloud of
    n_points; segment 3p + s runs from configuration s to s + 1 of path p.
    Returns (robot, points, q0 (3 n_paths, 6), q1 (3 n_paths, 6))."""
    robot = make_robot(1)
    paths = bin_paths(robot, n_paths, seed=seed)
    q0 = np.ascontiguousarray(paths[:, :3].reshape(-1, DOF))
    q1 = np.ascontiguousarray(paths[:, 1:].reshape(-1, DOF))
    return robot, bin_cloud(n_points, seed=seed), q0, q1


def inputs_digest(*arrays) -> str:
    """SHA-256 of the arrays' bytes (dtype, shape and values), to tell whether
    two machines drew the same inputs."""
    import hashlib
    h = hashlib.sha256()
    for a in arrays:
        a = np.ascontiguousarray(a)
        h.update(f"{a.dtype.str}{a.shape}".encode())
        h.update(a.tobytes())
    return h.hexdigest()


# --------------------------------------------------------------------------
# Network parameters
# --------------------------------------------------------------------------

IN_DIM = 3 + 2 * DOF   # [x, y, z, q0_1..q0_6, q1_1..q1_6]


def layer_shapes(width: int, n_hidden: int):
    """(out, in) of every linear layer: input 15 -> W, n_hidden W -> W, W -> 1."""
    return [(width, IN_DIM)] + [(width, width)] * n_hidden + [(1, width)]


def xavier_weights(width: int = 256, n_hidden: int = 4, seed: int = 2):
    """Glorot-uniform weights U(+-sqrt(6 / (fan_in + fan_out))), zero biases,
    drawn in float64 and stored as float32.  Returns a list of (W, b)."""
    r = Rng(seed, S_WEIGHTS)
    out = []
    for (o, i) in layer_shapes(width, n_hidden):
        lim = math.sqrt(6.0 / (i + o))
        W = r.uniform(o * i, -lim, lim).reshape(o, i).astype(np.float32)
        b = np.zeros(o, dtype=np.float32)
        out.append((W, b))
    return out


def block_weights(width: int = 512, n_blocks: int = 5, seed: int = 2, bn_scale: float = 1.0):
    """Parameters of the block architecture of Sec. IV-A: an initial layer
    15 -> width, n_blocks blocks (linear width (+15 for the jump input from
    the second block on) -> width, ReLU, BatchNorm, skip), a final layer
    width + 15 -> 1.  Glorot-uniform weights, small uniform biases and
    BatchNorm statistics (gamma, beta, running mean and variance) drawn in
    float64 and stored as float32.  Returns dict(init=(W, b), blocks=[(W, b,
    gamma, beta, mean, var)], final=(W, b))."""
    r = Rng(seed, S_WEIGHTS)

    def glorot(o, i):
        lim = math.sqrt(6.0 / (i + o))
        return r.uniform(o * i, -lim, lim).reshape(o, i).astype(np.float32)

    init = (glorot(width, IN_DIM), r.uniform(width, -0.05, 0.05).astype(np.float32))
    blocks = []
    for b in range(n_blocks):
        fan_in = width if b == 0 else width + IN_DIM
        W = glorot(width, fan_in)
        bias = r.uniform(width, -0.05, 0.05).astype(np.float32)
        gamma = (bn_scale * r.uniform(width, 0.5, 1.5)).astype(np.float32)
        beta = r.uniform(width, -0.1, 0.1).astype(np.float32)
        mean = r.uniform(width, 0.0, 0.3).astype(np.float32)
        var = r.uniform(width, 0.2, 1.0).astype(np.float32)
        blocks.append((W, bias, gamma, beta, mean, var))
    final = (glorot(1, width + IN_DIM), r.uniform(1, -0.05, 0.05).astype(np.float32))
    return {"init": init, "blocks": blocks, "final": final}


# Activation codes shared with the C interface.
ACT_RELU, ACT_SILU = 0, 1
