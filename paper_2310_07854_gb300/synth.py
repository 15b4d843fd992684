"""Seeded synthetic inputs for the batched cost-and-gradient path.

This module only *draws inputs*: the arm description, the obstacle set and
the joint configurations.  It computes nothing the method itself computes
(no kinematics, distances, costs or quantisation), so both the CUDA path and
the FP64 oracle may consume what it produces.

The paper evaluates on the Franka Panda arm and the MotionBenchMaker scenes
(Sec. III-A, Sec. VI); neither is available, so these generators stand in for
them with the same shapes:

* a 7-revolute-joint serial chain whose fixed joint transforms are
  ``F_i = Trans(0, 0, l_i) * Rx(alpha_i)`` with ``l_i ~ U[0.05, 0.4]`` m and
  ``alpha_i`` in ``{-pi/2, +pi/2}`` (a non-planar, Panda-like alternating arm);
* 52 collision spheres, 4-10 per link, radii ``U[0.03, 0.08]`` m, placed
  along each link's segment with up to 2 cm of lateral jitter;
* self-collision pairs: every sphere pair whose links differ by two or more
  (adjacent links are allowed to touch);
* oriented cuboids with centres ``U[-0.75, 0.75]^3`` m, orientation uniform on
  SO(3) (normalised Gaussian quaternion) and side lengths ``U[0.05, 0.6]`` m;
* joint configurations i.i.d. ``U[-2.8, 2.8]`` rad per joint.

All arrays are float32 / int32 and C-contiguous, in the layouts the C ABI
takes (``include/vapr.h``).
"""
from __future__ import annotations

import dataclasses

import numpy as np

N_JOINTS = 7
N_SPHERES = 52
JOINT_LIMIT = 2.8


@dataclasses.dataclass
class Robot:
    """A serial arm: fixed joint transforms, collision spheres, self pairs."""

    joint_fixed: np.ndarray   # [J, 12] float32: row-major 3x3 rotation then translation
    sphere_local: np.ndarray  # [S, 4] float32: x, y, z in the link frame, radius
    sphere_link: np.ndarray   # [S] int32: link index in 1..J
    pairs: np.ndarray         # [n_pairs, 2] int32: sphere indices (i < j)

    @property
    def n_joints(self) -> int:
        return int(self.joint_fixed.shape[0])

    @property
    def n_spheres(self) -> int:
        return int(self.sphere_local.shape[0])

    @property
    def n_pairs(self) -> int:
        return int(self.pairs.shape[0])


@dataclasses.dataclass
class Scene:
    """Oriented cuboids: pose = row-major rotation (9) then centre (3)."""

    pose: np.ndarray      # [O, 12] float32
    half_ext: np.ndarray  # [O, 3] float32

    @property
    def n_cuboids(self) -> int:
        return int(self.pose.shape[0])


@dataclasses.dataclass
class CostParams:
    """Collision margin, self-collision margin and the two cost weights."""

    eta: float = 0.02
    eta_self: float = 0.01
    w_coll: float = 1.0
    w_self: float = 1.0


def _fixed_transform(length: float, alpha_sign: int) -> np.ndarray:
    # Trans(0, 0, length) * Rx(alpha) with alpha = alpha_sign * pi/2, written
    # out with exact 0/+-1 entries so the table carries no rounding noise.
    s = float(alpha_sign)
    rot = np.array([[1.0, 0.0, 0.0],
                    [0.0, 0.0, -s],
                    [0.0, s, 0.0]])
    return np.concatenate([rot.reshape(9), [0.0, 0.0, length]]).astype(np.float32)


def self_pairs(sphere_link: np.ndarray, min_link_gap: int = 2) -> np.ndarray:
    """All sphere pairs (i < j) whose links differ by at least ``min_link_gap``."""
    out = []
    n = len(sphere_link)
    for i in range(n):
        for j in range(i + 1, n):
            if abs(int(sphere_link[i]) - int(sphere_link[j])) >= min_link_gap:
                out.append((i, j))
    return np.asarray(out, dtype=np.int32).reshape(-1, 2)


def make_robot(seed: int = 0, n_spheres: int = N_SPHERES,
               radius_jitter: float = 0.0, jitter_seed: int = 0) -> Robot:
    """Seeded 7-joint arm with ``n_spheres`` collision spheres (4-10 per link).

    ``radius_jitter`` scales every radius by ``U[1 - j, 1 + j]`` (per sphere,
    drawn from ``jitter_seed``): the same arm with per-problem radii, as the
    uneven batch uses.
    """
    rng = np.random.default_rng(seed)
    lengths = rng.uniform(0.05, 0.4, size=N_JOINTS)
    signs = rng.choice([-1, 1], size=N_JOINTS)
    joint_fixed = np.stack([_fixed_transform(lengths[i], int(signs[i]))
                            for i in range(N_JOINTS)])

    if not (4 * N_JOINTS <= n_spheres <= 10 * N_JOINTS):
        raise ValueError("n_spheres must allow 4..10 spheres per link")
    counts = np.full(N_JOINTS, 4, dtype=np.int64)
    for _ in range(n_spheres - counts.sum()):
        open_links = np.flatnonzero(counts < 10)
        counts[rng.choice(open_links)] += 1

    local, link = [], []
    for li in range(N_JOINTS):
        # link li+1 spans from its origin to the next joint's offset along z
        seg = lengths[li + 1] if li + 1 < N_JOINTS else 0.1
        n = int(counts[li])
        for k in range(n):
            z = seg * k / max(n - 1, 1)
            x, y = rng.uniform(-0.02, 0.02, size=2)
            r = rng.uniform(0.03, 0.08)
            local.append((x, y, z, r))
            link.append(li + 1)
    sphere_local = np.asarray(local, dtype=np.float64)
    if radius_jitter:
        jrng = np.random.default_rng(jitter_seed + 5_000_011)
        sphere_local[:, 3] *= jrng.uniform(1.0 - radius_jitter,
                                           1.0 + radius_jitter, size=n_spheres)
    sphere_local = sphere_local.astype(np.float32)
    sphere_link = np.asarray(link, dtype=np.int32)
    return Robot(joint_fixed=np.ascontiguousarray(joint_fixed),
                 sphere_local=sphere_local, sphere_link=sphere_link,
                 pairs=self_pairs(sphere_link))


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    # Uniform on SO(3): a normalised 4-D Gaussian is a uniform unit quaternion.
    quat = rng.normal(size=(n, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    w, x, y, z = quat.T
    return np.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y),
    ], axis=1)


def make_scene(seed: int = 0, n_cuboids: int = 8, extent: float = 0.75) -> Scene:
    """Seeded oriented cuboids in a ``2*extent`` m box around the arm base."""
    rng = np.random.default_rng(seed + 1_000_003)
    centres = rng.uniform(-extent, extent, size=(n_cuboids, 3))
    rot = _random_rotations(rng, n_cuboids)
    sides = rng.uniform(0.05, 0.6, size=(n_cuboids, 3))
    pose = np.concatenate([rot, centres], axis=1).astype(np.float32)
    return Scene(pose=np.ascontiguousarray(pose),
                 half_ext=np.ascontiguousarray((0.5 * sides).astype(np.float32)))


def make_q(seed: int, n: int, limit: float = JOINT_LIMIT) -> np.ndarray:
    """``n`` joint configurations, i.i.d. uniform within the joint limits."""
    rng = np.random.default_rng(seed + 2_000_029)
    return rng.uniform(-limit, limit, size=(n, N_JOINTS)).astype(np.float32)


def make_dcost(seed: int, n: int) -> np.ndarray:
    """Upstream cost gradients for the backward pass (positive, O(1))."""
    rng = np.random.default_rng(seed + 3_000_017)
    return rng.uniform(0.5, 1.5, size=n).astype(np.float32)


@dataclasses.dataclass
class Workload:
    """One batch: ``n_traj`` trajectories x ``horizon`` timesteps."""

    robot: Robot
    scene: Scene
    q: np.ndarray
    params: CostParams
    n_traj: int
    horizon: int

    @property
    def n(self) -> int:
        return int(self.q.shape[0])


# The five evaluation workloads: (trajectories, horizon, cuboids).
WORKLOADS = {
    "single_128": (4, 32, 8),       # plain FP32, one problem, 128 configurations
    "sweep_1024": (32, 32, 20),     # per-tensor format sweep
    "particle_32768": (1024, 32, 40),  # 1024 x 32 x 52 sphere evaluations
}


def make_workload(name: str, seed: int | None = None) -> Workload:
    n_traj, horizon, n_cub = WORKLOADS[name]
    if seed is None:
        seed = list(WORKLOADS).index(name) + 1
    robot = make_robot(seed)
    scene = make_scene(seed, n_cub)
    q = make_q(seed, n_traj * horizon)
    return Workload(robot=robot, scene=scene, q=q, params=CostParams(),
                    n_traj=n_traj, horizon=horizon)


def make_uneven_problems(seed: int = 4, n_problems: int = 64):
    """Problems for the uneven batch: 4-256 trajectories, horizon 16-64,
    4-60 cuboids, per-problem sphere radii jittered by +-10 %."""
    rng = np.random.default_rng(seed + 4_000_037)
    problems = []
    for p in range(n_problems):
        n_traj = int(rng.integers(4, 257))
        horizon = int(rng.integers(16, 65))
        n_cub = int(rng.integers(4, 61))
        pseed = int(rng.integers(0, 2**31 - 1))
        robot = make_robot(seed, radius_jitter=0.1, jitter_seed=pseed)
        scene = make_scene(pseed, n_cub)
        q = make_q(pseed, n_traj * horizon)
        problems.append(Workload(robot=robot, scene=scene, q=q,
                                 params=CostParams(), n_traj=n_traj,
                                 horizon=horizon))
    return problems


# ------------------------------------------------------ surrogate training data
def uniform_points(seed: int, lo, hi, n: int) -> np.ndarray:
    """``n`` points uniform in the box [lo, hi]."""
    rng = np.random.default_rng(seed + 5_000_011)
    return rng.uniform(np.asarray(lo, np.float64), np.asarray(hi, np.float64), size=(n, 3)).astype(np.float32)


def near_surface_points(seed: int, scene: Scene, n: int, sigma: float = 0.02) -> np.ndarray:
    """``n`` points near cuboid surfaces: a cuboid drawn uniformly, a face
    drawn by area, a point uniform on the face, then Gaussian noise of
    ``sigma`` metres per axis."""
    rng = np.random.default_rng(seed + 6_000_023)
    O = scene.n_cuboids
    R = scene.pose[:, :9].reshape(O, 3, 3).astype(np.float64)
    t = scene.pose[:, 9:].astype(np.float64)
    h = scene.half_ext.astype(np.float64)
    o = rng.integers(0, O, size=n)
    area = np.stack([h[:, 1] * h[:, 2], h[:, 0] * h[:, 2], h[:, 0] * h[:, 1]], 1)[o]
    u = rng.uniform(0.0, 1.0, size=n) * area.sum(1)
    axis = (u > area[:, 0]).astype(np.int64) + (u > area[:, 0] + area[:, 1]).astype(np.int64)
    local = rng.uniform(-1.0, 1.0, size=(n, 3)) * h[o]
    sign = np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    local[np.arange(n), axis] = sign * h[o, axis]
    world = t[o] + np.einsum("nij,nj->ni", R[o], local)
    return (world + rng.normal(0.0, sigma, size=(n, 3))).astype(np.float32)


def init_mlp_params(seed: int, hidden: int = 256, w1_scale: float = 4.0) -> np.ndarray:
    """Initial surrogate parameters in the library's order (W1, b1, W2, b2,
    W3, b3, w4, b4): W1 and b1 ~ N(0, w1_scale^2) so that the first-layer
    hyperplanes cut the [-1, 1]^3 domain at many offsets, W2 and W3 ~
    N(0, 2/hidden) (He), w4 ~ N(0, 1/hidden), other biases zero."""
    rng = np.random.default_rng(seed + 7_000_003)
    H = hidden
    parts = [rng.normal(0.0, w1_scale, 3 * H), rng.normal(0.0, w1_scale, H),
             rng.normal(0.0, np.sqrt(2.0 / H), H * H), np.zeros(H),
             rng.normal(0.0, np.sqrt(2.0 / H), H * H), np.zeros(H),
             rng.normal(0.0, np.sqrt(1.0 / H), H), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)
