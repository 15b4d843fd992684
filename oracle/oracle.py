"""numpy front end of the FP64 C oracle (``vapr_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product path.

Every function converts its float32 inputs once and hands them to the C
code, which computes in double precision.  See ``vapr_oracle.h`` for the
readings of the paper each function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vapr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

# Special-value classes, mirroring the OR_* constants of vapr_oracle.h.
IEEE = 1
FN = 2
SAT = 4

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (OpenMP when available)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(os.path.join(_HERE, "vapr_oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
            "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i32, i64, u32, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
        sig = {
            "or_exmy_encode": (u32, [ctypes.c_float, i32, i32, u32]),
            "or_exmy_decode": (dbl, [u32, i32, i32, u32]),
            "or_exmy_max_finite": (dbl, [i32, i32, u32]),
            "or_exmy_encode_batch": (None, [P, i64, i32, i32, u32, P]),
            "or_exmy_encode_bits_range": (None, [u32, i64, i32, i32, u32, P]),
            "or_exmy_decode_batch": (None, [P, i64, i32, i32, u32, P]),
            "or_pack_rows": (None, [P, i64, i64, i32, P, i64]),
            "or_unpack_rows": (None, [P, i64, i64, i32, i64, P]),
            "or_fk": (None, [i32, P, i32, P, P, P, i64, P, P]),
            "or_box_sdf_batch": (None, [P, P, P, i64, P, P]),
            "or_collision": (None, [i32, P, i32, P, i32, P, P, dbl, dbl, dbl,
                                    dbl, P, i64, P, P, P, P, dbl]),
            "or_backward": (None, [i32, P, i32, P, P, P, P, P, i64, P]),
            "or_scene_sdf": (None, [i32, P, P, P, i64, P]),
            "or_mlp_forward": (None, [P, i32, P, i64, P]),
            "or_mlp_forward_bf16act": (None, [P, i32, P, i64, P]),
            "or_mlp_grads": (dbl, [P, i32, P, P, i64, dbl, P]),
            "or_swept": (None, [i32, P, i32, P, P, dbl, dbl, P, i64, i32, i32, P, P, P, P, dbl]),
            "or_ik_costs": (None, [i32, P, i32, P, P, i32, P, i32, P, P, dbl, dbl, dbl, dbl, dbl, dbl,
                                   dbl, P, P, P, P, i64, P, P]),
            "or_lbfgs_direction": (None, [i32, i32, P, P, P, P]),
            "or_num_threads": (i32, []),
            "or_set_num_threads": (None, [i32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops over configurations from now on."""
    _load().or_set_num_threads(int(n))


# ----------------------------------------------------------------- formats
def default_flags(E: int, M: int) -> int:
    """Special-value class of each format (reading; Sec. IV-A is silent):
    float32/bfloat16/half are IEEE with overflow to Inf; E5M2 is IEEE with
    saturation; E4M3 is the OCP "fn" variant (no Inf, one NaN, saturation);
    every other ExMy format is finite-only and saturates."""
    if (E, M) in ((8, 23), (8, 7), (5, 10)):
        return IEEE
    if (E, M) == (5, 2):
        return IEEE | SAT
    if (E, M) == (4, 3):
        return FN | SAT
    if E == 8:
        # 8 exponent bits: Inf/NaN reserved as in bfloat16, saturating
        return IEEE | SAT
    return SAT


def encode(x, E: int, M: int, flags: int | None = None) -> np.ndarray:
    flags = default_flags(E, M) if flags is None else flags
    x = _c(x, np.float32)
    out = np.empty(x.shape, np.uint32)
    _load().or_exmy_encode_batch(_p(x), x.size, E, M, flags, _p(out))
    return out


def encode_bits_range(start: int, count: int, E: int, M: int,
                      flags: int | None = None) -> np.ndarray:
    flags = default_flags(E, M) if flags is None else flags
    out = np.empty(count, np.uint32)
    _load().or_exmy_encode_bits_range(start, count, E, M, flags, _p(out))
    return out


def decode(codes, E: int, M: int, flags: int | None = None) -> np.ndarray:
    flags = default_flags(E, M) if flags is None else flags
    codes = _c(codes, np.uint32)
    out = np.empty(codes.shape, np.float64)
    _load().or_exmy_decode_batch(_p(codes), codes.size, E, M, flags, _p(out))
    return out


def quantize(x, E: int, M: int, flags: int | None = None) -> np.ndarray:
    """float32 -> format -> exact value (float64)."""
    return decode(encode(x, E, M, flags), E, M, flags)


def max_finite(E: int, M: int, flags: int | None = None) -> float:
    flags = default_flags(E, M) if flags is None else flags
    return float(_load().or_exmy_max_finite(E, M, flags))


def packed_row_bytes(row_len: int, bits: int) -> int:
    """Bytes of one packed row: floor(32/bits) codes per 32-bit word, the
    row padded to a multiple of 16 bytes."""
    k = 32 // bits
    words = -(-row_len // k)
    return -(-4 * words // 16) * 16


def pack_rows(codes, bits: int, row_stride: int | None = None) -> np.ndarray:
    codes = _c(codes, np.uint32)
    rows, row_len = codes.shape
    stride = packed_row_bytes(row_len, bits) if row_stride is None else row_stride
    out = np.empty((rows, stride), np.uint8)
    _load().or_pack_rows(_p(codes), rows, row_len, bits, _p(out), stride)
    return out


def unpack_rows(packed, row_len: int, bits: int) -> np.ndarray:
    packed = _c(packed, np.uint8)
    rows, stride = packed.shape
    out = np.empty((rows, row_len), np.uint32)
    _load().or_unpack_rows(_p(packed), rows, row_len, bits, stride, _p(out))
    return out


# -------------------------------------------------------------- kinematics
def fk(robot, q, with_xform: bool = False):
    """-> pos [n, S, 3] (and xform [n, J, 12]) in float64."""
    q = _c(q, np.float32)
    n = q.shape[0]
    nj, ns = robot.joint_fixed.shape[0], robot.sphere_local.shape[0]
    pos = np.empty((n, ns, 3), np.float64)
    xf = np.empty((n, nj, 12), np.float64) if with_xform else None
    _load().or_fk(nj, _p(_c(robot.joint_fixed, np.float32)), ns,
                  _p(_c(robot.sphere_local, np.float32)),
                  _p(_c(robot.sphere_link, np.int32)), _p(q), n, _p(xf), _p(pos))
    return (pos, xf) if with_xform else pos


def box_sdf(pose, half, pts):
    """Per-row signed distance of point i to cuboid i -> (d [m], grad [m, 3])."""
    pose = _c(pose, np.float32).reshape(-1, 12)
    half = _c(half, np.float32).reshape(-1, 3)
    pts = _c(pts, np.float64).reshape(-1, 3)
    m = pts.shape[0]
    d = np.empty(m, np.float64)
    g = np.empty((m, 3), np.float64)
    _load().or_box_sdf_batch(_p(pose), _p(half), _p(pts), m, _p(d), _p(g))
    return d, g


def scene_sdf(scene, pts):
    pts = _c(pts, np.float64).reshape(-1, 3)
    out = np.empty(pts.shape[0], np.float64)
    _load().or_scene_sdf(scene.pose.shape[0], _p(_c(scene.pose, np.float32)),
                         _p(_c(scene.half_ext, np.float32)), _p(pts),
                         pts.shape[0], _p(out))
    return out


def collision(robot, scene, params, pos, kink_eps: float = 1e-4):
    """-> dict(cost [n], dist [n, S], grad [n, S, 3], kink [n, S])."""
    pos = _c(pos, np.float64)
    n, ns = pos.shape[0], pos.shape[1]
    cost = np.empty(n, np.float64)
    dist = np.empty((n, ns), np.float64)
    grad = np.empty((n, ns, 3), np.float64)
    kink = np.empty((n, ns), np.int32)
    pairs = _c(robot.pairs, np.int32).reshape(-1, 2)
    _load().or_collision(ns, _p(_c(robot.sphere_local, np.float32)),
                         pairs.shape[0], _p(pairs), scene.pose.shape[0],
                         _p(_c(scene.pose, np.float32)),
                         _p(_c(scene.half_ext, np.float32)),
                         params.eta, params.eta_self, params.w_coll,
                         params.w_self, _p(pos), n, _p(cost), _p(dist),
                         _p(grad), _p(kink), kink_eps)
    return {"cost": cost, "dist": dist, "grad": grad, "kink": kink.astype(bool)}


def swept(robot, scene, params, pos, horizon: int, samples: int, kink_eps: float = 1e-4):
    """Swept-sphere environment cost -> dict(cost [n], dist [n, S], grad [n, S, 3], kink [n, S])."""
    pos = _c(pos, np.float64)
    n, ns = pos.shape[0], pos.shape[1]
    cost = np.empty(n, np.float64)
    dist = np.empty((n, ns), np.float64)
    grad = np.empty((n, ns, 3), np.float64)
    kink = np.empty((n, ns), np.int32)
    _load().or_swept(ns, _p(_c(robot.sphere_local, np.float32)), scene.pose.shape[0],
                     _p(_c(scene.pose, np.float32)), _p(_c(scene.half_ext, np.float32)),
                     float(params.eta), float(params.w_coll), _p(pos), n, horizon, samples,
                     _p(cost), _p(dist), _p(grad), _p(kink), float(kink_eps))
    return {"cost": cost, "dist": dist, "grad": grad, "kink": kink.astype(bool)}


def backward(robot, q, grad, dcost=None):
    """-> jgrad [n, J] float64."""
    q = _c(q, np.float32)
    n = q.shape[0]
    nj, ns = robot.joint_fixed.shape[0], robot.sphere_local.shape[0]
    grad = _c(grad, np.float64)
    dc = None if dcost is None else _c(dcost, np.float64)
    out = np.empty((n, nj), np.float64)
    _load().or_backward(nj, _p(_c(robot.joint_fixed, np.float32)), ns,
                        _p(_c(robot.sphere_local, np.float32)),
                        _p(_c(robot.sphere_link, np.int32)), _p(q), _p(grad),
                        _p(dc), n, _p(out))
    return out


def cost_and_grad(robot, scene, params, q, dcost=None):
    """The whole path in FP64: q -> (pos, collision dict, jgrad)."""
    pos = fk(robot, q)
    col = collision(robot, scene, params, pos)
    jg = backward(robot, q, col["grad"], dcost)
    return pos, col, jg


# ------------------------------------------------------------- surrogate
def mlp_param_count(H: int = 256) -> int:
    return 2 * H * H + 7 * H + 1


def mlp_forward(params, x, H: int = 256, bf16_activations: bool = False):
    """f(x) for points x [n, 3] (float32 params in the documented order).
    bf16_activations rounds the inputs of the two H x H layers to bfloat16."""
    params = _c(params, np.float32)
    x = _c(x, np.float32).reshape(-1, 3)
    out = np.empty(x.shape[0], np.float64)
    fn = _load().or_mlp_forward_bf16act if bf16_activations else _load().or_mlp_forward
    fn(_p(params), H, _p(x), x.shape[0], _p(out))
    return out


def mlp_grads(params, x, y, H: int = 256, over_weight: float = 1.0):
    """(loss, dloss/dparams) of the squared error, residuals f > y weighted
    by over_weight (1: the mean squared error)."""
    params = _c(params, np.float32)
    x = _c(x, np.float32).reshape(-1, 3)
    y = _c(y, np.float32)
    g = np.empty(mlp_param_count(H), np.float64)
    loss = _load().or_mlp_grads(_p(params), H, _p(x), _p(y), x.shape[0], float(over_weight), _p(g))
    return float(loss), g


# ------------------------------------------------------------- IK iteration
def ik_costs(robot, scene, params, ik, goal, q):
    """Total cost [n] and gradient [n, J] of configurations q against goals
    [n, 12]; ik has w_pos, w_rot, w_bound, q_lo [J], q_hi [J]."""
    q = _c(q, np.float32).reshape(-1, robot.joint_fixed.shape[0])
    n, nj = q.shape
    goal = _c(goal, np.float32).reshape(n, 12)
    pairs = _c(robot.pairs, np.int32).reshape(-1, 2)
    cost = np.empty(n, np.float64)
    grad = np.empty((n, nj), np.float64)
    _load().or_ik_costs(nj, _p(_c(robot.joint_fixed, np.float32)), robot.sphere_local.shape[0],
                        _p(_c(robot.sphere_local, np.float32)), _p(_c(robot.sphere_link, np.int32)),
                        pairs.shape[0], _p(pairs), scene.pose.shape[0], _p(_c(scene.pose, np.float32)),
                        _p(_c(scene.half_ext, np.float32)), params.eta, params.eta_self, params.w_coll,
                        params.w_self, ik.w_pos, ik.w_rot, ik.w_bound,
                        _p(_c(ik.q_lo, np.float32)), _p(_c(ik.q_hi, np.float32)), _p(goal), _p(q), n,
                        _p(cost), _p(grad))
    return cost, grad


def lbfgs_direction(s, y, g):
    """-H g from stored pairs s, y [m, dim] (oldest first)."""
    g = _c(g, np.float64)
    dim = g.shape[0]
    s = _c(s, np.float64).reshape(-1, dim)
    y = _c(y, np.float64).reshape(-1, dim)
    d = np.empty(dim, np.float64)
    _load().or_lbfgs_direction(dim, s.shape[0], _p(s), _p(y), _p(g), _p(d))
    return d


def ik_initial_direction(g, step0: float):
    """Steepest descent scaled so that the largest joint move at step 1 is step0."""
    g = np.asarray(g, np.float64)
    return -g * (step0 / max(np.max(np.abs(g)), 1e-30))


def ik_iterate(robot, scene, params, ik, goal, q0, iters: int):
    """Batched IK optimisation in FP64 following Sec. III-B's iteration: N
    step scales along the direction, costs and gradients of every candidate,
    the lowest-cost candidate kept (a line search over the scales), then the
    L-BFGS direction from the updated history.  A step whose best scale is 0
    clears the history and restarts from steepest descent.  Candidates are
    rounded to float32 before evaluation, as a float32 solver holds them.
    ik: w_pos, w_rot, w_bound, q_lo, q_hi, scales, history, step0.
    Returns dict(q [iters+1, n, J], cost [iters+1, n], pick [iters, n])."""
    q = np.asarray(q0, np.float64).copy()
    n, J = q.shape
    goal = np.asarray(goal, np.float32)
    f, g = ik_costs(robot, scene, params, ik, goal, q.astype(np.float32))
    d = np.stack([ik_initial_direction(g[i], ik.step0) for i in range(n)])
    hist = [[] for _ in range(n)]
    scales = np.asarray(ik.scales, np.float64)
    N = len(scales)
    qs, fs, picks = [q.copy()], [f.copy()], []
    for _ in range(iters):
        cand = (q[:, None, :] + scales[None, :, None] * d[:, None, :]).astype(np.float32)
        fc, gc = ik_costs(robot, scene, params, ik, np.repeat(goal, N, 0), cand.reshape(-1, J))
        fc, gc = fc.reshape(n, N), gc.reshape(n, N, J)
        pick = np.argmin(fc, axis=1)
        for i in range(n):
            k = pick[i]
            qn, gn = cand[i, k].astype(np.float64), gc[i, k]
            if scales[k] == 0.0:
                hist[i] = []
                d[i] = ik_initial_direction(gn, ik.step0)
            else:
                s, y = qn - q[i], gn - g[i]
                if s @ y > 0.0:
                    hist[i].append((s, y))
                    hist[i] = hist[i][-ik.history:]
                if hist[i]:
                    S = np.array([h[0] for h in hist[i]])
                    Y = np.array([h[1] for h in hist[i]])
                    d[i] = lbfgs_direction(S, Y, gn)
                else:
                    d[i] = ik_initial_direction(gn, ik.step0)
            q[i], g[i], f[i] = qn, gn, fc[i, k]
        qs.append(q.copy())
        fs.append(f.copy())
        picks.append(pick)
    return {"q": np.array(qs), "cost": np.array(fs), "pick": np.array(picks)}
