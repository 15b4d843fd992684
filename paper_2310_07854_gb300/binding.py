"""Thin Python binding of libvapr.so (include/vapr.h).

Each ``vapr_*`` function here has the name and argument order of the C entry
point it calls; it only marshals arguments (torch tensors -> device
pointers, the current CUDA stream) and turns a non-OK status into
``VaprError``.  All computation happens in the CUDA library: there is no
CPU or PyTorch fallback, and loading fails loudly when the library is
missing.

``DeviceRobot`` / ``DeviceScene`` hold the device copies of the seeded
tables (``synth``) together with the C structs that point at them, and
``alloc_packed`` sizes packed buffers with ``vapr_packed_row_bytes``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import formats as F

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvapr.so")

OK = 0
STATUS_NAMES = {0: "VAPR_OK", 1: "VAPR_ERR_INVALID_ARG", 2: "VAPR_ERR_UNSUPPORTED_FORMAT",
                3: "VAPR_ERR_MISALIGNED", 4: "VAPR_ERR_CUDA", 5: "VAPR_ERR_TIMEOUT",
                6: "VAPR_ERR_TOO_LARGE"}
MAX_JOINTS, MAX_SPHERES, MAX_PAIRS, MAX_CUBOIDS = 16, 128, 8128, 1024


class VaprError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _load().vapr_status_string(status).decode()
        extra = ""
        if status == 4:
            extra = f" (cudaError {_load().vapr_last_cuda_error()})"
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}{extra}")


# ------------------------------------------------------------------ structs
class vapr_format(ctypes.Structure):
    _fields_ = [("exp_bits", ctypes.c_uint8), ("man_bits", ctypes.c_uint8),
                ("flags", ctypes.c_uint8), ("reserved", ctypes.c_uint8)]


class vapr_format_table(ctypes.Structure):
    _fields_ = [(n, vapr_format) for n in ("pos", "dist", "grad", "jgrad", "xform")]


class vapr_robot(ctypes.Structure):
    _fields_ = [("n_joints", ctypes.c_int32), ("n_spheres", ctypes.c_int32),
                ("n_pairs", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("joint_fixed", ctypes.c_void_p), ("sphere_local", ctypes.c_void_p),
                ("sphere_link", ctypes.c_void_p), ("pairs", ctypes.c_void_p),
                ("tables", ctypes.c_void_p)]


class vapr_scene(ctypes.Structure):
    _fields_ = [("n_cuboids", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("pose", ctypes.c_void_p), ("half_ext", ctypes.c_void_p),
                ("grid", ctypes.c_void_p)]


class vapr_cost_params(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_float), ("eta_self", ctypes.c_float),
                ("w_coll", ctypes.c_float), ("w_self", ctypes.c_float)]


class vapr_problem(ctypes.Structure):
    _fields_ = [("robot", vapr_robot), ("scene", vapr_scene), ("params", vapr_cost_params),
                ("q", ctypes.c_void_p), ("n", ctypes.c_int64), ("dcost", ctypes.c_void_p),
                ("cost", ctypes.c_void_p), ("dist_packed", ctypes.c_void_p),
                ("jgrad_packed", ctypes.c_void_p), ("deferred", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class vapr_batch_tuning(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("wait_limit_us", ctypes.c_int32)]


class vapr_train_params(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("over_weight", ctypes.c_float)]


class vapr_surrogate_domain(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3), ("pad", ctypes.c_float),
                ("margin", ctypes.c_float)]


class vapr_ik_params(ctypes.Structure):
    _fields_ = [("w_pos", ctypes.c_float), ("w_rot", ctypes.c_float), ("w_bound", ctypes.c_float),
                ("step0", ctypes.c_float), ("n_scales", ctypes.c_int32), ("history", ctypes.c_int32),
                ("scales", ctypes.c_float * 16), ("q_lo", ctypes.c_void_p), ("q_hi", ctypes.c_void_p)]


class vapr_batch_plan(ctypes.Structure):
    _fields_ = [("opaque", ctypes.c_uint64 * 160)]


# Every exported symbol, with (restype, argtypes).
_P = ctypes.c_void_p
_i64 = ctypes.c_int64
SIGNATURES = {
    "vapr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "vapr_last_cuda_error": (ctypes.c_int, []),
    "vapr_format_default": (vapr_format, [ctypes.c_int, ctypes.c_int]),
    "vapr_format_supported": (ctypes.c_int, [vapr_format]),
    "vapr_packed_row_bytes": (ctypes.c_size_t, [_i64, vapr_format]),
    "vapr_robot_check": (ctypes.c_int, [ctypes.POINTER(vapr_robot)]),
    "vapr_device_error": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32)]),
    "vapr_pack": (ctypes.c_int, [_P, _i64, _i64, vapr_format, _P, _P]),
    "vapr_unpack": (ctypes.c_int, [_P, _i64, _i64, vapr_format, _P, _P]),
    "vapr_fk": (ctypes.c_int, [ctypes.POINTER(vapr_robot), _P, _i64,
                               ctypes.POINTER(vapr_format_table), _P, _P, _P]),
    "vapr_collision_cost": (ctypes.c_int, [ctypes.POINTER(vapr_robot), ctypes.POINTER(vapr_scene),
                                           ctypes.POINTER(vapr_cost_params), _P, _i64,
                                           ctypes.POINTER(vapr_format_table), _P, _P, _P, _P]),
    "vapr_backward": (ctypes.c_int, [ctypes.POINTER(vapr_robot), _P, _P, _P, _P, _i64,
                                     ctypes.POINTER(vapr_format_table), _P, _P]),
    "vapr_gemm_bf16": (ctypes.c_int, [_P, _P, _P, _i64, _i64, _i64, _P]),
    "vapr_cost_grad_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(vapr_robot), _i64,
                                                         ctypes.POINTER(vapr_format_table)]),
    "vapr_cost_grad": (ctypes.c_int, [ctypes.POINTER(vapr_robot), ctypes.POINTER(vapr_scene),
                                      ctypes.POINTER(vapr_cost_params), _P, _i64,
                                      ctypes.POINTER(vapr_format_table), _P, _P, _P, _P, _P,
                                      ctypes.c_size_t, _P]),
    "vapr_cost_grad_fused": (ctypes.c_int, [ctypes.POINTER(vapr_robot), ctypes.POINTER(vapr_scene),
                                            ctypes.POINTER(vapr_cost_params), _P, _i64,
                                            ctypes.POINTER(vapr_format_table), _P, _P, _P, _P, _P]),
    "vapr_batched_plan_bytes": (ctypes.c_size_t, [ctypes.POINTER(vapr_problem), ctypes.c_int32,
                                                  ctypes.POINTER(vapr_format_table),
                                                  ctypes.POINTER(vapr_batch_tuning)]),
    "vapr_batched_plan": (ctypes.c_int, [ctypes.POINTER(vapr_problem), ctypes.c_int32,
                                         ctypes.POINTER(vapr_format_table),
                                         ctypes.POINTER(vapr_batch_tuning), _P, ctypes.c_size_t,
                                         ctypes.POINTER(vapr_batch_plan)]),
    "vapr_batched_publish": (ctypes.c_int, [ctypes.POINTER(vapr_batch_plan), ctypes.c_int32, _P]),
    "vapr_batched_eval": (ctypes.c_int, [ctypes.POINTER(vapr_batch_plan), _P, _P]),
    "vapr_cost_grad_noalloc": (ctypes.c_int, [ctypes.POINTER(vapr_robot), ctypes.POINTER(vapr_scene),
                                              ctypes.POINTER(vapr_cost_params), _P, _i64,
                                              ctypes.POINTER(vapr_format_table), _P, _P, _P, _P,
                                              _P]),
    "vapr_swept_cost": (ctypes.c_int, [ctypes.POINTER(vapr_robot), ctypes.POINTER(vapr_scene),
                                       ctypes.POINTER(vapr_cost_params), _P, _i64, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.POINTER(vapr_format_table), _P, _P, _P,
                                       _P]),
    "vapr_env_ceiling": (ctypes.c_int, [ctypes.POINTER(vapr_scene), _P, _i64, ctypes.c_float,
                                        ctypes.c_float, ctypes.c_int32, _P, _P]),
    "vapr_env_ceiling_warps": (ctypes.c_int64, [ctypes.c_int32]),
    "vapr_ik_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(vapr_robot), _i64,
                                                  ctypes.POINTER(vapr_ik_params),
                                                  ctypes.POINTER(vapr_format_table)]),
    "vapr_ik_init": (ctypes.c_int, [ctypes.POINTER(vapr_robot), ctypes.POINTER(vapr_scene),
                                    ctypes.POINTER(vapr_cost_params), ctypes.POINTER(vapr_ik_params), _P, _P,
                                    _i64, ctypes.POINTER(vapr_format_table), _P, ctypes.c_size_t, _P, _P]),
    "vapr_ik_step": (ctypes.c_int, [ctypes.POINTER(vapr_robot), ctypes.POINTER(vapr_scene),
                                    ctypes.POINTER(vapr_cost_params), ctypes.POINTER(vapr_ik_params), _P, _P,
                                    _i64, ctypes.POINTER(vapr_format_table), _P, ctypes.c_size_t, _P, _P,
                                    _P]),
    "vapr_mlp_state_bytes": (ctypes.c_size_t, []),
    "vapr_mlp_init": (ctypes.c_int, [_P, _P, _P]),
    "vapr_mlp_get_params": (ctypes.c_int, [_P, _P, _P]),
    "vapr_mlp_forward": (ctypes.c_int, [_P, _P, _i64, _P, _P]),
    "vapr_mlp_workspace_bytes": (ctypes.c_size_t, [_i64]),
    "vapr_mlp_grads": (ctypes.c_int, [_P, _P, _P, _i64, ctypes.c_float, _P, ctypes.c_size_t, _P,
                                      _P, _P]),
    "vapr_mlp_train_step": (ctypes.c_int, [_P, _P, _P, _i64, ctypes.POINTER(vapr_train_params),
                                           _P, ctypes.c_size_t, _P, _P]),
    "vapr_scene_sdf": (ctypes.c_int, [ctypes.POINTER(vapr_scene), _P, _i64, _P, _P]),
    "vapr_scene_grid_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32]),
    "vapr_robot_tables_bytes": (ctypes.c_size_t, [ctypes.POINTER(vapr_robot)]),
    "vapr_robot_tables_build": (ctypes.c_int, [ctypes.POINTER(vapr_robot), _P, ctypes.c_size_t, _P]),
    "vapr_scene_grid_build": (ctypes.c_int, [ctypes.POINTER(vapr_scene), ctypes.c_float, ctypes.c_float,
                                             ctypes.c_int32, _P, ctypes.c_size_t, _P]),
    "vapr_surrogate_samples": (ctypes.c_int, [ctypes.POINTER(vapr_scene),
                                              ctypes.POINTER(vapr_surrogate_domain), _P, _i64,
                                              ctypes.c_float, ctypes.c_float, _P, _P, _P]),
    "vapr_surrogate_collision_cost": (ctypes.c_int, [ctypes.POINTER(vapr_robot),
                                                     ctypes.POINTER(vapr_scene),
                                                     ctypes.POINTER(vapr_cost_params), _P,
                                                     ctypes.POINTER(vapr_surrogate_domain), _P,
                                                     _i64, ctypes.POINTER(vapr_format_table), _P,
                                                     _P, _P, _P, _P]),
}

_lib = None
_lock = threading.Lock()


def _load():
    """Loads libvapr.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libvapr.so is missing at {LIB_PATH}; run build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def lib():
    return _load()


# ----------------------------------------------------------------- helpers
def to_c_format(f: F.Fmt) -> vapr_format:
    return vapr_format(f.E, f.M, f.flags, 0)


def to_c_table(t) -> vapr_format_table:
    if isinstance(t, vapr_format_table):
        return t
    return vapr_format_table(*(to_c_format(getattr(t, n)) for n in F.TENSORS))


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int, where: str):
    if status != OK:
        raise VaprError(status, where)


class DeviceRobot:
    """Device copies of a ``synth.Robot`` and the ``vapr_robot`` pointing at
    them, with the robot's prebuilt tables attached (``tables=False``: none,
    every launch builds its own)."""

    def __init__(self, robot, device="cuda", tables=True):
        import torch
        self.host = robot
        self.joint_fixed = torch.as_tensor(np.ascontiguousarray(robot.joint_fixed, np.float32), device=device)
        self.sphere_local = torch.as_tensor(np.ascontiguousarray(robot.sphere_local, np.float32), device=device)
        self.sphere_link = torch.as_tensor(np.ascontiguousarray(robot.sphere_link, np.int32), device=device)
        pairs = np.ascontiguousarray(robot.pairs, np.int32).reshape(-1, 2)
        self.pairs = torch.as_tensor(pairs if pairs.size else np.zeros((1, 2), np.int32), device=device)
        self.c = vapr_robot(robot.n_joints, robot.n_spheres, int(pairs.shape[0]), 0,
                            self.joint_fixed.data_ptr(), self.sphere_local.data_ptr(),
                            self.sphere_link.data_ptr(), self.pairs.data_ptr(), None)
        self.tables = None
        if tables:
            self.build_tables()

    def build_tables(self, stream=None):
        """Builds the robot tables (``vapr_robot_tables_build``) and attaches
        them (``vapr_robot.tables``)."""
        import torch
        nb = vapr_robot_tables_bytes(self)
        buf = torch.empty(nb, dtype=torch.uint8, device=self.joint_fixed.device)
        self.c.tables = None
        vapr_robot_tables_build(self, buf, nb, stream)
        self.tables = buf
        self.c.tables = buf.data_ptr()
        return self

    def drop_tables(self):
        self.tables = None
        self.c.tables = None

    @property
    def n_joints(self):
        return self.c.n_joints

    @property
    def n_spheres(self):
        return self.c.n_spheres


class DeviceScene:
    def __init__(self, scene, device="cuda"):
        import torch
        self.host = scene
        n = scene.n_cuboids
        pose = np.ascontiguousarray(scene.pose, np.float32).reshape(-1, 12)
        half = np.ascontiguousarray(scene.half_ext, np.float32).reshape(-1, 3)
        if n == 0:  # keep valid (unused) pointers for an empty scene
            pose, half = np.zeros((1, 12), np.float32), np.zeros((1, 3), np.float32)
        self.pose = torch.as_tensor(pose, device=device)
        self.half_ext = torch.as_tensor(half, device=device)
        self.c = vapr_scene(n, 0, self.pose.data_ptr(), self.half_ext.data_ptr(), None)
        self.grid = None
        self.grid_cells = None

    def build_grid(self, reach: float, eta: float, cells: int = 64, stream=None):
        """Builds the broad-phase grid for spheres of radius <= reach and this
        eta and attaches it to the scene (``vapr_scene.grid``)."""
        import torch
        nb = vapr_scene_grid_bytes(self.c.n_cuboids, cells)
        if nb == 0:
            raise ValueError(f"no grid of {cells} cells per axis")
        buf = torch.empty(nb, dtype=torch.uint8, device=self.pose.device)
        vapr_scene_grid_build(self, reach, eta, cells, buf, nb, stream)
        self.grid = buf
        self.grid_cells = cells
        self.c.grid = buf.data_ptr()
        return self

    def drop_grid(self):
        self.grid = None
        self.grid_cells = None
        self.c.grid = None


def cost_params(p) -> vapr_cost_params:
    return vapr_cost_params(p.eta, p.eta_self, p.w_coll, p.w_self)


def packed_row_bytes(row_len: int, fmt: F.Fmt) -> int:
    return int(_load().vapr_packed_row_bytes(row_len, to_c_format(fmt)))


def alloc_packed(rows: int, row_len: int, fmt: F.Fmt, device="cuda"):
    """A uint8 tensor [rows, row_bytes] for packed rows (16-byte aligned)."""
    import torch
    rb = packed_row_bytes(row_len, fmt)
    return torch.empty((rows, rb), dtype=torch.uint8, device=device)


# ---------------------------------------------- entry points (same names)
def vapr_format_default(exp_bits: int, man_bits: int) -> vapr_format:
    return _load().vapr_format_default(exp_bits, man_bits)


def vapr_format_supported(f: vapr_format) -> bool:
    return bool(_load().vapr_format_supported(f))


def vapr_packed_row_bytes(row_len: int, f: vapr_format) -> int:
    return int(_load().vapr_packed_row_bytes(row_len, f))


def vapr_device_error() -> int:
    """Reads and clears the sticky device error word (0 = none)."""
    v = ctypes.c_int32(0)
    _check(_load().vapr_device_error(ctypes.byref(v)), "vapr_device_error")
    return int(v.value)


def vapr_robot_check(robot: DeviceRobot):
    _check(_load().vapr_robot_check(ctypes.byref(robot.c)), "vapr_robot_check")


def vapr_pack(src, rows, row_len, fmt: F.Fmt, dst, stream=None):
    _check(_load().vapr_pack(_ptr(src), rows, row_len, to_c_format(fmt), _ptr(dst),
                             _stream(stream)), "vapr_pack")


def vapr_unpack(src, rows, row_len, fmt: F.Fmt, dst, stream=None):
    _check(_load().vapr_unpack(_ptr(src), rows, row_len, to_c_format(fmt), _ptr(dst),
                               _stream(stream)), "vapr_unpack")


def vapr_fk(robot: DeviceRobot, q, n, table: F.FormatTable, pos_packed, xform_packed=None,
            stream=None):
    ct = to_c_table(table)
    _check(_load().vapr_fk(ctypes.byref(robot.c), _ptr(q), n, ctypes.byref(ct),
                           _ptr(pos_packed), _ptr(xform_packed), _stream(stream)), "vapr_fk")


def vapr_collision_cost(robot: DeviceRobot, scene: DeviceScene, params, pos_packed, n,
                        table: F.FormatTable, cost=None, dist_packed=None, grad_packed=None,
                        stream=None):
    ct = to_c_table(table)
    cp = params if isinstance(params, vapr_cost_params) else cost_params(params)
    _check(_load().vapr_collision_cost(ctypes.byref(robot.c), ctypes.byref(scene.c),
                                       ctypes.byref(cp), _ptr(pos_packed), n, ctypes.byref(ct),
                                       _ptr(cost), _ptr(dist_packed), _ptr(grad_packed),
                                       _stream(stream)), "vapr_collision_cost")


def vapr_swept_cost(robot: DeviceRobot, scene: DeviceScene, params, pos_packed, n, horizon, samples,
                    table, cost=None, dist_packed=None, grad_packed=None, stream=None):
    ct = to_c_table(table)
    cp = params if isinstance(params, vapr_cost_params) else cost_params(params)
    _check(_load().vapr_swept_cost(ctypes.byref(robot.c), ctypes.byref(scene.c), ctypes.byref(cp),
                                   _ptr(pos_packed), n, horizon, samples, ctypes.byref(ct), _ptr(cost),
                                   _ptr(dist_packed), _ptr(grad_packed), _stream(stream)),
           "vapr_swept_cost")


def vapr_env_ceiling(scene: DeviceScene, spheres, n, eta, w_coll, reps, out, stream=None):
    """spheres, out: float32 [n, 4] device tensors (x, y, z, r) -> (D, G)."""
    _check(_load().vapr_env_ceiling(ctypes.byref(scene.c), _ptr(spheres), n, eta, w_coll, reps,
                                    _ptr(out), _stream(stream)), "vapr_env_ceiling")


def vapr_env_ceiling_warps(n_cuboids: int) -> int:
    return int(_load().vapr_env_ceiling_warps(n_cuboids))


def vapr_backward(robot: DeviceRobot, q, xform_packed, grad_packed, dcost, n,
                  table: F.FormatTable, jgrad_packed, stream=None):
    ct = to_c_table(table)
    _check(_load().vapr_backward(ctypes.byref(robot.c), _ptr(q), _ptr(xform_packed),
                                 _ptr(grad_packed), _ptr(dcost), n, ctypes.byref(ct),
                                 _ptr(jgrad_packed), _stream(stream)), "vapr_backward")


def vapr_cost_grad_workspace_bytes(robot: DeviceRobot, n: int, table) -> int:
    ct = to_c_table(table)
    return int(_load().vapr_cost_grad_workspace_bytes(ctypes.byref(robot.c), n, ctypes.byref(ct)))


def alloc_workspace(robot: DeviceRobot, n: int, table, device="cuda"):
    """A device buffer of vapr_cost_grad_workspace_bytes (256-byte aligned:
    torch's allocator aligns blocks to at least 512 bytes)."""
    import torch
    nbytes = max(vapr_cost_grad_workspace_bytes(robot, n, table), 256)
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def vapr_cost_grad(robot: DeviceRobot, scene: DeviceScene, params, q, n, table, dcost, cost,
                   dist_packed, jgrad_packed, workspace, workspace_bytes=None, stream=None):
    ct = to_c_table(table)
    cp = params if isinstance(params, vapr_cost_params) else cost_params(params)
    nbytes = workspace.numel() if workspace_bytes is None else workspace_bytes
    _check(_load().vapr_cost_grad(ctypes.byref(robot.c), ctypes.byref(scene.c), ctypes.byref(cp),
                                  _ptr(q), n, ctypes.byref(ct), _ptr(dcost), _ptr(cost),
                                  _ptr(dist_packed), _ptr(jgrad_packed), _ptr(workspace),
                                  nbytes, _stream(stream)), "vapr_cost_grad")


def vapr_cost_grad_fused(robot: DeviceRobot, scene: DeviceScene, params, q, n, table, dcost, cost,
                         dist_packed, jgrad_packed, stream=None):
    """The step in one kernel, P and G kept on the SM (see include/vapr.h)."""
    ct = to_c_table(table)
    cp = params if isinstance(params, vapr_cost_params) else cost_params(params)
    _check(_load().vapr_cost_grad_fused(ctypes.byref(robot.c), ctypes.byref(scene.c), ctypes.byref(cp),
                                        _ptr(q), n, ctypes.byref(ct), _ptr(dcost), _ptr(cost),
                                        _ptr(dist_packed), _ptr(jgrad_packed), _stream(stream)),
           "vapr_cost_grad_fused")


NOALLOC_SCRATCH_BYTES = 64 << 20  # VAPR_NOALLOC_SCRATCH_BYTES


def vapr_cost_grad_noalloc(robot: DeviceRobot, scene: DeviceScene, params, q, n, table, dcost,
                           cost, dist_packed, jgrad_packed, stream=None):
    """vapr_cost_grad without a workspace argument: for callers that cannot
    allocate device memory while they run (see include/vapr.h)."""
    ct = to_c_table(table)
    cp = params if isinstance(params, vapr_cost_params) else cost_params(params)
    _check(_load().vapr_cost_grad_noalloc(ctypes.byref(robot.c), ctypes.byref(scene.c),
                                          ctypes.byref(cp), _ptr(q), n, ctypes.byref(ct),
                                          _ptr(dcost), _ptr(cost), _ptr(dist_packed),
                                          _ptr(jgrad_packed), _stream(stream)),
           "vapr_cost_grad_noalloc")


def vapr_batched_plan_bytes(problems, table, tuning) -> int:
    ct = to_c_table(table)
    return int(_load().vapr_batched_plan_bytes(problems, len(problems), ctypes.byref(ct),
                                               ctypes.byref(tuning)))


def vapr_batched_plan(problems, table, tuning, plan_dev, plan: "vapr_batch_plan"):
    ct = to_c_table(table)
    nbytes = plan_dev.numel() if hasattr(plan_dev, "numel") else int(plan_dev[1])
    _check(_load().vapr_batched_plan(problems, len(problems), ctypes.byref(ct),
                                     ctypes.byref(tuning), _ptr(plan_dev), nbytes,
                                     ctypes.byref(plan)), "vapr_batched_plan")


def vapr_batched_publish(plan: "vapr_batch_plan", problem: int, stream=None):
    _check(_load().vapr_batched_publish(ctypes.byref(plan), problem, _stream(stream)),
           "vapr_batched_publish")


def vapr_batched_eval(plan: "vapr_batch_plan", dev_status, stream=None):
    _check(_load().vapr_batched_eval(ctypes.byref(plan), _ptr(dev_status), _stream(stream)),
           "vapr_batched_eval")


def vapr_gemm_bf16(A, B_, C, M, N, K, stream=None):
    """C[M,N] (float32) = A[M,K] @ B_[N,K]^T with bfloat16 A, B_ on tcgen05."""
    _check(_load().vapr_gemm_bf16(_ptr(A), _ptr(B_), _ptr(C), M, N, K, _stream(stream)),
           "vapr_gemm_bf16")


# ---------------------------------------------------------------- surrogate
MLP_HIDDEN = 256
MLP_PARAMS = 2 * 256 * 256 + 7 * 256 + 1


def vapr_mlp_state_bytes() -> int:
    return int(_load().vapr_mlp_state_bytes())


def alloc_mlp_state(device="cuda"):
    """A uint8 tensor of vapr_mlp_state_bytes() bytes (256-byte aligned)."""
    import torch
    return torch.empty(vapr_mlp_state_bytes(), dtype=torch.uint8, device=device)


def vapr_mlp_init(state, params, stream=None):
    _check(_load().vapr_mlp_init(_ptr(state), _ptr(params), _stream(stream)), "vapr_mlp_init")


def vapr_mlp_get_params(state, params, stream=None):
    _check(_load().vapr_mlp_get_params(_ptr(state), _ptr(params), _stream(stream)),
           "vapr_mlp_get_params")


def vapr_mlp_forward(state, u, n, out, stream=None):
    _check(_load().vapr_mlp_forward(_ptr(state), _ptr(u), n, _ptr(out), _stream(stream)),
           "vapr_mlp_forward")


def vapr_mlp_workspace_bytes(batch: int) -> int:
    return int(_load().vapr_mlp_workspace_bytes(batch))


def alloc_mlp_workspace(batch: int, device="cuda"):
    import torch
    nb = vapr_mlp_workspace_bytes(batch)
    if nb == 0:
        raise VaprError(1, "vapr_mlp_workspace_bytes")
    return torch.empty(nb, dtype=torch.uint8, device=device)


def vapr_mlp_grads(state, u, y, batch, workspace, grads=None, loss=None, over_weight=1.0,
                   stream=None):
    _check(_load().vapr_mlp_grads(_ptr(state), _ptr(u), _ptr(y), batch, over_weight, _ptr(workspace),
                                  workspace.numel() if workspace is not None else 0, _ptr(grads),
                                  _ptr(loss), _stream(stream)), "vapr_mlp_grads")


def vapr_mlp_train_step(state, u, y, batch, hp, workspace, loss=None, stream=None):
    """hp: vapr_train_params or (lr, beta1, beta2, eps[, over_weight])."""
    if isinstance(hp, vapr_train_params):
        a = hp
    else:
        hp = tuple(hp)
        a = vapr_train_params(*(hp + (1.0,) * (5 - len(hp))))
    _check(_load().vapr_mlp_train_step(_ptr(state), _ptr(u), _ptr(y), batch, ctypes.byref(a),
                                       _ptr(workspace),
                                       workspace.numel() if workspace is not None else 0,
                                       _ptr(loss), _stream(stream)), "vapr_mlp_train_step")


def vapr_scene_sdf(scene: DeviceScene, pts, n, sdf, stream=None):
    _check(_load().vapr_scene_sdf(ctypes.byref(scene.c), _ptr(pts), n, _ptr(sdf), _stream(stream)),
           "vapr_scene_sdf")


def vapr_scene_grid_bytes(n_cuboids: int, cells_per_axis: int) -> int:
    return int(_load().vapr_scene_grid_bytes(n_cuboids, cells_per_axis))


def vapr_scene_grid_build(scene: DeviceScene, reach, eta, cells_per_axis, grid, grid_bytes, stream=None):
    _check(_load().vapr_scene_grid_build(ctypes.byref(scene.c), float(reach), float(eta), int(cells_per_axis),
                                         _ptr(grid), int(grid_bytes), _stream(stream)),
           "vapr_scene_grid_build")


def vapr_robot_tables_bytes(robot: "DeviceRobot") -> int:
    return int(_load().vapr_robot_tables_bytes(ctypes.byref(robot.c)))


def vapr_robot_tables_build(robot: "DeviceRobot", tables, nbytes, stream=None):
    _check(_load().vapr_robot_tables_build(ctypes.byref(robot.c), _ptr(tables), int(nbytes), _stream(stream)),
           "vapr_robot_tables_build")


def surrogate_domain(lo, hi, pad, margin) -> vapr_surrogate_domain:
    d = vapr_surrogate_domain()
    for j in range(3):
        d.lo[j] = float(lo[j])
        d.hi[j] = float(hi[j])
    d.pad = float(pad)
    d.margin = float(margin)
    return d


FLT_MAX = float(np.finfo(np.float32).max)


def vapr_surrogate_samples(scene: DeviceScene, domain: vapr_surrogate_domain, pts, n, u, y,
                           y_min=-FLT_MAX, y_max=FLT_MAX, stream=None):
    _check(_load().vapr_surrogate_samples(ctypes.byref(scene.c), ctypes.byref(domain), _ptr(pts), n,
                                          y_min, y_max, _ptr(u), _ptr(y), _stream(stream)),
           "vapr_surrogate_samples")


def vapr_surrogate_collision_cost(robot: DeviceRobot, scene: DeviceScene, params, state,
                                  domain: vapr_surrogate_domain, pos_packed, n, table, cost=None,
                                  dist_packed=None, grad_packed=None, estimate=None, stream=None):
    ct = to_c_table(table)
    cp = params if isinstance(params, vapr_cost_params) else cost_params(params)
    _check(_load().vapr_surrogate_collision_cost(
        ctypes.byref(robot.c), ctypes.byref(scene.c), ctypes.byref(cp), _ptr(state),
        ctypes.byref(domain), _ptr(pos_packed), n, ctypes.byref(ct), _ptr(cost),
        _ptr(dist_packed), _ptr(grad_packed), _ptr(estimate), _stream(stream)),
        "vapr_surrogate_collision_cost")


# ------------------------------------------------------------- IK iteration
IK_MAX_SCALES = 16


def ik_params(w_pos, w_rot, w_bound, step0, scales, history, q_lo, q_hi) -> vapr_ik_params:
    """q_lo, q_hi: device float32 tensors [J] (kept alive by the caller)."""
    p = vapr_ik_params()
    p.w_pos, p.w_rot, p.w_bound, p.step0 = float(w_pos), float(w_rot), float(w_bound), float(step0)
    p.n_scales, p.history = len(scales), int(history)
    for k, a in enumerate(scales):
        p.scales[k] = float(a)
    p.q_lo, p.q_hi = _ptr(q_lo), _ptr(q_hi)
    return p


def vapr_ik_workspace_bytes(robot: DeviceRobot, n_seeds: int, ik: vapr_ik_params, table) -> int:
    ct = to_c_table(table)
    return int(_load().vapr_ik_workspace_bytes(ctypes.byref(robot.c), n_seeds, ctypes.byref(ik), ctypes.byref(ct)))


def vapr_ik_init(robot: DeviceRobot, scene: DeviceScene, params, ik, goal, q, n_seeds, table, workspace,
                 cost=None, stream=None):
    ct = to_c_table(table)
    cp = params if isinstance(params, vapr_cost_params) else cost_params(params)
    _check(_load().vapr_ik_init(ctypes.byref(robot.c), ctypes.byref(scene.c), ctypes.byref(cp), ctypes.byref(ik),
                                _ptr(goal), _ptr(q), n_seeds, ctypes.byref(ct), _ptr(workspace),
                                workspace.numel(), _ptr(cost), _stream(stream)), "vapr_ik_init")


def vapr_ik_step(robot: DeviceRobot, scene: DeviceScene, params, ik, goal, q, n_seeds, table, workspace,
                 cost=None, pick=None, stream=None):
    ct = to_c_table(table)
    cp = params if isinstance(params, vapr_cost_params) else cost_params(params)
    _check(_load().vapr_ik_step(ctypes.byref(robot.c), ctypes.byref(scene.c), ctypes.byref(cp), ctypes.byref(ik),
                                _ptr(goal), _ptr(q), n_seeds, ctypes.byref(ct), _ptr(workspace),
                                workspace.numel(), _ptr(cost), _ptr(pick), _stream(stream)), "vapr_ik_step")
