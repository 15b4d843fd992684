"""Shared helpers of the GPU parity tests.

Inputs are drawn by ``synth``; every expected value comes from the FP64
oracle (``oracle/``), never from the CUDA path.  Packed tensors produced on
the GPU are decoded on the host by the oracle's own unpacker and decoder.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F

# The FP32 path must match FP64 to 1e-5 relative (normwise per tensor).
REL_TOL = 1e-5
# Float32 arithmetic error bound used when a float decides a quantised code:
# the GPU value before rounding lies within FP32_BAND * scale of the FP64 one.
FP32_BAND = 4e-6
# Spheres this close (metres) to a gradient discontinuity are left out of
# elementwise gradient comparisons (the float32 error is ~1e-7 m).
KINK_EPS = 1e-5


def torch():
    import torch as t
    return t


def to_dev(a):
    return torch().as_tensor(np.ascontiguousarray(a), device="cuda")


def decode_packed(packed, row_len: int, fmt: F.Fmt) -> np.ndarray:
    """GPU packed rows (torch uint8 [rows, stride]) -> exact float64 values."""
    host = packed.cpu().numpy()
    codes = oracle.unpack_rows(host, row_len, fmt.bits)
    return oracle.decode(codes, fmt.E, fmt.M, fmt.flags)


def oracle_packed(values64: np.ndarray, fmt: F.Fmt):
    """Oracle quantisation + packing of float64 values (rounded to float32
    first, as a float32 kernel holds them) -> (torch uint8 on device,
    exact quantised float64 values)."""
    v32 = values64.astype(np.float32)
    codes = oracle.encode(v32, fmt.E, fmt.M, fmt.flags)
    packed = oracle.pack_rows(codes.reshape(values64.shape[0], -1), fmt.bits)
    exact = oracle.decode(codes, fmt.E, fmt.M, fmt.flags).reshape(values64.shape)
    return to_dev(packed), exact


def check_quantized(got: np.ndarray, exact64: np.ndarray, fmt: F.Fmt, band: np.ndarray | float,
                    mask: np.ndarray | None = None, what: str = ""):
    """Each GPU value must be the format's rounding of some value within
    ``band`` of the FP64 value: Q(v - band) <= got <= Q(v + band)."""
    got = np.asarray(got, np.float64).reshape(exact64.shape)
    band = np.broadcast_to(np.asarray(band, np.float64), exact64.shape)
    lo = oracle.quantize((exact64 - band).astype(np.float32), fmt.E, fmt.M, fmt.flags)
    hi = oracle.quantize((exact64 + band).astype(np.float32), fmt.E, fmt.M, fmt.flags)
    ok = (got >= lo) & (got <= hi)
    if mask is not None:
        ok |= ~mask
    bad = np.flatnonzero(~ok.ravel())
    assert bad.size == 0, (f"{what} {fmt}: {bad.size} values outside the band; first "
                           f"{bad[:5]} got {got.ravel()[bad[:5]]} want "
                           f"{exact64.ravel()[bad[:5]]}")
    # and most values are exactly the rounding of the FP64 value itself
    q = oracle.quantize(exact64.astype(np.float32), fmt.E, fmt.M, fmt.flags)
    frac = np.mean(got == q) if got.size else 1.0
    assert frac > 0.98, f"{what} {fmt}: only {frac:.4f} exact"


def check_fp32(got: np.ndarray, exact64: np.ndarray, mask: np.ndarray | None = None,
               rel: float = REL_TOL, what: str = ""):
    """Normwise: max |got - exact| <= rel * max |exact| over unmasked entries."""
    got = np.asarray(got, np.float64).reshape(exact64.shape)
    err = np.abs(got - exact64)
    if mask is not None:
        err = np.where(mask, err, 0.0)
    scale = max(np.abs(exact64).max(), 1e-30) if exact64.size else 1.0
    worst = err.max() if err.size else 0.0
    assert worst <= rel * scale, f"{what}: max err {worst:.3e} > {rel:g} * {scale:.3e}"
    return worst / scale


class GpuPath:
    """Runs the three stages through the C ABI for one workload."""

    def __init__(self, robot, scene, params):
        self.robot, self.scene, self.params = robot, scene, params
        self.rd = B.DeviceRobot(robot)
        self.sd = B.DeviceScene(scene)

    def fk(self, q_dev, n, table, with_xform=False):
        S, J = self.robot.n_spheres, self.robot.n_joints
        pos = B.alloc_packed(n, 3 * S, table.pos)
        xf = B.alloc_packed(n, 12 * J, table.xform) if with_xform else None
        B.vapr_fk(self.rd, q_dev, n, table, pos, xf)
        return pos, xf

    def collision(self, pos, n, table):
        S = self.robot.n_spheres
        t = torch()
        cost = t.empty(n, dtype=t.float32, device="cuda")
        dist = B.alloc_packed(n, S, table.dist)
        grad = B.alloc_packed(n, 3 * S, table.grad)
        B.vapr_collision_cost(self.rd, self.sd, self.params, pos, n, table, cost, dist, grad)
        return cost, dist, grad

    def backward(self, q_dev, xf, grad, dcost_dev, n, table):
        J = self.robot.n_joints
        jg = B.alloc_packed(n, J, table.jgrad)
        B.vapr_backward(self.rd, q_dev, xf, grad, dcost_dev, n, table, jg)
        return jg
