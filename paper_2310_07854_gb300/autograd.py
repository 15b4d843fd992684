"""torch.autograd.Function around the CUDA path.

Forward runs FK and the collision cost (iteration steps 2-4 of Sec. III-B)
and keeps the packed gradient G = dC/dP (grad_out_spheres) for backward;
backward runs the backward-kinematics kernel (step 5) with the incoming
dL/dC, either recomputing FK from q or reading the link transforms T stored
in forward.  Every buffer is allocated per call from torch's caching
allocator and owned by the autograd graph, so several forwards may be
pending at once.
"""
from __future__ import annotations

import torch

from . import binding as B
from . import formats as F


class _VaprCostFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, mod):
        if not q.is_cuda or q.dtype != torch.float32:
            raise TypeError("q must be a float32 CUDA tensor [n, n_joints]")
        q = q.detach().contiguous()
        n = q.shape[0]
        S, J = mod.robot.n_spheres, mod.robot.n_joints
        t = mod.table
        pos = B.alloc_packed(n, 3 * S, t.pos)
        grad = B.alloc_packed(n, 3 * S, t.grad)
        dist = B.alloc_packed(n, S, t.dist) if mod.keep_dist else None
        xform = None if mod.recompute_fk else B.alloc_packed(n, 12 * J, t.xform)
        cost = torch.empty(n, dtype=torch.float32, device=q.device)
        B.vapr_fk(mod.robot, q, n, mod.ctable, pos, xform)
        B.vapr_collision_cost(mod.robot, mod.scene, mod.cparams, pos, n, mod.ctable, cost,
                              dist, grad)
        ctx.mod = mod
        ctx.save_for_backward(q, grad, *( [xform] if xform is not None else []))
        ctx.has_xform = xform is not None
        mod.last_dist = dist
        return cost

    @staticmethod
    def backward(ctx, dcost):
        mod = ctx.mod
        saved = ctx.saved_tensors
        q, grad = saved[0], saved[1]
        xform = saved[2] if ctx.has_xform else None
        n, J = q.shape[0], mod.robot.n_joints
        dc = dcost.detach().to(torch.float32).contiguous()
        jg = B.alloc_packed(n, J, mod.table.jgrad)
        B.vapr_backward(mod.robot, q, xform, grad, dc, n, mod.ctable, jg)
        out = torch.empty((n, J), dtype=torch.float32, device=q.device)
        B.vapr_unpack(jg, n, J, mod.table.jgrad, out)
        return out, None


class VaprCost(torch.nn.Module):
    """cost = VaprCost(robot, scene, params, table)(q): per-configuration
    collision cost C [n] of joint configurations q [n, J], differentiable in q.

    ``recompute_fk=True`` recomputes the joint chain in backward instead of
    storing the link transforms (12 values per joint and configuration).

    A scene given as host arrays gets the collision stage's broad-phase
    grid, as ``path.Evaluator`` builds it (``grid_cells``: "auto" for the
    finest up to 128 cells per axis that fits 32 MiB, a cell count, or None
    for no grid); a DeviceScene is used as it is.  The grid changes which
    cuboids the kernel visits, never a result bit."""

    def __init__(self, robot, scene, params, table: F.FormatTable = F.FP32_TABLE,
                 recompute_fk: bool = True, keep_dist: bool = False, device="cuda",
                 grid_cells="auto"):
        super().__init__()
        from .path import attach_grid
        self.robot = robot if isinstance(robot, B.DeviceRobot) else B.DeviceRobot(robot, device)
        if isinstance(scene, B.DeviceScene):
            self.scene = scene
        else:
            self.scene = B.DeviceScene(scene, device)
            attach_grid(self.scene, self.robot, params, grid_cells)
        self.cparams = B.cost_params(params)
        self.table = table
        self.ctable = B.to_c_table(table)
        self.recompute_fk = recompute_fk
        self.keep_dist = keep_dist
        self.last_dist = None

    def forward(self, q):
        return _VaprCostFn.apply(q, self)
