"""Batched IK optimisation around the cost-and-gradient path (Sec. III-B,
iteration steps 1-7) through vapr_ik_init / vapr_ik_step: every iteration
evaluates each seed at N step scales along its L-BFGS direction (FK,
collision cost, backward pass, pose and bound terms, all in the library's
kernels), keeps the lowest-cost scale and updates the direction.  This
module only holds the buffers and the loop."""
from __future__ import annotations

import numpy as np

from . import binding as B
from . import formats as F

SCALES = (0.0, 0.01, 0.05, 0.1, 0.2, 0.4, 0.7, 1.0)


class IkSolver:
    def __init__(self, robot: B.DeviceRobot, scene: B.DeviceScene, params, n_seeds: int,
                 w_pos=100.0, w_rot=10.0, w_bound=100.0, step0=0.2, scales=SCALES, history=6,
                 limit=2.8, table: F.FormatTable = F.FP32_TABLE, device="cuda"):
        import torch
        self.torch = torch
        self.robot, self.scene, self.params = robot, scene, params
        self.n = n_seeds
        self.table = table
        J = robot.n_joints
        self.q_lo = torch.full((J,), -limit, dtype=torch.float32, device=device)
        self.q_hi = torch.full((J,), limit, dtype=torch.float32, device=device)
        self.ik = B.ik_params(w_pos, w_rot, w_bound, step0, scales, history, self.q_lo, self.q_hi)
        nb = B.vapr_ik_workspace_bytes(robot, n_seeds, self.ik, table)
        if nb == 0:
            raise ValueError("vapr_ik_workspace_bytes rejected the arguments")
        self.ws = torch.empty(nb, dtype=torch.uint8, device=device)
        self.cost = torch.empty(n_seeds, dtype=torch.float32, device=device)
        self.pick = torch.empty(n_seeds, dtype=torch.int32, device=device)

    def init(self, goal, q):
        """goal [n, 12], q [n, J] device float32 (q is updated in place by step)."""
        self.goal, self.q = goal, q
        B.vapr_ik_init(self.robot, self.scene, self.params, self.ik, goal, q, self.n, self.table, self.ws,
                       self.cost)

    def step(self, stream=None):
        B.vapr_ik_step(self.robot, self.scene, self.params, self.ik, self.goal, self.q, self.n, self.table,
                       self.ws, self.cost, self.pick, stream)

    def solve(self, iters: int):
        for _ in range(iters):
            self.step()
        return self.q, self.cost
