"""Many uneven planning problems in one persistent launch (vapr_batched_*).

``BatchedEvaluator`` holds each problem's device tables, configurations and
outputs, builds the device plan once (``vapr_batched_plan``), and evaluates
every problem with one launch (``vapr_batched_eval``), directly or as a
captured CUDA graph.
"""
from __future__ import annotations

import ctypes

from . import binding as B
from . import formats as F


class BatchedEvaluator:
    def __init__(self, problems, table: F.FormatTable = F.FP32_TABLE, tile: int = 128,
                 wait_limit_us: int = 0, deferred=(), keep_dist: bool = False, device="cuda",
                 grid_cells: int | None = 32):
        """Each problem's scene gets a broad-phase grid of grid_cells cells per
        axis (None: none); it changes no result."""
        import numpy as np
        import torch
        self.torch = torch
        self.table = table
        self.tile = tile
        self.problems = problems
        self.robots, self.scenes, self.q, self.cost, self.dist, self.jgrad = [], [], [], [], [], []
        arr = (B.vapr_problem * len(problems))()
        for i, w in enumerate(problems):
            rd, sd = B.DeviceRobot(w.robot, device), B.DeviceScene(w.scene, device)
            if grid_cells and w.scene.n_cuboids > 0:
                sd.build_grid(float(np.max(w.robot.sphere_local[:, 3])), w.params.eta, grid_cells)
            q = torch.as_tensor(w.q, device=device)
            cost = torch.full((w.n,), float("nan"), dtype=torch.float32, device=device)
            dist = B.alloc_packed(w.n, w.robot.n_spheres, table.dist, device) if keep_dist else None
            jg = B.alloc_packed(w.n, w.robot.n_joints, table.jgrad, device)
            jg.zero_()
            self.robots.append(rd)
            self.scenes.append(sd)
            self.q.append(q)
            self.cost.append(cost)
            self.dist.append(dist)
            self.jgrad.append(jg)
            arr[i] = B.vapr_problem(rd.c, sd.c, B.cost_params(w.params), q.data_ptr(), w.n, None,
                                    cost.data_ptr(), dist.data_ptr() if dist is not None else None,
                                    jg.data_ptr(), 1 if i in deferred else 0, 0)
        self.c_problems = arr
        self.tuning = B.vapr_batch_tuning(tile, wait_limit_us)
        nbytes = B.vapr_batched_plan_bytes(arr, table, self.tuning)
        if nbytes == 0:
            raise ValueError("vapr_batched_plan_bytes rejected the batch")
        self.plan_dev = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.plan = B.vapr_batch_plan()
        B.vapr_batched_plan(arr, table, self.tuning, self.plan_dev, self.plan)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)

    @property
    def n_configs(self) -> int:
        return sum(w.n for w in self.problems)

    def eval(self, stream=None):
        B.vapr_batched_eval(self.plan, self.status, stream)

    def publish(self, problem: int, stream=None):
        B.vapr_batched_publish(self.plan, problem, stream)

    def capture(self):
        """A CUDA graph whose replay is one eval (two memsets + one launch)."""
        torch = self.torch
        self.eval()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.eval()
        return g

    def device_status(self) -> int:
        return int(self.status.item())
