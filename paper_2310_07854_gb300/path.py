"""The whole cost-and-gradient step through the C ABI.

``Evaluator`` owns the packed intermediate tensors of one batch size and
runs FK -> collision cost -> backward (iteration steps 2, 3-4 and 5 of
Sec. III-B) with a per-tensor format table.  ``step_host`` is the end-to-end
call: joint configurations in pinned host memory go to the device, the path
runs, and costs and joint gradients come back to the host.
"""
from __future__ import annotations

from . import binding as B
from . import formats as F


def auto_grid_cells(n_cuboids: int, budget: int = 32 << 20) -> int:
    """The finest grid (at most 128 cells per axis) whose bytes fit the budget."""
    cells = 128
    while cells > 8 and B.vapr_scene_grid_bytes(n_cuboids, cells) > budget:
        cells -= 8
    return cells


def attach_grid(scene, robot, params, grid_cells="auto") -> None:
    """Builds the broad-phase grid of a DeviceScene for the robot's largest
    sphere radius and the margin eta: grid_cells cells per axis ("auto":
    auto_grid_cells; None or 0: no grid)."""
    import numpy as np
    if grid_cells == "auto":
        grid_cells = auto_grid_cells(scene.c.n_cuboids)
    if grid_cells:
        reach = float(np.max(robot.host.sphere_local[:, 3]))
        scene.build_grid(reach, params.eta, grid_cells)


class Evaluator:
    def __init__(self, robot, scene, params, n_max: int, table: F.FormatTable = F.FP32_TABLE,
                 recompute_fk: bool = True, device: str = "cuda", grid_cells: int | str | None = "auto"):
        """A scene given as host arrays gets a broad-phase grid of grid_cells
        cells per axis ("auto": the finest up to 128 whose grid fits 32 MiB;
        None: no grid); a DeviceScene is used as it is."""
        import torch
        self.torch = torch
        self.robot = robot if isinstance(robot, B.DeviceRobot) else B.DeviceRobot(robot, device)
        if isinstance(scene, B.DeviceScene):
            self.scene = scene
        else:
            self.scene = B.DeviceScene(scene, device)
            attach_grid(self.scene, self.robot, params, grid_cells)
        self.params = B.cost_params(params)
        self.table = table
        self.ctable = B.to_c_table(table)  # built once: calls pass the C struct
        self.recompute_fk = recompute_fk
        self.n_max = n_max
        S, J = self.robot.n_spheres, self.robot.n_joints
        self.pos = B.alloc_packed(n_max, 3 * S, table.pos, device)
        self.dist = B.alloc_packed(n_max, S, table.dist, device)
        self.grad = B.alloc_packed(n_max, 3 * S, table.grad, device)
        self.jgrad = B.alloc_packed(n_max, J, table.jgrad, device)
        self.xform = None if recompute_fk else B.alloc_packed(n_max, 12 * J, table.xform, device)
        self.cost = torch.empty(n_max, dtype=torch.float32, device=device)
        self.jgrad_f32 = torch.empty((n_max, J), dtype=torch.float32, device=device)
        self.workspace = B.alloc_workspace(self.robot, n_max, table, device)

    # ---- device-resident stages
    def forward(self, q, n: int, stream=None):
        self.fk(q, n, stream)
        self.collision(n, stream)
        return self.cost[:n]

    def fk(self, q, n: int, stream=None):
        B.vapr_fk(self.robot, q, n, self.ctable, self.pos, self.xform, stream)

    def collision(self, n: int, stream=None):
        B.vapr_collision_cost(self.robot, self.scene, self.params, self.pos, n, self.ctable,
                              self.cost, self.dist, self.grad, stream)

    def backward(self, q, n: int, dcost=None, stream=None):
        B.vapr_backward(self.robot, q, self.xform, self.grad, dcost, n, self.ctable,
                        self.jgrad, stream)
        return self.jgrad[:n]

    def unpack_jgrad(self, n: int, stream=None):
        B.vapr_unpack(self.jgrad, n, self.robot.n_joints, self.table.jgrad, self.jgrad_f32, stream)
        return self.jgrad_f32[:n]

    def step(self, q, n: int, dcost=None, stream=None):
        """FK, collision cost, backward: three kernel launches."""
        self.forward(q, n, stream)
        self.backward(q, n, dcost, stream)

    def capture(self, q, n: int, dcost=None, timing_events: bool = False):
        """Captures one step in a CUDA graph (replay = three kernel launches,
        no host work in between).  With ``timing_events`` the graph also
        records four external timing events at the kernel boundaries;
        returns (graph, events or None)."""
        torch = self.torch
        self.step(q, n, dcost)  # first launches fill the library's launch caches
        torch.cuda.synchronize()
        evs = None
        if timing_events:
            try:
                evs = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(4)]
            except TypeError:  # a torch without external events
                evs = None
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            if evs:
                evs[0].record()
            self.fk(q, n)
            if evs:
                evs[1].record()
            self.collision(n)
            if evs:
                evs[2].record()
            self.backward(q, n, dcost)
            if evs:
                evs[3].record()
        return g, evs

    def cost_grad(self, q, n: int, dcost=None, stream=None):
        """The whole step in one library call (vapr_cost_grad): cost [n] and
        packed joint gradients, P and G in the evaluator's workspace."""
        B.vapr_cost_grad(self.robot, self.scene, self.params, q, n, self.ctable, dcost,
                         self.cost, self.dist, self.jgrad, self.workspace, stream=stream)

    # ---- end to end from host memory
    def step_host(self, q_host, cost_host, jgrad_host, q_dev, stream=None):
        """q_host (pinned float32 [n, J]) -> cost_host [n], jgrad_host [n, J]
        float32 (pinned).  Copies and kernels are enqueued on one stream;
        the call returns after the results are on the host."""
        torch = self.torch
        n = q_host.shape[0]
        st = stream or torch.cuda.current_stream()
        with torch.cuda.stream(st):
            q_dev[:n].copy_(q_host, non_blocking=True)
            self.cost_grad(q_dev, n, None, st)
            self.unpack_jgrad(n, st)
            cost_host.copy_(self.cost[:n], non_blocking=True)
            jgrad_host.copy_(self.jgrad_f32[:n], non_blocking=True)
        st.synchronize()
        return cost_host, jgrad_host

    def host_step_graph(self, q_host, cost_host, jgrad_host, q_dev):
        """The end-to-end step of ``step_host`` captured once in a CUDA graph:
        the host-to-device copy of q, the path, the joint-gradient unpack and
        the device-to-host copies of C and J replay as one launch.  Returns a
        function that runs one step on the current contents of q_host and
        returns after cost_host and jgrad_host hold the results.  The buffers
        are bound at capture time."""
        torch = self.torch
        n = q_host.shape[0]
        st = torch.cuda.Stream()
        self.step_host(q_host, cost_host, jgrad_host, q_dev, st)  # fills the launch caches
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            q_dev[:n].copy_(q_host, non_blocking=True)
            self.cost_grad(q_dev, n, None, st)
            self.unpack_jgrad(n, st)
            cost_host.copy_(self.cost[:n], non_blocking=True)
            jgrad_host.copy_(self.jgrad_f32[:n], non_blocking=True)

        def run():
            with torch.cuda.stream(st):
                g.replay()
            st.synchronize()
            return cost_host, jgrad_host
        run.graph = g
        return run

    def host_pipeline(self, n: int):
        """Streaming end to end from pinned host memory: returns run(batches),
        where batches is a sequence of (q_host [n, J], cost_host [n],
        jgrad_host [n, J]) pinned float32 tensors; run processes them in
        order, each batch with its own host-to-device copy of q and
        device-to-host copies of C and J, and returns once every result is on
        the host.  Two batches are in flight: the path of batch k (one CUDA
        graph: vapr_cost_grad and the J unpack) runs while the copy of batch
        k+1's q and the copies of batch k-1's results move on streams of
        their own, ordered by events; the two batches in flight use two
        evaluators (this one and a twin sharing its robot, scene and table),
        so no copy touches a buffer that a running kernel uses."""
        torch = self.torch
        J = self.robot.n_joints
        dev = self.cost.device
        evs = [self, self._twin(n)]
        qd = [torch.empty((n, J), dtype=torch.float32, device=dev) for _ in range(2)]
        sc, si, so = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        cur = torch.cuda.current_stream()
        for st in (sc, si, so):  # the evaluators' tables and buffers were made on the current stream
            st.wait_stream(cur)
        graphs = []
        for b in range(2):
            with torch.cuda.stream(sc):
                qd[b].zero_()
                evs[b].cost_grad(qd[b], n, None, sc)  # fills the launch caches
                evs[b].unpack_jgrad(n, sc)
            sc.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=sc):
                evs[b].cost_grad(qd[b], n, None, sc)
                evs[b].unpack_jgrad(n, sc)
            graphs.append(g)
        in_done = [torch.cuda.Event() for _ in range(2)]
        comp_done = [torch.cuda.Event() for _ in range(2)]
        out_done = [torch.cuda.Event() for _ in range(2)]

        def run(batches):
            for k, (qh, ch, jh) in enumerate(batches):
                b = k & 1
                if k >= 2:
                    si.wait_event(comp_done[b])  # batch k-2's kernels have read qd[b]
                with torch.cuda.stream(si):
                    qd[b].copy_(qh, non_blocking=True)
                in_done[b].record(si)
                sc.wait_event(in_done[b])
                if k >= 2:
                    sc.wait_event(out_done[b])  # batch k-2's results are out of evs[b]
                with torch.cuda.stream(sc):
                    graphs[b].replay()
                comp_done[b].record(sc)
                so.wait_event(comp_done[b])
                with torch.cuda.stream(so):
                    ch.copy_(evs[b].cost[:n], non_blocking=True)
                    jh.copy_(evs[b].jgrad_f32[:n], non_blocking=True)
                out_done[b].record(so)
            so.synchronize()
        run.graphs = graphs
        return run

    def _twin(self, n: int):
        """An evaluator for n configurations sharing this one's robot, scene,
        parameters and table, with buffers of its own."""
        t = object.__new__(Evaluator)
        t.torch = self.torch
        t.robot, t.scene, t.params = self.robot, self.scene, self.params
        t.table, t.ctable, t.recompute_fk, t.n_max = self.table, self.ctable, self.recompute_fk, n
        torch = self.torch
        dev = self.cost.device
        S, J = self.robot.n_spheres, self.robot.n_joints
        t.pos = B.alloc_packed(n, 3 * S, self.table.pos, dev)
        t.dist = B.alloc_packed(n, S, self.table.dist, dev)
        t.grad = B.alloc_packed(n, 3 * S, self.table.grad, dev)
        t.jgrad = B.alloc_packed(n, J, self.table.jgrad, dev)
        t.xform = None if self.recompute_fk else B.alloc_packed(n, 12 * J, self.table.xform, dev)
        t.cost = torch.empty(n, dtype=torch.float32, device=dev)
        t.jgrad_f32 = torch.empty((n, J), dtype=torch.float32, device=dev)
        t.workspace = B.alloc_workspace(self.robot, n, self.table, dev)
        return t

    def bytes_per_config(self) -> dict:
        """Algorithmic bytes per configuration of each stage (packed rows,
        unpadded; robot and scene tables excluded)."""
        S, J = self.robot.n_spheres, self.robot.n_joints
        t = self.table
        P = t.pos.row_bytes_unpadded(3 * S)
        D = t.dist.row_bytes_unpadded(S)
        G = t.grad.row_bytes_unpadded(3 * S)
        Jb = t.jgrad.row_bytes_unpadded(J)
        T = t.xform.row_bytes_unpadded(12 * J)
        q = 4 * J
        fk = q + P + (0 if self.recompute_fk else T)
        coll = P + D + G + 4
        bw = q + G + 4 + Jb + (0 if self.recompute_fk else T)
        return {"fk": fk, "collision": coll, "backward": bw, "total": fk + coll + bw}
