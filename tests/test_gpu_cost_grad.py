"""vapr_cost_grad (the whole step in one call, intermediates in a caller
workspace) against the three entry points called one by one, and against
the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from parity import KINK_EPS, GpuPath, check_fp32, decode_packed, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("spec", ["", "P=E5M10,D=E2M1,G=E2M1,J=E4M3", "P=E6M6,G=E3M1,J=BF16"])
@pytest.mark.parametrize("name", ["single_128", "particle_32768"])
def test_cost_grad_equals_three_calls(name, spec):
    import torch
    w = synth.make_workload(name)
    table = F.FormatTable.parse(spec) if spec else F.FP32_TABLE
    gp = GpuPath(w.robot, w.scene, w.params)
    q = to_dev(w.q)
    dc = to_dev(synth.make_dcost(2, w.n))
    pos, _ = gp.fk(q, w.n, table)
    cost, dist, grad = gp.collision(pos, w.n, table)
    jg = gp.backward(q, None, grad, dc, w.n, table)
    ws = B.alloc_workspace(gp.rd, w.n, table)
    ws.fill_(0x5A)  # scratch contents must not matter
    cost2 = torch.empty_like(cost)
    dist2 = torch.empty_like(dist)
    jg2 = torch.empty_like(jg)
    B.vapr_cost_grad(gp.rd, gp.sd, w.params, q, w.n, table, dc, cost2, dist2, jg2, ws)
    assert torch.equal(cost, cost2) and torch.equal(dist, dist2) and torch.equal(jg, jg2)
    assert B.vapr_device_error() == 0


def test_cost_grad_fp32_parity():
    import torch
    w = synth.make_workload("sweep_1024")
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    q = to_dev(w.q)
    cost = torch.empty(w.n, device="cuda")
    jg = B.alloc_packed(w.n, 7, F.FP32)
    ws = B.alloc_workspace(rd, w.n, F.FP32_TABLE)
    B.vapr_cost_grad(rd, sd, w.params, q, w.n, F.FP32_TABLE, None, cost, None, jg, ws)
    pos = oracle.fk(w.robot, w.q)
    col = oracle.collision(w.robot, w.scene, w.params, pos, kink_eps=KINK_EPS)
    want = oracle.backward(w.robot, w.q, col["grad"])
    check_fp32(cost.cpu().numpy(), col["cost"], what="C")
    ok = ~col["kink"].any(1)
    check_fp32(decode_packed(jg, 7, F.FP32), want, mask=np.repeat(ok[:, None], 7, 1), what="J")


def test_host_step_and_its_graph():
    """step_host (pinned host q in, C and J out) and its captured graph give
    the device path's results, and each replay reads the current q_host."""
    import torch
    from paper_2310_07854_gb300.path import Evaluator
    w = synth.make_workload("sweep_1024")
    n, J = w.n, w.robot.n_joints
    ev = Evaluator(w.robot, w.scene, w.params, n)
    qh = torch.empty((n, J), dtype=torch.float32).pin_memory()
    ch = torch.empty(n, dtype=torch.float32).pin_memory()
    jh = torch.empty((n, J), dtype=torch.float32).pin_memory()
    qd = torch.empty((n, J), dtype=torch.float32, device="cuda")

    def device_path(qnp):
        q = to_dev(qnp)
        ev.cost_grad(q, n)
        return ev.cost[:n].cpu().clone(), ev.unpack_jgrad(n).cpu().clone()

    qh.copy_(torch.as_tensor(w.q))
    c1, j1 = ev.step_host(qh, ch, jh, qd)
    want_c, want_j = device_path(w.q)
    assert torch.equal(c1, want_c) and torch.equal(j1, want_j)
    run = ev.host_step_graph(qh, ch, jh, qd)
    for seed in (31, 32):
        qn = synth.make_q(seed, n)
        qh.copy_(torch.as_tensor(qn))
        c2, j2 = run()
        want_c, want_j = device_path(qn)
        assert torch.equal(c2, want_c) and torch.equal(j2, want_j), seed


@pytest.mark.parametrize("batches", [1, 2, 5])
def test_host_pipeline(batches):
    """host_pipeline: every batch's C and J, copied out while the next
    batch's kernels run, equal the device path's bytes for that batch's q
    (distinct q per batch, distinct host buffers)."""
    import torch
    from paper_2310_07854_gb300.path import Evaluator
    w = synth.make_workload("sweep_1024")
    n, J = w.n, w.robot.n_joints
    ev = Evaluator(w.robot, w.scene, w.params, n)
    run = ev.host_pipeline(n)
    qs = [synth.make_q(40 + k, n) for k in range(batches)]
    bufs = []
    for qn in qs:
        qh = torch.as_tensor(qn).pin_memory()
        ch = torch.full((n,), float("nan")).pin_memory()
        jh = torch.full((n, J), float("nan")).pin_memory()
        bufs.append((qh, ch, jh))
    run(bufs)
    ref = Evaluator(w.robot, w.scene, w.params, n)
    for qn, (_, ch, jh) in zip(qs, bufs):
        ref.cost_grad(to_dev(qn), n)
        assert torch.equal(ch, ref.cost[:n].cpu()) and torch.equal(jh, ref.unpack_jgrad(n).cpu())
