"""vapr_cost_grad_fused: the whole step in one kernel with P and G kept on
the SM.  Cost, D and the joint gradient equal vapr_cost_grad's bytes with
any table (the same collision code on the same rounded centres, and the
backward sums taken in the same order with the same operations); the joint
gradient also matches the FP64 oracle to 1e-5 relative (normwise) with
float32 storage."""
import numpy as np
import pytest

import oracle
from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from parity import KINK_EPS, check_fp32, decode_packed, to_dev

pytestmark = pytest.mark.gpu

TABLES = ["", "P=E5M10,D=E2M1,G=E2M1,J=E4M3", "P=BF16,D=E4M3,G=E6M3,J=E8M23"]


def _run(fn, rd, sd, w, q, n, table, dc):
    import torch
    S, J = w.robot.n_spheres, w.robot.n_joints
    cost = torch.full((n,), float("nan"), device="cuda")
    dist = B.alloc_packed(n, S, table.dist)
    jg = B.alloc_packed(n, J, table.jgrad)
    fn(cost, dist, jg)
    torch.cuda.synchronize()
    return cost, dist, jg


def _both(w, table, q, n, dc=None):
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    if w.scene.n_cuboids > 0:
        sd.build_grid(float(np.max(w.robot.sphere_local[:, 3])), w.params.eta, 64)
    ws = B.alloc_workspace(rd, n, table)
    staged = _run(lambda c, d, j: B.vapr_cost_grad(rd, sd, w.params, q, n, table, dc, c, d, j, ws),
                  rd, sd, w, q, n, table, dc)
    fused = _run(lambda c, d, j: B.vapr_cost_grad_fused(rd, sd, w.params, q, n, table, dc, c, d, j),
                 rd, sd, w, q, n, table, dc)
    return staged, fused


@pytest.mark.parametrize("name", ["single_128", "sweep_1024", "particle_32768"])
@pytest.mark.parametrize("spec", TABLES)
def test_fused_equals_staged(name, spec):
    import torch
    w = synth.make_workload(name)
    table = F.FormatTable.parse(spec) if spec else F.FP32_TABLE
    q = to_dev(w.q)
    dc = to_dev(synth.make_dcost(3, w.n))
    (c0, d0, j0), (c1, d1, j1) = _both(w, table, q, w.n, dc)
    assert torch.equal(c0, c1) and torch.equal(d0, d1)
    assert torch.equal(j0, j1), f"{name} {spec}"
    assert B.vapr_device_error() == 0


@pytest.mark.parametrize("name", ["sweep_1024", "particle_32768"])
def test_fused_matches_oracle(name):
    w = synth.make_workload(name)
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    sd.build_grid(float(np.max(w.robot.sphere_local[:, 3])), w.params.eta, 64)
    import torch
    n, J = w.n, w.robot.n_joints
    dcost = synth.make_dcost(7, n)
    cost = torch.empty(n, device="cuda")
    jg = B.alloc_packed(n, J, F.FP32)
    B.vapr_cost_grad_fused(rd, sd, w.params, to_dev(w.q), n, F.FP32_TABLE, to_dev(dcost), cost, None, jg)
    torch.cuda.synchronize()
    pos = oracle.fk(w.robot, w.q)
    col = oracle.collision(w.robot, w.scene, w.params, pos, kink_eps=KINK_EPS)
    want = oracle.backward(w.robot, w.q, col["grad"], dcost.astype(np.float64))
    check_fp32(cost.cpu().numpy(), col["cost"], what="C")
    ok = ~col["kink"].any(1)
    assert ok.mean() > 0.5
    check_fp32(decode_packed(jg, J, F.FP32), want, mask=np.repeat(ok[:, None], J, 1), what="J")


@pytest.mark.parametrize("case", ["n1", "n33", "shuffled_spheres", "no_cuboids", "no_pairs"])
def test_fused_edge_cases(case):
    import torch
    robot, n, O = synth.make_robot(2), 97, 8
    if case == "n1":
        n = 1
    elif case == "n33":
        n = 33
    elif case == "shuffled_spheres":
        perm = np.random.default_rng(5).permutation(robot.n_spheres)
        inv = np.argsort(perm)
        robot = synth.Robot(robot.joint_fixed, robot.sphere_local[perm], robot.sphere_link[perm],
                            np.sort(inv[robot.pairs], axis=1).astype(np.int32))
    elif case == "no_cuboids":
        O = 0
    elif case == "no_pairs":
        robot = synth.Robot(robot.joint_fixed, robot.sphere_local, robot.sphere_link, np.zeros((0, 2), np.int32))
    w = synth.Workload(robot=robot, scene=synth.make_scene(4, O), q=synth.make_q(9, n, limit=np.pi),
                       params=synth.CostParams(), n_traj=n, horizon=1)
    (c0, d0, j0), (c1, d1, j1) = _both(w, F.FP32_TABLE, to_dev(w.q), n)
    assert torch.equal(c0, c1) and torch.equal(d0, d1) and torch.equal(j0, j1)
    # J against the FP64 oracle, as the staged path's edge cases are checked
    pos = oracle.fk(robot, w.q)
    col = oracle.collision(robot, w.scene, w.params, pos, kink_eps=KINK_EPS)
    want = oracle.backward(robot, w.q, col["grad"])
    ok = ~col["kink"].any(1)
    J = robot.n_joints
    check_fp32(decode_packed(j1, J, F.FP32), want, mask=np.repeat(ok[:, None], J, 1), what=f"J {case}")
