"""Prebuilt robot tables (vapr_robot_tables_build): launches that copy them
give the bytes of launches that build their own, for every kernel that runs
the collision stage; tables that do not match the robot's current contents
are ignored."""
import numpy as np
import pytest

from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from parity import to_dev

pytestmark = pytest.mark.gpu

TABLES = [F.FP32_TABLE, F.FormatTable.parse("P=E5M10,D=E2M1,G=E6M3,J=E3M4")]


def _robots():
    base = synth.make_robot(2)
    perm = np.random.default_rng(5).permutation(base.n_spheres)
    inv = np.argsort(perm)
    rng = np.random.default_rng(8)
    dup = np.concatenate([base.pairs, base.pairs[rng.integers(0, len(base.pairs), 40)]])
    S = 128
    big = synth.Robot(np.tile(base.joint_fixed[:1], (16, 1)),
                      np.concatenate([rng.uniform(-0.1, 0.1, (S, 3)), rng.uniform(0.02, 0.06, (S, 1))],
                                     1).astype(np.float32),
                      (np.arange(S) % 16 + 1).astype(np.int32),
                      np.array([(i, j) for i in range(S) for j in range(i + 1, S)], np.int32))
    return {
        "particle": synth.make_workload("particle_32768").robot,
        "single": synth.make_workload("single_128").robot,
        "shuffled": synth.Robot(base.joint_fixed, base.sphere_local[perm], base.sphere_link[perm],
                                np.sort(inv[base.pairs], axis=1).astype(np.int32)),
        "duplicate_pairs": synth.Robot(base.joint_fixed, base.sphere_local, base.sphere_link, dup.astype(np.int32)),
        "no_pairs": synth.Robot(base.joint_fixed, base.sphere_local, base.sphere_link, np.zeros((0, 2), np.int32)),
        "max_size": big,
    }


def _run(robot, scene, params, q, n, table, with_tables, fused=False):
    import torch
    rd = B.DeviceRobot(robot, tables=with_tables)
    sd = B.DeviceScene(scene)
    if scene.n_cuboids:
        sd.build_grid(float(np.max(robot.sphere_local[:, 3])), params.eta, 32)
    S, J = robot.n_spheres, robot.n_joints
    cost = torch.full((n,), float("nan"), device="cuda")
    dist = B.alloc_packed(n, S, table.dist)
    jg = B.alloc_packed(n, J, table.jgrad)
    if fused:
        B.vapr_cost_grad_fused(rd, sd, params, q, n, table, None, cost, dist, jg)
    else:
        ws = B.alloc_workspace(rd, n, table)
        B.vapr_cost_grad(rd, sd, params, q, n, table, None, cost, dist, jg, ws)
    torch.cuda.synchronize()
    return cost, dist, jg


@pytest.mark.parametrize("name", list(_robots()))
@pytest.mark.parametrize("fused", [False, True], ids=["staged", "fused"])
def test_copied_tables_equal_built(name, fused):
    import torch
    robot = _robots()[name]
    n = 777
    q = to_dev(np.random.default_rng(4).uniform(-2.8, 2.8, (n, robot.n_joints)).astype(np.float32))
    scene = synth.make_scene(6, 24)
    params = synth.CostParams()
    for table in TABLES:
        a = _run(robot, scene, params, q, n, table, True, fused)
        b = _run(robot, scene, params, q, n, table, False, fused)
        for x, y in zip(a, b):
            assert torch.equal(x, y), (name, str(table))
    assert B.vapr_device_error() == 0


def test_stale_tables_are_ignored():
    """Tables built for one robot, attached to a robot of the same sizes with
    other radii (and to the first robot after its pairs change on the
    device), are detected and the launch builds its own."""
    import torch
    w = synth.make_workload("sweep_1024")
    r0 = w.robot
    r1 = synth.Robot(r0.joint_fixed, (r0.sphere_local * np.float32([1, 1, 1, 1.25])).astype(np.float32),
                     r0.sphere_link, r0.pairs)
    n, q, table = w.n, to_dev(w.q), F.FP32_TABLE
    want = _run(r1, w.scene, w.params, q, n, table, False)
    rd0, rd1 = B.DeviceRobot(r0), B.DeviceRobot(r1, tables=False)
    rd1.c.tables = rd0.tables.data_ptr()  # another robot's tables
    sd = B.DeviceScene(w.scene)
    sd.build_grid(float(np.max(r1.sphere_local[:, 3])), w.params.eta, 32)
    S, J = r1.n_spheres, r1.n_joints
    cost = torch.empty(n, device="cuda")
    dist = B.alloc_packed(n, S, table.dist)
    jg = B.alloc_packed(n, J, table.jgrad)
    B.vapr_cost_grad(rd1, sd, w.params, q, n, table, None, cost, dist, jg, B.alloc_workspace(rd1, n, table))
    torch.cuda.synchronize()
    for x, y in zip((cost, dist, jg), want):
        assert torch.equal(x, y)
    # the robot's own tables, then its pair list edited in place
    rd2 = B.DeviceRobot(r1)
    rd2.pairs[0, 1] = int(r1.pairs[1, 1])
    edited = synth.Robot(r1.joint_fixed, r1.sphere_local, r1.sphere_link, rd2.pairs.cpu().numpy())
    want2 = _run(edited, w.scene, w.params, q, n, table, False)
    B.vapr_cost_grad(rd2, sd, w.params, q, n, table, None, cost, dist, jg, B.alloc_workspace(rd2, n, table))
    torch.cuda.synchronize()
    for x, y in zip((cost, dist, jg), want2):
        assert torch.equal(x, y)


def test_damaged_tables_are_ignored():
    """A tables buffer whose body was overwritten after the build (the
    header left alone) fails the body hash, and the launch builds its own."""
    import torch
    w = synth.make_workload("sweep_1024")
    n, q, table = w.n, to_dev(w.q), F.FP32_TABLE
    want = _run(w.robot, w.scene, w.params, q, n, table, False)
    rd = B.DeviceRobot(w.robot)
    body = rd.tables[64:]
    body[: body.numel() // 2] = 0xFF  # cluster and pair tables out of range
    sd = B.DeviceScene(w.scene)
    sd.build_grid(float(np.max(w.robot.sphere_local[:, 3])), w.params.eta, 32)
    S, J = w.robot.n_spheres, w.robot.n_joints
    cost = torch.empty(n, device="cuda")
    dist = B.alloc_packed(n, S, table.dist)
    jg = B.alloc_packed(n, J, table.jgrad)
    B.vapr_cost_grad(rd, sd, w.params, q, n, table, None, cost, dist, jg, B.alloc_workspace(rd, n, table))
    torch.cuda.synchronize()
    for x, y in zip((cost, dist, jg), want):
        assert torch.equal(x, y)
    assert B.vapr_device_error() == 0
