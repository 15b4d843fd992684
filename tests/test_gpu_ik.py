"""The batched IK iteration on the GPU against the FP64 oracle iteration:
initial cost and gradient, the kept step scale and the iterates over a few
iterations, and that the cost never rises and the pose error falls."""
import types

import numpy as np
import pytest

import oracle
from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import ik as IK
from paper_2310_07854_gb300 import synth
from parity import to_dev

pytestmark = pytest.mark.gpu


def _problem(n=256, seed=7):
    w = synth.make_workload("single_128")
    goal_q = synth.make_q(seed, n) * 0.8
    x = oracle.fk(w.robot, goal_q, with_xform=True)[1]
    goal = x[:, -1, :].astype(np.float32)
    q0 = synth.make_q(seed + 1, n) * 0.8
    return w, goal, q0


def _oik(solver):
    J = solver.robot.n_joints
    return types.SimpleNamespace(w_pos=100.0, w_rot=10.0, w_bound=100.0, q_lo=np.full(J, -2.8, np.float32),
                                 q_hi=np.full(J, 2.8, np.float32), scales=list(IK.SCALES), history=6,
                                 step0=0.2)


def test_init_matches_oracle():
    import torch
    w, goal, q0 = _problem()
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    s = IK.IkSolver(rd, sd, w.params, len(q0))
    q = to_dev(q0)
    s.init(to_dev(goal), q)
    f64, g64 = oracle.ik_costs(w.robot, w.scene, w.params, _oik(s), goal, q0)
    f = s.cost.cpu().numpy()
    assert np.max(np.abs(f - f64)) <= 1e-5 * np.max(np.abs(f64))
    assert torch.equal(q, to_dev(q0))  # init leaves q alone


def test_iterations_match_oracle():
    w, goal, q0 = _problem()
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    s = IK.IkSolver(rd, sd, w.params, len(q0))
    q = to_dev(q0)
    s.init(to_dev(goal), q)
    iters = 3
    ref = oracle.ik_iterate(w.robot, w.scene, w.params, _oik(s), goal, q0, iters)
    same = np.ones(len(q0), bool)
    for it in range(iters):
        s.step()
        pick = s.pick.cpu().numpy()
        same &= pick == ref["pick"][it]
        qg = q.cpu().numpy().astype(np.float64)
        err = np.abs(qg - ref["q"][it + 1])[same]
        # float32 state against float64: iterates agree to 1e-4 rad while the
        # two sides keep choosing the same step scales
        assert np.max(err) <= 1e-4 * (it + 1), (it, np.max(err))
    assert same.mean() > 0.9
    f = s.cost.cpu().numpy()
    assert np.max(np.abs(f - ref["cost"][-1])[same]) <= 1e-4 * np.max(np.abs(ref["cost"][-1]))


def test_solver_descends():
    import torch
    w, goal, q0 = _problem(1024, seed=11)
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    s = IK.IkSolver(rd, sd, w.params, len(q0))
    q = to_dev(q0)
    s.init(to_dev(goal), q)
    f0 = s.cost.clone()
    prev = f0.clone()
    for _ in range(30):
        s.step()
        assert bool((s.cost <= prev).all())
        prev = s.cost.clone()
    assert float(s.cost.mean()) < 0.25 * float(f0.mean())
    assert B.vapr_device_error() == 0


def test_reduced_table_descends():
    """The solver with the path's tensors in reduced formats still descends."""
    from paper_2310_07854_gb300 import formats as F
    w, goal, q0 = _problem(512, seed=21)
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    s = IK.IkSolver(rd, sd, w.params, len(q0), table=F.FormatTable.parse("P=E5M10,D=E2M1,G=E4M3,J=E5M10"))
    q = to_dev(q0)
    s.init(to_dev(goal), q)
    f0 = float(s.cost.mean())
    for _ in range(20):
        s.step()
    assert float(s.cost.mean()) < 0.5 * f0
    assert B.vapr_device_error() == 0
