"""Pins of the oracle's IK iteration pieces: the pose and bound terms and
their gradient (closed forms, central finite differences), the collision
part (equal to the collision cost and backward pass), and the L-BFGS
two-loop direction against the dense BFGS inverse-Hessian update."""
import dataclasses
import types

import numpy as np
import pytest

from paper_2310_07854_gb300 import synth


def _ik(J, w_pos=100.0, w_rot=10.0, w_bound=100.0, lim=2.8):
    return types.SimpleNamespace(w_pos=w_pos, w_rot=w_rot, w_bound=w_bound,
                                 q_lo=np.full(J, -lim, np.float32), q_hi=np.full(J, lim, np.float32),
                                 scales=[0.0, 0.05, 0.25, 1.0], history=5, step0=0.2)


def _goal_from(orc, robot, q):
    """End-effector pose T_J of configurations q: R row-major, then t."""
    x = orc.fk(robot, q, with_xform=True)[1]  # [n, J, 12]
    return x[:, -1, :].astype(np.float32)


def test_zero_error_goal_costs_nothing(orc):
    robot = dataclasses.replace(synth.make_robot(0), pairs=np.zeros((0, 2), np.int32))
    empty = synth.make_scene(0, 0)
    q = synth.make_q(1, 16) * 0.5
    goal = _goal_from(orc, robot, q)
    f, g = orc.ik_costs(robot, empty, synth.CostParams(), _ik(7), goal, q)
    # the goal is stored in float32: |t - t*| <= 6e-8 m, so the cost is
    # ~1e-13 and the gradient 2 w |t - t*| x (lever <= 3 m) <= 4e-5
    assert np.max(np.abs(f)) < 1e-11 and np.max(np.abs(g)) < 1e-4


def test_bound_term_closed_form(orc):
    robot = dataclasses.replace(synth.make_robot(0), pairs=np.zeros((0, 2), np.int32))
    empty = synth.make_scene(0, 0)
    q = np.zeros((1, 7), np.float32)
    q[0, 2], q[0, 5] = 3.0, -3.25
    goal = _goal_from(orc, robot, q)
    ik = _ik(7, w_pos=0.0, w_rot=0.0, w_bound=7.0)
    f, g = orc.ik_costs(robot, empty, synth.CostParams(), ik, goal, q)
    lim = float(np.float32(2.8))
    assert f[0] == pytest.approx(7.0 * ((3.0 - lim) ** 2 + (3.25 - lim) ** 2), rel=1e-12)
    assert g[0, 2] == pytest.approx(14.0 * (3.0 - lim), rel=1e-12)
    assert g[0, 5] == pytest.approx(-14.0 * (3.25 - lim), rel=1e-12)
    assert np.count_nonzero(g[0]) == 2


def test_pose_gradient_matches_finite_differences(orc):
    robot = dataclasses.replace(synth.make_robot(2), pairs=np.zeros((0, 2), np.int32))
    empty = synth.make_scene(0, 0)
    q = synth.make_q(3, 6) * 0.8
    goal = _goal_from(orc, robot, synth.make_q(4, 6) * 0.8)
    ik = _ik(7)
    f, g = orc.ik_costs(robot, empty, synth.CostParams(), ik, goal, q)
    for c in range(len(q)):
        for j in range(7):
            qp, qm = q.copy(), q.copy()
            qp[c, j] += np.float32(2.0 ** -12)
            qm[c, j] -= np.float32(2.0 ** -12)
            dh = float(qp[c, j]) - float(qm[c, j])
            fd = (orc.ik_costs(robot, empty, synth.CostParams(), ik, goal[c:c + 1], qp[c:c + 1])[0][0]
                  - orc.ik_costs(robot, empty, synth.CostParams(), ik, goal[c:c + 1], qm[c:c + 1])[0][0]) / dh
            assert fd == pytest.approx(g[c, j], rel=1e-6, abs=1e-8), (c, j)


def test_collision_part_is_the_path(orc):
    w = synth.make_workload("single_128")
    ik = _ik(7, w_pos=0.0, w_rot=0.0, w_bound=0.0)
    goal = np.zeros((w.n, 12), np.float32)
    f, g = orc.ik_costs(w.robot, w.scene, w.params, ik, goal, w.q)
    pos, col, jg = orc.cost_and_grad(w.robot, w.scene, w.params, w.q)
    assert np.allclose(f, col["cost"], rtol=1e-13, atol=1e-15)
    assert np.allclose(g, jg, rtol=1e-13, atol=1e-13)


def test_lbfgs_two_loop_equals_dense_bfgs(orc):
    rng = np.random.default_rng(0)
    dim = 7
    for m in (0, 1, 3, 6):
        S = rng.normal(size=(m, dim))
        A = rng.normal(size=(dim, dim))
        A = A @ A.T + dim * np.eye(dim)  # s.y > 0 for y = A s
        Y = S @ A.T
        g = rng.normal(size=dim)
        d = orc.lbfgs_direction(S, Y, g)
        # textbook BFGS inverse update from H0 = gamma I (newest pair)
        if m == 0:
            H = np.eye(dim)
        else:
            H = (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1]) * np.eye(dim)
            for s, y in zip(S, Y):
                rho = 1.0 / (y @ s)
                V = np.eye(dim) - rho * np.outer(y, s)
                H = V.T @ H @ V + rho * np.outer(s, s)
        assert np.allclose(d, -H @ g, rtol=1e-10, atol=1e-12), m


def test_iteration_never_increases_the_cost(orc):
    w = synth.make_workload("single_128")
    ik = _ik(7)
    goal = _goal_from(orc, w.robot, synth.make_q(9, w.n))
    out = orc.ik_iterate(w.robot, w.scene, w.params, ik, goal[:32], w.q[:32], iters=4)
    assert np.all(np.diff(out["cost"], axis=0) <= 1e-12)
    assert np.mean(out["cost"][-1]) < np.mean(out["cost"][0])


def _bfgs_direction(pairs, g):
    """-H g with H the textbook BFGS inverse update from H0 = gamma I
    (gamma from the newest pair), pairs oldest first."""
    dim = g.shape[0]
    if not pairs:
        return -g
    s_n, y_n = pairs[-1]
    H = (s_n @ y_n) / (y_n @ y_n) * np.eye(dim)
    for s, y in pairs:
        rho = 1.0 / (y @ s)
        V = np.eye(dim) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return -H @ g


def test_iteration_steps_follow_the_rules(orc):
    """Each step of the iteration, re-derived from its outputs: the kept
    scale is the lowest-cost candidate (costs recomputed one by one); the
    first step and every step after keeping scale 0 follow steepest descent
    scaled so that scale 1 moves the largest joint by step0; otherwise the
    direction is the BFGS step from the newest `history` pairs with
    positive curvature, and a pair without positive curvature is skipped."""
    w = synth.make_workload("single_128")
    ik = _ik(7)
    ik.history = 2
    ik.scales = [0.0, 0.1, 0.5, 2.0]  # long steps overshoot: scale 0 is kept now and then
    n, iters = 24, 6
    goal = _goal_from(orc, w.robot, synth.make_q(9, w.n))[:n]
    out = orc.ik_iterate(w.robot, w.scene, w.params, ik, goal, w.q[:n], iters=iters)
    scales = np.asarray(ik.scales)
    restarts = curv_steps = trims = after_restart = 0
    for i in range(n):
        qs = out["q"][:, i]
        g = [orc.ik_costs(w.robot, w.scene, w.params, ik, goal[i:i + 1], qs[k:k + 1].astype(np.float32))[1][0]
             for k in range(iters + 1)]
        d = -g[0] * ik.step0 / np.abs(g[0]).max()
        pairs = []
        for k in range(iters):
            cand = (qs[k][None] + scales[:, None] * d[None]).astype(np.float32)
            fc = orc.ik_costs(w.robot, w.scene, w.params, ik, np.repeat(goal[i:i + 1], len(scales), 0), cand)[0]
            pick = out["pick"][k, i]
            assert pick == np.argmin(fc)
            assert np.array_equal(qs[k + 1], cand[pick].astype(np.float64))
            if scales[pick] == 0.0:
                pairs = []
                d = -g[k + 1] * ik.step0 / np.abs(g[k + 1]).max()
                restarts += 1
                continue
            s, y = qs[k + 1] - qs[k], g[k + 1] - g[k]
            if s @ y > 0:
                pairs.append((s, y))
                trims += len(pairs) > ik.history
                after_restart += k > 0 and out["pick"][k - 1, i] == 0
                pairs = pairs[-ik.history:]
                curv_steps += 1
            d = _bfgs_direction(pairs, g[k + 1]) if pairs else -g[k + 1] * ik.step0 / np.abs(g[k + 1]).max()
    assert restarts > 0 and curv_steps > 0 and trims > 0 and after_restart > 0  # every rule exercised
