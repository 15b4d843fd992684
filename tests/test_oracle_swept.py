"""Pins of the oracle's swept-sphere environment cost (closest_pt_swept):
one sample per row reduces to the plain environment term, a static
trajectory scales it by closed-form weights, the sample points are the
stated interpolation, and the gradient is the derivative of the total
swept cost (central finite differences)."""
import dataclasses

import numpy as np
import pytest

from paper_2310_07854_gb300 import synth


def _setup(seed=0, n_traj=3, H=5, O=6):
    robot = synth.make_robot(seed)
    robot = dataclasses.replace(robot, pairs=np.zeros((0, 2), np.int32))
    scene = synth.make_scene(seed, O, extent=0.4)
    q = synth.make_q(seed, n_traj * H)
    return robot, scene, synth.CostParams(), q, H


def test_one_sample_is_the_environment_term(orc):
    robot, scene, params, q, H = _setup()
    pos = orc.fk(robot, q)
    sw = orc.swept(robot, scene, params, pos, H, 1)
    env = orc.collision(robot, scene, params, pos)
    assert np.array_equal(sw["dist"], env["dist"])
    assert np.array_equal(sw["grad"], env["grad"])
    assert np.array_equal(sw["cost"], env["cost"])
    assert (env["dist"] > 0).any()


@pytest.mark.parametrize("K", [2, 3, 5])
def test_static_trajectory_weights(orc, K):
    robot, scene, params, q, H = _setup(1, n_traj=2, H=4)
    q = np.repeat(q[::H], H, axis=0)  # every row of a trajectory the same
    pos = orc.fk(robot, q)
    env = orc.collision(robot, scene, params, pos)
    sw = orc.swept(robot, scene, params, pos, H, K)
    assert np.allclose(sw["dist"], K * env["dist"], rtol=1e-12, atol=1e-15)
    # own weights sum(1 - k/K) = (K+1)/2, previous row's sum(k/K) = (K-1)/2
    h = np.arange(len(q)) % H
    w = np.where(h == 0, (K + 1) / 2, np.where(h == H - 1, K + (K - 1) / 2, K))
    assert np.allclose(sw["grad"], w[:, None, None] * env["grad"], rtol=1e-12, atol=1e-13)


def test_sample_points_are_the_interpolation(orc):
    robot, scene, params, q, H = _setup(2, n_traj=1, H=3, O=4)
    pos = orc.fk(robot, q)
    K = 4
    sw = orc.swept(robot, scene, params, pos, H, K)
    r = robot.sphere_local[:, 3].astype(np.float64)
    for h in range(H):
        nxt = min(h + 1, H - 1)
        want = np.zeros(robot.n_spheres)
        for k in range(K):
            a = k / K
            x = (1 - a) * pos[h] + a * pos[nxt]  # [S, 3]
            for o in range(scene.n_cuboids):
                d, _ = orc.box_sdf(np.repeat(scene.pose[o:o + 1], len(x), 0),
                                   np.repeat(scene.half_ext[o:o + 1], len(x), 0), x)
                want += np.maximum(0.0, r + params.eta - d)
        assert np.allclose(sw["dist"][h], want, rtol=1e-12, atol=1e-14)


def test_gradient_matches_finite_differences(orc):
    robot, scene, params, q, H = _setup(3, n_traj=2, H=4, O=8)
    pos = orc.fk(robot, q)
    K = 3
    sw = orc.swept(robot, scene, params, pos, H, K, kink_eps=1e-5)
    rng = np.random.default_rng(0)
    h_fd = 1e-6
    checked = 0
    active = np.argwhere((np.linalg.norm(sw["grad"], axis=2) > 0) & ~sw["kink"])
    for c, s in active[rng.permutation(len(active))[:40]]:
        for i in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[c, s, i] += h_fd
            pm[c, s, i] -= h_fd
            fd = (orc.swept(robot, scene, params, pp, H, K)["cost"].sum()
                  - orc.swept(robot, scene, params, pm, H, K)["cost"].sum()) / (2 * h_fd)
            assert fd == pytest.approx(sw["grad"][c, s, i], rel=1e-5, abs=1e-7), (c, s, i)
            checked += 1
    assert checked >= 30
