"""The seeded synthetic inputs follow the stated recipe: a 7-joint arm with
link offsets in [0.05, 0.4] m and alternating +-90 degree twists, 52 spheres
(4-10 per link, radii in [0.03, 0.08] m), self pairs on links two or more
apart; oriented cuboids with sides in [0.05, 0.6] m centred in a 1.5 m box;
joint configurations within +-2.8 rad; the workload sizes; the uneven batch's
ranges; and the surrogate's training points."""
import numpy as np

import oracle
from paper_2310_07854_gb300 import synth


def test_arm():
    for seed in range(5):
        r = synth.make_robot(seed)
        assert r.joint_fixed.shape == (7, 12) and r.sphere_local.shape == (52, 4)
        R = r.joint_fixed[:, :9].reshape(7, 3, 3).astype(np.float64)
        t = r.joint_fixed[:, 9:].astype(np.float64)
        assert np.allclose(R @ R.transpose(0, 2, 1), np.eye(3), atol=0)
        assert np.allclose(np.linalg.det(R), 1.0)
        # Rx(+-pi/2): x fixed, z maps to -+y
        assert np.array_equal(R[:, :, 0], np.tile([1.0, 0.0, 0.0], (7, 1)))
        assert np.all(np.abs(R[:, 1, 2]) == 1.0) and np.all(R[:, 2, 1] == -R[:, 1, 2])
        assert np.all(t[:, :2] == 0) and np.all((t[:, 2] >= 0.05) & (t[:, 2] <= 0.4))
        counts = np.bincount(r.sphere_link, minlength=8)[1:]
        assert counts.sum() == 52 and counts.min() >= 4 and counts.max() <= 10
        assert np.all(np.diff(r.sphere_link) >= 0)  # grouped by link
        rad = r.sphere_local[:, 3]
        assert np.all((rad >= 0.03) & (rad <= 0.08))
        assert np.all(np.abs(r.sphere_local[:, :2]) <= 0.02)
        # self pairs: every pair two or more links apart, each once, i < j
        want = {(i, j) for i in range(52) for j in range(i + 1, 52)
                if abs(int(r.sphere_link[i]) - int(r.sphere_link[j])) >= 2}
        assert {tuple(p) for p in r.pairs.tolist()} == want and len(r.pairs) == len(want)
        assert 800 <= len(want) <= 1000


def test_radius_jitter_keeps_the_arm():
    a = synth.make_robot(4)
    b = synth.make_robot(4, radius_jitter=0.1, jitter_seed=77)
    assert np.array_equal(a.joint_fixed, b.joint_fixed)
    assert np.array_equal(a.sphere_local[:, :3], b.sphere_local[:, :3])
    ratio = b.sphere_local[:, 3].astype(np.float64) / a.sphere_local[:, 3]
    assert np.all((ratio >= 0.9 - 1e-6) & (ratio <= 1.1 + 1e-6)) and ratio.std() > 0.02


def test_scene():
    s = synth.make_scene(3, 400)
    R = s.pose[:, :9].reshape(-1, 3, 3).astype(np.float64)
    assert np.allclose(R @ R.transpose(0, 2, 1), np.eye(3), atol=1e-6)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-6)
    assert np.all(np.abs(s.pose[:, 9:]) <= 0.75)
    assert np.all((s.half_ext >= 0.025) & (s.half_ext <= 0.3))
    # orientations are spread over SO(3): the mean rotation is near zero
    assert np.abs(R.mean(0)).max() < 0.15


def test_configurations_and_workloads():
    q = synth.make_q(0, 10000)
    assert q.shape == (10000, 7) and np.abs(q).max() <= 2.8 and np.abs(q).max() > 2.79
    assert np.array_equal(q, synth.make_q(0, 10000)) and not np.array_equal(q, synth.make_q(1, 10000))
    sizes = {name: (synth.make_workload(name).n, synth.make_workload(name).scene.n_cuboids)
             for name in synth.WORKLOADS}
    assert sizes == {"single_128": (128, 8), "sweep_1024": (1024, 20), "particle_32768": (32768, 40)}
    w = synth.make_workload("particle_32768")
    assert w.n * w.robot.n_spheres == 1_703_936  # sphere evaluations per step


def test_uneven_batch_ranges():
    probs = synth.make_uneven_problems()
    assert len(probs) == 64
    traj = [p.n_traj for p in probs]
    hor = [p.horizon for p in probs]
    cub = [p.scene.n_cuboids for p in probs]
    assert min(traj) >= 4 and max(traj) <= 256 and min(hor) >= 16 and max(hor) <= 64
    assert min(cub) >= 4 and max(cub) <= 60
    assert len(set(traj)) > 20 and len(set(cub)) > 20  # uneven
    assert all(p.n == p.n_traj * p.horizon for p in probs)


def test_surrogate_training_points():
    scene = synth.make_scene(2, 40)
    lo, hi = np.array([-1.0, -1.2, -0.9]), np.array([1.1, 1.0, 1.3])
    u = synth.uniform_points(5, lo, hi, 20000)
    assert np.all((u >= lo) & (u <= hi))
    near = synth.near_surface_points(5, scene, 4000)
    # points drawn on cuboid faces plus N(0, 2 cm) noise: the nearest cuboid
    # surface is at most the noise away (|d_o| of the face's own cuboid), and
    # the noise along a face normal exceeds 6 cm (3 sigma) in 0.3 % of draws
    O = scene.n_cuboids
    d_all = np.stack([oracle.box_sdf(np.repeat(scene.pose[o:o + 1], len(near), 0),
                                     np.repeat(scene.half_ext[o:o + 1], len(near), 0), near)[0]
                      for o in range(O)])
    to_surface = np.abs(d_all).min(0)
    assert np.mean(to_surface < 0.06) > 0.99
    assert np.median(to_surface) < 0.02
