"""Pins of the oracle's kinematics, box distance, collision cost and joint
gradient (Sec. II-B kernels; Sec. III-B iteration steps 2, 3 and 5) against
facts fixed outside it: closed forms, central finite differences,
rigid-motion invariance, brute-force surface sampling and special cases."""
import numpy as np
import pytest

from paper_2310_07854_gb300 import synth


def _robot(joint_fixed, sphere_local, sphere_link, pairs=None):
    sphere_link = np.asarray(sphere_link, np.int32)
    if pairs is None:
        pairs = synth.self_pairs(sphere_link)
    return synth.Robot(np.asarray(joint_fixed, np.float32),
                       np.asarray(sphere_local, np.float32), sphere_link,
                       np.asarray(pairs, np.int32).reshape(-1, 2))


def _tf(R=np.eye(3), t=(0, 0, 0)):
    return np.concatenate([np.asarray(R, float).reshape(9), t]).astype(np.float32)


def _scene(boxes):
    pose = np.stack([_tf(R, t) for R, t, _ in boxes])
    half = np.asarray([h for _, _, h in boxes], np.float32)
    return synth.Scene(pose, half)


def _dyadic(x, bits=20):
    """Round to a multiple of 2^-bits so that small dyadic steps stay exact."""
    return (np.round(np.asarray(x, np.float64) * 2**bits) / 2**bits).astype(np.float32)


# ------------------------------------------------------------- closed forms
def test_two_link_planar_fk_and_gradient(orc):
    l1, l2, r = 0.5, float(np.float32(0.3)), float(np.float32(0.05))
    robot = _robot([_tf(), _tf(t=(l1, 0, 0))], [[l2, 0, 0, r]], [2], pairs=[])
    rng = np.random.default_rng(0)
    q = rng.uniform(-2.8, 2.8, (64, 2)).astype(np.float32)
    pos = orc.fk(robot, q)
    q1, q2 = q[:, 0].astype(float), q[:, 1].astype(float)
    want = np.stack([l1 * np.cos(q1) + l2 * np.cos(q1 + q2),
                     l1 * np.sin(q1) + l2 * np.sin(q1 + q2), 0 * q1], 1)
    assert np.abs(pos[:, 0] - want).max() < 1e-14

    # an axis-aligned box 3 cm beyond the tip along +x, face region:
    # d = 0.03, penetration 0.05 + 0.02 - 0.03 = 0.04, dd/dc = (-1, 0, 0)
    params = synth.CostParams(eta=0.02, eta_self=0.01, w_coll=1.0, w_self=1.0)
    for i in range(8):
        c = want[i]
        hx = 0.2
        scene = _scene([(np.eye(3), (c[0] + 0.03 + hx, c[1], c[2]), (hx, 0.5, 0.5))])
        col = orc.collision(robot, scene, params, pos[i:i + 1])
        assert col["dist"][0, 0] == pytest.approx(r + 0.02 - 0.03, abs=1e-7)
        assert col["cost"][0] == pytest.approx(r + 0.02 - 0.03, abs=1e-7)
        assert np.allclose(col["grad"][0, 0], [1.0, 0.0, 0.0], atol=1e-12)
        jg = orc.backward(robot, q[i:i + 1], col["grad"])[0]
        s1, s12 = np.sin(q1[i]), np.sin(q1[i] + q2[i])
        assert jg == pytest.approx([-l1 * s1 - l2 * s12, -l2 * s12], abs=1e-12)


def test_box_sdf_special_cases(orc):
    # dyadic sizes and offsets: every input and expected value is exact
    R = np.eye(3)
    h = np.array([0.125, 0.25, 0.375])
    t = np.array([1.0, -2.0, 0.5])
    pose = _tf(R, t)
    pts = np.array([
        t + [0.125, 0.0, 0.0],        # on the +x face
        t + [0.0, 0.0, 0.0],          # centre: nearest faces are +-x
        t + [0.25, 0.375, 0.5],       # corner region
        t + [0.0625, -0.125, 0.0],    # inside, 0.0625 from the +x face
        t + [0.0, 0.0, -0.625],       # outside below the -z face
    ])
    d, g = orc.box_sdf(np.repeat(pose[None], 5, 0), np.repeat(h[None], 5, 0), pts)
    assert d[0] == 0.0
    assert d[1] == -0.125
    assert d[2] == pytest.approx(np.linalg.norm([0.125, 0.125, 0.125]), abs=1e-15)
    assert d[3] == -0.0625
    assert d[4] == 0.25
    assert np.allclose(g[2], np.ones(3) / np.sqrt(3), atol=1e-15)
    assert np.array_equal(g[1], [1, 0, 0])        # tie: lowest axis, sgn(0) = +1
    assert np.array_equal(g[3], [1, 0, 0]) and np.array_equal(g[4], [0, 0, -1])
    # a rotated box: same answers for the rotated points
    Rz = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], float)
    pose_r = _tf(Rz, t)
    pts_r = (pts - t) @ Rz.T + t
    d_r, g_r = orc.box_sdf(np.repeat(pose_r[None], 5, 0), np.repeat(h[None], 5, 0), pts_r)
    assert np.array_equal(d_r, d)
    assert np.allclose(g_r, g @ Rz.T, atol=1e-15)


def _box_surface(h, step):
    """Points on the six faces of a box of half extents h (its own frame),
    on a grid of the given spacing that includes the edges."""
    faces = []
    for k in range(3):
        a, b = [j for j in range(3) if j != k]
        ua = np.arange(-h[a], h[a] + 1e-12, step)
        ub = np.arange(-h[b], h[b] + 1e-12, step)
        A, B = np.meshgrid(np.append(ua, h[a]), np.append(ub, h[b]))
        for sgn in (-1, 1):
            P = np.zeros((A.size, 3))
            P[:, a], P[:, b], P[:, k] = A.ravel(), B.ravel(), sgn * h[k]
            faces.append(P)
    return np.concatenate(faces)


def test_box_sdf_brute_force_sampling(orc):
    """|d| equals the distance to a dense sample of the surface (within the
    grid's half-diagonal) and its sign is the containment test."""
    rng = np.random.default_rng(5)
    scene = synth.make_scene(7, 3)
    for o in range(3):
        R = scene.pose[o, :9].reshape(3, 3).astype(float)
        t = scene.pose[o, 9:].astype(float)
        h = scene.half_ext[o].astype(float)
        step = 0.004
        surf = _box_surface(h, step)
        local = rng.uniform(-1.6, 1.6, (200, 3)) * h
        world = local @ R.T + t
        d, _ = orc.box_sdf(np.repeat(scene.pose[o:o + 1], 200, 0),
                           np.repeat(scene.half_ext[o:o + 1], 200, 0), world)
        near = np.sqrt(((local[:, None, :] - surf[None]) ** 2).sum(-1)).min(1)
        inside = np.all(np.abs(local) <= h, axis=1)
        tol = step * np.sqrt(2) / 2 + 1e-6
        assert np.all(np.abs(np.abs(d) - near) <= tol)
        assert np.all((d <= 1e-12) == inside)


def test_scene_sdf_brute_force(orc):
    """The scene distance (the surrogate's training label, the least box
    distance over the cuboids): outside every cuboid it is the distance to
    the nearest sampled surface point of any cuboid, inside exactly one it
    is minus the distance to that cuboid's surface; a one-cuboid scene gives
    the box distance itself."""
    rng = np.random.default_rng(9)
    scene = synth.make_scene(11, 4, extent=0.4)
    O = scene.n_cuboids
    Rs = scene.pose[:, :9].reshape(O, 3, 3).astype(float)
    ts = scene.pose[:, 9:].astype(float)
    hs = scene.half_ext.astype(float)
    # half the points anywhere around the scene, half near a chosen cuboid
    pick = rng.integers(0, O, 150)
    near_box = np.einsum("nij,nj->ni", Rs[pick], rng.uniform(-1.2, 1.2, (150, 3)) * hs[pick]) + ts[pick]
    pts = np.concatenate([rng.uniform(-0.9, 0.9, (150, 3)), near_box])
    sdf = orc.scene_sdf(scene, pts)
    step = 0.006
    near = np.empty((O, len(pts)))
    inside = np.zeros((O, len(pts)), bool)
    for o in range(O):
        surf = _box_surface(hs[o], step)
        local = (pts - ts[o]) @ Rs[o]  # R^T (p - t) for each point
        for c in range(0, len(pts), 50):
            diff = local[c:c + 50, None, :] - surf[None]
            near[o, c:c + 50] = np.sqrt((diff ** 2).sum(-1)).min(1)
        inside[o] = np.all(np.abs(local) <= hs[o], axis=1)
    tol = step * np.sqrt(2) / 2 + 1e-6
    out = ~inside.any(0)
    assert out.sum() > 100
    assert np.all(sdf[out] > 0)
    assert np.all(np.abs(sdf[out] - near[:, out].min(0)) <= tol)
    one = inside.sum(0) == 1
    assert one.sum() > 20
    own = np.argmax(inside, 0)
    assert np.all(sdf[one] <= 0)
    assert np.all(np.abs(-sdf[one] - near[own[one], one]) <= tol)
    single = synth.Scene(scene.pose[:1].copy(), scene.half_ext[:1].copy())
    d, _ = orc.box_sdf(np.repeat(scene.pose[:1], len(pts), 0), np.repeat(scene.half_ext[:1], len(pts), 0),
                       pts)
    assert np.array_equal(orc.scene_sdf(single, pts), d)


def test_self_collision_closed_form(orc):
    """Three spheres on links 1, 2, 3 at chosen points: only the listed
    (non-adjacent) pair counts; penetration r_i + r_j + eta_s - |c_i - c_j|."""
    robot = _robot([_tf()] * 3, [[0, 0, 0, 0.05], [0, 0, 0, 0.05], [0, 0, 0, 0.04]],
                   [1, 2, 3])
    assert robot.pairs.tolist() == [[0, 2]]
    scene = _scene([(np.eye(3), (10.0, 10.0, 10.0), (0.1, 0.1, 0.1))])
    pos = np.array([[[0, 0, 0], [0.05, 0, 0], [0.06, 0.02, 0.0]]])
    params = synth.CostParams(eta_self=0.01, w_self=2.0)
    col = orc.collision(robot, scene, params, pos)
    dist = np.hypot(0.06, 0.02)
    assert col["cost"][0] == pytest.approx(2.0 * (0.05 + 0.04 + 0.01 - dist))
    u = np.array([0.06, 0.02, 0.0]) / dist
    assert np.allclose(col["grad"][0, 0], 2.0 * u)
    assert np.allclose(col["grad"][0, 2], -2.0 * u)
    assert np.allclose(col["grad"][0, 1], 0.0)
    assert np.all(col["dist"] == 0)


def test_cost_weights_scale_their_terms(orc):
    """Sphere 0 is 3 cm outside the -x face of an axis-aligned box and in
    the one non-adjacent pair (0, 2); weights w_coll = 0.7, w_self = 1.9:
    C = w_coll (r_0 + eta - 0.03) + w_self (r_0 + r_2 + eta_s - |c_0 - c_2|),
    D is the unweighted penetration, and each term's gradient carries its
    own weight (environment: -w_coll e_x on sphere 0)."""
    robot = _robot([_tf()] * 3, [[0, 0, 0, 0.05], [0, 0, 0, 0.05], [0, 0, 0, 0.04]],
                   [1, 2, 3])
    hx = 0.2
    scene = _scene([(np.eye(3), (-0.03 - hx, 0.0, 0.0), (hx, 0.05, 0.05))])
    pos = np.array([[[0, 0, 0], [0.05, 0, 0], [0.06, 0.02, 0.0]]])
    params = synth.CostParams(eta=0.02, eta_self=0.01, w_coll=0.7, w_self=1.9)
    col = orc.collision(robot, scene, params, pos)
    r0, r2 = float(np.float32(0.05)), float(np.float32(0.04))
    dist = np.hypot(0.06, 0.02)
    face = float(np.float32(-0.03 - hx)) + float(np.float32(hx))  # the -x face as stored
    pen_env = r0 + 0.02 + face  # d = -face: sphere 0 sits at the origin
    pen_self = r0 + r2 + 0.01 - dist
    assert col["dist"][0] == pytest.approx([pen_env, 0.0, 0.0], abs=1e-9)
    assert col["cost"][0] == pytest.approx(0.7 * pen_env + 1.9 * pen_self, rel=1e-9)
    u = np.array([0.06, 0.02, 0.0]) / dist
    assert np.allclose(col["grad"][0, 0], [-0.7, 0.0, 0.0] + 1.9 * u, atol=1e-9)
    assert np.allclose(col["grad"][0, 1], 0.0)
    assert np.allclose(col["grad"][0, 2], -1.9 * u, atol=1e-9)


# ------------------------------------------------------- finite differences
def test_gradient_wrt_sphere_centres_fd(orc):
    w = synth.make_workload("single_128")
    pos = orc.fk(w.robot, w.q)
    col = orc.collision(w.robot, w.scene, w.params, pos, kink_eps=1e-4)
    h = 1e-7
    rng = np.random.default_rng(1)
    checked = 0
    for c in rng.choice(w.n, 24, replace=False):
        for s in range(w.robot.n_spheres):
            if col["kink"][c, s]:
                continue
            for k in range(3):
                p1, p2 = pos[c:c + 1].copy(), pos[c:c + 1].copy()
                p1[0, s, k] += h
                p2[0, s, k] -= h
                fd = (orc.collision(w.robot, w.scene, w.params, p1)["cost"][0]
                      - orc.collision(w.robot, w.scene, w.params, p2)["cost"][0]) / (2 * h)
                assert abs(fd - col["grad"][c, s, k]) < 1e-6, (c, s, k)
                checked += 1
    assert checked > 1000


def test_joint_gradient_fd(orc):
    """Central differences of C(q) (h = 2^-16, exact in float32) against the
    analytic backward pass; configurations within reach of a kink skipped."""
    w = synth.make_workload("sweep_1024")
    q = _dyadic(w.q[:400])
    h = 2.0 ** -16
    dcost = synth.make_dcost(0, 400).astype(np.float64)
    pos = orc.fk(w.robot, q)
    # a step of h moves a sphere by < 2e-5 m; skip anything within 2e-4
    col = orc.collision(w.robot, w.scene, w.params, pos, kink_eps=2e-4)
    jg = orc.backward(w.robot, q, col["grad"], dcost)
    ok = ~col["kink"].any(1)
    assert ok.sum() > 100
    fd = np.empty_like(jg)
    for j in range(7):
        qp, qm = q.copy(), q.copy()
        qp[:, j] += np.float32(h)
        qm[:, j] -= np.float32(h)
        cp = orc.collision(w.robot, w.scene, w.params, orc.fk(w.robot, qp))["cost"]
        cm = orc.collision(w.robot, w.scene, w.params, orc.fk(w.robot, qm))["cost"]
        fd[:, j] = dcost * (cp - cm) / (2 * h)
    err = np.abs(fd - jg)[ok]
    assert err.max() <= 1e-6 * max(1.0, np.abs(jg[ok]).max()), err.max()


# ------------------------------------------------------------- invariances
def _transform_inputs(robot, scene, Rx, tx):
    jf = robot.joint_fixed.astype(np.float64).copy()
    R1, t1 = jf[0, :9].reshape(3, 3), jf[0, 9:]
    jf[0, :9] = (Rx @ R1).ravel()
    jf[0, 9:] = Rx @ t1 + tx
    pose = scene.pose.astype(np.float64).copy()
    for o in range(pose.shape[0]):
        Ro, to = pose[o, :9].reshape(3, 3), pose[o, 9:]
        pose[o, :9] = (Rx @ Ro).ravel()
        pose[o, 9:] = Rx @ to + tx
    r2 = synth.Robot(jf.astype(np.float32), robot.sphere_local,
                     robot.sphere_link, robot.pairs)
    return r2, synth.Scene(pose.astype(np.float32), scene.half_ext)


def test_rigid_motion_invariance_exact(orc):
    """A signed-permutation rotation and a dyadic shift of the base and of
    every cuboid (exact in float32) leave D, C and J unchanged and rotate G."""
    w = synth.make_workload("single_128")
    robot = synth.Robot(_dyadic(w.robot.joint_fixed), w.robot.sphere_local,
                        w.robot.sphere_link, w.robot.pairs)
    scene = synth.Scene(np.concatenate([w.scene.pose[:, :9],
                                        _dyadic(w.scene.pose[:, 9:])], 1),
                        w.scene.half_ext)
    Rx = np.array([[0, -1, 0], [0, 0, 1], [-1, 0, 0]], float)
    assert np.linalg.det(Rx) == pytest.approx(1.0)
    tx = np.array([0.25, -0.5, 0.125])
    r2, s2 = _transform_inputs(robot, scene, Rx, tx)
    assert np.array_equal(r2.joint_fixed.astype(np.float64)[0, 9:],
                          Rx @ robot.joint_fixed[0, 9:].astype(float) + tx)
    a = orc.cost_and_grad(robot, scene, w.params, w.q)
    b = orc.cost_and_grad(r2, s2, w.params, w.q)
    assert np.abs(a[1]["dist"] - b[1]["dist"]).max() < 1e-12
    assert np.abs(a[1]["cost"] - b[1]["cost"]).max() < 1e-12
    assert np.abs(a[1]["grad"] @ Rx.T - b[1]["grad"]).max() < 1e-10
    assert np.abs(a[2] - b[2]).max() < 1e-10
    assert np.abs(a[0] @ Rx.T + tx - b[0]).max() < 1e-12


def test_rigid_motion_invariance_general(orc):
    """A random SE(3): equal up to the float32 rounding of moved inputs."""
    w = synth.make_workload("single_128")
    rng = np.random.default_rng(9)
    Qm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    Rx = Qm * np.sign(np.linalg.det(Qm))
    tx = rng.uniform(-0.3, 0.3, 3)
    r2, s2 = _transform_inputs(w.robot, w.scene, Rx, tx)
    a = orc.cost_and_grad(w.robot, w.scene, w.params, w.q)
    b = orc.cost_and_grad(r2, s2, w.params, w.q)
    ok = ~(a[1]["kink"].any(1) | b[1]["kink"].any(1))
    assert np.abs(a[1]["cost"] - b[1]["cost"]).max() < 1e-5
    assert np.abs(a[2] - b[2])[ok].max() < 1e-4


def test_backward_respects_chain_structure(orc):
    """A sphere on link k moves only with joints 1..k."""
    w = synth.make_workload("single_128")
    pos = orc.fk(w.robot, w.q)
    g = np.zeros_like(pos)
    on3 = w.robot.sphere_link == 3
    g[:, on3] = np.random.default_rng(2).normal(size=g[:, on3].shape)
    jg = orc.backward(w.robot, w.q, g)
    assert np.all(jg[:, 3:] == 0)
    assert np.all(np.abs(jg[:, :3]).sum(1) > 0)
    # linear in G and in dC
    jg2 = orc.backward(w.robot, w.q, 2 * g, np.full(w.n, 0.5))
    assert np.allclose(jg, jg2, rtol=1e-14, atol=1e-15)


def test_self_pairs_rule():
    link = np.array([1, 1, 2, 3, 3, 5], np.int32)
    p = synth.self_pairs(link)
    for i, j in p:
        assert abs(link[i] - link[j]) >= 2 and i < j
    n_all = sum(1 for i in range(6) for j in range(i + 1, 6) if abs(link[i] - link[j]) >= 2)
    assert len(p) == n_all == 9
