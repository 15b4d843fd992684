"""Parity of the CUDA path (vapr_fk, vapr_collision_cost, vapr_backward)
with the FP64 oracle on seeded inputs: FP32 storage to 1e-5 relative
(normwise), reduced formats code by code within the float32 error band,
edge cases, and determinism."""
import numpy as np
import pytest

import oracle
from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from parity import (FP32_BAND, KINK_EPS, GpuPath, check_fp32, check_quantized,
                    decode_packed, oracle_packed, to_dev)

pytestmark = pytest.mark.gpu

WORKLOADS = ["single_128", "sweep_1024", "particle_32768"]


@pytest.fixture(scope="module", params=WORKLOADS)
def wl(request):
    w = synth.make_workload(request.param)
    pos64, xf64 = oracle.fk(w.robot, w.q, with_xform=True)
    col = oracle.collision(w.robot, w.scene, w.params, pos64, kink_eps=KINK_EPS)
    dcost = synth.make_dcost(7, w.n)
    jg = oracle.backward(w.robot, w.q, col["grad"], dcost.astype(np.float64))
    return dict(w=w, pos64=pos64, xf64=xf64, col=col, dcost=dcost, jg=jg,
                gp=GpuPath(w.robot, w.scene, w.params), q=to_dev(w.q), dc=to_dev(dcost))


def test_fk_fp32(wl):
    w, gp = wl["w"], wl["gp"]
    pos, xf = gp.fk(wl["q"], w.n, F.FP32_TABLE, with_xform=True)
    S, J = w.robot.n_spheres, w.robot.n_joints
    check_fp32(decode_packed(pos, 3 * S, F.FP32), wl["pos64"].reshape(w.n, -1), what="P")
    check_fp32(decode_packed(xf, 12 * J, F.FP32), wl["xf64"].reshape(w.n, -1), what="T")


def test_fk_large_angles():
    """Joint angles far outside [-pi, pi] (the kernels reduce an angle by
    multiples of 2 pi before taking its sine and cosine), at +-pi and at
    multiples of 2 pi, against the FP64 oracle; the backward pass recomputes
    the same chain, so its joint gradient is checked on the same angles."""
    w = synth.make_workload("sweep_1024")
    J, S, n = w.robot.n_joints, w.robot.n_spheres, 256
    rng = np.random.default_rng(41)
    q = rng.uniform(-300.0, 300.0, size=(n, J)).astype(np.float32)
    q[:16] = np.float32(np.pi) * rng.choice([-1.0, 1.0], size=(16, J)).astype(np.float32)
    q[16:32] = (2.0 * np.pi * rng.integers(-40, 40, size=(16, J))).astype(np.float32)
    q[32:48] = np.nextafter(q[:16], np.float32(0.0))  # just inside +-pi
    gp = GpuPath(w.robot, w.scene, w.params)
    pos, xf = gp.fk(to_dev(q), n, F.FP32_TABLE, with_xform=True)
    pos64, xf64 = oracle.fk(w.robot, q, with_xform=True)
    check_fp32(decode_packed(pos, 3 * S, F.FP32), pos64.reshape(n, -1), what="P")
    check_fp32(decode_packed(xf, 12 * J, F.FP32), xf64.reshape(n, -1), what="T")
    g = synth.make_dcost(5, n * 3 * S).reshape(n, S, 3) - 1.0  # any sphere gradient
    g_dev, g32 = oracle_packed(g.reshape(n, -1), F.FP32)
    jg = gp.backward(to_dev(q), None, g_dev, None, n, F.FP32_TABLE)
    check_fp32(decode_packed(jg, J, F.FP32), oracle.backward(w.robot, q, g32.reshape(n, S, 3)), what="J")


@pytest.mark.parametrize("fmt", [F.BF16, F.FP16, F.E4M3, F.E5M2, F.E3M2, F.E2M1, F.fmt(3, 1),
                                 F.fmt(2, 2), F.fmt(6, 6), F.fmt(4, 5)], ids=str)
def test_fk_reduced(wl, fmt):
    w, gp = wl["w"], wl["gp"]
    table = F.FormatTable(pos=fmt, xform=fmt)
    pos, xf = gp.fk(wl["q"], w.n, table, with_xform=True)
    S, J = w.robot.n_spheres, w.robot.n_joints
    p64 = wl["pos64"].reshape(w.n, -1)
    check_quantized(decode_packed(pos, 3 * S, fmt), p64, fmt,
                    FP32_BAND * np.abs(p64).max(), what="P")
    x64 = wl["xf64"].reshape(w.n, -1)
    check_quantized(decode_packed(xf, 12 * J, fmt), x64, fmt,
                    FP32_BAND * np.abs(x64).max(), what="T")


TABLES = [
    F.FP32_TABLE,
    F.FormatTable.parse("P=E5M10,D=E2M1,G=E2M1,J=E4M3"),
    F.FormatTable.parse("P=BF16,D=E4M3,G=E5M2,J=FP16"),
    F.FormatTable.parse("P=E6M6,D=E3M2,G=E3M1,J=E2M3"),
]


@pytest.mark.parametrize("table", TABLES, ids=str)
def test_collision(wl, table):
    """P is the oracle's FP64 positions quantised and packed by the oracle."""
    w, gp = wl["w"], wl["gp"]
    S = w.robot.n_spheres
    pos_dev, pq = oracle_packed(wl["pos64"].reshape(w.n, -1), table.pos)
    ref = oracle.collision(w.robot, w.scene, w.params, pq.reshape(w.n, S, 3), kink_eps=KINK_EPS)
    cost, dist, grad = gp.collision(pos_dev, w.n, table)
    ok = ~ref["kink"]
    check_fp32(cost.cpu().numpy(), ref["cost"], what="C")
    gD = decode_packed(dist, S, table.dist)
    gG = decode_packed(grad, 3 * S, table.grad).reshape(w.n, S, 3)
    if table.dist == F.FP32:
        check_fp32(gD, ref["dist"], what="D")
    else:
        check_quantized(gD, ref["dist"], table.dist, FP32_BAND * max(ref["dist"].max(), 1e-3),
                        what="D")
    if table.grad == F.FP32:
        check_fp32(gG, ref["grad"], mask=np.repeat(ok[:, :, None], 3, 2), what="G")
    else:
        check_quantized(gG, ref["grad"], table.grad, FP32_BAND * np.abs(ref["grad"]).max(),
                        mask=np.repeat(ok[:, :, None], 3, 2), what="G")


@pytest.mark.parametrize("table", TABLES, ids=str)
@pytest.mark.parametrize("stored_xform", [False, True], ids=["recompute", "stored"])
def test_backward(wl, table, stored_xform):
    """G (and T) are the oracle's values quantised and packed by the oracle."""
    w, gp = wl["w"], wl["gp"]
    S, J = w.robot.n_spheres, w.robot.n_joints
    g_dev, gq = oracle_packed(wl["col"]["grad"].reshape(w.n, -1), table.grad)
    xf_dev = None
    if stored_xform:
        xf_dev, _ = oracle_packed(wl["xf64"].reshape(w.n, -1), F.FP32)
    want = oracle.backward(w.robot, w.q, gq.reshape(w.n, S, 3), wl["dcost"].astype(np.float64))
    jg = gp.backward(wl["q"], xf_dev, g_dev, wl["dc"], w.n, table)
    got = decode_packed(jg, J, table.jgrad)
    if table.jgrad == F.FP32:
        check_fp32(got, want, what="J")
    else:
        check_quantized(got, want, table.jgrad, FP32_BAND * np.abs(want).max(), what="J")


def test_whole_path_fp32(wl):
    """q -> P -> (C, D, G) -> J, all on the GPU, against FP64 throughout."""
    w, gp = wl["w"], wl["gp"]
    S, J = w.robot.n_spheres, w.robot.n_joints
    pos, _ = gp.fk(wl["q"], w.n, F.FP32_TABLE)
    cost, dist, grad = gp.collision(pos, w.n, F.FP32_TABLE)
    jg = gp.backward(wl["q"], None, grad, wl["dc"], w.n, F.FP32_TABLE)
    col = wl["col"]
    check_fp32(cost.cpu().numpy(), col["cost"], what="C")
    check_fp32(decode_packed(dist, S, F.FP32), col["dist"], what="D")
    ok = ~col["kink"]
    check_fp32(decode_packed(grad, 3 * S, F.FP32).reshape(w.n, S, 3), col["grad"],
               mask=np.repeat(ok[:, :, None], 3, 2), what="G")
    cfg_ok = ok.all(1)
    assert cfg_ok.mean() > 0.5
    check_fp32(decode_packed(jg, J, F.FP32), wl["jg"], mask=np.repeat(cfg_ok[:, None], J, 1),
               what="J")
    assert B.vapr_device_error() == 0  # no device-side wait timed out


def test_whole_path_reduced_reports_error(wl):
    """A reduced table runs end to end; its error against FP64 is measured
    (a report, not a pin) and must stay finite and bounded."""
    w, gp = wl["w"], wl["gp"]
    table = F.FormatTable.parse("P=E5M10,D=E2M1,G=E2M1,J=E4M3")
    pos, _ = gp.fk(wl["q"], w.n, table)
    cost, dist, grad = gp.collision(pos, w.n, table)
    jg = gp.backward(wl["q"], None, grad, wl["dc"], w.n, table)
    c = cost.cpu().numpy()
    assert np.all(np.isfinite(c))
    rel = np.abs(c - wl["col"]["cost"]).max() / np.abs(wl["col"]["cost"]).max()
    assert rel < 0.05, rel
    j = decode_packed(jg, w.robot.n_joints, table.jgrad)
    assert np.all(np.isfinite(j))


# ------------------------------------------------------------------ edges
def _tiny_robot(n_spheres=1, n_joints=7):
    r = synth.make_robot(3)
    if n_spheres == 1:
        sl = r.sphere_local[-1:].copy()
        link = np.array([7], np.int32)
        return synth.Robot(r.joint_fixed, sl, link, np.zeros((0, 2), np.int32))
    return r


def _big_robot():
    """16 joints, 128 spheres (8 per link), all 8128 pairs listed."""
    rng = np.random.default_rng(11)
    jf = []
    for i in range(16):
        s = 1.0 if i % 2 else -1.0
        jf.append([1, 0, 0, 0, 0, -s, 0, s, 0, 0, 0, rng.uniform(0.03, 0.12)])
    local, link = [], []
    for L in range(16):
        for k in range(8):
            local.append([rng.uniform(-.02, .02), rng.uniform(-.02, .02), 0.01 * k, rng.uniform(.02, .05)])
            link.append(L + 1)
    pairs = np.array([(i, j) for i in range(128) for j in range(i + 1, 128)], np.int32)
    return synth.Robot(np.asarray(jf, np.float32), np.asarray(local, np.float32),
                       np.asarray(link, np.int32), pairs)


@pytest.mark.parametrize("case", ["n1", "n129", "n1000_no_pairs", "one_sphere", "no_cuboids",
                                  "max_sizes", "shuffled_spheres", "reversed_pairs", "duplicate_pairs",
                                  "heavy_duplicates"])
def test_edge_cases(case):
    robot, n, O = synth.make_robot(2), 64, 8
    if case == "n1":
        n = 1
    elif case == "n129":
        n = 129
    elif case == "n1000_no_pairs":
        robot = synth.Robot(robot.joint_fixed, robot.sphere_local, robot.sphere_link,
                            np.zeros((0, 2), np.int32))
        n = 1000
    elif case == "one_sphere":
        robot = _tiny_robot(1)
    elif case == "no_cuboids":
        O = 0
    elif case == "max_sizes":
        robot, n, O = _big_robot(), 200, 1024
    elif case == "shuffled_spheres":
        perm = np.random.default_rng(5).permutation(robot.n_spheres)
        inv = np.argsort(perm)
        robot = synth.Robot(robot.joint_fixed, robot.sphere_local[perm], robot.sphere_link[perm],
                            np.sort(inv[robot.pairs], axis=1).astype(np.int32))
    elif case == "reversed_pairs":  # every pair listed as (j, i), in reverse order
        robot = synth.Robot(robot.joint_fixed, robot.sphere_local, robot.sphere_link,
                            np.ascontiguousarray(robot.pairs[::-1, ::-1]))
    elif case == "duplicate_pairs":  # some pairs named twice, one of them reversed: each counts
        pr = np.asarray(robot.pairs)
        extra = np.concatenate([pr[:40], pr[100:101, ::-1]])
        robot = synth.Robot(robot.joint_fixed, robot.sphere_local, robot.sphere_link,
                            np.ascontiguousarray(np.concatenate([pr, extra]).astype(np.int32)))
    elif case == "heavy_duplicates":  # one always-overlapping pair named 6000 times: the
        # fixed-point self sums of its two spheres take a coarse exponent and must not
        # overflow.  Its spheres are on links 1 and 2, so the pair turns joint 2 (a pair
        # within one link would cancel in J, leaving float32 rounding of 6000-fold terms)
        pr = np.asarray(robot.pairs)
        extra = np.tile(np.array([[4, 5]], np.int32), (6000, 1))
        robot = synth.Robot(robot.joint_fixed, robot.sphere_local, robot.sphere_link,
                            np.ascontiguousarray(np.concatenate([pr, extra]).astype(np.int32)))
    scene = synth.make_scene(4, O)
    q = synth.make_q(9, n, limit=np.pi) if robot.n_joints == 7 else \
        np.random.default_rng(9).uniform(-2.8, 2.8, (n, robot.n_joints)).astype(np.float32)
    params = synth.CostParams()
    gp = GpuPath(robot, scene, params)
    B.vapr_robot_check(gp.rd)
    pos64 = oracle.fk(robot, q)
    col = oracle.collision(robot, scene, params, pos64, kink_eps=KINK_EPS)
    jg64 = oracle.backward(robot, q, col["grad"])
    qd = to_dev(q)
    pos, _ = gp.fk(qd, n, F.FP32_TABLE)
    cost, dist, grad = gp.collision(pos, n, F.FP32_TABLE)
    jg = gp.backward(qd, None, grad, None, n, F.FP32_TABLE)
    S, J = robot.n_spheres, robot.n_joints
    check_fp32(decode_packed(pos, 3 * S, F.FP32), pos64.reshape(n, -1), what="P")
    check_fp32(cost.cpu().numpy(), col["cost"], what="C")
    ok = ~col["kink"]
    check_fp32(decode_packed(grad, 3 * S, F.FP32).reshape(n, S, 3), col["grad"],
               mask=np.repeat(ok[:, :, None], 3, 2), what="G")
    cfg = ok.all(1)
    if case == "heavy_duplicates":
        # the 6000-fold pair forces cancel within link 1: float32 rounding of those terms,
        # not the method, bounds J's error, so the scale is the sum of the torques' sizes
        # (1e-6 of it: about 16 float32 ulps; 1e-3 of max |J| here)
        gj = decode_packed(jg, J, F.FP32)[cfg]
        scale = (np.abs(col["grad"]).sum(2) * (1.0 + np.linalg.norm(pos64, axis=2))).sum(1)[cfg].max()
        assert np.abs(gj - jg64[cfg]).max() <= 1e-6 * scale, "J beyond the float32 bound of its sums"
    else:
        check_fp32(decode_packed(jg, J, F.FP32), jg64, mask=np.repeat(cfg[:, None], J, 1), what="J")
    if O == 0 and robot.n_pairs == 0:
        assert np.all(cost.cpu().numpy() == 0)


def test_optional_outputs_and_determinism():
    import torch
    w = synth.make_workload("sweep_1024")
    gp = GpuPath(w.robot, w.scene, w.params)
    q = to_dev(w.q)
    table = F.FormatTable.parse("P=E5M10,D=E2M1,G=E2M1,J=E4M3")
    pos, _ = gp.fk(q, w.n, table)
    c1, d1, g1 = gp.collision(pos, w.n, table)
    c2, d2, g2 = gp.collision(pos, w.n, table)
    assert torch.equal(c1, c2) and torch.equal(d1, d2) and torch.equal(g1, g2)
    # each output can be left out; the others do not change
    only_cost = torch.empty_like(c1)
    B.vapr_collision_cost(gp.rd, gp.sd, w.params, pos, w.n, table, only_cost, None, None)
    assert torch.equal(only_cost, c1)
    only_grad = torch.empty_like(g1)
    B.vapr_collision_cost(gp.rd, gp.sd, w.params, pos, w.n, table, None, None, only_grad)
    assert torch.equal(only_grad, g1)
    # a batch split into pieces gives the same bytes as one call
    parts = torch.empty_like(g1)
    cuts = [0, 100, 129, 700, w.n]
    for a, b in zip(cuts[:-1], cuts[1:]):
        B.vapr_collision_cost(gp.rd, gp.sd, w.params, pos[a:b], b - a, table, None, None, parts[a:b])
    assert torch.equal(parts, g1)
    jg1 = gp.backward(q, None, g1, None, w.n, table)
    jparts = torch.empty_like(jg1)
    for a, b in zip(cuts[:-1], cuts[1:]):
        B.vapr_backward(gp.rd, q[a:b], None, g1[a:b], None, b - a, table, jparts[a:b])
    assert torch.equal(jparts, jg1)
