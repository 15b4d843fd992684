"""Swept-sphere environment cost (closest_pt_swept) on the GPU against the
FP64 oracle: one sample per row equals the environment term of the
collision stage bit for bit, the FP32 path matches FP64 to 1e-5 normwise
(gradients away from discontinuities), horizon 1 scales the environment
term by K, and reduced-format outputs are the format's rounding of the
FP32 results."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from parity import KINK_EPS, REL_TOL, to_dev

pytestmark = pytest.mark.gpu


def _setup(name="sweep_1024"):
    w = synth.make_workload(name)
    robot = dataclasses.replace(w.robot, pairs=np.zeros((0, 2), np.int32))
    rd, sd = B.DeviceRobot(robot), B.DeviceScene(w.scene)
    pos = B.alloc_packed(w.n, 3 * robot.n_spheres, F.FP32)
    B.vapr_fk(rd, to_dev(w.q), w.n, F.FP32_TABLE, pos)
    return w, robot, rd, sd, pos


def _swept(rd, sd, w, pos, H, K, table=F.FP32_TABLE):
    import torch
    S = rd.n_spheres
    cost = torch.empty(w.n, device="cuda")
    dist = B.alloc_packed(w.n, S, table.dist)
    grad = B.alloc_packed(w.n, 3 * S, table.grad)
    B.vapr_swept_cost(rd, sd, w.params, pos, w.n, H, K, table, cost, dist, grad)
    return cost, dist, grad


def test_one_sample_equals_environment_term():
    import torch
    w, robot, rd, sd, pos = _setup()
    S = robot.n_spheres
    cost = torch.empty(w.n, device="cuda")
    dist = B.alloc_packed(w.n, S, F.FP32)
    grad = B.alloc_packed(w.n, 3 * S, F.FP32)
    B.vapr_collision_cost(rd, sd, w.params, pos, w.n, F.FP32_TABLE, cost, dist, grad)
    c1, d1, g1 = _swept(rd, sd, w, pos, w.horizon, 1)
    assert torch.equal(cost, c1) and torch.equal(dist, d1) and torch.equal(grad, g1)


@pytest.mark.parametrize("K", [2, 4])
def test_matches_oracle(K):
    w, robot, rd, sd, pos = _setup()
    S = robot.n_spheres
    c, d, g = _swept(rd, sd, w, pos, w.horizon, K)
    p32 = pos.cpu().numpy().view(np.float32)[:, :3 * S]
    p64 = p32.reshape(w.n, S, 3).astype(np.float64)
    ref = oracle.swept(robot, w.scene, w.params, p64, w.horizon, K, kink_eps=KINK_EPS)
    got_d = d.cpu().numpy().view(np.float32)[:, :S]
    got_g = g.cpu().numpy().view(np.float32)[:, :3 * S].reshape(w.n, S, 3)
    got_c = c.cpu().numpy()
    assert np.max(np.abs(got_c - ref["cost"])) <= REL_TOL * np.max(np.abs(ref["cost"]))
    assert np.max(np.abs(got_d - ref["dist"])) <= REL_TOL * np.max(np.abs(ref["dist"]))
    ok = ~ref["kink"]
    assert ok.mean() > 0.8
    err = np.abs(got_g - ref["grad"])[ok]
    assert np.max(err) <= REL_TOL * np.max(np.abs(ref["grad"]))
    assert (ref["dist"] > 0).mean() > 0.1


def test_horizon_one_scales_by_samples():
    import torch
    w, robot, rd, sd, pos = _setup()
    c1, d1, g1 = _swept(rd, sd, w, pos, 1, 1)
    c3, d3, g3 = _swept(rd, sd, w, pos, 1, 3)
    S = robot.n_spheres
    f = lambda t, L: t.view(torch.float32)[:, :L]
    assert torch.allclose(f(d3, S), 3 * f(d1, S), rtol=1e-6, atol=1e-7)
    assert torch.allclose(f(g3, 3 * S), 3 * f(g1, 3 * S), rtol=1e-5, atol=1e-6)


def test_reduced_formats_round_the_fp32_results():
    import torch
    w, robot, rd, sd, pos = _setup()
    S = robot.n_spheres
    t = F.FormatTable(pos=F.FP32, dist=F.E2M1, grad=F.E4M3)
    c32, d32, g32 = _swept(rd, sd, w, pos, w.horizon, 3)
    cr, dr, gr = _swept(rd, sd, w, pos, w.horizon, 3, t)
    assert torch.equal(c32, cr)
    dp = B.alloc_packed(w.n, S, F.E2M1)
    gp = B.alloc_packed(w.n, 3 * S, F.E4M3)
    B.vapr_pack(d32.view(torch.float32)[:, :S].contiguous(), w.n, S, F.E2M1, dp)
    B.vapr_pack(g32.view(torch.float32)[:, :3 * S].contiguous(), w.n, 3 * S, F.E4M3, gp)
    assert torch.equal(dp, dr) and torch.equal(gp, gr)
    assert B.vapr_device_error() == 0


def test_reduced_position_format_matches_oracle_on_decoded_centres():
    """P stored in E5M10: the swept cost equals the FP64 swept cost of the
    decoded (rounded) centres to the FP32 tolerance."""
    import torch
    w, robot, rd, sd, _ = _setup()
    S = robot.n_spheres
    t = F.FormatTable(pos=F.FP16)
    pos = B.alloc_packed(w.n, 3 * S, F.FP16)
    B.vapr_fk(rd, to_dev(w.q), w.n, t, pos)
    c, d, g = _swept(rd, sd, w, pos, w.horizon, 3, t)
    dec = torch.empty((w.n, 3 * S), device="cuda")
    B.vapr_unpack(pos, w.n, 3 * S, F.FP16, dec)
    p64 = dec.cpu().numpy().astype(np.float64).reshape(w.n, S, 3)
    ref = oracle.swept(robot, w.scene, w.params, p64, w.horizon, 3, kink_eps=KINK_EPS)
    got_c = c.cpu().numpy()
    assert np.max(np.abs(got_c - ref["cost"])) <= REL_TOL * np.max(np.abs(ref["cost"]))
