"""The pair-test compute ceiling (vapr_env_ceiling) does the collision
stage's work: its per-sphere (D, G) match the FP64 oracle's environment
term to 1e-5 normwise and the collision stage's FP32 outputs to rounding,
with a ragged last group; repetitions change nothing; spheres clear of
every cuboid (the bench's timed case) give exact zeros, also in the launch
configuration the bench times."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from parity import KINK_EPS, check_fp32, to_dev

pytestmark = pytest.mark.gpu


def _setup(name):
    """FP32 sphere centres of the workload from the library's FK, and the
    (x, y, z, r) rows the ceiling takes."""
    w = synth.make_workload(name)
    robot = dataclasses.replace(w.robot, pairs=np.zeros((0, 2), np.int32))
    rd, sd = B.DeviceRobot(robot), B.DeviceScene(w.scene)
    S = robot.n_spheres
    pos = B.alloc_packed(w.n, 3 * S, F.FP32)
    B.vapr_fk(rd, to_dev(w.q), w.n, F.FP32_TABLE, pos)
    p32 = pos.cpu().numpy().view(np.float32)[:, :3 * S].reshape(w.n, S, 3)
    r = np.asarray(robot.sphere_local, np.float32)[:, 3]
    sph = np.concatenate([p32, np.broadcast_to(r[None, :, None], (w.n, S, 1))], axis=2)
    return w, robot, rd, sd, pos, p32, np.ascontiguousarray(sph.reshape(-1, 4))


def _ceiling(sd, sph, eta, w_c, reps):
    import torch
    m = sph.shape[0]
    out = torch.full((m, 4), float("nan"), device="cuda")
    B.vapr_env_ceiling(sd, to_dev(sph), m, eta, w_c, reps, out)
    torch.cuda.synchronize()
    return out


def test_matches_oracle_and_collision_stage():
    import torch
    w, robot, rd, sd, pos, p32, sph = _setup("sweep_1024")
    S, n = robot.n_spheres, w.n
    m = n * S - 37  # the last 64-sphere group is ragged
    out = _ceiling(sd, sph[:m], w.params.eta, w.params.w_coll, 1).cpu().numpy().astype(np.float64)
    assert np.count_nonzero(out[:, 0]) > 0.05 * m  # many spheres touch a cuboid

    ref = oracle.collision(robot, w.scene, w.params, p32.astype(np.float64), kink_eps=KINK_EPS)
    keep = ~ref["kink"].reshape(-1)[:m, None]
    check_fp32(out[:, 0], ref["dist"].reshape(-1)[:m], what="D vs oracle")
    check_fp32(out[:, 1:], ref["grad"].reshape(-1, 3)[:m], mask=keep, what="G vs oracle")

    # the collision stage on the same centres (no self pairs, no grid)
    cost = torch.empty(n, device="cuda")
    dist = B.alloc_packed(n, S, F.FP32)
    grad = B.alloc_packed(n, 3 * S, F.FP32)
    B.vapr_collision_cost(rd, sd, w.params, pos, n, F.FP32_TABLE, cost, dist, grad)
    cd = dist.cpu().numpy().view(np.float32)[:, :S].reshape(-1)[:m].astype(np.float64)
    cg = grad.cpu().numpy().view(np.float32)[:, :3 * S].reshape(-1, 3)[:m].astype(np.float64)
    check_fp32(out[:, 0], cd, rel=1e-6, what="D vs collision stage")
    check_fp32(out[:, 1:], cg, rel=1e-6, what="G vs collision stage")


def test_repetitions_change_nothing():
    import torch
    w, robot, rd, sd, pos, p32, sph = _setup("single_128")
    a = _ceiling(sd, sph, w.params.eta, w.params.w_coll, 1)
    b = _ceiling(sd, sph, w.params.eta, w.params.w_coll, 7)
    assert torch.equal(a, b)


def test_edge_cases():
    import torch
    w, robot, rd, sd, pos, p32, sph = _setup("single_128")
    # no cuboids: every term is zero
    empty = B.DeviceScene(dataclasses.replace(w.scene, pose=np.zeros((0, 12), np.float32),
                                              half_ext=np.zeros((0, 3), np.float32)))
    out = _ceiling(empty, sph[:100], w.params.eta, w.params.w_coll, 2)
    assert torch.count_nonzero(out) == 0
    # n = 0 launches nothing and leaves the output alone
    o = torch.full((4, 4), 7.0, device="cuda")
    B.vapr_env_ceiling(sd, to_dev(sph[:4]), 0, w.params.eta, w.params.w_coll, 1, o)
    torch.cuda.synchronize()
    assert torch.all(o == 7.0)
    # a single sphere (one lane of one group)
    one = _ceiling(sd, sph[:1], w.params.eta, w.params.w_coll, 3).cpu().numpy()
    assert np.array_equal(one, _ceiling(sd, sph, w.params.eta, w.params.w_coll, 1).cpu().numpy()[:1])


def test_bench_launch_configuration():
    """The bench's timed case: the particle workload's spheres moved 100 m
    away, tiled to 64 x resident warps x 4 spheres, clear every cuboid
    (exact zeros); the same tiling of the real centres matches the oracle
    on a sample."""
    import torch
    w, robot, rd, sd, pos, p32, sph = _setup("particle_32768")
    W = B.vapr_env_ceiling_warps(w.scene.n_cuboids)
    props = torch.cuda.get_device_properties(0)
    assert W > 0 and W % 8 == 0 and W % props.multi_processor_count == 0
    nc = 64 * W * 4
    tiled = sph[np.arange(nc) % sph.shape[0]]
    far = tiled.copy()
    far[:, 0] += 100.0
    out = _ceiling(sd, far, w.params.eta, w.params.w_coll, 16)
    assert torch.count_nonzero(out) == 0
    out = _ceiling(sd, tiled, w.params.eta, w.params.w_coll, 2).cpu().numpy().astype(np.float64)
    idx = np.random.default_rng(3).choice(nc, 2000, replace=False)
    src = idx % sph.shape[0]
    cfg, s = src // robot.n_spheres, src % robot.n_spheres
    ref = oracle.collision(robot, w.scene, w.params, p32[cfg].astype(np.float64), kink_eps=KINK_EPS)
    pick = np.arange(idx.size)
    check_fp32(out[idx, 0], ref["dist"][pick, s], what="D sample")
    check_fp32(out[idx, 1:], ref["grad"][pick, s], mask=~ref["kink"][pick, s][:, None], what="G sample")
