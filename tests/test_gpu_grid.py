"""The broad-phase grid of a scene (vapr_scene_grid_build): the collision
stage gives the same bits with and without it, the cell of every point lists
each cuboid that a sphere centred there can penetrate (box distance below
reach + eta, from the FP64 oracle), a grid that does not match the scene,
eta or radii is ignored, and a matching one is the grid the kernel reads."""
import numpy as np
import pytest

import oracle

from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from paper_2310_07854_gb300.path import Evaluator
from parity import GpuPath, to_dev

pytestmark = pytest.mark.gpu

TABLES = [F.FP32_TABLE, F.FormatTable.parse("P=E5M10,D=E2M1,G=E2M1,J=E4M3"),
          F.FormatTable.parse("P=BF16,D=E4M3,G=E5M2,J=FP16")]


def reach_of(robot):
    return float(np.max(robot.sphere_local[:, 3]))


def outputs(gp, pos, n, table):
    """cost, D, G of the collision stage as raw bytes."""
    cost, dist, grad = gp.collision(pos, n, table)
    return cost.cpu().numpy().view(np.uint32), dist.cpu().numpy(), grad.cpu().numpy()


def assert_same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def with_grid(gp, cells, reach=None, eta=None):
    gp.sd.build_grid(reach_of(gp.robot) if reach is None else reach,
                     gp.params.eta if eta is None else eta, cells)
    return gp


@pytest.mark.parametrize("name", ["single_128", "sweep_1024", "particle_32768"])
@pytest.mark.parametrize("table", TABLES, ids=str)
@pytest.mark.parametrize("cells", [1, 7, 48, 128])
def test_grid_outputs_bit_identical(name, table, cells):
    w = synth.make_workload(name)
    gp = GpuPath(w.robot, w.scene, w.params)
    pos, _ = gp.fk(to_dev(w.q), w.n, table)
    plain = outputs(gp, pos, w.n, table)
    with_grid(gp, cells)
    assert_same(outputs(gp, pos, w.n, table), plain)


@pytest.mark.parametrize("n_cuboids,extent", [(0, 0.75), (1, 0.3), (65, 0.9), (200, 1.2), (130, 0.2),
                                               (1024, 1.5)])
@pytest.mark.parametrize("cells", [5, 32, 100])
def test_grid_random_scenes(n_cuboids, extent, cells):
    """Several 64-cuboid chunks (up to the 1024-cuboid maximum), an empty
    scene, a scene far smaller than the arm's reach (most spheres outside
    the grid), a dense one."""
    w = synth.make_workload("sweep_1024")
    w.scene = synth.make_scene(11 + n_cuboids, n_cuboids, extent=extent)
    gp = GpuPath(w.robot, w.scene, w.params)
    for table in TABLES[:2]:
        pos, _ = gp.fk(to_dev(w.q), w.n, table)
        gp.sd.drop_grid()
        plain = outputs(gp, pos, w.n, table)
        with_grid(gp, cells)
        assert_same(outputs(gp, pos, w.n, table), plain)


def decode_grid(buf):
    raw = buf.cpu().numpy()
    f = raw[:128].view(np.float32)
    i = raw[:128].view(np.int32)
    u = raw[:128].view(np.uint32)
    hdr = dict(lo=f[0:3].copy(), inv_h=np.float32(f[3]), dims=i[4:7].copy(), words=int(i[7]), O=int(i[8]),
               eta_bits=int(u[9]), reach=float(f[10]), h=float(f[12]), magic=int(i[13]))
    ncell = int(np.prod(hdr["dims"]))
    cells = raw[128:128 + ncell * hdr["words"] * 4].view(np.uint32).reshape(ncell, hdr["words"])
    return hdr, cells


def cell_bits(hdr, cells, p):
    """Candidate mask of the cell holding p (float32 index arithmetic as the
    kernel does it), or None outside the grid."""
    p = np.asarray(p, np.float32)
    fidx = (p - hdr["lo"]) * hdr["inv_h"]
    if not np.all((fidx >= 0) & (fidx < hdr["dims"].astype(np.float32))):
        return None
    ix, iy, iz = np.minimum(fidx.astype(np.int64), hdr["dims"] - 1)
    return cells[(iz * hdr["dims"][1] + iy) * hdr["dims"][0] + ix]


@pytest.mark.parametrize("cells_n", [3, 24, 64])
def test_grid_lists_every_cuboid_a_sphere_can_penetrate(cells_n):
    """Points spread over the region and points around each cuboid, many of
    them near the threshold: wherever the box distance d_o(p) < reach + eta
    (some sphere of radius <= reach centred at p penetrates o with margin
    eta), the cell of p lists o."""
    w = synth.make_workload("particle_32768")
    sd = B.DeviceScene(w.scene)
    reach, eta = reach_of(w.robot), w.params.eta
    sd.build_grid(reach, eta, cells_n)
    hdr, cells = decode_grid(sd.grid)
    assert hdr["magic"] == 0x56475244 and hdr["O"] == w.scene.n_cuboids
    pose = np.asarray(w.scene.pose, np.float32).reshape(-1, 12)
    half = np.asarray(w.scene.half_ext, np.float32).reshape(-1, 3)
    O = pose.shape[0]
    rng = np.random.default_rng(cells_n)
    lo = hdr["lo"].astype(np.float64)
    hi = lo + hdr["dims"] * hdr["h"]
    pts = [rng.uniform(lo - 0.1, hi + 0.1, size=(4000, 3))]
    for o in range(O):  # around cuboid o, out to beyond the threshold
        ext = np.abs(pose[o, :9].reshape(3, 3)).astype(np.float64) @ half[o] + reach + eta + 0.03
        pts.append(pose[o, 9:12] + rng.uniform(-1, 1, size=(300, 3)) * ext)
    pts = np.concatenate(pts).astype(np.float32)
    m = pts.shape[0]
    d = np.empty((m, O))
    for o in range(O):
        d[:, o] = oracle.box_sdf(np.repeat(pose[o:o + 1], m, 0), np.repeat(half[o:o + 1], m, 0), pts)[0]
    must = d < (reach + eta) * (1 - 1e-6)
    near = (np.abs(d - (reach + eta)) < 0.01) & must
    assert near.sum() > 200  # many pairs close to the threshold
    checked = 0
    for p, row in zip(pts, must):
        if not row.any():
            continue
        bits = cell_bits(hdr, cells, p)
        assert bits is not None, p
        for o in np.nonzero(row)[0]:
            assert (int(bits[o // 32]) >> (o % 32)) & 1, (p, o)
            checked += 1
    assert checked > 1000
    # and the grid narrows: a cell lists far fewer than all cuboids on average
    pop = np.array([bin(int(x)).count("1") for x in cells.reshape(-1)]).reshape(cells.shape[0], -1).sum(1)
    if cells_n >= 24:
        assert pop.mean() < 0.5 * w.scene.n_cuboids


def _moved_scene(scene, o, shift):
    pose = np.array(scene.pose, np.float32).reshape(-1, 12)
    pose[o, 9:12] += shift
    return synth.Scene(pose=pose, half_ext=np.array(scene.half_ext, np.float32).reshape(-1, 3))


def _poisoned(gp, cells=16, **kw):
    """A grid whose header matches what it was built for, over empty cells:
    if the kernel accepted it, no sphere would meet a cuboid."""
    with_grid(gp, cells, **kw)
    gp.sd.grid[128:].zero_()


def test_stale_grids_are_ignored():
    """Grids built for other scene contents, another eta or too small a
    reach (and emptied, so that using one would show) are not used."""
    import torch
    w = synth.make_workload("sweep_1024")
    table = F.FP32_TABLE
    gp = GpuPath(w.robot, w.scene, w.params)
    pos, _ = gp.fk(to_dev(w.q), w.n, table)
    plain = outputs(gp, pos, w.n, table)
    empty = outputs(GpuPath(w.robot, synth.make_scene(0, 0), w.params), pos, w.n, table)
    assert not np.array_equal(plain[0], empty[0])
    # (a) scene contents changed after the build
    _poisoned(gp)
    moved = _moved_scene(w.scene, 0, np.float32(1e-3))
    gp.sd.pose.copy_(torch.as_tensor(np.asarray(moved.pose, np.float32).reshape(-1, 12)))
    assert_same(outputs(gp, pos, w.n, table), outputs(GpuPath(w.robot, moved, w.params), pos, w.n, table))
    # (b) built for another eta
    gp = GpuPath(w.robot, w.scene, w.params)
    _poisoned(gp, eta=w.params.eta + 0.01)
    assert_same(outputs(gp, pos, w.n, table), plain)
    # (c) built for smaller spheres
    _poisoned(gp, reach=0.5 * reach_of(w.robot))
    assert_same(outputs(gp, pos, w.n, table), plain)
    # (d) a grid the builder marked unusable is not used either
    with_grid(gp, 16)
    gp.sd.grid[52:56].zero_()  # magic
    gp.sd.grid[128:].zero_()
    assert_same(outputs(gp, pos, w.n, table), plain)


def test_matching_grid_is_read():
    """A valid header over empty cells: the kernel believes it, so no sphere
    meets a cuboid and the outputs are those of the empty scene."""
    w = synth.make_workload("sweep_1024")
    table = F.FP32_TABLE
    gp = GpuPath(w.robot, w.scene, w.params)
    pos, _ = gp.fk(to_dev(w.q), w.n, table)
    with_grid(gp, 16)
    gp.sd.grid[128:].zero_()
    emptied = outputs(gp, pos, w.n, table)
    empty = GpuPath(w.robot, synth.make_scene(0, 0), w.params)
    assert_same(emptied, outputs(empty, pos, w.n, table))
    assert not np.array_equal(emptied[0], outputs(GpuPath(w.robot, w.scene, w.params), pos, w.n, table)[0])


def test_grid_in_cost_grad_ik_and_surrogate():
    """The entry points that run the collision stage inside them."""
    import torch
    from paper_2310_07854_gb300 import ik as IK
    from paper_2310_07854_gb300 import surrogate as SG
    w = synth.make_workload("sweep_1024")
    table = F.FormatTable.parse("P=E5M10,D=E2M1,G=E2M1,J=E4M3")
    res = []
    for grid in (False, True):
        sd = B.DeviceScene(w.scene)
        if grid:
            sd.build_grid(reach_of(w.robot), w.params.eta, 48)
        ev = Evaluator(w.robot, sd, w.params, w.n, table)
        q = to_dev(w.q)
        ev.step(q, w.n)
        out = [ev.cost[:w.n].cpu().numpy().view(np.uint32), ev.jgrad[:w.n].cpu().numpy()]
        # IK: a few iterations from the same seeds
        n_seeds = 256
        goal = torch.zeros(n_seeds, 12, device="cuda")
        goal[:, 0] = goal[:, 4] = goal[:, 8] = 1.0
        goal[:, 9:12] = torch.tensor([0.3, 0.2, 0.5])
        qi = to_dev(synth.make_q(5, n_seeds))
        s = IK.IkSolver(ev.robot, sd, w.params, n_seeds)
        s.init(goal, qi)
        s.solve(3)
        out.append(qi.cpu().numpy().view(np.uint32))
        # surrogate gate (an untrained network: the gate is the same either way)
        sg = SG.Surrogate(sd, synth.init_mlp_params(3))
        pos = B.alloc_packed(w.n, 3 * w.robot.n_spheres, F.FP32)
        B.vapr_fk(ev.robot, q, w.n, F.FP32_TABLE, pos)
        S = w.robot.n_spheres
        cost = torch.empty(w.n, device="cuda")
        dist = B.alloc_packed(w.n, S, F.FP32)
        grad = B.alloc_packed(w.n, 3 * S, F.FP32)
        sg.collision_cost(ev.robot, w.params, pos, w.n, F.FP32_TABLE, cost, dist, grad)
        out += [cost.cpu().numpy().view(np.uint32), dist.cpu().numpy(), grad.cpu().numpy()]
        res.append(out)
    assert_same(res[0], res[1])


@pytest.mark.parametrize("name,K", [("sweep_1024", 4), ("particle_32768", 3), ("single_128", 1)])
def test_grid_in_swept_cost(name, K):
    """The swept points go through the same grid: same bits with and without."""
    import torch
    w = synth.make_workload(name)
    rd = B.DeviceRobot(w.robot)
    S = w.robot.n_spheres
    pos = B.alloc_packed(w.n, 3 * S, F.FP32)
    B.vapr_fk(rd, to_dev(w.q), w.n, F.FP32_TABLE, pos)
    res = []
    for grid in (False, True):
        sd = B.DeviceScene(w.scene)
        if grid:
            sd.build_grid(reach_of(w.robot), w.params.eta, 48)
        for table in TABLES[:2]:
            cost = torch.empty(w.n, device="cuda")
            dist = B.alloc_packed(w.n, S, table.dist)
            grad = B.alloc_packed(w.n, 3 * S, table.grad)
            B.vapr_swept_cost(rd, sd, w.params, pos, w.n, w.horizon, K, table, cost, dist, grad)
            res.append([cost.cpu().numpy().view(np.uint32), dist.cpu().numpy(), grad.cpu().numpy()])
    assert_same(res[0], res[2])
    assert_same(res[1], res[3])
