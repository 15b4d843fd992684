"""The uneven multi-problem launch (vapr_batched_*) on the 64-problem batch
(4-256 trajectories, horizon 16-64, 4-60 cuboids, radii +-10 %): results
equal vapr_cost_grad per problem, a captured CUDA graph replays them, an
unpublished problem times out with a status (the others still run), and
the tile autotuner persists its choice."""
import json
import os

import numpy as np
import pytest

from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problems():
    return synth.make_uneven_problems()


def _reference(w, table):
    import torch
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    q = torch.as_tensor(w.q, device="cuda")
    cost = torch.empty(w.n, device="cuda")
    jg = B.alloc_packed(w.n, w.robot.n_joints, table.jgrad)
    ws = B.alloc_workspace(rd, w.n, table)
    B.vapr_cost_grad(rd, sd, w.params, q, w.n, table, None, cost, None, jg, ws)
    return cost, jg


@pytest.mark.parametrize("spec,tile,grid", [("", 128, 32), ("", 32, 32), ("", 256, 32),
                                            ("P=E5M10,D=E2M1,G=E2M1,J=E4M3", 64, 32), ("", 128, None),
                                            ("", 64, 96)])
def test_batched_equals_per_problem(problems, spec, tile, grid):
    """Each problem's scene grid (or none) leaves the results as the plain
    per-problem path gives them."""
    import torch
    from paper_2310_07854_gb300.batched import BatchedEvaluator
    table = F.FormatTable.parse(spec) if spec else F.FP32_TABLE
    ev = BatchedEvaluator(problems, table, tile=tile, grid_cells=grid)
    ev.eval()
    torch.cuda.synchronize()
    assert ev.device_status() == 0
    for i, w in enumerate(problems):
        cost, jg = _reference(w, table)
        assert torch.equal(ev.cost[i], cost), i
        assert torch.equal(ev.jgrad[i], jg), i


def test_graph_replay(problems):
    import torch
    from paper_2310_07854_gb300.batched import BatchedEvaluator
    ev = BatchedEvaluator(problems, F.FP32_TABLE, tile=128)
    ev.eval()
    torch.cuda.synchronize()
    want = [c.clone() for c in ev.cost]
    wantj = [j.clone() for j in ev.jgrad]
    for c in ev.cost:
        c.fill_(float("nan"))
    g = ev.capture()
    for c in ev.cost:
        c.fill_(float("nan"))
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(ev.cost, want))
    assert all(torch.equal(a, b) for a, b in zip(ev.jgrad, wantj))


def test_unpublished_problem_times_out(problems):
    """A deferred problem nobody publishes: the bounded wait gives up after
    20 ms, the status says VAPR_ERR_TIMEOUT, its outputs stay untouched and
    every other problem is still evaluated; after publishing, all run."""
    import torch
    from paper_2310_07854_gb300.batched import BatchedEvaluator
    sub = problems[:12]
    ev = BatchedEvaluator(sub, F.FP32_TABLE, tile=128, wait_limit_us=20000, deferred=(3,))
    ev.eval()
    torch.cuda.synchronize()
    assert ev.device_status() == 5  # VAPR_ERR_TIMEOUT
    assert torch.isnan(ev.cost[3]).all()
    for i, w in enumerate(sub):
        if i != 3:
            cost, jg = _reference(w, F.FP32_TABLE)
            assert torch.equal(ev.cost[i], cost), i
    ev.publish(3)
    ev.eval()
    torch.cuda.synchronize()
    assert ev.device_status() == 0
    cost, jg = _reference(sub[3], F.FP32_TABLE)
    assert torch.equal(ev.cost[3], cost) and torch.equal(ev.jgrad[3], jg)


def test_autotuner_picks_and_caches(problems, tmp_path):
    from paper_2310_07854_gb300 import autotune
    cache = str(tmp_path / "tiles.json")
    r1 = autotune.tune(problems, F.FP32_TABLE, cache_path=cache)
    assert r1["tile"] in autotune.CANDIDATES and not r1["cached"]
    assert r1["ms"][str(r1["tile"])] == min(r1["ms"].values())
    r2 = autotune.tune(problems, F.FP32_TABLE, cache_path=cache)
    assert r2["cached"] and r2["tile"] == r1["tile"]
    data = json.load(open(cache))
    assert len(data) == 1 and len(next(iter(data.values()))) == 1
    out_dir = os.environ.get("VAPR_REPORT_DIR")
    if out_dir:
        with open(os.path.join(out_dir, "autotune_uneven64.json"), "w") as f:
            json.dump(r1, f)
