"""Ticket scheduling of the collision stage: every configuration is
evaluated exactly once per launch, whether the launch is replayed from a
captured graph, runs beside others on several streams, or follows more
launches than there are round-robin ticket slots."""
import numpy as np
import pytest

from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from parity import GpuPath, to_dev

pytestmark = pytest.mark.gpu


def _path(name="sweep_1024"):
    w = synth.make_workload(name)
    return w, GpuPath(w.robot, w.scene, w.params)


def _collide(gp, pos, n, cost, dist, grad, stream=None):
    B.vapr_collision_cost(gp.rd, gp.sd, gp.params, pos, n, F.FP32_TABLE, cost, dist, grad, stream)


def _bufs(w, n):
    import torch
    S = w.robot.n_spheres
    return (torch.full((n,), float("nan"), device="cuda"), B.alloc_packed(n, S, F.FP32),
            B.alloc_packed(n, 3 * S, F.FP32))


def test_graph_replays_see_new_inputs():
    """A captured launch keeps its ticket slot; each replay must start from
    ticket zero again, so new inputs give new outputs on every replay."""
    import torch
    w, gp = _path()
    n = w.n
    pos = B.alloc_packed(n, 3 * w.robot.n_spheres, F.FP32)
    out = _bufs(w, n)
    s = torch.cuda.Stream()
    gp.fk(to_dev(w.q), n, F.FP32_TABLE)  # warm the launch caches
    with torch.cuda.stream(s):
        _collide(gp, pos, n, *out, stream=s)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            _collide(gp, pos, n, *out, stream=s)
    for seed in (3, 4, 5, 6):
        q = to_dev(synth.make_q(seed, n))
        B.vapr_fk(gp.rd, q, n, F.FP32_TABLE, pos)
        torch.cuda.synchronize()
        for t in out:
            t.fill_(0) if t.dtype == torch.uint8 else t.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        want = _bufs(w, n)
        _collide(gp, pos, n, *want)
        torch.cuda.synchronize()
        for a, b in zip(out, want):
            assert torch.equal(a.view(torch.uint8), b.view(torch.uint8)), seed


def test_concurrent_streams_and_slot_wraparound():
    """1300 launches (more than the 1024 round-robin slots) over four streams
    at once, each on its own inputs."""
    import torch
    w, gp = _path("single_128")
    n, S = w.n, w.robot.n_spheres
    streams = [torch.cuda.Stream() for _ in range(4)]
    poss, wants, outs = [], [], []
    for k in range(4):
        pos = B.alloc_packed(n, 3 * S, F.FP32)
        B.vapr_fk(gp.rd, to_dev(synth.make_q(20 + k, n)), n, F.FP32_TABLE, pos)
        poss.append(pos)
        want = _bufs(w, n)
        _collide(gp, pos, n, *want)
        wants.append(want)
        outs.append(_bufs(w, n))
    torch.cuda.synchronize()
    for it in range(1300):
        k = it % 4
        with torch.cuda.stream(streams[k]):
            _collide(gp, poss[k], n, *outs[k], stream=streams[k])
        if it % 260 == 259:
            torch.cuda.synchronize()
            for k2 in range(4):
                for a, b in zip(outs[k2], wants[k2]):
                    assert torch.equal(a.view(torch.uint8), b.view(torch.uint8)), (it, k2)
                for t in outs[k2]:
                    t.zero_()
            torch.cuda.synchronize()
