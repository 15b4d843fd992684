"""Replica host logic with two gloo ranks on CPU: distinct per-rank batches,
max over ranks, whole-job throughput."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_2310_07854_gb300 import replicas, synth
    w_, r_, l_ = replicas.dist_env()
    dist.init_process_group("gloo", rank=r_, world_size=w_, init_method="env://")
    w = synth.make_workload("single_128")
    q = replicas.rank_batch(w, r_)
    t = replicas.max_over_ranks(1.0 + r_, dist)
    out.put((r_, w_, l_, q.sum(), q.shape, t, replicas.job_throughput(w_, w.n, 10, t)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, sh0, t0, v0), (r1, w1, l1, s1, sh1, t1, v1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert sh0 == sh1 and s0 != s1          # same size, different configurations
    assert t0 == t1 == 2.0                  # the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 128 * 10 / 2.0)
