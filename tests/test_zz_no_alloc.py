"""vapr_cost_grad_noalloc -- the whole step for callers that cannot allocate
device memory while they run (a real-time loop that cannot absorb
cudaMalloc, or a program whose device memory is fixed or owned by another
allocator).  Its scratch is a fixed array inside the library; the results
must match vapr_cost_grad with a caller workspace, on two calls in a row
(the second one finds the first one's leftovers in the array).

This file is collected last, so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from parity import check_fp32, decode_packed, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("spec", ["", "P=E5M10,D=E2M1,G=E2M1,J=E4M3"])
def test_noalloc_matches_cost_grad(spec):
    import torch
    w = synth.make_workload("particle_32768")
    table = F.FormatTable.parse(spec) if spec else F.FP32_TABLE
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    S, J, n = w.robot.n_spheres, w.robot.n_joints, w.n
    assert B.vapr_cost_grad_workspace_bytes(rd, n, table) <= B.NOALLOC_SCRATCH_BYTES
    q = to_dev(w.q)
    dc = to_dev(synth.make_dcost(5, n))

    # the existing entry point, with a workspace the caller allocated
    ref_cost = torch.empty(n, device="cuda")
    ref_dist = B.alloc_packed(n, S, table.dist)
    ref_jg = B.alloc_packed(n, J, table.jgrad)
    ws = B.alloc_workspace(rd, n, table)
    B.vapr_cost_grad(rd, sd, w.params, q, n, table, dc, ref_cost, ref_dist, ref_jg, ws)
    want_c = ref_cost.cpu().numpy().astype(np.float64)
    want_d = decode_packed(ref_dist, S, table.dist)
    want_j = decode_packed(ref_jg, J, table.jgrad)

    for call in range(2):  # two calls in a row share the library's scratch
        cost = torch.full((n,), float("nan"), device="cuda")
        dist = B.alloc_packed(n, S, table.dist)
        jg = B.alloc_packed(n, J, table.jgrad)
        B.vapr_cost_grad_noalloc(rd, sd, w.params, q, n, table, dc, cost, dist, jg)
        torch.cuda.synchronize()
        check_fp32(cost.cpu().numpy(), want_c, what=f"cost, call {call}")
        check_fp32(decode_packed(dist, S, table.dist), want_d, what=f"dist, call {call}")
        check_fp32(decode_packed(jg, J, table.jgrad), want_j, what=f"jgrad, call {call}")
    assert B.vapr_device_error() == 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """53,773 FP32 configurations of the 52-sphere arm fill the 64 MiB
    array exactly; one more is refused before any device work."""
    import torch
    w = synth.make_workload("single_128")
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    assert B.vapr_cost_grad_workspace_bytes(rd, 53773, F.FP32_TABLE) <= B.NOALLOC_SCRATCH_BYTES
    assert B.vapr_cost_grad_workspace_bytes(rd, 53774, F.FP32_TABLE) > B.NOALLOC_SCRATCH_BYTES
    q = torch.zeros((53774, 7), device="cuda")
    cost = torch.empty(53774, device="cuda")
    jg = B.alloc_packed(53774, 7, F.FP32)
    with pytest.raises(B.VaprError) as err:
        B.vapr_cost_grad_noalloc(rd, sd, w.params, q, 53774, F.FP32_TABLE, None, cost, None, jg)
    assert err.value.status == 6  # VAPR_ERR_TOO_LARGE
