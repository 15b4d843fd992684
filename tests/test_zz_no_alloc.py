"""vapr_cost_grad_noalloc -- the whole step for callers that cannot allocate
device memory while they run (a real-time loop that cannot absorb
cudaMalloc, or a program whose device memory is fixed or owned by another
allocator).  Its scratch is a fixed array inside the library.

Both entry points run the same kernels on the same inputs, and the path is
deterministic, so the outputs must match vapr_cost_grad with a caller
workspace byte for byte.  Between the checked calls another call runs on a
different batch of a different size, so the array holds other P and G rows
(at other offsets) when the checked call starts: a word that a checked call
failed to write would keep a wrong value and show up.  One call fills the
array to its last byte.

This file is collected last, so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import pytest

from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from parity import to_dev

pytestmark = pytest.mark.gpu

FULL = 53773  # FP32 configurations of the 52-sphere arm that fill the 64 MiB array


def _outputs(n, S, J, table):
    import torch
    cost = torch.full((n,), float("nan"), device="cuda")
    return cost, B.alloc_packed(n, S, table.dist), B.alloc_packed(n, J, table.jgrad)


def _reference(rd, sd, params, q, n, table, dc, S, J):
    """vapr_cost_grad with a workspace the caller allocated."""
    cost, dist, jg = _outputs(n, S, J, table)
    ws = B.alloc_workspace(rd, n, table)
    B.vapr_cost_grad(rd, sd, params, q, n, table, dc, cost, dist, jg, ws)
    return cost, dist, jg


def _noalloc(rd, sd, params, q, n, table, dc, S, J):
    cost, dist, jg = _outputs(n, S, J, table)
    B.vapr_cost_grad_noalloc(rd, sd, params, q, n, table, dc, cost, dist, jg)
    return cost, dist, jg


def _assert_same(got, want, what):
    import torch
    torch.cuda.synchronize()
    for name, g, w in zip(("cost", "dist", "jgrad"), got, want):
        assert torch.equal(g, w), f"{name} differs from vapr_cost_grad ({what})"


@pytest.mark.parametrize("spec", ["", "P=E5M10,D=E2M1,G=E2M1,J=E4M3"])
def test_noalloc_matches_cost_grad(spec):
    w = synth.make_workload("particle_32768")
    table = F.FormatTable.parse(spec) if spec else F.FP32_TABLE
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    S, J, n = w.robot.n_spheres, w.robot.n_joints, w.n
    assert B.vapr_cost_grad_workspace_bytes(rd, n, table) <= B.NOALLOC_SCRATCH_BYTES
    q = to_dev(w.q)
    dc = to_dev(synth.make_dcost(5, n))
    # another batch, of another size: its P and G rows land at other offsets
    n2 = n - 4093
    q2 = to_dev(synth.make_q(77, n2))
    dc2 = to_dev(synth.make_dcost(78, n2))

    want = _reference(rd, sd, w.params, q, n, table, dc, S, J)
    want2 = _reference(rd, sd, w.params, q2, n2, table, dc2, S, J)
    for call in range(2):  # two checked calls in a row, another batch between them
        _assert_same(_noalloc(rd, sd, w.params, q, n, table, dc, S, J), want, f"call {call}")
        _assert_same(_noalloc(rd, sd, w.params, q2, n2, table, dc2, S, J), want2, f"between, call {call}")
    assert B.vapr_device_error() == 0


def test_noalloc_fills_the_whole_array():
    """53,773 FP32 configurations use the array up to its last bytes; the
    results still equal vapr_cost_grad's, after a smaller call and before one."""
    w = synth.make_workload("particle_32768")
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    S, J = w.robot.n_spheres, w.robot.n_joints
    table = F.FP32_TABLE
    need = B.vapr_cost_grad_workspace_bytes(rd, FULL, table)
    assert B.NOALLOC_SCRATCH_BYTES - 512 < need <= B.NOALLOC_SCRATCH_BYTES
    q = to_dev(synth.make_q(91, FULL))
    want = _reference(rd, sd, w.params, q, FULL, table, None, S, J)
    small = to_dev(synth.make_q(92, 1000))
    want_small = _reference(rd, sd, w.params, small, 1000, table, None, S, J)
    _assert_same(_noalloc(rd, sd, w.params, small, 1000, table, None, S, J), want_small, "small, first")
    _assert_same(_noalloc(rd, sd, w.params, q, FULL, table, None, S, J), want, "full array")
    _assert_same(_noalloc(rd, sd, w.params, small, 1000, table, None, S, J), want_small, "small, after")
    assert B.vapr_device_error() == 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """One configuration more than fits is refused before any device work."""
    import torch
    w = synth.make_workload("single_128")
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    assert B.vapr_cost_grad_workspace_bytes(rd, FULL, F.FP32_TABLE) <= B.NOALLOC_SCRATCH_BYTES
    assert B.vapr_cost_grad_workspace_bytes(rd, FULL + 1, F.FP32_TABLE) > B.NOALLOC_SCRATCH_BYTES
    q = torch.zeros((FULL + 1, 7), device="cuda")
    cost = torch.empty(FULL + 1, device="cuda")
    jg = B.alloc_packed(FULL + 1, 7, F.FP32)
    with pytest.raises(B.VaprError) as err:
        B.vapr_cost_grad_noalloc(rd, sd, w.params, q, FULL + 1, F.FP32_TABLE, None, cost, None, jg)
    assert err.value.status == 6  # VAPR_ERR_TOO_LARGE
