"""The uneven multi-problem launch against the FP64 oracle, problem by
problem, on each problem's own jittered-radius arm and scene: every eighth of
the 64 uneven problems (4-256 trajectories, horizon 16-64, 4-60 cuboids,
radii +-10 %), and the particle workload run as one problem of the
persistent launch.

FP32 storage: cost and joint gradient to 1e-5 relative (normwise), the
gradient away from configurations next to a kink.  A reduced table with
float32 sphere centres and reduced D and G: the oracle quantises its own
FP64 gradient rows to the table's G format and runs its backward pass on
them; configurations where float32 rounding could pick a neighbouring code
(an FP64 value within the float32 error band of a rounding midpoint) are
left out, and every other one must match to 1e-5 relative."""
import numpy as np
import pytest

import oracle
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from parity import FP32_BAND, KINK_EPS, REL_TOL, decode_packed

pytestmark = pytest.mark.gpu

REDUCED = "P=E8M23,D=E2M1,G=E2M1,J=E8M23"


@pytest.fixture(scope="module")
def problems():
    return synth.make_uneven_problems()[::8]


def _normwise(got, want, mask, what):
    err = np.abs(got - want)[mask].max() if mask.any() else 0.0
    scale = np.abs(want[mask]).max() if mask.any() else 1.0
    assert err <= REL_TOL * scale, f"{what}: max error {err:.3e} vs {REL_TOL:.0e} x {scale:.3e}"


def _ambiguous_rows(values64, fmt):
    """Rows holding a value whose rounding to fmt could differ within the
    float32 error band (4e-6 of the row's scale)."""
    v = values64.reshape(values64.shape[0], -1)
    band = FP32_BAND * np.abs(v).max()
    lo = oracle.quantize((v - band).astype(np.float32), fmt.E, fmt.M, fmt.flags)
    hi = oracle.quantize((v + band).astype(np.float32), fmt.E, fmt.M, fmt.flags)
    return (lo != hi).any(1)


def _check(ev, i, w, table):
    import torch
    torch.cuda.synchronize()
    S, J = w.robot.n_spheres, w.robot.n_joints
    pos = oracle.fk(w.robot, w.q)
    col = oracle.collision(w.robot, w.scene, w.params, pos, kink_eps=KINK_EPS)
    cost = ev.cost[i].cpu().numpy().astype(np.float64)
    jg = decode_packed(ev.jgrad[i], J, table.jgrad)
    _normwise(cost, col["cost"], np.ones(w.n, bool), f"problem {i} cost")
    ok = ~col["kink"].any(1)
    grad = col["grad"]
    if table.grad != F.FP32:  # the oracle's own rows in the table's G format
        grad = oracle.quantize(grad.astype(np.float32), table.grad.E, table.grad.M,
                               table.grad.flags).reshape(grad.shape)
        ok &= ~_ambiguous_rows(col["grad"], table.grad)
    want = oracle.backward(w.robot, w.q, grad)
    assert ok.mean() > 0.5, f"problem {i}: too few configurations to compare"
    _normwise(jg, want, np.repeat(ok[:, None], J, 1), f"problem {i} jgrad")


@pytest.mark.parametrize("spec", ["", REDUCED])
def test_uneven_batch_matches_oracle(problems, spec):
    from paper_2310_07854_gb300.batched import BatchedEvaluator
    table = F.FormatTable.parse(spec) if spec else F.FP32_TABLE
    ev = BatchedEvaluator(problems, table, tile=128, grid_cells=32)
    ev.eval()
    assert ev.device_status() == 0
    assert len({w.scene.n_cuboids for w in problems}) > 4  # uneven obstacle counts
    assert len({float(w.robot.sphere_local[0, 3]) for w in problems}) == len(problems)  # jittered radii
    for i, w in enumerate(problems):
        _check(ev, i, w, table)


@pytest.mark.parametrize("spec", ["", REDUCED])
def test_single_problem_fused_launch_matches_oracle(spec):
    """FK, collision and backward of the particle workload in one persistent
    launch (the multi-problem kernel on a single problem)."""
    from paper_2310_07854_gb300.batched import BatchedEvaluator
    w = synth.make_workload("particle_32768")
    table = F.FormatTable.parse(spec) if spec else F.FP32_TABLE
    ev = BatchedEvaluator([w], table, tile=128)
    ev.eval()
    assert ev.device_status() == 0
    _check(ev, 0, w, table)
