"""Guard canaries: no entry point writes outside the buffers it is given.

Every output and workspace sits between two guard regions filled with a
byte pattern; after the calls (and a synchronize) the guards must be
unchanged.  The cases are ragged batch sizes and formats whose bit widths
do not divide 32 (E2M2 packs 6 values per word, E3M2 5, E2M3 5), where the
last word of a row is partly used and the row is padded to 16 bytes.  This
stands in for a device memory checker."""
import numpy as np
import pytest

from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from parity import to_dev

pytestmark = pytest.mark.gpu

FRONT, BACK, PATTERN = 256, 4096, 0xA5  # FRONT keeps 256-byte alignment


class Guarded:
    """nbytes of device memory with guard bytes on both sides."""

    def __init__(self, nbytes: int):
        import torch
        self.n = int(nbytes)
        self.buf = torch.full((FRONT + self.n + BACK,), PATTERN, dtype=torch.uint8, device="cuda")

    def view(self, shape=None, dtype=None):
        v = self.buf[FRONT:FRONT + self.n]
        if dtype is not None:
            v = v.view(dtype)
        return v.view(shape) if shape is not None else v

    def intact(self) -> bool:
        return bool((self.buf[:FRONT] == PATTERN).all()) and bool((self.buf[FRONT + self.n:] == PATTERN).all())


def _packed(rows, row_len, fmt):
    rb = B.packed_row_bytes(row_len, fmt)
    g = Guarded(rows * rb)
    return g, g.view((rows, rb))


def _floats(*shape):
    import torch
    g = Guarded(4 * int(np.prod(shape)))
    return g, g.view(shape, torch.float32)


TABLES = ["", "P=E2M2,D=E3M2,G=E2M1,J=E2M3,T=E5M10", "P=E5M10,D=E2M3,G=E3M4,J=E2M2,T=E8M7"]


@pytest.mark.parametrize("spec", TABLES, ids=lambda s: s or "fp32")
@pytest.mark.parametrize("n", [1, 37, 1031])
def test_path_entry_points_stay_inside_their_buffers(spec, n):
    import torch
    w = synth.make_workload("single_128")
    table = F.FormatTable.parse(spec) if spec else F.FP32_TABLE
    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    S, J = w.robot.n_spheres, w.robot.n_joints
    q = to_dev(synth.make_q(11, n))
    dc = to_dev(synth.make_dcost(12, n))
    guards = []

    def packed(row_len, fmt):
        g, v = _packed(n, row_len, fmt)
        guards.append(g)
        return v

    def floats(*shape):
        g, v = _floats(*shape)
        guards.append(g)
        return v

    pos, xf = packed(3 * S, table.pos), packed(12 * J, table.xform)
    B.vapr_fk(rd, q, n, table, pos, xf)
    cost, dist, grad = floats(n), packed(S, table.dist), packed(3 * S, table.grad)
    B.vapr_collision_cost(rd, sd, w.params, pos, n, table, cost, dist, grad)
    B.vapr_backward(rd, q, xf, grad, dc, n, table, packed(J, table.jgrad))
    B.vapr_backward(rd, q, None, grad, None, n, table, packed(J, table.jgrad))
    B.vapr_swept_cost(rd, sd, w.params, pos, n, n, 3, table, floats(n), packed(S, table.dist),
                      packed(3 * S, table.grad))
    ws = Guarded(max(B.vapr_cost_grad_workspace_bytes(rd, n, table), 1))
    guards.append(ws)
    B.vapr_cost_grad(rd, sd, w.params, q, n, table, dc, floats(n), packed(S, table.dist),
                     packed(J, table.jgrad), ws.view(), workspace_bytes=ws.n)
    B.vapr_cost_grad_noalloc(rd, sd, w.params, q, n, table, dc, floats(n), packed(S, table.dist),
                             packed(J, table.jgrad))
    spheres = torch.rand((n, 4), device="cuda") * 0.5
    B.vapr_env_ceiling(sd, spheres, n, w.params.eta, w.params.w_coll, 2, floats(n, 4))
    torch.cuda.synchronize()
    assert B.vapr_device_error() == 0
    bad = [i for i, g in enumerate(guards) if not g.intact()]
    assert not bad, f"guards overwritten: {bad}"


@pytest.mark.parametrize("fmt", list(F.SWEEP) + [F.fmt(2, 2), F.fmt(2, 3), F.fmt(3, 1), F.fmt(6, 1),
                                                 F.fmt(5, 10), F.fmt(4, 5)], ids=str)
@pytest.mark.parametrize("rows,row_len", [(1, 1), (3, 7), (129, 61)])
def test_pack_unpack_stay_inside_their_buffers(fmt, rows, row_len):
    import torch
    src = torch.randn((rows, row_len), device="cuda") * 3.0
    gp, dst = _packed(rows, row_len, fmt)
    B.vapr_pack(src, rows, row_len, fmt, dst)
    gu, back = _floats(rows, row_len)
    B.vapr_unpack(dst, rows, row_len, fmt, back)
    torch.cuda.synchronize()
    assert gp.intact() and gu.intact()
