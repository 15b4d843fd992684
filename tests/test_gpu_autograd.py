"""The autograd wrapper on the particle workload: gradients through
torch.autograd against central finite differences of the FP64 oracle
(h = 2^-13 ~ 1.2e-4, exact in float32), with FK recomputed in backward and
with stored transforms, plus a reduced-precision table."""
import numpy as np
import pytest

import oracle
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from parity import check_fp32, to_dev

pytestmark = pytest.mark.gpu


def _dyadic(x, bits=20):
    return (np.round(np.asarray(x, np.float64) * 2**bits) / 2**bits).astype(np.float32)


@pytest.fixture(scope="module")
def fd_case():
    w = synth.make_workload("particle_32768")
    n = 512
    q = _dyadic(w.q[:n])
    weights = synth.make_dcost(3, n).astype(np.float64)
    h = 2.0 ** -13
    pos = oracle.fk(w.robot, q)
    # a step of h moves a sphere by < 2.5e-4 m: skip configurations within 5e-4 of a kink
    col = oracle.collision(w.robot, w.scene, w.params, pos, kink_eps=5e-4)
    fd = np.empty((n, 7))
    for j in range(7):
        qp, qm = q.copy(), q.copy()
        qp[:, j] += np.float32(h)
        qm[:, j] -= np.float32(h)
        cp = oracle.collision(w.robot, w.scene, w.params, oracle.fk(w.robot, qp))["cost"]
        cm = oracle.collision(w.robot, w.scene, w.params, oracle.fk(w.robot, qm))["cost"]
        fd[:, j] = weights * (cp - cm) / (2 * h)
    ok = ~col["kink"].any(1)
    return dict(w=w, q=q, weights=weights, fd=fd, ok=ok, cost=col["cost"])


@pytest.mark.parametrize("recompute", [True, False], ids=["recompute_fk", "stored_T"])
def test_autograd_matches_fd(fd_case, recompute):
    import torch
    from paper_2310_07854_gb300.autograd import VaprCost
    c = fd_case
    w = c["w"]
    mod = VaprCost(w.robot, w.scene, w.params, recompute_fk=recompute)
    q = to_dev(c["q"]).requires_grad_(True)
    cost = mod(q)
    loss = (cost.double() * torch.as_tensor(c["weights"], device="cuda")).sum()
    loss.backward()
    g = q.grad.cpu().numpy().astype(np.float64)
    assert c["ok"].sum() > 50
    # FD truncation error (h^2 f''') and float32 error are both far below this
    check_fp32(g, c["fd"], mask=np.repeat(c["ok"][:, None], 7, 1), rel=2e-5, what="dL/dq")
    check_fp32(cost.detach().cpu().numpy(), c["cost"], what="C")


def test_autograd_reduced_table(fd_case):
    """A reduced table still gives a usable gradient: report its error."""
    import torch
    from paper_2310_07854_gb300.autograd import VaprCost
    c = fd_case
    w = c["w"]
    mod = VaprCost(w.robot, w.scene, w.params, F.FormatTable.parse("P=E5M10,G=E4M3,J=BF16"))
    q = to_dev(c["q"]).requires_grad_(True)
    mod(q).mul(torch.as_tensor(c["weights"], dtype=torch.float32, device="cuda")).sum().backward()
    g = q.grad.cpu().numpy().astype(np.float64)
    ok = c["ok"]
    rel = np.abs(g - c["fd"])[ok].max() / np.abs(c["fd"][ok]).max()
    cos = (g[ok] * c["fd"][ok]).sum() / np.linalg.norm(g[ok]) / np.linalg.norm(c["fd"][ok])
    assert cos > 0.99 and rel < 0.2, (cos, rel)


def test_two_pending_forwards():
    """Buffers belong to each graph: a second forward does not disturb the
    first one's backward."""
    import torch
    from paper_2310_07854_gb300.autograd import VaprCost
    w = synth.make_workload("single_128")
    mod = VaprCost(w.robot, w.scene, w.params)
    qa = to_dev(w.q).requires_grad_(True)
    qb = to_dev(synth.make_q(99, w.n)).requires_grad_(True)
    ca = mod(qa)
    cb = mod(qb)
    ca.sum().backward()
    ga = qa.grad.clone()
    qa2 = to_dev(w.q).requires_grad_(True)
    mod(qa2).sum().backward()
    assert torch.equal(ga, qa2.grad)
    cb.sum().backward()
    assert torch.isfinite(qb.grad).all()


def test_autograd_uses_the_scene_grid():
    """VaprCost builds the broad-phase grid for a host scene, and its cost and
    gradient equal the grid-less module's bit for bit (the grid only narrows
    which cuboids the kernel visits)."""
    import torch
    from paper_2310_07854_gb300.autograd import VaprCost
    w = synth.make_workload("particle_32768")
    with_grid = VaprCost(w.robot, w.scene, w.params)
    plain = VaprCost(w.robot, w.scene, w.params, grid_cells=None)
    assert with_grid.scene.grid is not None and plain.scene.grid is None
    out = []
    for mod in (with_grid, plain):
        q = to_dev(w.q).requires_grad_(True)
        c = mod(q)
        c.sum().backward()
        out.append((c.detach(), q.grad))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
