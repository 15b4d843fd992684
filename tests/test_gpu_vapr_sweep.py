"""The per-tensor format sweep on the 32 x 32-configuration, 20-cuboid
workload: every combination of {FP32, BF16, FP16, E4M3, E5M2, E3M2, E2M1}
for P, D, G and J (7^4 = 2401 tables) runs through the whole path on the
GPU, and each table reports its max error per tensor against one FP64
oracle evaluation (Sec. V-A's search measures the effect of each tensor's
format; success rates are not available here, so error is the measure).

Checks, besides producing the report:
* the FP32 table matches FP64 to 1e-5 (normwise) on every tensor;
* each tensor's error depends only on the formats upstream of it
  (P on P; D on P, D; G on P, G; J on P, G, J), which is the data flow of
  the staged path;
* a tensor's own rounding error is bounded by half a unit in the last place
  of its format at the tensor's largest magnitude, plus the propagated error,
  plus how far the tensor exceeds the format's largest value (saturation).
Set VAPR_REPORT_DIR to write the report as JSON.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth
from parity import KINK_EPS, to_dev

pytestmark = pytest.mark.gpu

TENSORS = ("pos", "dist", "grad", "jgrad")


def _half_ulp(f, mag):
    """Largest rounding error of format f on values up to magnitude mag:
    half a spacing at mag, or the distance past the largest finite value."""
    if f == F.FP32:
        return float(np.spacing(np.float32(mag))) / 2
    top = oracle.max_finite(f.E, f.M, f.flags)
    e = np.floor(np.log2(max(min(mag, top), 1e-30)))
    half = 2.0 ** (e - f.M) / 2
    return max(half, mag - top)


def test_vapr_sweep_1024():
    import torch
    w = synth.make_workload("sweep_1024")
    n, S, J = w.n, w.robot.n_spheres, w.robot.n_joints
    pos64 = oracle.fk(w.robot, w.q)
    col = oracle.collision(w.robot, w.scene, w.params, pos64, kink_eps=KINK_EPS)
    jg64 = oracle.backward(w.robot, w.q, col["grad"])
    ok_cfg = ~col["kink"].any(1)
    ref = {
        "pos": torch.as_tensor(pos64.reshape(n, -1), device="cuda"),
        "dist": torch.as_tensor(col["dist"], device="cuda"),
        "grad": torch.as_tensor(col["grad"].reshape(n, -1), device="cuda"),
        "jgrad": torch.as_tensor(jg64, device="cuda"),
        "cost": torch.as_tensor(col["cost"], device="cuda"),
    }
    # G and J are compared away from gradient discontinuities (float32 vs
    # float64 may fall on either side of one)
    gmask = torch.as_tensor(np.repeat(~col["kink"], 3, 1), device="cuda")
    jmask = torch.as_tensor(np.repeat(ok_cfg[:, None], J, 1), device="cuda")
    scale = {k: float(v.abs().max()) for k, v in ref.items()}

    rd, sd = B.DeviceRobot(w.robot), B.DeviceScene(w.scene)
    q = to_dev(w.q)
    lens = {"pos": 3 * S, "dist": S, "grad": 3 * S, "jgrad": J}
    report = {}
    for combo in itertools.product(F.SWEEP, repeat=4):
        t = F.FormatTable(**dict(zip(TENSORS, combo)))
        bufs = {k: B.alloc_packed(n, lens[k], getattr(t, k)) for k in TENSORS}
        cost = torch.empty(n, device="cuda")
        B.vapr_fk(rd, q, n, t, bufs["pos"])
        B.vapr_collision_cost(rd, sd, w.params, bufs["pos"], n, t, cost, bufs["dist"], bufs["grad"])
        B.vapr_backward(rd, q, None, bufs["grad"], None, n, t, bufs["jgrad"])
        errs = {}
        for k in TENSORS:
            out = torch.empty((n, lens[k]), device="cuda")
            B.vapr_unpack(bufs[k], n, lens[k], getattr(t, k), out)
            d = (out.double() - ref[k]).abs()
            if k == "grad":
                d = d * gmask
            if k == "jgrad":
                d = d * jmask
            errs[k] = float(d.max())
        errs["cost"] = float((cost.double() - ref["cost"]).abs().max())
        report["|".join(f.name for f in combo)] = errs

    def err(p, d, g, j, k):
        return report[f"{p.name}|{d.name}|{g.name}|{j.name}"][k]

    fp32 = F.FP32
    for k in ("pos", "dist", "grad", "jgrad", "cost"):
        assert err(fp32, fp32, fp32, fp32, k) <= 1e-5 * scale[k], k
    for p, d, g, j in itertools.product(F.SWEEP, repeat=4):
        # data flow: an output's error ignores formats downstream of it
        assert err(p, d, g, j, "pos") == err(p, fp32, fp32, fp32, "pos")
        assert err(p, d, g, j, "dist") == err(p, d, fp32, fp32, "dist")
        assert err(p, d, g, j, "grad") == err(p, fp32, g, fp32, "grad")
        assert err(p, d, g, j, "jgrad") == err(p, fp32, g, j, "jgrad")
        assert err(p, d, g, j, "cost") == err(p, fp32, fp32, fp32, "cost")
    for f in F.SWEEP:
        # P's error is its own rounding (the tensor is bounded by ~1.6 m)
        bound = _half_ulp(f, scale["pos"]) + 1e-5 * scale["pos"]
        assert err(f, fp32, fp32, fp32, "pos") <= bound, f
        # with exact P and G, J's error is the rounding of J itself
        assert err(fp32, fp32, fp32, f, "jgrad") <= _half_ulp(f, scale["jgrad"]) + 1e-5 * scale["jgrad"]
    out_dir = os.environ.get("VAPR_REPORT_DIR")
    if out_dir:
        with open(os.path.join(out_dir, "vapr_sweep_1024.json"), "w") as fh:
            json.dump({"workload": "sweep_1024", "n": n, "scale": scale, "errors": report}, fh)
