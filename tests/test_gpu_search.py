"""The VaPr format search (Sec. V-A) on the GPU path: per-tensor binary
search then the combinatorial search, with an error budget on the step's
outputs (cost and joint gradient) against the FP32 path."""
import json
import os

import pytest

from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import search as S
from paper_2310_07854_gb300 import synth

pytestmark = pytest.mark.gpu
TENSORS = ("pos", "dist", "grad", "jgrad")


def test_search_on_sweep_workload():
    w = synth.make_workload("sweep_1024")
    ev = S.CachedEvaluator(S.PathEvaluator(w.robot, w.scene, w.params, w.q, rel_c=0.05, rel_j=0.05))
    assert ev(F.FP32_TABLE).feasible and ev(F.FP32_TABLE).error == 0.0
    per = S.per_tensor_search(ev, TENSORS)
    n1 = ev.count
    space = S.reduced_space(per)
    assert S.space_size(space) < 21 ** 4
    start = F.FormatTable(**{k: space[k][0] for k in TENSORS})
    best, e, hist = S.combinatorial_search(ev, space, samples=300, seed=0, seeds=[start])
    assert best is not None and e.feasible
    # the chosen table really meets the budget when evaluated afresh
    again = S.PathEvaluator(w.robot, w.scene, w.params, w.q)(best)
    assert again.feasible and again.error == pytest.approx(e.error)
    # narrower than FP32 on the four searched tensors, and no narrower than
    # the per-tensor minima
    bits = {k: getattr(best, k).bits for k in TENSORS}
    assert sum(bits.values()) < 4 * 32
    assert all(bits[k] >= per[k][0] for k in TENSORS)
    report = {"per_tensor": {k: [w_, [f.name for f in fs]] for k, (w_, fs) in per.items()},
              "reduced_space": S.space_size(space), "phase1_evals": n1, "evals": ev.count,
              "best": str(best), "bits": bits, "error": e.error}
    print(json.dumps(report))
    out = os.environ.get("VAPR_REPORT_DIR")
    if out:
        with open(os.path.join(out, "vapr_search_1024.json"), "w") as fh:
            json.dump(report, fh)
