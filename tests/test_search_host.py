"""Host logic of the VaPr format search (Sec. V-A) against a synthetic
evaluator whose optimum is known by brute force."""
import itertools

import pytest

from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import search as S

TENSORS = ("pos", "dist", "grad", "jgrad")
NEED = {"pos": 16, "dist": 4, "grad": 5, "jgrad": 8}  # per-tensor minimum widths


def synthetic(t: F.FormatTable) -> S.Evaluation:
    """Each tensor alone needs NEED bits (and a mantissa of at least 2 for
    jgrad); in combination the shortfalls add up, error = sum over tensors of
    2^(need - bits) / 3, so the all-minimum table is infeasible (4/3) and
    some tensors must widen, as the paper observes of its combined search."""
    err = 0.0
    for k in TENSORS:
        f = getattr(t, k)
        if f.bits < NEED[k] or (k == "jgrad" and f.M < 2):
            return S.Evaluation(False, 10.0)
        err += 2.0 ** (NEED[k] - f.bits) / 3
    return S.Evaluation(err <= 1.0, err)


def test_per_tensor_binary_search_finds_minimum_widths():
    ev = S.CachedEvaluator(synthetic)
    # phase 1 holds the other tensors at FP32 (their terms are tiny)
    res = S.per_tensor_search(ev, TENSORS)
    assert {k: w for k, (w, _) in res.items()} == NEED
    assert all(f.M >= 2 for f in res["jgrad"][1])
    # binary search: about log2(7) widths per tensor, each all formats of that width
    assert ev.count < 4 * 3 * 6


def test_reduced_space_counts():
    res = {"pos": (16, []), "dist": (4, []), "grad": (5, []), "jgrad": (8, [])}
    space = S.reduced_space(res)
    assert [len(space[k]) for k in TENSORS] == [3, 21, 20, 15]
    assert S.space_size(space) == 3 * 21 * 20 * 15


def test_combinatorial_search_reaches_the_optimum():
    ev = S.CachedEvaluator(synthetic)
    space = S.reduced_space(S.per_tensor_search(ev, TENSORS))
    # brute force optimum over the reduced space
    best_bits = min(F.FormatTable(**dict(zip(TENSORS, c))).total_bits
                    for c in itertools.product(*(space[k] for k in TENSORS))
                    if synthetic(F.FormatTable(**dict(zip(TENSORS, c)))).feasible)
    t, e, hist = S.combinatorial_search(ev, space, samples=500, seed=1)
    assert e.feasible and synthetic(t).feasible
    assert best_bits <= t.total_bits <= best_bits + 2
    assert len(hist) > 0
    # from the per-tensor minima as a starting point it reaches the optimum
    start = F.FormatTable(**{k: space[k][0] for k in TENSORS})
    t2, e2, _ = S.combinatorial_search(S.CachedEvaluator(synthetic), space, samples=500, seed=1,
                                       seeds=[start])
    assert e2.feasible and t2.total_bits == best_bits


def test_combinatorial_search_is_seeded():
    space = S.reduced_space(S.per_tensor_search(S.CachedEvaluator(synthetic), TENSORS))
    a = S.combinatorial_search(S.CachedEvaluator(synthetic), space, samples=120, seed=3)
    b = S.combinatorial_search(S.CachedEvaluator(synthetic), space, samples=120, seed=3)
    assert str(a[0]) == str(b[0]) and [str(x[0]) for x in a[2]] == [str(x[0]) for x in b[2]]


def test_domination_is_constraint_first():
    assert S._dominates((True, 100, 0.9), (False, 10, 0.0))
    assert not S._dominates((False, 10, 0.0), (True, 100, 0.9))
    assert S._dominates((True, 40, 0.5), (True, 44, 0.5))
    assert not S._dominates((True, 40, 0.6), (True, 44, 0.5))
    assert S._dominates((False, 99, 2.0), (False, 10, 3.0))
