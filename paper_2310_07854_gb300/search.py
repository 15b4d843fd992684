"""VaPr format search (Sec. V-A) on the cost-and-gradient path.

Two phases, as the paper describes them:
  1. per-tensor search: for each large tensor, with every other tensor in
     FP32, the narrowest bit width at which some candidate format meets the
     accuracy constraint, found by binary search over the widths of the
     21-format set; every narrower format is then dropped for that tensor;
  2. combinatorial search across tensors over what is left: an NSGA-II
     style evolutionary search (non-dominated sorting and crowding distance,
     constraint-first ranking) minimising the total bit width of the tensors
     while the constraint holds.

The paper's constraint is the planner's success rate on its benchmark
tasks, which this library has no planner or dataset for; here the
constraint is an error budget of the path's outputs against the FP32 path
on a validation batch (the evaluator decides; ``PathEvaluator`` measures the
cost C and the joint gradient J on the GPU).  Both phases are host logic;
every evaluation runs the CUDA path.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Sequence

import numpy as np

from . import formats as F

WIDTHS = (4, 5, 6, 8, 10, 16, 32)


@dataclasses.dataclass
class Evaluation:
    feasible: bool
    error: float  # the evaluator's normalised error (<= 1 means within budget)


Evaluator = Callable[[F.FormatTable], Evaluation]


class CachedEvaluator:
    """Memoises an evaluator on the table and counts distinct evaluations."""

    def __init__(self, fn: Evaluator):
        self.fn = fn
        self.cache: dict[str, Evaluation] = {}

    def __call__(self, t: F.FormatTable) -> Evaluation:
        k = str(t)
        if k not in self.cache:
            self.cache[k] = self.fn(t)
        return self.cache[k]

    @property
    def count(self) -> int:
        return len(self.cache)


def _by_width(cands: Sequence[F.Fmt]) -> dict[int, list[F.Fmt]]:
    out: dict[int, list[F.Fmt]] = {}
    for f in cands:
        out.setdefault(f.bits, []).append(f)
    return out


def per_tensor_search(evaluate: Evaluator, tensors: Sequence[str], base: F.FormatTable = F.FP32_TABLE,
                      candidates: Sequence[F.Fmt] | None = None):
    """Phase 1.  For each tensor: binary search over the bit widths for the
    narrowest width at which at least one format of that width (others held
    at ``base``) is feasible, assuming wider widths stay feasible.  Returns
    {tensor: (min_width, feasible formats of that width)}."""
    cands = list(candidates or F.search_set())
    groups = _by_width(cands)
    widths = sorted(groups)
    out = {}
    for t in tensors:
        def ok_at(w):
            good = [f for f in groups[w] if evaluate(dataclasses.replace(base, **{t: f})).feasible]
            return good
        lo, hi = 0, len(widths) - 1  # widths[hi] (FP32) is feasible by definition
        best = (widths[hi], groups[widths[hi]])
        while lo <= hi:
            mid = (lo + hi) // 2
            good = ok_at(widths[mid])
            if good:
                best = (widths[mid], good)
                hi = mid - 1
            else:
                lo = mid + 1
        out[t] = best
    return out


def reduced_space(per_tensor: dict, candidates: Sequence[F.Fmt] | None = None) -> dict[str, list[F.Fmt]]:
    """Formats left for each tensor: those at least as wide as its phase-1 width."""
    cands = list(candidates or F.search_set())
    return {t: [f for f in cands if f.bits >= w] for t, (w, _) in per_tensor.items()}


def space_size(space: dict[str, list]) -> int:
    n = 1
    for v in space.values():
        n *= len(v)
    return n


# ---------------------------------------------------------------- NSGA-II
def _dominates(a, b) -> bool:
    """Constraint-first domination on (feasible, bits, error)."""
    if a[0] != b[0]:
        return a[0]
    if not a[0]:  # both infeasible: smaller violation wins
        return a[2] < b[2]
    return (a[1] <= b[1] and a[2] <= b[2]) and (a[1] < b[1] or a[2] < b[2])


def _fronts(objs):
    n = len(objs)
    dom_by = [[] for _ in range(n)]
    count = [0] * n
    for i in range(n):
        for j in range(n):
            if i != j and _dominates(objs[i], objs[j]):
                dom_by[i].append(j)
            elif i != j and _dominates(objs[j], objs[i]):
                count[i] += 1
    fronts, cur = [], [i for i in range(n) if count[i] == 0]
    while cur:
        fronts.append(cur)
        nxt = []
        for i in cur:
            for j in dom_by[i]:
                count[j] -= 1
                if count[j] == 0:
                    nxt.append(j)
        cur = nxt
    return fronts


def _crowding(objs, front):
    d = {i: 0.0 for i in front}
    for k in (1, 2):
        srt = sorted(front, key=lambda i: objs[i][k])
        lo, hi = objs[srt[0]][k], objs[srt[-1]][k]
        d[srt[0]] = d[srt[-1]] = float("inf")
        if hi > lo:
            for a, b, c in zip(srt, srt[1:], srt[2:]):
                d[b] += (objs[c][k] - objs[a][k]) / (hi - lo)
    return d


def combinatorial_search(evaluate: Evaluator, space: dict[str, list[F.Fmt]], base: F.FormatTable = F.FP32_TABLE,
                         samples: int = 500, population: int = 20, seed: int = 0,
                         seeds: Sequence[F.FormatTable] = ()):
    """Phase 2: NSGA-II over the reduced space (uniform crossover, per-tensor
    mutation to a neighbouring candidate).  Objectives: total bit width and
    normalised error, infeasible tables ranked after feasible ones.  Stops
    after ``samples`` distinct evaluations.  Returns (best feasible table or
    None, its evaluation, history [(table, evaluation)])."""
    rng = np.random.default_rng(seed)
    tensors = list(space)
    cached = evaluate if isinstance(evaluate, CachedEvaluator) else CachedEvaluator(evaluate)
    start = cached.count

    def table(genes):
        return dataclasses.replace(base, **{t: space[t][g] for t, g in zip(tensors, genes)})

    def obj(genes):
        t = table(genes)
        e = cached(t)
        return (e.feasible, t.total_bits, e.error)

    pop = [tuple(space[t].index(getattr(s, t)) for t in tensors) for s in seeds
           if all(getattr(s, t) in space[t] for t in tensors)]
    while len(pop) < population:
        pop.append(tuple(int(rng.integers(len(space[t]))) for t in tensors))
    history = []
    budget_left = lambda: cached.count - start < samples

    def ranking(genes_list):
        objs = [obj(g) for g in genes_list]
        rank, crowd = {}, {}
        for r, front in enumerate(_fronts(objs)):
            cd = _crowding(objs, front)
            for i in front:
                rank[i], crowd[i] = r, cd[i]
        return rank, crowd

    def tournament(rank, crowd):
        i, j = (int(x) for x in rng.integers(len(pop), size=2))
        return pop[i] if (rank[i], -crowd[i]) <= (rank[j], -crowd[j]) else pop[j]

    while budget_left():
        rank, crowd = ranking(pop)
        children = []
        tries = 0
        while len(children) < population and tries < 50 * population:
            tries += 1
            a, b = tournament(rank, crowd), tournament(rank, crowd)
            child = [a[k] if rng.random() < 0.5 else b[k] for k in range(len(tensors))]
            for k in range(len(tensors)):
                if rng.random() < 1.0 / len(tensors):
                    child[k] = int(np.clip(child[k] + rng.choice((-1, 1)), 0, len(space[tensors[k]]) - 1))
            child = tuple(child)
            if child not in pop and child not in children:
                children.append(child)
        if not children:
            break
        union = pop + children
        uobjs = [obj(g) for g in union]
        for g in children:
            history.append((table(g), cached(table(g))))
        nxt = []
        for front in _fronts(uobjs):
            if len(nxt) + len(front) <= population:
                nxt.extend(front)
            else:
                cd = _crowding(uobjs, front)
                nxt.extend(sorted(front, key=lambda i: -cd[i])[:population - len(nxt)])
                break
        pop = [union[i] for i in nxt]
        if not budget_left():
            break
    best = None
    for k, e in cached.cache.items():
        if not e.feasible:
            continue
        t = F.FormatTable.parse(k)
        if any(getattr(t, x) not in space[x] for x in tensors):
            continue
        if best is None or (t.total_bits, e.error) < (best[0].total_bits, best[1].error):
            best = (t, e)
    return (best[0] if best else None), (best[1] if best else None), history


# ------------------------------------------------------------ GPU evaluator
class PathEvaluator:
    """Runs the whole step (vapr_cost_grad) with a candidate table on a
    validation batch and compares C and J with the FP32 path:
    error = max(max|C - C32| / (rel_c max|C32|), max|J - J32| / (rel_j max|J32|));
    feasible when error <= 1 and every output is finite."""

    def __init__(self, robot, scene, params, q, rel_c: float = 0.05, rel_j: float = 0.05,
                 tensors=("pos", "dist", "grad", "jgrad")):
        import torch
        from . import binding as B
        self.torch, self.B = torch, B
        self.q = torch.as_tensor(q, device="cuda")
        self.n = self.q.shape[0]
        self.robot = robot if isinstance(robot, B.DeviceRobot) else B.DeviceRobot(robot)
        self.scene = scene if isinstance(scene, B.DeviceScene) else B.DeviceScene(scene)
        self.params = params
        self.rel_c, self.rel_j = rel_c, rel_j
        self.tensors = tensors
        ref = self._run(F.FP32_TABLE)
        self.c32, self.j32 = ref
        self.cscale = float(self.c32.abs().max()) or 1.0
        self.jscale = float(self.j32.abs().max()) or 1.0

    def _run(self, t: F.FormatTable):
        from .path import Evaluator as PathEv
        ev = PathEv(self.robot, self.scene, self.params, self.n, t)
        ev.cost_grad(self.q, self.n)
        j = ev.unpack_jgrad(self.n).clone()
        c = ev.cost[:self.n].clone()
        return c, j

    def __call__(self, t: F.FormatTable) -> Evaluation:
        c, j = self._run(t)
        ec = float((c - self.c32).abs().max()) / (self.rel_c * self.cscale)
        ej = float((j - self.j32).abs().max()) / (self.rel_j * self.jscale)
        finite = bool(self.torch.isfinite(c).all() and self.torch.isfinite(j).all())
        err = max(ec, ej) if finite else float("inf")
        return Evaluation(finite and err <= 1.0, err)
