#!/usr/bin/env python
"""Throughput of the VaPr cost-and-gradient step on GB300.

One step = FK -> collision cost (environment + self) -> backward to joint
gradients over one batch of joint configurations, i.e. iteration steps 2,
3-4 and 5 of Sec. III-B, through the C ABI of libvapr.so.

Default workload: 1024 trajectories x 32 timesteps = 32768 configurations
of the seeded 7-joint, 52-sphere arm against 40 oriented cuboids (1.7 M
sphere evaluations per step).  Inputs are synthetic (the paper's Franka
model and MotionBenchMaker scenes are not available) and resident in HBM;
an L2-sized buffer is rewritten before every timed step, outside the timed
events.  Prints one JSON line (rank 0).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2310_07854_gb300 import formats as F  # noqa: E402
from paper_2310_07854_gb300 import replicas  # noqa: E402
from paper_2310_07854_gb300 import synth  # noqa: E402

WORKLOAD = "particle_32768"
# example reduced table for the single-stage profiling mode (--kernel)
EXAMPLE_TABLE = "P=E5M10,D=E2M1,G=E2M1,J=E4M3"
METRIC = "configs/s for FK+collision cost+grad, % of HBM roofline; VaPr vs FP32 at stated err"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="vapr", choices=["vapr", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=list(synth.WORKLOADS))
    ap.add_argument("--table", default="searched",
                    help="format table of the VaPr leg: 'searched' (the table the VaPr search finds within "
                         "its error budget) or a table string; with --kernel, 'searched' means " + EXAMPLE_TABLE)
    ap.add_argument("--grid-cells", type=int, default=-1,
                    help="cells per axis of the scene's broad-phase grid (0: none, -1: the evaluator's choice)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dram-scale", action="store_true", help="skip the DRAM-scale sweep")
    ap.add_argument("--no-config-baselines", action="store_true",
                    help="skip timing configs 1-3 beside the oracle (1 thread and all threads)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-surrogate", action="store_true",
                    help="skip the learned-surrogate leg (training + gated collision)")
    ap.add_argument("--surrogate-epochs", type=int, default=80)
    ap.add_argument("--kernel", choices=["fk", "collision", "backward", "mlp_infer", "step", "fused", "ceiling"],
                    default=None,
                    help="profiling mode: run only this stage (--warmup launches, then --steps timed) on "
                         "--configs configurations of the workload and print its CUDA-event time")
    ap.add_argument("--search-samples", type=int, default=300)
    ap.add_argument("--ceiling-reps", type=int, default=16,
                    help="repetitions per launch of the pair-test ceiling measurement")
    ap.add_argument("--configs", type=int, default=0,
                    help="override the batch size (configurations per GPU)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------ cpu baseline
def cpu_baseline(workload_name: str, seconds: float) -> dict:
    """The FP64 oracle, as it stands, on the host cores: whole batches of the
    same workload until at least ``seconds`` of CPU time have passed."""
    import oracle
    w = synth.make_workload(workload_name)
    oracle.build()
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.cost_and_grad(w.robot, w.scene, w.params, w.q)
        done += w.n
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": done / el, "unit": "configs/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{done // w.n} full batches of {w.n} configurations of {workload_name} "
                      f"(FP64 FK + collision + backward, OpenMP over configurations), "
                      f"{el:.1f} s"}


def workload_config(w, world: int) -> dict:
    """The `config` object of both arms' JSON lines."""
    return {"workload": w.name if hasattr(w, "name") else None, "global_batch": world * w.n,
            "trajectories": w.n_traj, "horizon": w.horizon, "spheres": w.robot.n_spheres,
            "cuboids": w.scene.n_cuboids, "self_pairs": w.robot.n_pairs, "table": str(F.FP32_TABLE),
            "parallelism": f"replicas{world}",
            "l2": "flushed before every step (2 x L2 buffer rewritten outside the timed events)"}


def run_reference(args):
    """The oracle as the reference arm: --warmup untimed batches, then
    --steps timed batches of the workload on the host cores (rank 0 only)."""
    world, rank, _ = replicas.dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = synth.make_workload(args.workload)
    w.name = args.workload
    for _ in range(args.warmup):
        oracle.cost_and_grad(w.robot, w.scene, w.params, w.q)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.cost_and_grad(w.robot, w.scene, w.params, w.q)
    el = time.perf_counter() - t0
    value = args.steps * w.n / el
    cfg = workload_config(w, 1)
    cfg["l2"] = "n/a (host CPU)"
    cb = {"value": value, "unit": "configs/s", "cores": oracle.num_threads(), "kind": "oracle",
          "sample": f"{args.steps} timed batches of {w.n} configurations of {args.workload} after "
                    f"{args.warmup} untimed (FP64 FK + collision + backward, OpenMP over configurations), "
                    f"{el:.1f} s"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "configs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * el / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "configs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ timing
def time_steps(ev, q, n, steps, warmup, flush_buf, torch):
    """Device times (ms) of each step and of each kernel in it.

    A step is one replay of a CUDA graph holding one vapr_cost_grad call
    (FK, collision, backward; the last two start while the stage before them
    finishes).  The per-kernel split comes from a second graph of the three
    stage calls with external events captured between them (which keeps the
    kernels from overlapping; its step time is kept as step_three_calls).
    CUDA events on the launching stream bracket each replay; the L2 flush
    runs before it, outside the events (none when flush_buf is None: inputs
    larger than L2)."""
    st = torch.cuda.current_stream()
    flush_buf = flush_buf if flush_buf is not None else torch.zeros(1, device="cuda")
    g, inner = ev.capture(q, n, timing_events=True)
    per = {"fk": [], "collision": [], "backward": [], "step": [], "step_three_calls": []}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for i in range(warmup + steps):
        flush_buf.add_(1)
        e0.record(st)
        g.replay()
        e1.record(st)
        st.synchronize()
        if i < warmup:
            continue
        per["step_three_calls"].append(e0.elapsed_time(e1))
        if inner:
            per["fk"].append(inner[0].elapsed_time(inner[1]))
            per["collision"].append(inner[1].elapsed_time(inner[2]))
            per["backward"].append(inner[2].elapsed_time(inner[3]))
    if not inner:  # per-kernel times from single-kernel graphs
        for name, fn in (("fk", lambda: ev.fk(q, n)), ("collision", lambda: ev.collision(n)),
                         ("backward", lambda: ev.backward(q, n))):
            gk = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gk):
                fn()
            for i in range(warmup + steps):
                flush_buf.add_(1)
                e0.record(st)
                gk.replay()
                e1.record(st)
                st.synchronize()
                if i >= warmup:
                    per[name].append(e0.elapsed_time(e1))
    ev.cost_grad(q, n)  # the whole step as one call
    torch.cuda.synchronize()
    gs = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gs):
        ev.cost_grad(q, n)
    for i in range(warmup + steps):
        flush_buf.add_(1)
        e0.record(st)
        gs.replay()
        e1.record(st)
        st.synchronize()
        if i >= warmup:
            per["step"].append(e0.elapsed_time(e1))
    return per


KERNEL_SOURCES = {
    "fk": ("fk.cu", "stages.cuh", "tcgen05.cuh", "exmy.cuh", "common.cuh"),
    "collision": ("collision.cu", "stages.cuh", "grid.cuh", "exmy.cuh", "common.cuh"),
    "backward": ("backward.cu", "stages.cuh", "exmy.cuh", "common.cuh"),
}


def kernel_source_sha(stage: str) -> str:
    """Hash of every source file the stage's kernel is compiled from, with
    comments and blank lines left out (a comment edit is not a kernel change)."""
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[stage]:
        text = open(os.path.join(ROOT, "paper_2310_07854_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("\n".join(l.rstrip() for l in text.splitlines() if l.strip()).encode())
    return h.hexdigest()[:16]


def kernel_traffic(stage: str, table: str, n: int):
    """DRAM bytes per configuration of one launch on n configurations, from
    a committed ncu capture of the current kernel source at that size (else
    None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return None
    h = kernel_source_sha(stage)
    ent = data.get(f"{stage}:{table}:{n}")
    if not ent or ent.get("source_sha") != h:
        return None
    return ent.get("dram_bytes_per_config")


def collision_flops_per_config(w) -> int:
    """Algorithmic FP32 work of the collision stage per configuration: the
    bounding test of every sphere/cuboid pair (|c - t|^2 < (r + R)^2: 3 sub,
    1 mul, 2 fma, 1 add, 1 mul = 10 FLOP) and of every self pair (3 sub,
    1 mul, 2 fma, 1 mul = 9 FLOP).  Exact distances of the pairs that pass
    come on top; they are data-dependent and not counted."""
    return 10 * w.robot.n_spheres * w.scene.n_cuboids + 9 * w.robot.n_pairs


def broad_phase_leg(w, ev32, q, n, args, flush, torch):
    """What the two broad phases buy: the same step with the plain loop over
    every cuboid (no grid), and the grid's build time.  (The self-pair
    clusters are part of the kernel and always on.)"""
    from paper_2310_07854_gb300.path import Evaluator
    import numpy as np
    if ev32.scene.grid is None:
        return {"grid_cells_per_axis": None}
    ev = Evaluator(ev32.robot, w.scene, w.params, n, F.FP32_TABLE, grid_cells=None)
    per = time_steps(ev, q, n, args.steps, args.warmup, flush, torch)
    reach = float(np.max(w.robot.sphere_local[:, 3]))
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(5):
        g0.record()
        ev.scene.build_grid(reach, w.params.eta, ev32.scene.grid_cells)
        g1.record()
        torch.cuda.synchronize()
        ts.append(g0.elapsed_time(g1))
    return {"grid_cells_per_axis": ev32.scene.grid_cells, "grid_bytes": int(ev32.scene.grid.numel()),
            "grid_build_ms": statistics.median(ts),
            "without_grid": {"configs_per_s": n * args.steps / (sum(per["step"]) / 1000.0),
                             "collision_ms": statistics.mean(per["collision"])}}


def sparsity(dist, grad, S: int) -> dict:
    """Fraction of nonzero per-sphere penetrations D and of spheres with a
    nonzero gradient G (the zero words the backward pass skips); dist
    [n, S] and grad [n, 3S] decoded float tensors."""
    n = dist.shape[0]
    g = grad[:, :3 * S].reshape(n, S, 3)
    return {"dist_nonzero": float((dist[:, :S] != 0).float().mean()),
            "grad_spheres_nonzero": float((g != 0).any(-1).float().mean())}


def speedup_pct(t_fp32: float, t_x: float) -> float:
    """Speedup in the paper's form (Appendix, Detailed Experimental
    Results): (T_FP32 / T_x - 1) x 100 %; negative when x is slower."""
    return (t_fp32 / t_x - 1.0) * 100.0


def fp32_peak_tflops(peaks) -> float:
    """152 SMs x 128 FP32 lanes x 2 FLOP (FMA) x max SM clock."""
    return 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def ceiling_leg(w, ev32, q, n, flush, torch, peak_alu, reps=16, rounds=5):
    """Measured compute ceiling of the collision stage's pair test
    (vapr_env_ceiling): the stage's own environment loop in registers on the
    workload's FP32 sphere centres moved 100 m away, so that every
    sphere/cuboid pair runs its bounding test (10 FLOP) and none passes;
    64 spheres x every resident warp x 4, `reps` repetitions per launch, L2
    flushed before each timed launch.  Also times the same loop on the real
    centres (bounding tests plus the exact distances that pass, no broad
    phase, no memory): the in-register cost of the plain environment term
    per configuration.  About 5 ms of GPU time in all, so that this
    measurement stays a small share of a bench run's launches."""
    from paper_2310_07854_gb300 import binding as B
    S, O = w.robot.n_spheres, w.scene.n_cuboids
    ev32.fk(q, n)
    cen = ev32.pos.view(torch.float32)[:n, :3 * S].reshape(n * S, 3)
    rad = torch.as_tensor(np.asarray(w.robot.sphere_local, np.float32)[:, 3], device="cuda").repeat(n)
    sph = torch.cat([cen, rad[:, None]], dim=1)
    W = B.vapr_env_ceiling_warps(O)
    if W <= 0:
        raise RuntimeError("vapr_env_ceiling_warps: no resident warps")
    nc = 64 * W * 4
    tiled = sph[torch.arange(nc, device="cuda") % sph.shape[0]].contiguous()
    far = tiled.clone()
    far[:, 0] += 100.0
    out = torch.empty_like(tiled)

    def timed(spheres, r):
        for _ in range(3):
            B.vapr_env_ceiling(ev32.scene, spheres, nc, w.params.eta, w.params.w_coll, r, out)
        ts = []
        for _ in range(rounds):
            flush.add_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            B.vapr_env_ceiling(ev32.scene, spheres, nc, w.params.eta, w.params.w_coll, r, out)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.mean(ts)

    ms = timed(far, reps)
    if int(torch.count_nonzero(out)) != 0:
        raise RuntimeError("vapr_env_ceiling: spheres 100 m away reported contact")
    tests_per_s = nc * O * reps / (ms / 1000.0)
    tflops = 10 * tests_per_s / 1e12
    r_w = max(1, reps // 8)
    ms_w = timed(tiled, r_w)
    return {"tflops": tflops, "bounding_tests_per_s": tests_per_s,
            "frac_of_derived_peak": tflops / peak_alu, "ms_per_launch": ms,
            "spheres": nc, "cuboids": O, "reps": reps, "resident_warps": W,
            "loop": "vapr_env_ceiling: the collision stage's environment loop (bounding test, exact box "
                    "term where it passes, 2 spheres per lane, cuboids in shared memory) on centres "
                    "held in registers; all spheres 100 m from the scene, so every pair runs the "
                    "10-FLOP bounding test and none passes",
            "plain_env_term_in_registers": {
                "ns_per_config": ms_w * 1e6 / (nc * r_w) * S,
                "note": "the same loop on the workload's real centres: bounding tests plus the exact "
                        "distances that pass, no scene grid, no packed rows"}}


def search_tables(w, ev32, args):
    """VaPr search (Sec. V-A) for the workload: per-tensor binary search and
    the combinatorial search on a 1024-configuration validation batch with a
    5 % budget on C and J against the FP32 path; then the same search over
    the formats with a one-instruction converter.  Returns (table, report,
    hardware-only table)."""
    from paper_2310_07854_gb300 import search as S
    tensors = ("pos", "dist", "grad", "jgrad")
    t0 = time.perf_counter()
    ev = S.CachedEvaluator(S.PathEvaluator(ev32.robot, ev32.scene, w.params, synth.make_q(901, 1024)))
    per = S.per_tensor_search(ev, tensors)
    space = S.reduced_space(per)
    start = F.FormatTable(**{k: space[k][0] for k in tensors})
    best, e, _ = S.combinatorial_search(ev, space, samples=args.search_samples, seed=0, seeds=[start])
    hw = F.hardware_formats()
    per_hw = S.per_tensor_search(ev, tensors, candidates=hw)
    space_hw = S.reduced_space(per_hw, hw)
    start_hw = F.FormatTable(**{k: space_hw[k][0] for k in tensors})
    best_hw, e_hw, _ = S.combinatorial_search(ev, space_hw, samples=args.search_samples, seed=0, seeds=[start_hw])
    report = {"budget": "max|C-C32| <= 5% max|C32| and max|J-J32| <= 5% max|J32| (1024 validation configs)",
              "per_tensor_min_bits": {k: v[0] for k, v in per.items()}, "reduced_space": S.space_size(space),
              "evaluations": ev.count, "search_s": time.perf_counter() - t0,
              "table": str(best) if best is not None else None,
              "bits_searched_tensors": sum(getattr(best, k).bits for k in tensors) if best is not None else None,
              "validation_error": e.error if best is not None else None,
              "hardware_formats_only": {"reduced_space": S.space_size(space_hw),
                                        "table": str(best_hw) if best_hw is not None else None,
                                        "validation_error": e_hw.error if best_hw is not None else None}}
    return best, report, best_hw


def dram_sweep(w, robot_dev, tables, flush, torch, peaks, exps=range(15, 21), counts=(8, 40)):
    """Per-stage time and HBM fraction from 2^15 to 2^20 configurations, with
    the 8-cuboid scene of the single-problem workload and the 40-cuboid
    scene of the benchmark, for each format table (median of 3 steps after 2
    untimed).  L2 is flushed before every step while a step's tensors fit in
    twice the L2 size; beyond that the inputs themselves are larger than L2
    and no flush runs (a flush by writing leaves the L2 full of dirty lines,
    whose write-back the next kernel would pay)."""
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    from paper_2310_07854_gb300.path import Evaluator
    nmax = 1 << max(exps)
    qmax = torch.as_tensor(synth.make_q(77, nmax), device="cuda")
    scenes = {w.scene.n_cuboids: w.scene, 8: synth.make_workload("single_128").scene}
    out = []
    for O in counts:
        scene = scenes.get(O) or synth.make_scene(1 + O, O)
        for tname, table in tables.items():
            ev = Evaluator(robot_dev, scene, w.params, nmax, table)
            bp = ev.bytes_per_config()
            for e in exps:
                n = 1 << e
                big = sum(bp[k] for k in ("fk", "collision", "backward")) * n > 2 * l2
                per = time_steps(ev, qmax, n, 3, 2, None if big else flush, torch)
                if big:  # each stage alone, 5 back-to-back launches per graph (no launch gaps)
                    for k, fn in (("fk", lambda: ev.fk(qmax, n)), ("collision", lambda: ev.collision(n)),
                                  ("backward", lambda: ev.backward(qmax, n))):
                        per[k] = time_reps(fn, 5, 3, torch)
                row = {"cuboids": O, "table": tname, "n_configs": n,
                       "configs_per_s": n / (statistics.median(per["step"]) / 1000.0),
                       "l2": ("inputs larger than L2: no flush; stage times from graphs of 5 back-to-back "
                              "launches of the stage" if big else "flushed before every step; stage times from "
                              "events between the stages of one step")}
                for k in ("fk", "collision", "backward"):
                    ms = statistics.median(per[k])
                    row[k] = {"ms": ms, "hbm_frac": bp[k] * n / (ms / 1000.0) / 1e9 / peaks["hbm_gbs"]}
                out.append(row)
            del ev
    del qmax
    return out


def config_baselines(args, flush, torch):
    """Configs 1-3 (single_128, sweep_1024, particle_32768): the FP32 step on
    the GPU (median of >= 20 steps, L2 flushed before each) beside the FP64
    oracle as it stands on one host thread and on all host threads (median
    of 5 runs each)."""
    import oracle
    from paper_2310_07854_gb300.path import Evaluator
    oracle.build()
    threads = oracle.num_threads()
    out = {}
    try:
        for name in ("single_128", "sweep_1024", "particle_32768"):
            w = synth.make_workload(name)
            q = torch.as_tensor(w.q, device="cuda")
            ev = Evaluator(w.robot, w.scene, w.params, w.n, F.FP32_TABLE)
            per = time_steps(ev, q, w.n, max(args.steps, 20), max(args.warmup, 3), flush, torch)
            ms = statistics.median(per["step"])
            res = {"configs": w.n, "cuboids": w.scene.n_cuboids,
                   "gpu_fp32": {"ms_median": ms, "configs_per_s": w.n / (ms / 1000.0)}}
            for label, th in (("oracle_1_thread", 1), ("oracle_all_threads", threads)):
                oracle.set_num_threads(th)
                ts = []
                for _ in range(5):
                    t0 = time.perf_counter()
                    oracle.cost_and_grad(w.robot, w.scene, w.params, w.q)
                    ts.append(time.perf_counter() - t0)
                res[label] = {"threads": th, "s_median_of_5": statistics.median(ts),
                              "configs_per_s": w.n / statistics.median(ts)}
            res["gpu_over_oracle_all_threads"] = (res["gpu_fp32"]["configs_per_s"]
                                                  / res["oracle_all_threads"]["configs_per_s"])
            out[name] = res
            del ev
    finally:
        oracle.set_num_threads(threads)
    out["host"] = {"threads": threads, "cpu": host_cpu_name()}
    return out


def host_cpu_name() -> str:
    """The host CPU's model name as /proc/cpuinfo gives it (x86: model name;
    Arm: implementer and part), else the machine type."""
    import platform
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return platform.machine()
    for key in ("model name", "Model"):
        for line in info:
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    parts = {l.split(":")[0].strip(): l.split(":", 1)[1].strip() for l in info if ":" in l}
    if "CPU part" in parts:
        return f"{platform.machine()} implementer {parts.get('CPU implementer')} part {parts['CPU part']}"
    return platform.machine()


def swept_leg(w, ev32, n, vtable, args, flush, torch, samples=4):
    """Swept-sphere environment cost (closest_pt_swept) on the workload's
    trajectories (K points per row), FP32 and the VaPr table's D/G formats."""
    from paper_2310_07854_gb300 import binding as B
    S = w.robot.n_spheres
    out = {"samples": samples, "horizon": w.horizon}
    for name, table in (("fp32", F.FP32_TABLE), ("vapr", vtable)):
        t = F.FormatTable(pos=F.FP32, dist=table.dist, grad=table.grad)
        cost = torch.empty(n, device="cuda")
        dist = B.alloc_packed(n, S, t.dist)
        grad = B.alloc_packed(n, 3 * S, t.grad)
        fn = lambda: B.vapr_swept_cost(ev32.robot, ev32.scene, w.params, ev32.pos, n, w.horizon, samples,
                                       t, cost, dist, grad)
        ms = time_graph(fn, args.steps, args.warmup, flush, torch)
        out[name] = {"table": str(t), "ms": ms, "configs_per_s": n / (ms / 1000.0)}
    return out


def ik_pose_only(w, ev32, torch, n_seeds=4096, iters=100):
    """The same solver with the collision weights at zero: how well the
    pose and bound terms alone are met (the L-BFGS solver's own accuracy)."""
    import dataclasses
    from paper_2310_07854_gb300 import binding as B
    from paper_2310_07854_gb300 import ik as IK
    J = w.robot.n_joints
    params = dataclasses.replace(w.params, w_coll=0.0, w_self=0.0)
    goal_q = torch.as_tensor(synth.make_q(4242, n_seeds) * 0.8, device="cuda")
    xf = B.alloc_packed(n_seeds, 12 * J, F.FP32)
    pos = B.alloc_packed(n_seeds, 3 * w.robot.n_spheres, F.FP32)
    B.vapr_fk(ev32.robot, goal_q, n_seeds, F.FP32_TABLE, pos, xf)
    goal = xf.view(torch.float32)[:, 12 * (J - 1):12 * J].contiguous()
    q = torch.as_tensor(synth.make_q(4343, n_seeds) * 0.8, device="cuda")
    s = IK.IkSolver(ev32.robot, ev32.scene, params, n_seeds)
    s.init(goal, q)
    s.solve(iters)
    B.vapr_fk(ev32.robot, q, n_seeds, F.FP32_TABLE, pos, xf)
    fin = xf.view(torch.float32)[:, 12 * (J - 1):12 * J]
    perr = (fin[:, 9:12] - goal[:, 9:12]).norm(dim=1)
    rerr = (fin[:, :9] - goal[:, :9]).norm(dim=1)
    return {"iterations": iters, "position_error_m_median": float(perr.median()),
            "frac_within_1cm_and_0.05_rot": float(((perr < 0.01) & (rerr < 0.05)).float().mean())}


def ik_leg(w, ev32, args, torch, n_seeds=4096, iters=50):
    """Batched IK (Sec. III-B iteration) on the workload's scene: n_seeds
    seeds x 8 step scales = one particle-sized batch of candidate
    configurations per iteration; goals are end-effector poses of random
    configurations.  The iterations run as one captured CUDA graph."""
    from paper_2310_07854_gb300 import binding as B
    from paper_2310_07854_gb300 import ik as IK
    J = w.robot.n_joints
    goal_q = torch.as_tensor(synth.make_q(4242, n_seeds) * 0.8, device="cuda")
    xf = B.alloc_packed(n_seeds, 12 * J, F.FP32)
    pos = B.alloc_packed(n_seeds, 3 * w.robot.n_spheres, F.FP32)
    B.vapr_fk(ev32.robot, goal_q, n_seeds, F.FP32_TABLE, pos, xf)
    goal = xf.view(torch.float32)[:, 12 * (J - 1):12 * J].contiguous()
    q0 = torch.as_tensor(synth.make_q(4343, n_seeds) * 0.8, device="cuda")
    s = IK.IkSolver(ev32.robot, ev32.scene, w.params, n_seeds)
    q = q0.clone()
    s.init(goal, q)
    f0 = s.cost.clone()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    qg = q0.clone()
    s.init(goal, qg)
    s.step()  # warm the launch caches before capture
    qg.copy_(q0)
    s.init(goal, qg)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        for _ in range(iters):
            s.step()
    qg.copy_(q0)
    s.init(goal, qg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # final end-effector error
    B.vapr_fk(ev32.robot, qg, n_seeds, F.FP32_TABLE, pos, xf)
    fin = xf.view(torch.float32)[:, 12 * (J - 1):12 * J]
    perr = (fin[:, 9:12] - goal[:, 9:12]).norm(dim=1)
    rerr = (fin[:, :9] - goal[:, :9]).norm(dim=1)
    cost = torch.empty(n_seeds, device="cuda")
    B.vapr_collision_cost(ev32.robot, ev32.scene, w.params, pos, n_seeds, F.FP32_TABLE, cost)
    return {"seeds": n_seeds, "scales": len(IK.SCALES), "iterations": iters, "ms": ms,
            "iterations_per_s": iters / (ms / 1000.0),
            "candidate_configs_per_s": iters * n_seeds * len(IK.SCALES) / (ms / 1000.0),
            "mean_cost_start_end": [float(f0.mean()), float(s.cost.mean())],
            "position_error_m_median": float(perr.median()),
            "frac_position_within_1cm": float((perr < 0.01).float().mean()),
            "frac_collision_free": float((cost <= 0).float().mean()),
            "goal_note": "goals are end-effector poses of random configurations, often themselves in collision "
                         "in this cluttered scene, so pose and collision terms compete",
            "pose_only": ik_pose_only(w, ev32, torch, n_seeds)}


def fused_leg(w, ev32, q, n, vtable, args, flush, torch, sizes=(None, 1 << 20)):
    """The step in one kernel with P and G kept on the SM (vapr_cost_grad_fused:
    the upper bound of not storing them at all) timed beside the staged
    step (vapr_cost_grad: FK, collision, backward with P and G stored in
    their formats), FP32 and the VaPr table, at the workload's size and at
    2^20 configurations; and the multi-problem persistent kernel run on this
    single problem (P and G in per-block scratch)."""
    from paper_2310_07854_gb300 import binding as B
    from paper_2310_07854_gb300.batched import BatchedEvaluator
    S, J = w.robot.n_spheres, w.robot.n_joints
    out = {"sizes": []}
    for size in sizes:
        nn = n if size is None else size
        qq = q if size is None else torch.as_tensor(synth.make_q(77, nn), device="cuda")
        row = {"n_configs": nn}
        for name, table in (("fp32", F.FP32_TABLE), ("vapr", vtable)):
            cost = torch.empty(nn, device="cuda")
            jg = B.alloc_packed(nn, J, table.jgrad)
            ws = B.alloc_workspace(ev32.robot, nn, table)
            staged = time_graph(lambda: B.vapr_cost_grad(ev32.robot, ev32.scene, w.params, qq, nn, table, None,
                                                         cost, None, jg, ws), args.steps, args.warmup, flush, torch)
            fused = time_graph(lambda: B.vapr_cost_grad_fused(ev32.robot, ev32.scene, w.params, qq, nn, table, None,
                                                              cost, None, jg), args.steps, args.warmup, flush, torch)
            row[name] = {"table": str(table), "staged_ms": staged, "fused_ms": fused,
                         "fused_configs_per_s": nn / (fused / 1000.0), "fused_over_staged": staged / fused}
            del ws, jg, cost
        out["sizes"].append(row)
    be = BatchedEvaluator([w], table=F.FP32_TABLE, tile=128)
    ms = time_graph(be.eval, args.steps, args.warmup, flush, torch)
    out["multi_problem_kernel_on_one_problem"] = {"configs_per_s": n / (ms / 1000.0), "ms": ms, "tile": 128,
                                                  "status": be.device_status()}
    del be
    return out


def time_reps(fn, reps, samples, torch):
    """Device ms per call of fn(), from `samples` replays of a CUDA graph of
    `reps` back-to-back calls (for inputs larger than L2: no flush)."""
    st = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(reps):
            fn()
    g.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(samples):
        e0.record(st)
        g.replay()
        e1.record(st)
        st.synchronize()
        ts.append(e0.elapsed_time(e1) / reps)
    return ts


def time_graph(fn, steps, warmup, flush_buf, torch):
    """Mean device ms of fn() captured in a CUDA graph, L2 flushed before
    each replay (outside the events)."""
    st = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ts = []
    for i in range(warmup + steps):
        flush_buf.add_(1)
        e0.record(st)
        g.replay()
        e1.record(st)
        st.synchronize()
        if i >= warmup:
            ts.append(e0.elapsed_time(e1))
    return statistics.mean(ts)


def surrogate_sweep(w, q, n, args, flush, torch, counts=(40, 160, 640)):
    """Obstacle-count sweep of the surrogate against the exact stage, cuboid
    density held constant (the scene's half-width grows as O^(1/3))."""
    from paper_2310_07854_gb300.path import Evaluator
    out = []
    for O in counts:
        scene = synth.make_scene(1 + O, O, extent=0.75 * (O / 40.0) ** (1.0 / 3.0))
        ev = Evaluator(w.robot, scene, w.params, n, F.FP32_TABLE)
        r = surrogate_leg(w, ev, q, n, args, flush, torch, None, None, light=True)
        out.append({"cuboids": O, "extent_m": 0.75 * (O / 40.0) ** (1.0 / 3.0), **r})
        del ev
    return out


def surrogate_leg(w, ev32, q, n, args, flush, torch, peaks, peak_kind, light=False):
    """Learned signed-distance surrogate of the workload's scene: trained on
    2M exact distances, then used as the broad phase of the collision stage
    on the workload's sphere centres.  Reports training time and loss, the
    network's distance error against the exact kernel, the share of spheres
    it clears, missed contacts (must be 0), and the gated collision stage's
    speed against the plain FP32 collision stage."""
    from paper_2310_07854_gb300 import binding as B
    from paper_2310_07854_gb300 import surrogate as SG
    S = w.robot.n_spheres
    sg = SG.Surrogate(ev32.scene, synth.init_mlp_params(5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u, y = sg.training_set(seed=5)
    losses = sg.train(u, y, epochs=args.surrogate_epochs)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del u, y
    delta = sg.calibrate(seed=99, eta=w.params.eta)
    ev32.fk(q, n)
    ev32.collision(n)
    exact = (ev32.cost[:n].clone(), ev32.dist[:n].clone(), ev32.grad[:n].clone())
    cost = torch.empty(n, device="cuda")
    dist = torch.empty_like(ev32.dist[:n])
    grad = torch.empty_like(ev32.grad[:n])
    est = torch.empty((n, S), device="cuda")
    gated = lambda: sg.collision_cost(ev32.robot, ev32.params, ev32.pos, n, F.FP32_TABLE, cost,
                                      dist, grad, est)
    gated()
    torch.cuda.synchronize()
    c = ev32.pos[:n].view(torch.float32)[:, :3 * S].reshape(-1, 3).contiguous()
    r = torch.as_tensor(np.tile(w.robot.sphere_local[:, 3], n), device="cuda")
    sdf = torch.empty(n * S, device="cuda")
    B.vapr_scene_sdf(ev32.scene, c, n * S, sdf)
    e = est.reshape(-1)
    skipped = (e - r) >= sg.domain.margin
    miss = int((skipped & (sdf < r + w.params.eta)).sum())
    uq, _ = sg.samples(c)
    inside = (uq.abs() <= 1).all(1)
    band = inside & (sdf >= SG.Y_MIN) & (sdf <= SG.Y_MAX)
    err = (e - sdf).abs()
    t_exact = time_graph(lambda: ev32.collision(n), args.steps, args.warmup, flush, torch)
    t_gated = time_graph(gated, args.steps, args.warmup, flush, torch)
    if light:
        return {"cleared": float(skipped.float().mean()),
                "clearable": float(((sdf - r) >= sg.domain.margin).float().mean()),
                "missed_contacts": miss,
                "equal_to_exact": all(torch.equal(a, b) for a, b in zip(exact, (cost, dist, grad))),
                "margin_m": sg.domain.margin, "train_s": train_s,
                "ms": {"exact_collision": t_exact, "gated_collision": t_gated},
                "speedup_vs_fp32_collision": t_exact / t_gated}
    f = torch.empty(n * S, device="cuda")
    t_net = time_graph(lambda: sg.forward_into(uq, f), args.steps, args.warmup, flush, torch)
    t_sdf = time_graph(lambda: B.vapr_scene_sdf(ev32.scene, c, n * S, sdf), args.steps, args.warmup,
                       flush, torch)
    nq = n * S
    tc_flops = 2.0 * 2 * 256 * 256 * nq  # the two tensor-core layers
    tflops = tc_flops / (t_net / 1000.0) / 1e12
    return {
        "queries": nq, "cuboids": w.scene.n_cuboids, "train_points": 2_000_000,
        "train_epochs": args.surrogate_epochs, "train_s": train_s, "loss_first_last": [losses[0], losses[-1]],
        "cleared": float(skipped.float().mean()),
        "clearable": float(((sdf - r) >= sg.domain.margin).float().mean()),
        "missed_contacts": miss,
        "equal_to_exact": all(torch.equal(a, b) for a, b in zip(exact, (cost, dist, grad))),
        "max_dist_err_band_m": float(err[band].max()), "rms_dist_err_band_m": float(err[band].square().mean().sqrt()),
        "band_m": [SG.Y_MIN, SG.Y_MAX], "margin_m": sg.domain.margin,
        "validation_max_overestimate_m": delta,
        "ms": {"exact_collision": t_exact, "gated_collision": t_gated, "network_only": t_net,
               "exact_sdf_min_over_cuboids": t_sdf},
        "speedup_vs_fp32_collision": t_exact / t_gated,
        "network_roofline": {"bound": "tensor", "achieved": tflops, "unit": "TFLOP/s",
                             "peak": peaks.get("bf16_tflops"), "frac": tflops / peaks["bf16_tflops"]
                             if peaks.get("bf16_tflops") else None, "peak_source": peak_kind,
                             "flops_per_query": 2 * 2 * 256 * 256},
    }


def kernel_mode(args):
    """One stage alone, for ncu captures: a fixed number of launches of one
    kernel on a chosen size (timed as one CUDA graph), no flush, no other
    legs."""
    import torch
    from paper_2310_07854_gb300 import binding as B
    from paper_2310_07854_gb300.path import Evaluator
    w = synth.make_workload(args.workload)
    n = args.configs or w.n
    q = torch.as_tensor(synth.make_q(500, n), device="cuda")
    spec = EXAMPLE_TABLE if args.table == "searched" else args.table
    table = F.FormatTable.parse(spec) if spec != "fp32" else F.FP32_TABLE
    if args.kernel == "ceiling":
        ev = Evaluator(w.robot, w.scene, w.params, n, F.FP32_TABLE)
        l2 = torch.cuda.get_device_properties(0).L2_cache_size
        flush = torch.zeros(max(2 * l2, 256 << 20) // 4, dtype=torch.float32, device="cuda")
        res = ceiling_leg(w, ev, q, n, flush, torch, fp32_peak_tflops(measured_peaks()[0]),
                          reps=args.ceiling_reps)
        print(json.dumps({"kernel": "ceiling", "workload": args.workload, **res,
                          "device_error": B.vapr_device_error()}))
        return
    if args.kernel == "mlp_infer":
        st = B.alloc_mlp_state()
        B.vapr_mlp_init(st, torch.as_tensor(synth.init_mlp_params(5), device="cuda"))
        u = torch.as_tensor(synth.uniform_points(3, [-1, -1, -1], [1, 1, 1], n), device="cuda")
        out = torch.empty(n, device="cuda")
        fn = lambda: B.vapr_mlp_forward(st, u, n, out)
    else:
        ev = Evaluator(w.robot, w.scene, w.params, n, table)
        ev.fk(q, n)
        ev.collision(n)
        if args.kernel == "fused":
            cost = torch.empty(n, device="cuda")
            jg = B.alloc_packed(n, w.robot.n_joints, table.jgrad)
            fn = lambda: B.vapr_cost_grad_fused(ev.robot, ev.scene, w.params, q, n, table, None, cost, None, jg)
        else:
            fn = {"fk": lambda: ev.fk(q, n), "collision": lambda: ev.collision(n),
                  "backward": lambda: ev.backward(q, n), "step": lambda: ev.step(q, n)}[args.kernel]
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    # the launches as one CUDA graph, so that host-side launch costs do not
    # show in the device time of small launches
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(args.steps):
            fn()
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"kernel": args.kernel, "workload": args.workload, "units": n, "table": str(table),
                      "ms_per_launch": ms, "device_error": B.vapr_device_error()}))


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel:
        return kernel_mode(args)
    world, rank, local = replicas.dist_env()
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CUDA library has no CPU fallback)")
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
        pg = dist
    from paper_2310_07854_gb300 import binding as B
    from paper_2310_07854_gb300.path import Evaluator
    B.lib()

    w = synth.make_workload(args.workload)
    w.name = args.workload
    if args.configs:
        w.q = synth.make_q(500, args.configs)
        w.n_traj = max(1, args.configs // w.horizon)
    w.q = replicas.rank_batch(w, rank)  # weak scaling: each rank its own batch
    n = w.n
    q = torch.as_tensor(w.q, device="cuda")
    l2 = torch.cuda.get_device_properties(local).L2_cache_size
    flush = torch.zeros(max(2 * l2, 256 << 20) // 4, dtype=torch.float32, device="cuda")
    ev32 = Evaluator(w.robot, w.scene, w.params, n, F.FP32_TABLE,
                     grid_cells="auto" if args.grid_cells < 0 else (args.grid_cells or None))
    found, vtable_hw = None, None
    if args.table == "searched":  # the VaPr leg times the table the search finds within its budget
        vtable, found, vtable_hw = search_tables(w, ev32, args)
        if vtable is None:
            raise SystemExit("the VaPr search found no table within its budget")
    else:
        vtable = F.FormatTable.parse(args.table)
    evv = Evaluator(ev32.robot, ev32.scene, w.params, n, vtable)

    def barrier():
        torch.cuda.synchronize()
        if pg:
            pg.barrier()

    def max_over_ranks(x):
        return replicas.max_over_ranks(x, pg, "cuda")

    peaks, peak_kind = measured_peaks()
    barrier()
    with ClockSampler(local) as clk:
        # keep the GPU busy while the sampler starts, so that its samples see
        # the clocks under this load (untimed)
        t_end = time.perf_counter() + 0.8
        while time.perf_counter() < t_end:
            for _ in range(20):
                ev32.step(q, n)
            torch.cuda.synchronize()
        per32 = time_steps(ev32, q, n, args.steps, args.warmup, flush, torch)
        perv = time_steps(evv, q, n, args.steps, args.warmup, flush, torch)
    barrier()
    clocks = clk.summary()
    t32 = max_over_ranks(sum(per32["step"]))
    tv = max_over_ranks(sum(perv["step"]))
    value = replicas.job_throughput(world, n, args.steps, t32 / 1000.0)
    value_v = replicas.job_throughput(world, n, args.steps, tv / 1000.0)

    # error of the VaPr table against the FP32 path (decoded by the CUDA unpacker)
    def decoded(ev):
        S, J = ev.robot.n_spheres, ev.robot.n_joints
        out = {}
        for name, buf, L, f in (("pos", ev.pos, 3 * S, ev.table.pos), ("dist", ev.dist, S, ev.table.dist),
                                ("grad", ev.grad, 3 * S, ev.table.grad), ("jgrad", ev.jgrad, J, ev.table.jgrad)):
            o = torch.empty((n, L), dtype=torch.float32, device="cuda")
            B.vapr_unpack(buf, n, L, f, o)
            out[name] = o
        out["cost"] = ev.cost[:n].clone()
        return out
    a, b = decoded(ev32), decoded(evv)
    err = {k: float((a[k] - b[k]).abs().max()) for k in a}
    err_scale = {k: float(a[k].abs().max()) for k in a}
    sparse = sparsity(a["dist"], a["grad"], w.robot.n_spheres)

    # roofline of the dominant kernel (FP32 table).  FK and backward are
    # HBM-bound stages; the collision stage is bound by FP32 ALU work (every
    # sphere/cuboid and self pair needs at least its bounding test).
    bpc = ev32.bytes_per_config()
    avg = {k: statistics.mean(per32[k]) for k in ("fk", "collision", "backward")}
    dom = max(avg, key=avg.get)
    traffic = kernel_traffic(dom, "fp32", n)
    if dom == "collision":
        fpc = collision_flops_per_config(w)
        ach = fpc * n / (avg[dom] / 1000.0) / 1e12
        peak_alu = fp32_peak_tflops(peaks)
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak_alu, "unit": "TFLOP/s",
                "frac": ach / peak_alu, "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x max SM clock",
                "work": "the method's bounding tests of all S*O sphere/cuboid pairs and all self pairs; "
                        "the kernel's broad phases (grid cells, sphere clusters) skip most of them, so this "
                        "is the rate of the method's work, not of instructions executed",
                "traffic": None if traffic is None else traffic * n,
                "algorithmic_flops_per_launch": fpc * n, "algorithmic_bytes_per_launch": bpc[dom] * n}
    else:
        ach = bpc[dom] * n / (avg[dom] / 1000.0) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "peak_source": peak_kind,
                "traffic": None if traffic is None else traffic * n,
                "algorithmic_bytes_per_launch": bpc[dom] * n}
    if dom == "collision":
        ceil = ceiling_leg(w, ev32, q, n, flush, torch, roof["peak"], reps=args.ceiling_reps)
        roof["measured_ceiling"] = {"tflops": ceil["tflops"], "frac": ach / ceil["tflops"],
                                    "source": "vapr_env_ceiling (see alu_ceiling)"}
    else:
        ceil = None
    stages = {}
    for ev_, per_, name in ((ev32, per32, "fp32"), (evv, perv, "vapr")):
        bp = ev_.bytes_per_config()
        stages[name] = {k: {"ms": statistics.mean(per_[k]),
                            "GB/s": bp[k] * n / (statistics.mean(per_[k]) / 1000.0) / 1e9,
                            "hbm_frac": bp[k] * n / (statistics.mean(per_[k]) / 1000.0) / 1e9 / peaks["hbm_gbs"],
                            "bytes_per_config": bp[k]} for k in ("fk", "collision", "backward")}

    # end to end: pinned host q -> device -> path -> cost and J back to the host
    qh = torch.as_tensor(w.q).pin_memory()
    ch = torch.empty(n, dtype=torch.float32).pin_memory()
    jh = torch.empty((n, w.robot.n_joints), dtype=torch.float32).pin_memory()
    qd = torch.empty_like(q)
    for _ in range(args.warmup):
        ev32.step_host(qh, ch, jh, qd)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ev32.step_host(qh, ch, jh, qd)
    barrier()
    te_eager = max_over_ranks(time.perf_counter() - t0)
    run = ev32.host_step_graph(qh, ch, jh, qd)  # the same step as one graph launch
    for _ in range(args.warmup):
        run()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    barrier()
    te_graph = max_over_ranks(time.perf_counter() - t0)
    # streaming: each step's copies overlap the neighbouring steps' kernels
    pipe = ev32.host_pipeline(n)
    outs = [(torch.empty(n, dtype=torch.float32).pin_memory(),
             torch.empty((n, w.robot.n_joints), dtype=torch.float32).pin_memory()) for _ in range(2)]
    batches = lambda k: [(qh, outs[i & 1][0], outs[i & 1][1]) for i in range(k)]
    pipe(batches(args.warmup))
    barrier()
    t0 = time.perf_counter()
    pipe(batches(args.steps))
    barrier()
    te = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * n * args.steps / te, "unit": "configs/s",
           "h2d_bytes_per_step": int(qh.numel() * 4), "d2h_bytes_per_step": int(ch.numel() * 4 + jh.numel() * 4),
           "call": "Evaluator.host_pipeline: per step H2D q, FK, collision, backward, unpack J, D2H C and J; "
                   "two steps in flight (copies on their own streams overlap the neighbouring steps' kernels), "
                   "timed from the first copy to the last result on the host",
           "l2": "not flushed between steps: the steps stream back to back as a caller's would (every step "
                 "rewrites P, D and G and moves q, C and J over the host link); the device-resident value "
                 "above flushes L2 by writing 2 x L2 before each step and pays that write-back",
           "serial_graph_step": {"value": world * n * args.steps / te_graph, "unit": "configs/s",
                                 "call": "Evaluator.host_step_graph: one graph launch and a host wait per step"},
           "eager_step_host": {"value": world * n * args.steps / te_eager, "unit": "configs/s",
                               "launches_per_step": 4, "copies_per_step": 3}}

    sweep = None
    if not args.no_dram_scale:
        sweep = dram_sweep(w, ev32.robot, {"fp32": F.FP32_TABLE, "vapr": vtable}, flush, torch, peaks)
        if "measured_ceiling" in roof:  # the same fraction at the sweep's largest batch (FP32, this scene)
            big = [r for r in sweep if r["table"] == "fp32" and r["cuboids"] == w.scene.n_cuboids]
            if big:
                r = max(big, key=lambda r: r["n_configs"])
                tf = collision_flops_per_config(w) * r["n_configs"] / (r["collision"]["ms"] / 1000.0) / 1e12
                roof["measured_ceiling"]["at_largest_sweep_batch"] = {
                    "n_configs": r["n_configs"], "achieved_tflops": tf, "frac": tf / roof["measured_ceiling"]["tflops"]}
    bases = None
    if rank == 0 and world == 1 and not args.no_config_baselines:
        bases = config_baselines(args, flush, torch)

    broad = broad_phase_leg(w, ev32, q, n, args, flush, torch)
    fused = fused_leg(w, ev32, q, n, vtable, args, flush, torch)
    ev32.fk(q, n)
    swept = swept_leg(w, ev32, n, vtable, args, flush, torch)
    ik_res = ik_leg(w, ev32, args, torch)

    if found is not None:  # the hardware-converter table, timed beside
        hw = found["hardware_formats_only"]
        if vtable_hw is not None:
            evh = Evaluator(ev32.robot, ev32.scene, w.params, n, vtable_hw)
            ph = time_steps(evh, q, n, args.steps, args.warmup, flush, torch)
            hw.update({"configs_per_s": n * args.steps / (sum(ph["step"]) / 1000.0),
                       "speedup_vs_fp32": sum(per32["step"]) / sum(ph["step"]),
                       "stage_ms": {k: statistics.mean(ph[k]) for k in ("fk", "collision", "backward") if ph[k]}})
            del evh

    sur = None
    if not args.no_surrogate:
        sur = surrogate_leg(w, ev32, q, n, args, flush, torch, peaks, peak_kind)
        sur["obstacle_sweep"] = surrogate_sweep(w, q, n, args, flush, torch)

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(args.workload, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "configs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t32 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(w, world),
            "roofline": roof,
            "vapr": {"table": str(vtable), "source": "VaPr search within its budget" if found else "--table",
                     "value": value_v, "unit": "configs/s",
                     "speedup_vs_fp32": value_v / value, "speedup_pct": speedup_pct(t32, tv),
                     "ms_per_step": tv / args.steps,
                     "max_abs_err_vs_fp32_path": err, "fp32_max_abs": err_scale,
                     "max_err_rel_to_fp32_max": {k: err[k] / err_scale[k] if err_scale[k] else None for k in err},
                     "stage_ms": {k: statistics.mean(perv[k]) for k in ("fk", "collision", "backward") if perv[k]}},
            "stages": stages,
            "step_three_separate_calls_ms": statistics.mean(per32["step_three_calls"]),
            "sparsity": sparse,
            "alu_ceiling": ceil,
            "broad_phase": broad,
            "fused": fused,
            "swept": swept,
            "ik": ik_res,
            "vapr_search": found,
            "e2e": e2e,
            "gpu_launches": 3 * args.steps,
            "clocks": clocks,
            "cpu_baseline": cb,
            "dram_sweep": sweep,
            "config_baselines": bases,
            "surrogate": sur,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
