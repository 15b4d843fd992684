"""Host-side helpers of bench.py, on the CPU: the sparsity report, the
collision stage's work count, the derived FP32 peak and the kernel-source
hash that keys the committed DRAM traffic."""
import os

import bench
from paper_2310_07854_gb300 import synth


def test_sparsity():
    import torch
    dist = torch.tensor([[0.0, 0.5], [0.0, 0.0]])
    grad = torch.zeros(2, 6)
    grad[0, 4] = -1.0   # sphere 1 of configuration 0
    grad[1, 0] = 2.0    # sphere 0 of configuration 1
    grad[1, 2] = 3.0    # the same sphere: counted once
    assert bench.sparsity(dist, grad, 2) == {"dist_nonzero": 0.25, "grad_spheres_nonzero": 0.5}


def test_collision_work_count():
    w = synth.make_workload("particle_32768")
    # 52 spheres x 40 cuboids bounding tests at 10 FLOP, every self pair at 9
    assert bench.collision_flops_per_config(w) == 10 * 52 * 40 + 9 * w.robot.n_pairs


def test_derived_fp32_peak():
    assert abs(bench.fp32_peak_tflops({"sm_max_mhz": 2070.0}) - 80.54784) < 1e-9


def test_kernel_source_hash_ignores_comments(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2310_07854_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES["fk"]:
        (csrc / f).write_text("int a;  // note\n\n/* block\n comment */ int b;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_sha("fk")
    (csrc / "fk.cu").write_text("int a;  // another note\n/* changed */ int b;\n")
    assert bench.kernel_source_sha("fk") == h0
    (csrc / "fk.cu").write_text("int a; int c;\n")
    assert bench.kernel_source_sha("fk") != h0


def test_traffic_only_for_the_captured_source(monkeypatch):
    """The roofline's DRAM traffic is taken from the committed capture only
    while the collision source hash matches the one captured; otherwise it
    is null."""
    import json
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        ent = json.load(f)["collision:fp32:32768"]
    monkeypatch.setattr(bench, "kernel_source_sha", lambda stage: ent["source_sha"])
    assert bench.kernel_traffic("collision", "fp32", 32768) == ent["dram_bytes_per_config"]
    assert bench.kernel_traffic("collision", "fp32", 12345) is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda stage: "0" * 16)
    assert bench.kernel_traffic("collision", "fp32", 32768) is None


def test_clock_summary():
    """Clock samples as nvidia-smi prints them (csv, no header, no units):
    median SM clock, the highest maximum, and every throttle reason seen."""
    s = bench.ClockSampler(0)
    s.out = "\n".join([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ])
    out = s.summary()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4}
    s.out = "0, 1200, 2070, 500.0, 0x8, Active, Not Active, Active, Not Active"
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.out = ""
    assert s.summary()["reasons"] == ["unsampled"]


def test_reference_arm_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the contract's keys; it needs no GPU."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--workload", "single_128"],
                       capture_output=True, text=True, timeout=300, cwd=bench.ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "configs/s" and line["value"] > 0
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True
    assert line["config"]["workload"] == "single_128" and line["config"]["global_batch"] == 128
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "configs/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_speedup_in_the_papers_form():
    assert bench.speedup_pct(1.0, 0.5) == 100.0
    assert abs(bench.speedup_pct(1.0, 1 / 1.0628) - 6.28) < 1e-9
    assert bench.speedup_pct(0.96, 1.0) < 0  # slower: negative
