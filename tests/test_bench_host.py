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
