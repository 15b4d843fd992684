"""The C ABI without a GPU: the library loads, exports every function that
include/vapr.h declares, and rejects bad arguments before any device work."""
import ctypes
import os
import re

import pytest

from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "vapr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vapr_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    lib = B.lib()
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
        assert name in B.SIGNATURES, f"binding lacks {name}"


def test_status_strings():
    lib = B.lib()
    for code in range(7):
        assert lib.vapr_status_string(code)
    assert b"unknown" in lib.vapr_status_string(99)


def test_default_formats_match_host_logic():
    for f in F.search_set() + [F.fmt(5, 9), F.fmt(6, 8), F.fmt(6, 6)]:
        c = B.vapr_format_default(f.E, f.M)
        assert (c.exp_bits, c.man_bits, c.flags) == (f.E, f.M, f.flags), f
        assert B.vapr_format_supported(c)
        for n in (0, 1, 7, 52, 156, 1000):
            assert B.vapr_packed_row_bytes(n, c) == (f.row_bytes(n) if n else 0)


def test_unsupported_formats():
    bad = [(1, 2, 4), (9, 2, 4), (5, 20, 1), (8, 3, 4), (8, 23, 4), (4, 3, 3), (4, 3, 8)]
    for E, M, fl in bad:
        assert not B.vapr_format_supported(B.vapr_format(E, M, fl, 0)), (E, M, fl)
    assert not B.vapr_format_supported(B.vapr_format(4, 3, 6, 1))  # reserved != 0
    assert B.vapr_packed_row_bytes(10, B.vapr_format(9, 2, 4, 0)) == 0


def _robot_struct(**kw):
    base = dict(n_joints=7, n_spheres=52, n_pairs=10, reserved=0, joint_fixed=256,
                sphere_local=512, sphere_link=768, pairs=1024)
    base.update(kw)
    return B.vapr_robot(**base)


def test_argument_checks_before_launch():
    lib = B.lib()
    t = B.to_c_table(F.FP32_TABLE)
    r = _robot_struct()
    byref = ctypes.byref
    INVALID, UNSUP, MIS, TOO = 1, 2, 3, 6
    # null robot / table
    assert lib.vapr_fk(None, 256, 4, byref(t), 256, None, None) == INVALID
    assert lib.vapr_fk(byref(r), 256, 4, None, 256, None, None) == INVALID
    # counts out of range
    for kw in (dict(n_joints=0), dict(n_joints=17), dict(n_spheres=129), dict(n_pairs=-1),
               dict(n_pairs=8129), dict(sphere_local=0)):
        assert lib.vapr_fk(byref(_robot_struct(**kw)), 256, 4, byref(t), 256, None, None) == INVALID
    # n == 0 is a no-op, n < 0 invalid
    assert lib.vapr_fk(byref(r), 256, 0, byref(t), 256, None, None) == 0
    assert lib.vapr_fk(byref(r), 256, -1, byref(t), 256, None, None) == INVALID
    # misaligned packed buffer / table
    assert lib.vapr_fk(byref(r), 256, 4, byref(t), 264, None, None) == MIS
    assert lib.vapr_fk(byref(_robot_struct(sphere_local=520)), 256, 4, byref(t), 256, None, None) == MIS
    # unsupported format in the table
    bad = B.to_c_table(F.FP32_TABLE)
    bad.grad = B.vapr_format(9, 1, 4, 0)
    assert lib.vapr_fk(byref(r), 256, 4, byref(bad), 256, None, None) == UNSUP
    # collision: too many cuboids, missing scene
    p = B.vapr_cost_params(0.02, 0.01, 1.0, 1.0)
    sc = B.vapr_scene(1025, 0, 256, 256)
    assert lib.vapr_collision_cost(byref(r), byref(sc), byref(p), 256, 4, byref(t),
                                   None, None, None, None) == TOO
    assert lib.vapr_collision_cost(byref(r), None, byref(p), 256, 4, byref(t),
                                   None, None, None, None) == INVALID
    sc = B.vapr_scene(8, 0, 256, 256)
    assert lib.vapr_collision_cost(byref(r), byref(sc), byref(p), 0, 4, byref(t),
                                   None, None, None, None) == INVALID
    # backward needs q or stored transforms, and aligned outputs
    assert lib.vapr_backward(byref(r), None, None, 256, None, 4, byref(t), 256, None) == INVALID
    assert lib.vapr_backward(byref(r), 256, None, 256, None, 4, byref(t), 260, None) == MIS
    # converters
    f = B.vapr_format(2, 1, 4, 0)
    assert lib.vapr_pack(256, 4, 10, f, 8, None) == MIS
    assert lib.vapr_pack(256, -1, 10, f, 256, None) == INVALID
    assert lib.vapr_pack(256, 0, 10, f, 256, None) == 0
    assert lib.vapr_unpack(256, 4, 10, B.vapr_format(9, 1, 4, 0), 256, None) == UNSUP


def test_cost_grad_workspace_and_checks():
    lib = B.lib()
    byref = ctypes.byref
    r = _robot_struct()
    for spec in ("", "P=E5M10,G=E2M1"):
        t = F.FormatTable.parse(spec) if spec else F.FP32_TABLE
        ct = B.to_c_table(t)
        for n in (1, 7, 1000):
            want = 0
            for f in (t.pos, t.grad):
                want += -(-f.row_bytes(156) * n // 256) * 256
            assert lib.vapr_cost_grad_workspace_bytes(byref(r), n, byref(ct)) == want
    ct = B.to_c_table(F.FP32_TABLE)
    need = lib.vapr_cost_grad_workspace_bytes(byref(r), 10, byref(ct))
    p = B.vapr_cost_params(0.02, 0.01, 1.0, 1.0)
    sc = B.vapr_scene(8, 0, 256, 256)
    args = lambda ws, nbytes, n=10: (byref(r), byref(sc), byref(p), 256, n, byref(ct), None, 256,
                                     None, 256, ws, nbytes, None)
    assert lib.vapr_cost_grad(*args(1024, need - 1)) == 1       # workspace too small
    assert lib.vapr_cost_grad(*args(1040, need)) == 3           # not 256-byte aligned
    assert lib.vapr_cost_grad(*args(None, need)) == 1
    assert lib.vapr_cost_grad(*args(1024, 0, n=0)) == 0         # n == 0: no-op


def test_batched_argument_checks():
    lib = B.lib()
    byref = ctypes.byref
    ct = B.to_c_table(F.FP32_TABLE)
    arr = (B.vapr_problem * 1)()
    for tile in (0, 16, 100, 512):
        assert lib.vapr_batched_plan_bytes(arr, 1, byref(ct), byref(B.vapr_batch_tuning(tile, 0))) == 0
    assert lib.vapr_batched_plan_bytes(arr, 0, byref(ct), byref(B.vapr_batch_tuning(128, 0))) == 0
    plan = B.vapr_batch_plan()
    assert lib.vapr_batched_eval(byref(plan), 256, None) == 1       # not a plan
    assert lib.vapr_batched_eval(None, 256, None) == 1
    assert lib.vapr_batched_publish(byref(plan), 0, None) == 1
    assert lib.vapr_batched_plan(arr, 1, byref(ct), byref(B.vapr_batch_tuning(128, 0)),
                                 264, 1 << 20, byref(plan)) == 3    # plan buffer misaligned


def test_gemm_argument_checks():
    lib = B.lib()
    assert lib.vapr_gemm_bf16(256, 256, 256, 100, 256, 64, None) == 1   # M % 128
    assert lib.vapr_gemm_bf16(256, 256, 256, 128, 128, 64, None) == 1   # N % 256
    assert lib.vapr_gemm_bf16(256, 256, 256, 128, 256, 32, None) == 1   # K % 64
    assert lib.vapr_gemm_bf16(256, 256, 264, 128, 256, 64, None) == 3   # misaligned C
    assert lib.vapr_gemm_bf16(256, 256, 256, 0, 256, 64, None) == 0     # empty


def test_surrogate_argument_checks():
    """Bad arguments of the surrogate entry points return a status before
    any CUDA call (fake device addresses are never dereferenced)."""
    lib = B.lib()
    assert lib.vapr_mlp_state_bytes() > 3 * 4 * B.MLP_PARAMS
    assert lib.vapr_mlp_workspace_bytes(0) == 0
    assert lib.vapr_mlp_workspace_bytes(100) == 0
    assert lib.vapr_mlp_workspace_bytes(1 << 21) == 0
    assert lib.vapr_mlp_workspace_bytes(128) > 0
    assert lib.vapr_mlp_workspace_bytes(256) > lib.vapr_mlp_workspace_bytes(128)
    st, p = 4096, 8192
    assert lib.vapr_mlp_init(None, p, None) == 1
    assert lib.vapr_mlp_init(st + 16, p, None) == 3
    assert lib.vapr_mlp_forward(st, p, -1, p, None) == 1
    assert lib.vapr_mlp_forward(st, p, 0, p, None) == 0
    assert lib.vapr_mlp_forward(st, p + 2, 10, p, None) == 3
    ws = lib.vapr_mlp_workspace_bytes(128)
    assert lib.vapr_mlp_grads(st, p, p, 100, 1.0, st, ws, None, None, None) == 1
    assert lib.vapr_mlp_grads(st, p, p, 128, 1.0, st, ws - 1, None, None, None) == 1
    assert lib.vapr_mlp_grads(st, p, p, 128, 0.0, st, ws, None, None, None) == 1
    assert lib.vapr_mlp_grads(st, p, p, 1 << 21, 1.0, st, ws, None, None, None) == 6
    bad = B.vapr_train_params(1e-3, 1.0, 0.999, 1e-8, 1.0)
    assert lib.vapr_mlp_train_step(st, p, p, 128, ctypes.byref(bad), st, ws, None, None) == 1
    bad = B.vapr_train_params(1e-3, 0.9, 0.999, 1e-8, -1.0)
    assert lib.vapr_mlp_train_step(st, p, p, 128, ctypes.byref(bad), st, ws, None, None) == 1
    scene = B.vapr_scene(1, 0, 4096, 8192)
    dom = B.surrogate_domain([0, 0, 0], [1, 1, 1], 0.1, 0.05)
    assert lib.vapr_scene_sdf(ctypes.byref(scene), None, 5, p, None) == 1
    assert lib.vapr_scene_sdf(ctypes.byref(scene), p, 0, p, None) == 0
    flat = B.surrogate_domain([0, 0, 0], [1, 0, 1], 0.1, 0.05)
    assert lib.vapr_surrogate_samples(ctypes.byref(scene), ctypes.byref(flat), p, 5, -1.0, 1.0, p, p,
                                      None) == 1
    assert lib.vapr_surrogate_samples(ctypes.byref(scene), ctypes.byref(dom), p, 5, 1.0, -1.0, p, p,
                                      None) == 1
    neg = B.surrogate_domain([0, 0, 0], [1, 1, 1], -0.1, 0.05)
    assert lib.vapr_surrogate_samples(ctypes.byref(scene), ctypes.byref(neg), p, 5, -1.0, 1.0, p, p,
                                      None) == 1
    big = B.vapr_scene(B.MAX_CUBOIDS + 1, 0, 4096, 8192)
    assert lib.vapr_surrogate_samples(ctypes.byref(big), ctypes.byref(dom), p, 5, -1.0, 1.0, p, p,
                                      None) == 6


def test_swept_argument_checks():
    lib = B.lib()
    import numpy as np
    from paper_2310_07854_gb300 import synth
    r = synth.make_robot(0)
    robot = B.vapr_robot(r.n_joints, r.n_spheres, 0, 0, 4096, 8192, 12288, 16384)
    scene = B.vapr_scene(2, 0, 4096, 8192)
    params = B.cost_params(synth.CostParams())
    t = B.to_c_table(F.FP32_TABLE)
    call = lambda n, H, K, pos=4096: lib.vapr_swept_cost(ctypes.byref(robot), ctypes.byref(scene),
                                                         ctypes.byref(params), pos, n, H, K,
                                                         ctypes.byref(t), None, None, None, None)
    assert call(64, 32, 0) == 1          # no samples
    assert call(64, 32, 65) == 6         # above VAPR_MAX_SWEPT_SAMPLES
    assert call(63, 32, 4) == 1          # n not a multiple of the horizon
    assert call(64, 0, 4) == 1
    assert call(0, 32, 4) == 0
    assert call(64, 32, 4, pos=4104) == 3
    assert lib.vapr_swept_cost(ctypes.byref(robot), None, ctypes.byref(params), 4096, 64, 32, 4,
                               ctypes.byref(t), None, None, None, None) == 1


def test_scene_grid_bytes_and_checks():
    lib = B.lib()
    byref = ctypes.byref
    # header + cells^3 x (2 words per 64 cuboids) x 4 bytes
    assert B.vapr_scene_grid_bytes(40, 48) == 128 + 48 ** 3 * 2 * 4
    assert B.vapr_scene_grid_bytes(0, 8) == 128 + 8 ** 3 * 2 * 4
    assert B.vapr_scene_grid_bytes(64, 8) == 128 + 8 ** 3 * 2 * 4
    assert B.vapr_scene_grid_bytes(65, 8) == 128 + 8 ** 3 * 4 * 4
    assert B.vapr_scene_grid_bytes(B.MAX_CUBOIDS, 128) == 128 + 128 ** 3 * 32 * 4
    for bad in ((-1, 8), (B.MAX_CUBOIDS + 1, 8), (40, 0), (40, 129)):
        assert B.vapr_scene_grid_bytes(*bad) == 0, bad
    sc = B.vapr_scene(8, 0, 256, 256)
    nb = B.vapr_scene_grid_bytes(8, 16)
    build = lambda scene, reach=0.1, eta=0.02, cells=16, grid=4096, nbytes=nb: lib.vapr_scene_grid_build(
        scene, reach, eta, cells, grid, nbytes, None)
    assert build(None) == 1
    assert build(byref(B.vapr_scene(B.MAX_CUBOIDS + 1, 0, 256, 256))) == 6   # too large
    assert build(byref(B.vapr_scene(8, 0, 260, 256))) == 3                    # pose misaligned
    assert build(byref(sc), reach=-0.1) == 1
    assert build(byref(sc), reach=float("nan")) == 1
    assert build(byref(sc), reach=float("inf")) == 1
    assert build(byref(sc), eta=float("nan")) == 1
    assert build(byref(sc), cells=0) == 1
    assert build(byref(sc), cells=129) == 1
    assert build(byref(sc), grid=None) == 1
    assert build(byref(sc), grid=4104) == 3                                   # grid misaligned
    assert build(byref(sc), nbytes=nb - 1) == 1
    # a scene whose grid pointer is misaligned is rejected by the collision stage
    r = _robot_struct()
    t = B.to_c_table(F.FP32_TABLE)
    p = B.vapr_cost_params(0.02, 0.01, 1.0, 1.0)
    sc_bad = B.vapr_scene(8, 0, 256, 256, 4104)
    assert lib.vapr_collision_cost(byref(r), byref(sc_bad), byref(p), 256, 4, byref(t),
                                   None, None, None, None) == 3


def test_auto_grid_cells():
    from paper_2310_07854_gb300.path import auto_grid_cells
    assert auto_grid_cells(40) == 128                 # 17 MB
    assert auto_grid_cells(0) == 128
    c = auto_grid_cells(1024)                         # 32 words per cell
    assert B.vapr_scene_grid_bytes(1024, c) <= 32 << 20 < B.vapr_scene_grid_bytes(1024, c + 8)


def test_env_ceiling_argument_checks():
    """The pair-test ceiling rejects bad arguments before touching a device."""
    lib = B.lib()
    scene = B.vapr_scene(2, 0, 4096, 8192)
    call = lambda n, reps=4, sp=4096, out=8192, sc=ctypes.byref(scene): lib.vapr_env_ceiling(
        sc, sp, n, 0.02, 1.0, reps, out, None)
    assert call(0) == 0                  # nothing to do
    assert call(-1) == 1
    assert call(64, reps=0) == 1
    assert call(64, sp=None) == 1
    assert call(64, out=None) == 1
    assert call(64, sp=4100) == 3        # spheres not 16-byte aligned
    assert call(64, out=8200) == 3
    assert call(64, sc=None) == 1
    big = B.vapr_scene(B.MAX_CUBOIDS + 1, 0, 4096, 8192)
    assert call(64, sc=ctypes.byref(big)) == 6
    assert lib.vapr_env_ceiling_warps(-1) == 0
    assert lib.vapr_env_ceiling_warps(B.MAX_CUBOIDS + 1) == 0


def test_configuration_count_limit():
    """n above VAPR_MAX_CONFIGS (2^31) is refused before any device work,
    by every entry point that takes a configuration count (fake device
    addresses, never dereferenced)."""
    lib = B.lib()
    byref = ctypes.byref
    big, TOO = (1 << 31) + 1, 6
    t = B.to_c_table(F.FP32_TABLE)
    r = _robot_struct()
    p = B.vapr_cost_params(0.02, 0.01, 1.0, 1.0)
    sc = B.vapr_scene(8, 0, 256, 256)
    assert lib.vapr_fk(byref(r), 256, big, byref(t), 256, None, None) == TOO
    assert lib.vapr_collision_cost(byref(r), byref(sc), byref(p), 256, big, byref(t),
                                   None, None, None, None) == TOO
    assert lib.vapr_backward(byref(r), 256, None, 256, None, big, byref(t), 256, None) == TOO
    assert lib.vapr_cost_grad_workspace_bytes(byref(r), big, byref(t)) == 0
    assert lib.vapr_cost_grad(byref(r), byref(sc), byref(p), 256, big, byref(t), None, 256, None,
                              256, 256, 1 << 20, None) == TOO
    assert lib.vapr_cost_grad_noalloc(byref(r), byref(sc), byref(p), 256, big, byref(t), None, 256,
                                      None, 256, None) == TOO
    assert lib.vapr_swept_cost(byref(r), byref(sc), byref(p), 256, big, 1, 4, byref(t),
                               None, None, None, None) == TOO
    dom = B.surrogate_domain([-1, -1, -1], [1, 1, 1], 0.1, 0.05)
    assert lib.vapr_surrogate_collision_cost(byref(r), byref(sc), byref(p), 4096, byref(dom), 256, big,
                                             byref(t), None, None, None, 256, None) == TOO
    ik = B.vapr_ik_params(100.0, 10.0, 100.0, 0.2, 8, 6, (ctypes.c_float * 16)(*([0.0] * 16)), 256, 256)
    assert lib.vapr_ik_init(byref(r), byref(sc), byref(p), byref(ik), 256, 256, big, byref(t), 256,
                            1 << 20, 256, None) == TOO
    arr = (B.vapr_problem * 1)()
    arr[0].robot, arr[0].scene, arr[0].params = r, sc, p
    arr[0].q, arr[0].cost, arr[0].jgrad_packed, arr[0].n = 256, 256, 256, big
    plan = B.vapr_batch_plan()
    assert lib.vapr_batched_plan(arr, 1, byref(t), byref(B.vapr_batch_tuning(128, 0)), 256, 1 << 20,
                                 byref(plan)) == TOO


def test_noalloc_statuses():
    """The no-allocation step names each fault: a bad robot, a bad format
    and a batch beyond its array each get their own status."""
    lib = B.lib()
    byref = ctypes.byref
    t = B.to_c_table(F.FP32_TABLE)
    p = B.vapr_cost_params(0.02, 0.01, 1.0, 1.0)
    sc = B.vapr_scene(8, 0, 256, 256)
    call = lambda robot, table, n: lib.vapr_cost_grad_noalloc(robot, byref(sc), byref(p), 256, n, table,
                                                              None, 256, None, 256, None)
    assert call(byref(_robot_struct(n_joints=0)), byref(t), 4) == 1
    assert call(None, byref(t), 4) == 1
    bad = B.to_c_table(F.FP32_TABLE)
    bad.dist = B.vapr_format(9, 1, 4, 0)
    assert call(byref(_robot_struct()), byref(bad), 4) == 2
    assert call(byref(_robot_struct()), byref(t), -1) == 1
    assert call(byref(_robot_struct()), byref(t), 0) == 0
    assert call(byref(_robot_struct()), byref(t), 1 << 20) == 6   # beyond the 64 MiB array


def test_packed_row_bytes_agree_with_the_oracle():
    """Row sizes of the packed layout, three ways: the library's
    vapr_packed_row_bytes, the oracle's packer and the host format table,
    for every format of the search set and the extra ones, at every row
    length up to 300 and a few large ones."""
    import oracle
    fmts = F.search_set() + [F.fmt(5, 9), F.fmt(6, 8), F.fmt(6, 6)]
    lengths = list(range(1, 301)) + [1023, 1 << 16, (1 << 20) + 3]
    for f in fmts:
        c = B.to_c_format(f)
        for L in lengths:
            want = oracle.packed_row_bytes(L, f.bits)
            assert B.vapr_packed_row_bytes(L, c) == want == f.row_bytes(L), (str(f), L)
    assert B.vapr_packed_row_bytes(0, B.to_c_format(F.FP32)) == 0


def test_missing_library_fails_loudly():
    """Without libvapr.so every call raises: there is no CPU or PyTorch
    fallback (run in a child process so this one's loaded library stays)."""
    import subprocess
    import sys
    code = (
        "import paper_2310_07854_gb300.binding as B, paper_2310_07854_gb300.build as bld\n"
        "from paper_2310_07854_gb300 import formats as F\n"
        "bld.up_to_date = lambda: True\n"
        "B.LIB_PATH = '/nonexistent/libvapr.so'\n"
        "try:\n"
        "    B.packed_row_bytes(156, F.FP32)\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e)\n"
    )
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "raised: libvapr.so is missing" in r.stdout


def test_robot_tables_argument_checks():
    """vapr_robot_tables_bytes / _build reject bad robots and buffers on the
    host (no device work on these paths); a misaligned tables pointer on a
    robot is rejected by every entry point's robot check."""
    lib = B.lib()
    byref = ctypes.byref
    INVALID, MIS = 1, 3
    r = _robot_struct()
    nb = lib.vapr_robot_tables_bytes(byref(r))
    assert nb > 0 and nb % 16 == 0
    # more pairs, more bytes; a bad robot has none
    assert lib.vapr_robot_tables_bytes(byref(_robot_struct(n_pairs=100))) > nb
    assert lib.vapr_robot_tables_bytes(byref(_robot_struct(n_joints=0))) == 0
    assert lib.vapr_robot_tables_bytes(None) == 0
    assert lib.vapr_robot_tables_build(byref(r), None, nb, None) == INVALID
    assert lib.vapr_robot_tables_build(byref(r), 4104, nb, None) == MIS
    assert lib.vapr_robot_tables_build(byref(r), 4096, nb - 16, None) == INVALID
    assert lib.vapr_robot_tables_build(byref(_robot_struct(n_spheres=0)), 4096, nb, None) == INVALID
    t = B.to_c_table(F.FP32_TABLE)
    assert lib.vapr_fk(byref(_robot_struct(tables=4100)), 256, 4, byref(t), 256, None, None) == MIS
