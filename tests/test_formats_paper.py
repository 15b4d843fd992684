"""Host logic of the format set, pinned to the numbers the paper prints
(Sec. I, Sec. IV-A, Sec. V-A, Table II) -- fixtures in tests/golden/."""
import math
import os

from paper_2310_07854_gb300 import formats as F

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _kv(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            out[k] = int(v)
    return out


def _rows(name):
    rows = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            env, *fmts = line.split()
            rows[env] = [F.parse(f) for f in fmts]
    return rows


def test_search_set_counts():
    g = _kv("search_space.txt")
    s = F.search_set()
    assert len(s) == g["n_formats"]
    assert len(set(s)) == len(s)
    assert len(s) ** g["n_tensors"] == g["space"]
    assert {f.name for f in F.formats_at_least(16)} == {"E5M10", "E8M7", "E8M23"}
    assert len(F.formats_at_least(16)) == g["at_least_fp16"]
    # widths are exactly the paper's FP4..FP32 list
    assert sorted({f.bits for f in s}) == [4, 5, 6, 8, 10, 16, 32]


def test_per_tensor_reduction_reproduces_paper():
    """Sec. V-A: dropping every format narrower than each tensor's per-tensor
    result shrinks 4,084,101 to 555,660 (two environments) or 583,443."""
    g = _kv("search_space.txt")
    rows = _rows("table2_per_tensor.txt")
    sizes = {}
    for env, fmts in rows.items():
        sizes[env] = math.prod(len(F.formats_at_least(f.bits)) for f in fmts)
    assert sizes["table_pick_panda"] == g["reduced_hard"]
    assert sizes["table_under_pick_panda"] == g["reduced_hard"]
    for env, n in sizes.items():
        if env not in ("table_pick_panda", "table_under_pick_panda"):
            assert n == g["reduced_other"], env
    assert round(g["space"] / g["reduced_hard"], 2) == 7.35
    assert round(g["space"] / g["reduced_other"], 2) == 7.0


def test_combinatorial_bit_totals():
    """Sec. I: five FP32 tensors are 160 bits; the search ends at <= 43."""
    g = _kv("search_space.txt")
    rows = _rows("table2_combinatorial.txt")
    assert 5 * F.FP32.bits == g["bits_fp32_total"]
    totals = {env: sum(f.bits for f in fmts) for env, fmts in rows.items()}
    assert max(totals.values()) == g["bits_vapr_max"]
    assert totals["bookshelf_tall_panda"] == 34


def test_register_packing_counts():
    """Sec. IV-A: a 32-bit register holds 1 FP32, 2 FP16, 3 FP10, 4 FP8,
    5 FP6, 6 FP5 or 8 FP4 values."""
    per = {f.bits: f.per_word for f in F.search_set()}
    assert per == {32: 1, 16: 2, 10: 3, 8: 4, 6: 5, 5: 6, 4: 8}


def test_table_parse_roundtrip():
    t = F.FormatTable.parse("P=E5M10,D=E2M1,G=e2m1,J=E4M3")
    assert t.pos == F.FP16 and t.dist == F.E2M1 and t.jgrad == F.E4M3
    assert t.xform == F.FP32
    assert F.FormatTable.parse(str(t)) == t
    assert F.parse("bf16") == F.BF16
    assert len(list(F.sweep_tables())) == 7 ** 4


def test_row_bytes():
    assert F.FP32.row_bytes(156) == 624
    assert F.FP16.row_bytes(156) == 320      # 78 words -> 312 B -> 320 B
    assert F.E2M1.row_bytes(156) == 80       # 20 words
    assert F.fmt(2, 3).row_bytes(156) == 128  # 5 per word: 32 words
    assert F.FP32.row_bytes(7) == 32
    assert F.FP32.row_bytes(0) == 0
