"""The oracle's pins catch plausible mistakes in it.

Each case plants one mistake -- a dropped term, a wrong sign, a transposed
operand, an index off by one, a wrong rounding rule -- in a temporary copy
of the C oracle (or of its Python front end), builds that copy, and runs the pins of the part it touches
(the ``test_oracle_*`` modules, called with the mutant in place of the
oracle).  At least one pin must fail.  A control case builds the unchanged
source the same way and must pass every pin, so a harness error cannot pass
for a caught mistake.  The committed oracle is never modified; everything
runs on the CPU.
"""
import importlib.util
import os
import shutil

import pytest

import test_oracle_exmy
import test_oracle_ik
import test_oracle_kinematics
import test_oracle_mlp
import test_oracle_swept

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")
PINS = {"exmy": test_oracle_exmy, "kin": test_oracle_kinematics, "swept": test_oracle_swept,
        "mlp": test_oracle_mlp, "ik": test_oracle_ik}

# (what the mistake is, pin modules, text in vapr_oracle.c, replacement)
MUTANTS = [
    # ExMy emulator (Sec. IV-A formats, Sec. V-B round to nearest even)
    ("exmy ties away from zero", ["exmy"],
     "double n = nearbyint(ldexp(a, -quantum_exp));", "double n = round(ldexp(a, -quantum_exp));"),
    ("exmy exponent bias off by one", ["exmy"],
     "f.bias = (1 << (E - 1)) - 1;", "f.bias = (1 << (E - 1));"),
    ("exmy no subnormal spacing", ["exmy"],
     "int quantum_exp = (e < f.emin ? f.emin : e) - M;", "int quantum_exp = e - M;"),
    ("exmy subnormal decode scale", ["exmy"],
     "if (ef == 0) return sign * ldexp((double)mf, f.emin - M);",
     "if (ef == 0) return sign * ldexp((double)mf, f.emin - M - 1);"),
    ("exmy fn format keeps the NaN mantissa", ["exmy"],
     "mmax = f.all_m - 1u;", "mmax = f.all_m;"),
    ("exmy overflow decided before rounding", ["exmy"],
     "if (v > f.max_val) return", "if (a > f.max_val) return"),
    ("pack most significant value first", ["exmy"],
     "int sh = bits * (int)(i % k);", "int sh = bits * (int)(k - 1 - i % k);"),
    # forward kinematics (Sec. III-B step 2)
    ("fk joint rotation before the fixed transform", ["kin"],
     "mat4_mul(F, Rz, A);", "mat4_mul(Rz, F, A);"),
    ("fk rotation transposed", ["kin"],
     "A[1] = -sin(q);\n  A[4] = sin(q);", "A[1] = sin(q);\n  A[4] = -sin(q);"),
    ("fk chain multiplied on the wrong side", ["kin"],
     "mat4_mul(prev, A, T + 16 * i);", "mat4_mul(A, prev, T + 16 * i);"),
    # box distance and collision cost (Sec. III-B step 3)
    ("box frame R instead of R^T", ["kin"],
     "x[k] += R[3 * i + k] * (c[i] - t[i]);", "x[k] += R[3 * k + i] * (c[i] - t[i]);"),
    ("box inside term dropped", ["kin"], "    d = u[ks];\n", "    d = 0.0;\n"),
    ("box outside test with and", ["kin"],
     "int outside = u[0] > 0.0 || u[1] > 0.0 || u[2] > 0.0;",
     "int outside = u[0] > 0.0 && u[1] > 0.0 && u[2] > 0.0;"),
    ("box gradient sign dropped", ["kin"],
     "gl[k] = (x[k] >= 0.0 ? 1.0 : -1.0) * v[k] / nrm;", "gl[k] = v[k] / nrm;"),
    ("box gradient rotated by R^T", ["kin"],
     "grad[i] = R[3 * i] * gl[0] + R[3 * i + 1] * gl[1] + R[3 * i + 2] * gl[2];",
     "grad[i] = R[i] * gl[0] + R[3 + i] * gl[1] + R[6 + i] * gl[2];"),
    ("box inside face of the smallest u", ["kin"],
     "if (u[k] > u[ks]) ks = k;", "if (u[k] < u[ks]) ks = k;"),
    ("collision margin subtracted", ["kin"],
     "        double pen = r + eta - d;\n        if (fabs(pen) < kink_eps) flag = 1;",
     "        double pen = r - eta - d;\n        if (fabs(pen) < kink_eps) flag = 1;"),
    ("collision gradient sign", ["kin"],
     "for (int k = 0; k < 3; ++k) gs[k] -= gd[k];", "for (int k = 0; k < 3; ++k) gs[k] += gd[k];"),
    ("collision weight dropped from the gradient", ["kin"],
     "for (int k = 0; k < 3; ++k) G[3 * s + k] = w_c * gs[k];",
     "for (int k = 0; k < 3; ++k) G[3 * s + k] = gs[k];"),
    ("collision weight dropped from the cost", ["kin"],
     "total += w_c * Ds;\n      if (K) K[s] = flag;", "total += Ds;\n      if (K) K[s] = flag;"),
    ("scene distance starts from zero", ["kin"],
     "double best = INFINITY, g[3], margin;", "double best = 0.0, g[3], margin;"),
    ("scene distance skips the last cuboid", ["kin"],
     "      double d = box_sdf(pose + 12 * o, half + 3 * o, pts + 3 * i, g, &margin);\n"
     "      if (d < best) best = d;",
     "      double d = box_sdf(pose + 12 * o, half + 3 * o, pts + 3 * i, g, &margin);\n"
     "      if (d < best && o + 1 < no) best = d;"),
    # self-collision (Sec. III-C out_vec)
    ("self radius of one sphere dropped", ["kin"],
     "(double)sphere_local[4 * i + 3] + (double)sphere_local[4 * j + 3] + eta_s - dd",
     "(double)sphere_local[4 * i + 3] + eta_s - dd"),
    ("self gradient directions swapped", ["kin"],
     "G[3 * i + k] -= w_s * diff[k] / dd;\n            G[3 * j + k] += w_s * diff[k] / dd;",
     "G[3 * i + k] += w_s * diff[k] / dd;\n            G[3 * j + k] -= w_s * diff[k] / dd;"),
    ("self weight dropped from the cost", ["kin"], "total += w_s * pen;", "total += pen;"),
    # backward pass (Sec. III-B step 5)
    ("backward cross product reversed", ["kin"],
     "dc[0] = a[1] * rel[2] - a[2] * rel[1];\n          dc[1] = a[2] * rel[0] - a[0] * rel[2];\n"
     "          dc[2] = a[0] * rel[1] - a[1] * rel[0];",
     "dc[0] = a[2] * rel[1] - a[1] * rel[2];\n          dc[1] = a[0] * rel[2] - a[2] * rel[0];\n"
     "          dc[2] = a[1] * rel[0] - a[0] * rel[1];"),
    ("backward link filter off by one", ["kin"],
     "if (sphere_link[s] - 1 < j) continue;", "if (sphere_link[s] - 1 <= j) continue;"),
    ("backward joint origin dropped", ["kin"],
     "double o[3] = {Tj[3], Tj[7], Tj[11]};  /* origin */", "double o[3] = {0.0, 0.0, 0.0};"),
    ("backward upstream gradient dropped", ["kin"],
     "jgrad[(int64_t)nj * c + j] = scale * acc;", "jgrad[(int64_t)nj * c + j] = acc;"),
    # swept spheres (Sec. III-C closest_pt_swept)
    ("swept own-point weight", ["swept"],
     "const double wown = nxt == c ? 1.0 : 1.0 - a;", "const double wown = nxt == c ? 1.0 : a;"),
    ("swept previous-row weight", ["swept"],
     "for (int i = 0; i < 3; ++i) gs[i] += a * gp[i];",
     "for (int i = 0; i < 3; ++i) gs[i] += (1.0 - a) * gp[i];"),
    ("swept interpolation reversed", ["swept"],
     "x[i] = (1.0 - a) * P[3 * s + i] + a * Pn[3 * s + i];",
     "x[i] = a * P[3 * s + i] + (1.0 - a) * Pn[3 * s + i];"),
    # surrogate network
    ("mlp SiLU derivative term dropped", ["mlp"],
     "return sg * (1.0 + z * (1.0 - sg));", "return sg;"),
    ("mlp layer 2 weights transposed", ["mlp"],
     "z2[i] += (double)v->W2[(int64_t)H * i + k] * a1[k];",
     "z2[i] += (double)v->W2[(int64_t)H * k + i] * a1[k];"),
    ("mlp layer 3 bias dropped", ["mlp"], "z3[i] = v->b3[i];", "z3[i] = 0.0;"),
    ("mlp overestimate weight on the wrong side", ["mlp"],
     "const double wt = r > 0.0 ? over_weight : 1.0;", "const double wt = r < 0.0 ? over_weight : 1.0;"),
    ("mlp bf16 rounding of a1 dropped", ["mlp"],
     "a1[i] = round_bf16(silu(z));", "a1[i] = silu(z);"),
    ("mlp layer 1 weight gradient without the input", ["mlp"],
     "for (int k = 0; k < 3; ++k) gW1[3 * i + k] += d1[i] * xs[k];",
     "for (int k = 0; k < 3; ++k) gW1[3 * i + k] += d1[i];"),
    ("mlp layer 2 delta without SiLU'", ["mlp"],
     "d2[k] = acc * silu_grad(z2[k]);", "d2[k] = acc;"),
    # IK iteration (Sec. III-B steps 1-7)
    ("ik rotation gradient halved", ["ik"],
     "gj += 2.0 * w_rot * dR[3 * i + k] * v[i];", "gj += w_rot * dR[3 * i + k] * v[i];"),
    ("ik lower bound gradient sign", ["ik"],
     "gj -= 2.0 * w_bound * (q_lo[j] - qj);", "gj += 2.0 * w_bound * (q_lo[j] - qj);"),
    ("ik position term dropped", ["ik"],
     "for (int i = 0; i < 3; ++i) total += w_pos * dt[i] * dt[i];", ""),
    ("lbfgs initial scaling inverted", ["ik"],
     "for (int i = 0; i < dim; ++i) d[i] *= sy / yy;", "for (int i = 0; i < dim; ++i) d[i] *= yy / sy;"),
    ("lbfgs second loop newest first", ["ik"],
     "for (int k = 0; k < m; ++k) { /* oldest to newest */", "for (int k = m - 1; k >= 0; --k) {"),
    ("lbfgs first loop sign", ["ik"],
     "for (int i = 0; i < dim; ++i) d[i] -= alpha[k] * y[k * dim + i];",
     "for (int i = 0; i < dim; ++i) d[i] += alpha[k] * y[k * dim + i];"),
]


# The same for the oracle's Python part (format classes, row sizes and the
# IK iteration loop of oracle.py).
PY_MUTANTS = [
    ("ik keeps the highest-cost candidate", ["ik"],
     "pick = np.argmin(fc, axis=1)", "pick = np.argmax(fc, axis=1)"),
    ("ik keeps the oldest pairs", ["ik"],
     "hist[i] = hist[i][-ik.history:]", "hist[i] = hist[i][:ik.history]"),
    ("ik restart keeps the history", ["ik"], "                hist[i] = []\n", "                pass\n"),
    ("ik first step unscaled", ["ik"],
     "return -g * (step0 / max(np.max(np.abs(g)), 1e-30))", "return -g"),
    ("ik pairs kept without positive curvature", ["ik"], "if s @ y > 0.0:", "if True:"),
    ("exmy E5M2 overflows to Inf", ["exmy"],
     "    if (E, M) == (5, 2):\n        return IEEE | SAT", "    if (E, M) == (5, 2):\n        return IEEE"),
    ("exmy E4M3 with Inf", ["exmy"], "        return FN | SAT", "        return IEEE | SAT"),
    ("exmy bfloat16 saturates", ["exmy"],
     "if (E, M) in ((8, 23), (8, 7), (5, 10)):", "if (E, M) in ((8, 23), (5, 10)):"),
    ("pack rows padded to 8 bytes", ["exmy"],
     "return -(-4 * words // 16) * 16", "return -(-4 * words // 8) * 8"),
    ("ik candidates not rounded to float32", ["ik"],
     "cand = (q[:, None, :] + scales[None, :, None] * d[:, None, :]).astype(np.float32)",
     "cand = q[:, None, :] + scales[None, :, None] * d[:, None, :]"),
]


def _oracle_copy(tmp_path, replace=None, py_replace=None):
    """The oracle's Python front end over a C library built from a copy of
    vapr_oracle.c in tmp_path, with `replace` = (old, new) applied to the C
    source and `py_replace` to the Python front end."""
    src = open(os.path.join(ORACLE_DIR, "vapr_oracle.c")).read()
    if replace:
        assert src.count(replace[0]) == 1, replace[0]
        src = src.replace(*replace)
    shutil.copy(os.path.join(ORACLE_DIR, "vapr_oracle.h"), tmp_path / "vapr_oracle.h")
    (tmp_path / "vapr_oracle.c").write_text(src)
    py = open(os.path.join(ORACLE_DIR, "oracle.py")).read()
    if py_replace:
        assert py.count(py_replace[0]) == 1, py_replace[0]
        py = py.replace(*py_replace)
    (tmp_path / "oracle_copy.py").write_text(py)
    spec = importlib.util.spec_from_file_location(f"oracle_copy_{tmp_path.name}",
                                                  str(tmp_path / "oracle_copy.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._HERE = str(tmp_path)
    mod._SRC = str(tmp_path / "vapr_oracle.c")
    mod._LIB_PATH = str(tmp_path / "liboracle.so")
    mod._lib = None
    mod.build(force=True)
    return mod


def _pin_cases(module):
    """(name, function, keyword arguments) of every pin of the module that
    takes the oracle, its parametrisations expanded, in definition order."""
    for name, fn in list(vars(module).items()):
        if not (name.startswith("test_") and callable(fn)):
            continue
        if "orc" not in fn.__code__.co_varnames[:fn.__code__.co_argcount]:
            continue
        combos = [{}]
        for mark in getattr(fn, "pytestmark", []):
            if mark.name != "parametrize":
                continue
            names = [s.strip() for s in mark.args[0].split(",")]
            rows = []
            for v in mark.args[1]:
                if hasattr(v, "values") and hasattr(v, "marks"):  # pytest.param(...)
                    rows.append(tuple(v.values))
                else:
                    rows.append(tuple(v) if len(names) > 1 else (v,))
            combos = [{**c, **dict(zip(names, row))} for c in combos for row in rows]
        for kw in combos:
            yield name, fn, kw


def _first_failing_pin(orc, modules):
    for key in modules:
        for name, fn, kw in _pin_cases(PINS[key]):
            try:
                fn(orc=orc, **kw)
            except pytest.skip.Exception:
                continue
            except Exception as e:  # an assertion, or an error the mistake provokes
                return f"{key}:{name}{kw or ''}: {type(e).__name__}"
    return None


def test_unmutated_copy_passes_every_pin(tmp_path):
    orc = _oracle_copy(tmp_path)
    assert _first_failing_pin(orc, list(PINS)) is None


@pytest.mark.parametrize("what,modules,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, what, modules, old, new):
    orc = _oracle_copy(tmp_path, (old, new))
    assert _first_failing_pin(orc, modules) is not None, f"no pin catches: {what}"


@pytest.mark.parametrize("what,modules,old,new", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pins_catch_planted_mistake_in_python(tmp_path, what, modules, old, new):
    orc = _oracle_copy(tmp_path, py_replace=(old, new))
    assert _first_failing_pin(orc, modules) is not None, f"no pin catches: {what}"
