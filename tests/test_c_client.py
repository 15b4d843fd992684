"""The C ABI from plain C: tests/c_client.c compiles as C99 against
include/vapr.h with warnings as errors, links libvapr.so directly (no
Python, no torch) and passes its checks, none of which needs a GPU."""
import os
import shutil
import subprocess

import pytest

from paper_2310_07854_gb300 import binding as B

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_plain_c_client(tmp_path):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no C compiler")
    B.lib()  # builds libvapr.so when its sources are newer
    lib_dir = os.path.dirname(B.LIB_PATH)
    exe = str(tmp_path / "c_client")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "c_client.c"),
                    "-o", exe, "-L", lib_dir, "-l:libvapr.so", f"-Wl,-rpath,{lib_dir}"],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout
