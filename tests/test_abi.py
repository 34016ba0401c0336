"""The C ABI library loads and exports every symbol include/lsq.h declares; the ctypes
mirrors of its structs have the C layout.  No compute calls (runs without a GPU)."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsq.h")


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"LSQ_API\s+[\w\s\*]+?\b(lsq_\w+)\s*\(", src)))


def test_header_declares_the_paper_calls():
    names = declared()
    for n in ["lsq_sample_rows", "lsq_build_precond", "lsq_pcg_solve", "lsq_pcg_adjoint",
              "lsq_precond_destroy", "lsq_status_string"]:
        assert n in names


def test_library_builds_loads_and_exports(lsq):
    L = lsq.L.load()
    for name in declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lsq.L.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lsq_\w+)", out))
    assert set(declared()) <= exported
    assert L.lsq_status_string(4) == b"not converged"
    assert L.lsq_sample_size(100, 4.0) == 1843


def test_ctypes_struct_layout_matches_c(lsq, tmp_path):
    c = tmp_path / "layout.c"
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lsq.h"\n'
                 'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(lsq_matrix), '
                 'offsetof(lsq_matrix, vals_f64), sizeof(lsq_opts), offsetof(lsq_opts, device_loop), '
                 'sizeof(lsq_info), offsetof(lsq_info, solve_ms), offsetof(lsq_opts, seed));'
                 'printf("%zu %zu %zu\\n", sizeof(lsq_batch_problem), offsetof(lsq_batch_problem, P), '
                 'offsetof(lsq_batch_problem, ldx));return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    L = lsq.L
    want = [ctypes.sizeof(L.LsqMatrix), L.LsqMatrix.vals_f64.offset, ctypes.sizeof(L.LsqOpts),
            L.LsqOpts.device_loop.offset, ctypes.sizeof(L.LsqInfo), L.LsqInfo.solve_ms.offset,
            L.LsqOpts.seed.offset, ctypes.sizeof(L.LsqBatchProblem), L.LsqBatchProblem.P.offset,
            L.LsqBatchProblem.ldx.offset]
    assert got == want


def test_package_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_1806_02968_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.lower().replace("oracle-free", ""), f


def test_missing_library_raises_instead_of_falling_back(tmp_path):
    """Without liblsq.so the package refuses to run: there is no CPU or Python path."""
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1806_02968_gb300 import _lib\n"
            "try:\n    _lib.load(%r)\nexcept RuntimeError as e:\n    print('raised', e)\n"
            "else:\n    print('loaded')\n") % (ROOT, str(tmp_path / "liblsq.so"))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("raised") and "is missing" in out.stdout
