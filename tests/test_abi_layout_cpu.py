"""The ctypes mirrors of the C-ABI structs match include/wproj.h: a small C
program compiled against the header prints every struct's size and each
member's offset, and they must equal the ctypes layout the binding uses."""
import ctypes
import keyword
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _pairs():
    # import the binding module without loading the library
    from paper_1307_3424_gb300 import wproj as W
    return [("wproj_grid_desc", W.GridDesc), ("wproj_csr", W.CSR), ("wproj_dr_params", W.DRParams),
            ("wproj_solve_info", W.SolveInfo), ("wproj_stats", W.Stats), ("wproj_learned_info", W.LearnedInfo),
            ("wproj_batch_schedule", W.BatchSchedule), ("wproj_batch_info", W.BatchInfo)]


def _cname(field):
    # a C member named like a Python keyword is bound with a trailing underscore
    return field[:-1] if field.endswith("_") and keyword.iskeyword(field[:-1]) else field


def test_struct_layouts_match_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = _pairs()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "wproj.h"', "int main(void) {"]
    for cname, cls in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {_cname(fname)}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        parts = ln.split()
        if len(parts) == 3:
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, cls in pairs:
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
