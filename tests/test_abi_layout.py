"""The ctypes mirrors of the C-ABI structs (paper_1810_07323_gb300/_lib.py) against the header:
a small C program built from include/corutv.h prints sizeof and the offset of every field the
binding declares, and each must equal what ctypes computes.  A field the header lacks fails the
compile; a field added on one side only moves an offset or the size."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1810_07323_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# binding field names that differ from the header's (Python keywords)
C_NAME = {"lam": "lambda"}

PAIRS = [
    ("corutv_params", _lib.Params),
    ("corutv_batch_tuning", _lib.BatchTuning),
    ("corutv_problem", _lib.Problem),
    ("corutv_info", _lib.Info),
    ("corutv_trace", _lib.Trace),
    ("corutv_rpca_params", _lib.RpcaParams),
    ("corutv_rpca_info", _lib.RpcaInfo),
]


def _c_layout(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "corutv.h"', "int main(void) {"]
    for cname, cls in PAIRS:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {C_NAME.get(f, f)}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    return got


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a C compiler")
def test_ctypes_structs_match_the_header(tmp_path):
    got = _c_layout(tmp_path)
    for cname, cls in PAIRS:
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
