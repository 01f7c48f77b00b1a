"""The ctypes mirrors of acr_opts / acr_stats have the C structs' layout:
size and every field offset, measured by compiling a probe against
include/acr.h with the host C compiler (no GPU)."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_layout(struct, fields):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "acr.h"', "int main(void) {",
           '  printf("%%zu\\n", sizeof(%s));' % struct]
    src += ['  printf("%%zu\\n", offsetof(%s, %s));' % (struct, f) for f in fields]
    src += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        cpath, exe = os.path.join(d, "p.c"), os.path.join(d, "p")
        with open(cpath, "w") as fh:
            fh.write("\n".join(src) + "\n")
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), cpath, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return [int(v) for v in out]


@pytest.mark.parametrize("cls,cname", [("AcrOpts", "acr_opts"), ("AcrStats", "acr_stats")])
def test_ctypes_struct_matches_c(cls, cname):
    import paper_1701_00182_gb300 as acr

    S = getattr(acr, cls)
    names = [f[0] for f in S._fields_]
    got = _c_layout(cname, names)
    assert got[0] == C.sizeof(S)
    for name, off in zip(names, got[1:]):
        assert getattr(S, name).offset == off, name
