"""The binding's ctypes structures mirror include/ckfwi.h field by field:
a plain C program built against the header prints every field's offset and
every structure's size, which must equal the ctypes layout (a mismatch would
pass wrong values across the boundary without any error); the status, memory,
storage and gradient-kind constants equal the header's."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_1810_05268_gb300 import _lib as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = [("ckfwi_grid", B.Grid), ("ckfwi_shot", B.Shot), ("ckfwi_grad_opts", B.GradOpts),
           ("ckfwi_stats", B.Stats)]


def _program():
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ckfwi.h"', "int main(void) {"]
    for cname, py in STRUCTS:
        lines.append('    printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in py._fields_:
            lines.append('    printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f[0], cname, f[0]))
    lines += ["    return 0;", "}"]
    return "\n".join(lines) + "\n"


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("layout")
    src = d / "layout.c"
    exe = d / "layout"
    src.write_text(_program())
    subprocess.run([cc, "-std=c11", "-Wall", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    lay = {}
    for line in out.splitlines():
        s, field, v = line.split()
        lay[(s, field)] = int(v)
    return lay


@pytest.mark.parametrize("cname,py", STRUCTS, ids=[s for s, _ in STRUCTS])
def test_struct_layout_matches_header(c_layout, cname, py):
    assert c_layout[(cname, "sizeof")] == ctypes.sizeof(py)
    for f in py._fields_:
        assert c_layout[(cname, f[0])] == getattr(py, f[0]).offset, f[0]


def test_constants_match_header():
    from paper_1810_05268_gb300 import ckfwi as C
    txt = open(os.path.join(ROOT, "include", "ckfwi.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define CKFWI_(\w+)\s+(-?\d+)\b", txt)}
    defs.pop("H", None)
    assert len(defs) >= 17
    for name, v in defs.items():
        assert getattr(C, name) == v, name
