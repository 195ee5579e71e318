"""The Python binding's view of include/occri.h: every ctypes structure has the size and field
offsets the C compiler gives the header's struct, and every OCCRI_* constant the binding defines
has the header's value (no GPU and no library needed; needs a C compiler)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

import paper_2207_09028_gb300 as occri

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "occri.h")
STRUCTS = [occri.occri_cell, occri.occri_basis, occri.occri_kmesh, occri.occri_kernel,
           occri.occri_tune_t, occri.occri_plan_info_t]


def _header_text():
    src = open(HEADER).read()
    return re.sub(r"/\*.*?\*/", "", src, flags=re.S)


def _constants():
    """OCCRI_* integers of the binding that the header also names."""
    src = _header_text()
    return sorted(n for n, v in vars(occri).items()
                  if n.startswith("OCCRI_") and isinstance(v, int) and not isinstance(v, bool)
                  and re.search(r"\b%s\b" % n, src))


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "occri.h"', 'int main(void) {']
    for s in STRUCTS:
        name = s.__name__
        lines.append('  printf("size %s %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in s._fields_:
            lines.append('  printf("off %s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    for n in _constants():
        lines.append('  printf("const %s %%lld\\n", (long long)(%s));' % (n, n))
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi_layout")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run([cc, "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for ln in out.splitlines():
        kind, key, val = ln.split()
        got[(kind, key)] = int(val)
    return got


@pytest.mark.parametrize("struct", STRUCTS, ids=lambda s: s.__name__)
def test_struct_layout_matches_header(c_layout, struct):
    name = struct.__name__
    assert ctypes.sizeof(struct) == c_layout[("size", name)], name
    for f, _ in struct._fields_:
        assert getattr(struct, f).offset == c_layout[("off", f"{name}.{f}")], (name, f)


def test_constants_match_header(c_layout):
    names = _constants()
    assert len(names) >= 15   # statuses, kernels, precisions, tuner and fault flags
    for n in names:
        assert getattr(occri, n) == c_layout[("const", n)], n
