"""The Python binding's ctypes structures have the layout of the C ABI's
structs: every field at the offset and with the size that a C compiler gives
it from include/mithra.h, and the same total size (a mismatch would pass
garbage through the ABI without any error).  The oracle's wrapper is held to
its own header (oracle/orc.h) the same way."""
import ctypes as C
import os
import subprocess

import pytest

from paper_1612_03310_gb300 import mithra

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PAIRS = [("mithra_grid", mithra.Grid), ("mithra_undulator", mithra.Undulator),
         ("mithra_bunch", mithra.Bunch), ("mithra_tuning", mithra.Tuning),
         ("mithra_lab_case", mithra.LabCase), ("mithra_rest_frame", mithra.RestFrame),
         ("mithra_bunch_spec", mithra.BunchSpec)]


def _layout(tmp_path_factory, header, incdir, pairs):
    d = tmp_path_factory.mktemp("layout")
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{header}"',
             'int main(void) {']
    for cname, py in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu %zu\\n", offsetof({cname}, {f[0]}), '
                         f'sizeof((({cname}*)0)->{f[0]}));')
    lines += ['  return 0;', '}']
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", incdir, "-o", str(exe), str(src)])
    out = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        parts = line.split()
        out[tuple(parts[:2])] = tuple(int(v) for v in parts[2:])
    return out


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    return _layout(tmp_path_factory, "mithra.h", os.path.join(ROOT, "include"), PAIRS)


def _check(layout, cname, py):
    assert layout[(cname, "size")] == (C.sizeof(py),)
    for f in py._fields_:
        desc = getattr(py, f[0])
        assert layout[(cname, f[0])] == (desc.offset, desc.size), f[0]


@pytest.mark.parametrize("cname,py", PAIRS, ids=[p[0] for p in PAIRS])
def test_struct_layout_matches_header(c_layout, cname, py):
    _check(c_layout, cname, py)


def test_oracle_struct_layout_matches_its_header(orc, tmp_path_factory):
    pairs = [("orc_grid", orc._Grid), ("orc_undulator", orc._Und)]
    lay = _layout(tmp_path_factory, "orc.h", os.path.join(ROOT, "oracle"), pairs)
    for cname, py in pairs:
        _check(lay, cname, py)
