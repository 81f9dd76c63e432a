"""The Python binding's ctypes structures against the C header, on the CPU.

For every structure the binding passes through the C-ABI (snp_allocator,
snp_options, snp_desc, snp_info, snp_device_system, snp_batch_info), a small
C program compiled with gcc against include/snp.h prints sizeof and the
offset of every field the binding declares; each must equal the ctypes
layout, so a field added to one side only (or in another order) fails here
instead of corrupting a call."""
import ctypes as ct
import os
import shutil
import subprocess

import pytest

from paper_2408_04343_gb300 import libsnp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["snp_allocator", "snp_options", "snp_desc", "snp_info", "snp_device_system", "snp_batch_info"]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "snp.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(libsnp, name)
        lines.append(f'    printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    lay = {}
    for line in out.splitlines():
        s, f, v = line.split()
        lay[(s, f)] = int(v)
    return lay


@pytest.mark.parametrize("name", STRUCTS)
def test_ctypes_struct_matches_the_header(c_layout, name):
    cls = getattr(libsnp, name)
    assert ct.sizeof(cls) == c_layout[(name, "sizeof")], name
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == c_layout[(name, field)], (name, field)
