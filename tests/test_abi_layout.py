"""The binding's ctypes structures have the layout include/rise.h gives them.

A small C program built with the host compiler from the header alone prints
sizeof and every field's offsetof for each public struct; the ctypes mirror
in rise.py must match field for field, so a field added to one side only (or
in another order) fails here on the CPU instead of corrupting a call.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _pairs():
    from paper_2603_20481_gb300 import rise
    return [("rise_config", rise.Config), ("rise_thresholds", rise.Thresholds),
            ("rise_capture", rise.Capture), ("rise_server_config", rise.ServerConfig),
            ("rise_result", rise.Result), ("rise_box", rise.Box)]


def _dtypes():
    """numpy record types the binding reads arrays of C structs into"""
    from paper_2603_20481_gb300 import rise
    return [("rise_box", rise.BOX_DTYPE), ("rise_colstat", rise.COLSTAT_DTYPE)]


def test_binding_layouts_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "rise.h"', "int main(void) {"]
    fields = {}
    for cname, cls in _pairs():
        fields.setdefault(cname, set()).update(f[0] for f in cls._fields_)
    for cname, dt in _dtypes():
        fields.setdefault(cname, set()).update(dt.names)
    for cname, names in fields.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for name in sorted(names):
            lines.append(f'  printf("{cname} {name} %zu\\n", offsetof({cname}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, cls in _pairs():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f in cls._fields_:
            assert got[(cname, f[0])] == getattr(cls, f[0]).offset, (cname, f[0])
    for cname, dt in _dtypes():
        assert got[(cname, "sizeof")] == dt.itemsize, cname
        for name in dt.names:
            assert got[(cname, name)] == dt.fields[name][1], (cname, name)
