"""The binding's ctypes mirrors of the C ABI's structs have the layout the
header gives them: a C program compiled against include/wiresim.h prints
every struct's size and each field's offset, and they must equal ctypes'
(a field added to the header but not to the binding, or in another order,
would otherwise shift every later field silently)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2203_02479_gb300 import wiresim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "ws_plane_desc": wiresim.WsPlaneDesc,
    "ws_depos": wiresim.WsDepos,
    "ws_params": wiresim.WsParams,
    "ws_patches": wiresim.WsPatches,
    "ws_plane_info": wiresim.WsPlaneInfo,
    "ws_trace_stat": wiresim.WsTraceStat,
}


def _c_layout(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "wiresim.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'    printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        parts = line.split()
        got[(parts[0], parts[1])] = int(parts[2])
    return got


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ctypes_structs_match_the_header(tmp_path):
    c = _c_layout(tmp_path)
    for cname, py in STRUCTS.items():
        assert c[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert c[(cname, f)] == getattr(py, f).offset, (cname, f)
