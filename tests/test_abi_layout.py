"""The binding's ctypes structures have the C header's layout: a C program
compiled against include/als.h prints every struct's size and each field's
offset, and the ctypes classes must agree (no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _structs():
    from paper_1508_03110_gb300 import _lib
    # C struct name -> (ctypes class, {ctypes field name: C member name})
    return {
        "als_config": (_lib.Config, {"lam": "lambda"}),
        "als_iter_info": (_lib.IterInfo, {}),
        "als_launch": (_lib.Launch, {}),
        "als_tune_report": (_lib.TuneReport, {}),
        "als_server_config": (_lib.ServerConfig, {}),
        "als_sweep_timing": (_lib.SweepTiming, {}),
    }


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_struct_layouts_match_the_header(tmp_path):
    structs = _structs()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "als.h"', "int main(void) {"]
    for cname, (cls, ren) in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            member = ren.get(fname, fname)
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {member}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                          text=True).stdout.splitlines())
    for cname, (cls, _) in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(cls, fname).offset, f"{cname}.{fname}"
