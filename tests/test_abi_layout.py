"""The Python binding's structures against the C header's: a small C program
compiled here against include/flz.h prints sizeof and every field's offset of
flz_params, flz_stats and flz_check, and each must equal the ctypes layout
(a field added on one side only would shift every later field)."""

import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2409_15053_gb300 as flz

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not found")
def test_struct_layouts_match_the_header(tmp_path):
    structs = {"flz_params": flz.flz_params, "flz_stats": flz.flz_stats, "flz_check": flz.flz_check}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "flz.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
