"""The binding's ctypes structures have the layout of the C structures of include/dmrg.h:
a host C program compiled with gcc against the header prints sizeof and offsetof of every
field the binding names, and both must equal ctypes' sizeof and field offsets (a field
renamed, reordered, added or dropped on one side only fails here, without a GPU)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C typedef name -> binding class name
PAIRS = [("dmrg_problem", "Problem"), ("dmrg_options", "Options"),
         ("dmrg_mps_init", "MpsInit"), ("dmrg_dav_stats", "DavStats"),
         ("dmrg_step_stats", "StepStats"), ("dmrg_counters", "Counters"),
         ("dmrg_tuning", "Tuning"), ("dmrg_batch_stats", "BatchStats")]


def _binding():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_dmrg_binding_layout", os.path.join(ROOT, "paper_1507_00161_gb300", "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ctypes_structures_match_the_header(tmp_path):
    B = _binding()
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dmrg.h"', "int main(void) {"]
    expect = []
    for cname, pname in PAIRS:
        cls = getattr(B, pname)
        lines.append('  printf("%%zu\\n", sizeof(%s));' % cname)
        expect.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            lines.append('  printf("%%zu\\n", offsetof(%s, %s));' % (cname, fname))
            expect.append(getattr(cls, fname).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got == expect
