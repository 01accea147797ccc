"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/mm.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+(mm_[a-z0-9_A-Z]+)\s*\(",
                            src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2112_03370_gb300.build import build
    path = build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 11, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_match_header():
    import paper_2112_03370_gb300.mm as m
    assert set(declared_functions()) <= set(m.EXPORTS) | {"mm_last_error"}


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's sizes and field offsets."""
    import shutil
    import subprocess

    import pytest

    import paper_2112_03370_gb300.mm as m
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"mm_problem_desc": m.ProblemDesc, "mm_solve_opts": m.SolveOpts,
               "mm_solve_info": m.SolveInfo, "mm_tune_info": m.TuneInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mm.h"', "int main(void){"]
    for cname, cls in structs.items():
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            cf = "lambda" if fname == "lambda_" else fname
            lines.append(f'printf("%zu\\n", offsetof({cname}, {cf}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = []
    for cls in structs.values():
        want.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            want.append(getattr(cls, fname).offset)
    assert got == want
