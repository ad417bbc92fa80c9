"""CPU checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point that include/bpm.h declares.  No compute calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bpm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bpm_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("bpm_create", "bpm_forces", "bpm_step", "bpm_energy", "bpm_destroy"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2603_27279_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_2603_27279_gb300 import bpm
    assert sorted(bpm.EXPORTED) == _declared()
    assert "sm_103a" in bpm.bpm_version()


def test_binding_refuses_to_run_without_library(tmp_path):
    from paper_2603_27279_gb300 import bpm
    with pytest.raises(RuntimeError):
        bpm._lib_saved = bpm._lib
        try:
            bpm._lib = None
            bpm.load(str(tmp_path / "missing.so"))
        finally:
            bpm._lib = bpm._lib_saved


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2603_27279_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "bpm_oracle" not in txt, f


def test_binding_structs_match_the_header(tmp_path):
    """sizeof / offsetof of bpm_desc, bpm_contact, bpm_lbm and
    bpm_device_state as the C compiler lays them out equal the ctypes mirrors
    of the binding."""
    import ctypes as C
    import subprocess
    from paper_2603_27279_gb300 import bpm as B
    structs = [("bpm_desc", B.bpm_desc), ("bpm_contact", B.bpm_contact), ("bpm_lbm", B.bpm_lbm),
               ("bpm_device_state", B.bpm_device_state)]
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bpm.h"', "int main(void) {"]
    want = []
    for cname, cls in structs:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        want.append(C.sizeof(cls))
        for f, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f}));')
            want.append(getattr(cls, f).offset)
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == want


def test_binding_constants_match_the_header():
    """Every integer macro BPM_* of include/bpm.h has the same value in the
    binding (precisions, dipole modes, plan kinds, error codes)."""
    from paper_2603_27279_gb300 import bpm as B
    src = open(os.path.join(ROOT, "include", "bpm.h")).read()
    macros = dict(re.findall(r"#define\s+(BPM_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", src))
    assert "BPM_FF" in macros and "BPM_ERR_NONFINITE" in macros
    for name, val in macros.items():
        assert getattr(B, name) == int(val), name
