"""The C-ABI library builds and exports every entry point include/sv.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sv_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["sv_create", "sv_destroy", "sv_bind_stream", "sv_run", "sv_sample", "sv_expval",
                 "sv_prepare", "sv_launch", "sv_get_amplitudes", "sv_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2604_11599_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.sv_version.restype = ctypes.c_char_p
    assert lib.sv_version().startswith(b"libsv")


def test_binding_covers_every_declared_symbol():
    """The Python binding gives every declared entry point a ctypes signature."""
    from paper_2604_11599_gb300 import sv

    L = sv.lib()
    unbound = [n for n in declared_functions() if getattr(L, n).argtypes is None]
    assert not unbound, unbound


def test_op_record_layout_matches_header():
    """sv_op is 120 bytes in both the header (C compiler) and the IR dtype."""
    import subprocess
    import tempfile

    from paper_2604_11599_gb300.ir import OP_DTYPE, PAULI_DTYPE

    code = r'''
#include <stdio.h>
#include <stddef.h>
#include "sv.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(sv_op), offsetof(sv_op, q), offsetof(sv_op, angle),
         offsetof(sv_op, mask), offsetof(sv_op, then_len), offsetof(sv_op, dense_off), sizeof(sv_pauli));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(code)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    f = OP_DTYPE.fields
    assert got == [OP_DTYPE.itemsize, f["q"][1], f["angle"][1], f["mask"][1], f["then_len"][1],
                   f["dense_off"][1], PAULI_DTYPE.itemsize]


def test_python_binding_fails_loudly_without_library(monkeypatch):
    from paper_2604_11599_gb300 import sv

    monkeypatch.setattr(sv, "_lib", None)
    monkeypatch.setattr(sv, "LIB_PATH", "/nonexistent/libsv.so")
    with pytest.raises(RuntimeError, match="not built"):
        sv.lib()
