"""The C ABI library loads and exports every symbol include/dda.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dda.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dda_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("dda_target_create", "dda_set_polarizability", "dda_solve", "dda_matvec",
              "dda_target_destroy", "dda_status_string", "dda_target_num_dipoles",
              "dda_solve_hbm_bytes", "dda_last_error", "dda_target_grid"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1305_6497_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n


def test_status_strings_without_gpu():
    from paper_1305_6497_gb300 import binding as B
    assert B.dda_status_string(0) == "ok"
    assert "converged" in B.dda_status_string(B.DDA_ERR_NOCONV)
