"""The C-ABI library loads on a machine without a GPU and exports every function
that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(vi_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["vi_problem_create", "vi_problem_create_desc", "vi_problem_destroy", "vi_solve",
                     "vi_simulate", "vi_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2303_10672_b300 as vi
    lib = ctypes.CDLL(vi.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    import paper_2303_10672_b300 as vi
    L = vi.lib()
    assert L.vi_status_string(0) == b"ok"
    assert L.vi_status_string(3).startswith(b"not converged")
