"""Host-side checks of the C-ABI library: it builds, loads and exports every
entry point that include/stm.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "stm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int32_t|const char \*)\s*(stm_\w+)\s*\(", src, re.M)))


def test_library_exports_header_symbols():
    from paper_1307_5310_gb300 import build, stm

    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert "stm_residual_apply" in declared and "stm_slab_solve" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) <= set(stm.EXPORTS)


def test_binding_loads():
    from paper_1307_5310_gb300 import stm

    L = stm.lib()
    assert L.stm_last_error(None) == b"null context"
