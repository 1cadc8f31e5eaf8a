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


@pytest.mark.parametrize("n_elem,p,q", [(1 << 60, 4, 3), ((1 << 63) - 1, 7, 6), (1 << 40, 0, 1), (10 ** 6, 4, 3),
                                        (5, 2, 7), (5, 8, 1), (0, 2, 1)])
def test_noalloc_rejects_before_any_device_call(n_elem, p, q):
    """Element counts whose scratch cannot fit (including ones whose byte count would wrap
    around 64 bits) and degrees out of range return STM_EINVAL before any CUDA call: the
    pointers below are never dereferenced, so this runs without a GPU."""
    from paper_1307_5310_gb300 import stm

    L = stm.lib()
    fake = ctypes.c_void_p(256)
    rc = L.stm_residual_apply_noalloc(n_elem, p, q, 0.1, fake, fake, fake, fake, fake, fake, 0)
    assert rc == stm.STM_EINVAL
