"""The C-ABI library loads and exports every entry point the header declares
(no GPU needed: nothing here launches a kernel)."""
import os
import re

import pytest

from paper_1712_07297_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "hsolve.h")).read()
    return sorted(set(re.findall(r"\b(hsolve_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_1712_07297_gb300 import hsolve
    return hsolve.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header(lib):
    from paper_1712_07297_gb300 import hsolve
    assert set(_declared()) == set(hsolve.EXPORTS)


def test_default_opts(lib):
    from paper_1712_07297_gb300 import hsolve
    o = hsolve.default_opts()
    assert o.leaf_size == 128 and o.symmetric == -1 and o.gmres_restart == 50


def test_analyze_rejects_bad_csr(lib):
    import ctypes as C
    import numpy as np
    from paper_1712_07297_gb300 import hsolve
    rp = np.array([0, 1, 2], dtype=np.int64)
    col = np.array([0, 5], dtype=np.int32)   # column out of range
    val = np.ones(2)
    csr = hsolve.Csr(2, 2, rp.ctypes.data, col.ctypes.data, val.ctypes.data)
    h = C.c_void_p()
    assert lib.hsolve_analyze(C.byref(csr), None, 0, None, None, C.byref(h)) == -1
    assert lib.hsolve_analyze(None, None, 0, None, None, C.byref(h)) == -1
    rp2 = np.array([0, 2, 1], dtype=np.int64)  # decreasing row pointer
    csr2 = hsolve.Csr(2, 1, rp2.ctypes.data, col.ctypes.data, val.ctypes.data)
    assert lib.hsolve_analyze(C.byref(csr2), None, 0, None, None, C.byref(h)) == -1


def test_null_handle_calls(lib):
    assert lib.hsolve_factor(None, 1e-2, 0) == -1
    assert lib.hsolve_apply(None, None, None, 1, 1) == -1
    lib.hsolve_destroy(None)
    assert lib.hsolve_last_error(None) == b"null handle"
