"""Host-side checks of the C ABI: the library loads and exports every declared call.

No CUDA compute call is made here (this suite runs without a GPU).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qeq.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qeq_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_17978_b300 import build, qeq
    build.build()
    return qeq.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "qeq_solve" in names and "qeq_plan_create" in names and "qeq_energy" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_the_header_functions():
    from paper_2607_17978_b300 import qeq
    assert sorted(qeq.EXPORTED) == declared_functions()


def test_status_strings(lib):
    for s in range(8):
        assert len(lib.qeq_status_str(s)) > 0
    assert lib.qeq_status_str(99) == b"unknown status"


def test_invalid_descriptions_are_rejected_before_any_device_work(lib):
    from paper_2607_17978_b300 import qeq
    import numpy as np
    offs = np.array([0, 4], np.int64)
    cell = np.eye(3).reshape(-1) * 10.0
    sig = np.array([1.0, 1.8])
    h = ctypes.c_void_p()

    def desc(**kw):
        d = qeq.PlanDesc(1, offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                         cell.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2,
                         sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0)
        for k, v in kw.items():
            setattr(d, k, v)
        return d

    for bad in (dict(n_struct=0), dict(n_species=0), dict(n_species=9), dict(spline_order=5),
                dict(precision=7), dict(preconditioner=3)):
        assert lib.qeq_plan_create(ctypes.byref(desc(**bad)), None, ctypes.byref(h)) == qeq.QEQ_ERR_INVALID
    assert lib.qeq_plan_create(None, None, ctypes.byref(h)) == qeq.QEQ_ERR_INVALID
    assert lib.qeq_last_error(None) == b"null plan"
    assert lib.qeq_solve(None, None, None, None, None, None, 0, None, None, None) == qeq.QEQ_ERR_INVALID


def test_missing_library_fails_loudly(tmp_path):
    from paper_2607_17978_b300 import qeq
    with pytest.raises(ImportError):
        qeq.load_library(str(tmp_path / "libqeq.so"))
