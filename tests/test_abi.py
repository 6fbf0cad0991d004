"""The C-ABI library builds, loads and exports every symbol the header declares.

These tests make no compute call: they run on a machine without a GPU.  The
CSR validation of ``gabp_setup`` runs on the host before any CUDA call, so
malformed matrices are rejected here too.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gabp.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b((?:gabp|mg)_[a-z_]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1904_04093_gb300 import build
    build.build()
    import paper_1904_04093_gb300 as g
    return g.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["gabp_setup", "gabp_sweep", "gabp_solve", "mg_vcycle", "gabp_solve_transpose",
                     "gabp_edge_grad", "mg_setup", "mg_solve", "gabp_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), f"{name} declared in gabp.h but not exported"


def test_status_strings_and_defaults(lib):
    import paper_1904_04093_gb300 as g
    for s in range(9):
        assert lib.gabp_status_str(s)
    opt = g.Options()
    lib.gabp_default_options(ctypes.byref(opt))
    assert opt.precision == 0 and opt.check_every == 10 and opt.use_graphs == 1
    assert opt.ir_inner_max == 0 and abs(opt.ir_inner_tol - 1e-3) < 1e-18  # 0: by schedule
    assert opt.freeze_lambda == -1 and opt.block_size == 0


def _setup_status(lib, n, indptr, indices, data):
    indptr = np.ascontiguousarray(indptr, dtype=np.int64)
    indices = np.ascontiguousarray(indices, dtype=np.int32)
    data = np.ascontiguousarray(data, dtype=np.float64)
    h = ctypes.c_void_p()
    st = lib.gabp_setup(n, int(indptr[-1]), indptr.ctypes.data, indices.ctypes.data,
                        data.ctypes.data, None, None, ctypes.byref(h))
    assert not h.value  # nothing is created for a rejected matrix
    return st, lib.gabp_last_error().decode()


@pytest.mark.parametrize("case,expect", [
    ("unsorted", 2), ("duplicate", 2), ("out_of_range", 2), ("nan", 2),
    ("missing_diag", 3), ("zero_diag", 3), ("bad_indptr", 2),
])
def test_malformed_csr_rejected_on_host(lib, case, expect):
    # 3x3 tridiagonal base
    indptr = [0, 2, 5, 7]
    indices = [0, 1, 0, 1, 2, 1, 2]
    data = [4.0, -1.0, -1.0, 4.0, -1.0, -1.0, 4.0]
    if case == "unsorted":
        indices[3], indices[4] = 2, 1
    elif case == "duplicate":
        indices[4] = 1
    elif case == "out_of_range":
        indices[6] = 3
    elif case == "nan":
        data[1] = float("nan")
    elif case == "missing_diag":
        indices[3] = 2
        indices[4] = 2
        indptr = [0, 2, 4, 6]
        indices = [0, 1, 0, 2, 1, 2]
        data = [4.0, -1.0, -1.0, -1.0, -1.0, 4.0]
    elif case == "zero_diag":
        data[3] = 0.0
    elif case == "bad_indptr":
        indptr = [0, 2, 1, 7]
    st, msg = _setup_status(lib, 3, indptr, indices, data)
    assert st == expect, msg
    assert msg


def test_invalid_arguments_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.gabp_setup(-1, 0, None, None, None, None, None, ctypes.byref(h)) == 1
    assert lib.gabp_setup(0, 0, None, None, None, None, None, None) == 1
    assert lib.gabp_solve(None, None, None, 1e-10, 10, None, None) == 1
    assert lib.mg_setup(0, None, None, 4.0, 0, None, None) == 1
