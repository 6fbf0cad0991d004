"""The allocation-free sweep entry point agrees with the regular one.

``gabp_sweep_noalloc`` is for callers that cannot call cudaMalloc (for
example code running while another component owns every device allocation,
or a loop that forbids allocation after start-up): it keeps all its working
state in a fixed array inside the library.  This file is collected last so a
stop-at-first-failure run has already run every other test; it also passes on
its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1904_04093_gb300 as g
    g.load()
    assert torch.cuda.is_available()
    return g


def _noalloc(lib, A, b_dev, nsweeps, x_dev, stream=None):
    ip = torch.as_tensor(np.asarray(A.indptr, np.int64), device="cuda")
    ix = torch.as_tensor(np.asarray(A.indices, np.int32), device="cuda")
    dv = torch.as_tensor(np.asarray(A.data, np.float64), device="cuda")
    sh = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream if stream is None else stream)
    st = lib.gabp_sweep_noalloc(ctypes.c_int32(A.n), ctypes.c_int64(A.nnz),
                                ctypes.c_void_p(ip.data_ptr()), ctypes.c_void_p(ix.data_ptr()),
                                ctypes.c_void_p(dv.data_ptr()), ctypes.c_void_p(b_dev.data_ptr()),
                                ctypes.c_int(nsweeps), ctypes.c_void_p(x_dev.data_ptr()), sh)
    torch.cuda.synchronize()
    return st


def _lib(g):
    lib = g.load()
    fn = lib.gabp_sweep_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int32, ctypes.c_int64] + [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return lib


@pytest.mark.parametrize("name", ["c1_32", "lognormal_33", "random_200"])
def test_noalloc_matches_regular_sweep_twice(g, name):
    rng = np.random.default_rng(3)
    A = {"c1_32": lambda: P.config_c1()[0],
         "lognormal_33": lambda: P.convdiff_5pt(33, P.lognormal_field(33, 0.5, rng), (1.91, 0.59)),
         "random_200": lambda: P.random_m_matrix(200, 0.03, 9, nonsym_pattern=True)}[name]()
    lib = _lib(g)
    solver = g.GabpSolver(A, "fp64")
    for call, (seed, nsweeps) in enumerate([(1, 7), (2, 12)]):
        b = torch.as_tensor(np.random.default_rng(seed).uniform(-1, 1, A.n), device="cuda")
        x_na = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
        st = _noalloc(lib, A, b, nsweeps, x_na)
        assert st == 0, lib.gabp_last_error().decode()
        solver.reset()
        x_ref = solver.sweep(b, nsweeps)
        torch.cuda.synchronize()
        err = (x_na - x_ref).abs().max().item() / x_ref.abs().max().item()
        assert err <= 1e-12, f"call {call}: {err}"


def test_noalloc_rejects_oversized_input(g):
    lib = _lib(g)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.gabp_sweep_noalloc(70000, 70000, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1,
                                ctypes.c_void_p(x.data_ptr()), None)
    assert st == 1
    assert b"too large" in lib.gabp_last_error()


def _csr(n, rows):
    """CSR from per-row lists of (column, value), kept in the order given."""
    indptr = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for r, row in enumerate(rows):
        indptr[r + 1] = indptr[r] + len(row)
        cols += [c for c, _ in row]
        vals += [v for _, v in row]
    return P.CSR(n, indptr, np.asarray(cols, np.int32), np.asarray(vals, np.float64))


def test_noalloc_one_sweep_matches_regular(g):
    """nsweeps = 1: the beliefs come from the zero-message aggregates, x = b / diag."""
    A = P.config_c1()[0]
    lib = _lib(g)
    b = torch.as_tensor(np.random.default_rng(4).uniform(-1, 1, A.n), device="cuda")
    x_na = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, A, b, 1, x_na) == 0, lib.gabp_last_error().decode()
    solver = g.GabpSolver(A, "fp64")
    x_ref = solver.sweep(b, 1)
    torch.cuda.synchronize()
    assert torch.equal(x_na, x_ref)
    assert torch.equal(x_na, b / torch.as_tensor(A.to_dense().diagonal().copy(), device="cuda"))


def test_noalloc_device_detected_statuses(g):
    """The statuses the kernel finds on the device, each with in-range indices:
    a stored zero diagonal (GABP_E_ZERO_DIAG), a zero message denominator at
    the second sweep (GABP_E_BREAKDOWN: on the path 0 - 1 - 2 with unit entries
    the message 1 -> 2 divides by A_11 - A_10 A_01 / A_00 = 0), and rows whose
    columns do not ascend (GABP_E_BAD_CSR).  Each sets gabp_last_error, and a
    valid call right after each one succeeds."""
    lib = _lib(g)
    good = P.config_c1(m=8)[0]
    cases = [
        (3, _csr(3, [[(0, 2.0), (1, -1.0)], [(0, -1.0), (1, 0.0), (2, -1.0)], [(1, -1.0), (2, 2.0)]]),
         1, b"diagonal"),
        (4, P.dense_to_csr(np.array([[1.0, 1.0, 0.0], [1.0, 1.0, 1.0], [0.0, 1.0, 1.0]])), 2,
         b"denominator"),
        (2, _csr(3, [[(0, 2.0), (2, -1.0), (1, -1.0)], [(0, -1.0), (1, 2.0)], [(0, -1.0), (2, 2.0)]]),
         1, b"ascending"),
        (2, _csr(3, [[(0, 2.0), (1, -1.0)], [(0, -1.0), (1, 2.0), (1, -0.5)], [(2, 2.0)]]),
         1, b"ascending"),
    ]
    for want, A, nsweeps, msg in cases:
        b = torch.ones(A.n, dtype=torch.float64, device="cuda")
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        st = _noalloc(lib, A, b, nsweeps, x)
        assert st == want, (want, st, lib.gabp_last_error())
        assert msg in lib.gabp_last_error()
        bg = torch.ones(good.n, dtype=torch.float64, device="cuda")
        xg = torch.zeros(good.n, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, good, bg, 3, xg) == 0
    # the path matrix is fine for one sweep: the zero pivot needs the message 0 -> 1 first
    A = cases[1][1]
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, A, torch.ones(3, dtype=torch.float64, device="cuda"), 1, x) == 0
