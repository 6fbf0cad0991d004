"""GPU parity of the CSR layout's edge-parallel sweeps against the FP64 oracle.

The CSR sweep splits a block's slots into tiles that ignore row boundaries
and adds each row's new messages from shared memory, tile by tile.  These
cases exercise what that split depends on: every slots-per-thread width
(mean row lengths below 1 to above 8), rows longer than a tile (hub rows),
rows without off-diagonal entries, sizes that leave a ragged last block, and
full-size grids in natural and in randomly permuted node order.

Tolerances as in the other parity tests: one sweep from an identical state
<= 1e-12 relative, normwise and element by element (tests/parity_util.py),
trajectories and converged solutions <= 1e-10 (double); float messages within
1e-5 of the oracle after 50 sweeps.
"""
import numpy as np
import pytest

import oracle
import problems as P
from parity_util import sweep_scales, worst_elementwise

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _rhs(n, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


MATS = {
    # mean symmetrised row length < 1: one slot per thread
    "short_rows_2000": P.sparse_random_m_matrix(2000, 0.3, 21, isolated=50),
    # hub rows of ~2900 slots cross tile boundaries; 40 rows are diagonal only
    "hubs_6001": P.sparse_random_m_matrix(6001, 1.5, 22, hubs=3, hub_degree=4000, isolated=40),
    # mean row length ~24: eight slots per thread and three tiles per block
    "long_rows_1500": P.sparse_random_m_matrix(1500, 12.0, 23),
    # grid operators stored as CSR: four (5-point) and eight (9-point) slots per thread
    "lognormal_45": P.convdiff_5pt(45, P.lognormal_field(45, 0.5, np.random.default_rng(24)),
                                   (1.91, 0.59)),
    "aniso9_31": P.convdiff_9pt_aniso(31, 0.01, (1.91, 0.59)),
}


@pytest.fixture(scope="module")
def g():
    import paper_1904_04093_gb300 as g
    g.load()
    assert torch.cuda.is_available()
    return g


def test_cases_cover_every_width():
    """The matrices above reach every slots-per-thread width of the kernel
    (1, 2 or 4, 8) and a row longer than one tile (256 threads x 8 slots)."""
    widths = set()
    longest = 0
    for A in MATS.values():
        sym = {(int(r), int(c)) for r, c in zip(np.repeat(np.arange(A.n), np.diff(A.indptr)), A.indices)
               if r != c}
        sym |= {(c, r) for r, c in sym}
        mean = len(sym) / A.n
        w = 1
        while w < 8 and w < mean:
            w *= 2
        widths.add(w)
        longest = max(longest, max(np.bincount([r for r, _ in sym], minlength=A.n)))
    assert {1, 8} <= widths and len(widths) >= 3
    assert longest > 256 * 8


@pytest.mark.parametrize("name", list(MATS))
def test_single_sweep_from_injected_state(g, name):
    A = MATS[name]
    b = _rhs(A.n, 1)
    lt, mm = oracle.zero_state(A)
    oracle.sweeps(A, _rhs(A.n, 2), 3, lt, mm)
    edge = (A.data != 0) & (np.repeat(np.arange(A.n), np.diff(A.indptr)) != A.indices)
    mm = np.where(edge, np.random.default_rng(3).uniform(-1, 1, A.nnz), 0.0)
    x_o, beta_o = oracle.beliefs(A, b, lt, mm)
    lt2, mm2, st = oracle.update(A, b, lt, mm)
    assert st == oracle.OK
    lc, lc2 = oracle.diag_contrib(A, lt), oracle.diag_contrib(A, lt2)
    s = g.GabpSolver(A, "fp64", layout="csr")
    assert s.info()["layout"] == "csr"
    s.set_state(dev(lc), dev(mm))
    x = s.sweep(dev(b), 1)
    lam, m = s.get_state()
    assert rel(host(x), x_o) <= 1e-12
    assert rel(host(lam), lc2) <= 1e-12
    assert rel(host(m), mm2) <= 1e-12
    sx, sl, sm = sweep_scales(A, b, lc, mm, x_o, beta_o, lc2, mm2)
    assert worst_elementwise(host(x), x_o, sx) <= 1e-12
    assert worst_elementwise(host(lam), lc2, sl) <= 1e-12
    assert worst_elementwise(host(m), mm2, sm) <= 1e-12
    s.close()


@pytest.mark.parametrize("name", list(MATS))
def test_trajectory_30_sweeps(g, name):
    A = MATS[name]
    b = _rhs(A.n, 4)
    lt, mm = oracle.zero_state(A)
    x_o, _, _ = oracle.sweeps(A, b, 30, lt, mm)
    s = g.GabpSolver(A, "fp64", layout="csr")
    x = s.sweep(dev(b), 30)
    lam, m = s.get_state()
    assert rel(host(x), x_o) <= 1e-10
    assert rel(host(lam), oracle.diag_contrib(A, lt)) <= 1e-10
    assert rel(host(m), mm) <= 1e-10
    s.close()


@pytest.mark.parametrize("name", list(MATS))
def test_solve_and_frozen_solve_match_oracle(g, name):
    """Plain solve (full sweeps) and the solve with frozen precision messages
    (mean-only sweeps, Sec. 4.2) reach the oracle's solution."""
    A = MATS[name]
    b = _rhs(A.n, 5)
    ref = oracle.solve(A, b, 1e-10, 5000)
    assert ref["status"] == oracle.OK
    for freeze in (0, 1):
        s = g.GabpSolver(A, "fp64", layout="csr", check_every=1, freeze_lambda=freeze)
        x, it, rr, st = s.solve(dev(b), 1e-10, 5000)
        assert st == g.OK and rr <= 1e-10
        assert abs(it - ref["iters"]) <= freeze
        assert rel(host(x), ref["x"]) <= (1e-10 if freeze == 0 else 1e-9)
        s.close()


@pytest.mark.parametrize("name", list(MATS))
def test_fp32_sweeps_error_against_oracle(g, name):
    A = MATS[name]
    b = _rhs(A.n, 9)
    lt, mm = oracle.zero_state(A)
    x_o, _, _ = oracle.sweeps(A, b, 50, lt, mm)
    s = g.GabpSolver(A, "fp32", layout="csr")
    x = host(s.sweep(dev(b), 50))
    assert rel(x, x_o) <= 1e-5
    s.close()


@pytest.mark.parametrize("name", ["hubs_6001", "lognormal_45"])
def test_mixed_precision_csr(g, name):
    A = MATS[name]
    b = _rhs(A.n, 10)
    s = g.GabpSolver(A, "fp32_ir", layout="csr", check_every=5)
    x, it, rr, st = s.solve(dev(b), 1e-10, 20000)
    assert st == g.OK and rr <= 1e-10
    r = b - A.matvec(host(x))
    assert np.max(np.abs(r)) / np.max(np.abs(b)) <= 1.05e-10
    s.close()


def test_relabelled_nodes_give_the_relabelled_solution(g):
    """Flood GaBP does not depend on the node numbering: on Q A Q^T with Q
    b the sweep count is the same and the solution is Q x."""
    A, b = P.config_c2(m=64, seed=31)
    B, perm = P.permute_symmetric(A, 32)
    s = g.GabpSolver(A, "fp64", layout="csr", check_every=1)
    x, it, rr, st = s.solve(dev(b), 1e-10, 20000)
    q = g.GabpSolver(B, "fp64", check_every=1)
    assert q.info()["layout"] == "csr"
    xq, itq, rrq, stq = q.solve(dev(b[perm]), 1e-10, 20000)
    assert st == stq == g.OK
    assert abs(it - itq) <= 1
    assert rel(host(xq), host(x)[perm]) <= 1e-9


# --------------------------------------------------------------------------
# full size: the 2048 x 2048 convection-diffusion system as CSR, in natural
# and in randomly permuted node order
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c2():
    return P.config_c2()


@pytest.mark.parametrize("order", ["natural", "permuted"])
def test_fullsize_csr_first_sweeps_elementwise(g, c2, order):
    A, b = c2
    if order == "permuted":
        A, perm = P.permute_symmetric(A, 1002)
        b = b[perm]
    lt, mm = oracle.zero_state(A)
    oracle.sweeps(A, b, 2, lt, mm)
    x_o, beta_o = oracle.beliefs(A, b, lt, mm)
    lt3, mm3, st = oracle.update(A, b, lt, mm)
    assert st == oracle.OK
    lc, lc3 = oracle.diag_contrib(A, lt), oracle.diag_contrib(A, lt3)
    sx, sl, sm = sweep_scales(A, b, lc, mm, x_o, beta_o, lc3, mm3)
    s = g.GabpSolver(A, "fp64", layout="csr")
    assert s.info()["layout"] == "csr"
    x = host(s.sweep(dev(b), 3))
    lam, m = (host(t) for t in s.get_state())
    assert rel(x, x_o) <= 1e-12
    assert rel(m, mm3) <= 1e-12
    assert rel(lam, lc3) <= 1e-12
    assert worst_elementwise(x, x_o, sx) <= 1e-12
    assert worst_elementwise(lam, lc3, sl) <= 1e-12
    assert worst_elementwise(m, mm3, sm) <= 1e-12
    s.close()


@pytest.mark.parametrize("n", [1, 31, 1000])
def test_csr_without_off_diagonals(g, n):
    """A diagonal matrix on the CSR layout: no slots at all, every warp's
    slot range empty; the belief is b / diag after one sweep and the solve
    converges at once."""
    d = np.random.default_rng(n).uniform(0.5, 2.0, n)
    A = P.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), d)
    b = np.random.default_rng(n + 1).uniform(-1, 1, n)
    s = g.GabpSolver(A, "fp64", layout="csr", check_every=1)
    assert s.info()["layout"] == "csr" and s.info()["slots"] == 0
    x = host(s.sweep(dev(b), 1))
    np.testing.assert_allclose(x, b / d, rtol=1e-15, atol=0)
    xs, it, rr, st = s.solve(dev(b), 1e-14, 10)
    assert st == g.OK and it == 1
    s.close()


def test_csr_single_edge_pair(g):
    """Two unknowns, one pair of edges (a path of length one: GaBP is exact
    after diameter + 1 = 2 sweeps, Sec. 2.2)."""
    M = np.array([[3.0, -1.2], [0.7, 2.0]])
    A = P.dense_to_csr(M)
    b = np.array([1.0, -2.0])
    s = g.GabpSolver(A, "fp64", layout="csr")
    x = host(s.sweep(dev(b), 2))
    assert rel(x, np.linalg.solve(M, b)) <= 1e-15


def test_internal_renumbering_is_invisible(g):
    """Reverse Cuthill-McKee renumbering of a CSR context (gabp_options
    reorder) is invisible at the interface: on a randomly numbered grid every
    call returns in the caller's order what the unrenumbered context returns,
    up to the rounding of a different summation order."""
    A0, b = P.config_c2(m=48, seed=41)
    A, perm = P.permute_symmetric(A0, 42)
    b = b[perm]
    gv = np.random.default_rng(43).uniform(-1, 1, A.n)
    ctx = {}
    for reorder in (0, 1):
        s = g.GabpSolver(A, "fp64", layout="csr", check_every=1, reorder=reorder)
        assert s.info()["reordered"] == reorder
        ctx[reorder] = s
    out = {}
    for reorder, s in ctx.items():
        r = {}
        x, r["it"], _, st = s.solve(dev(b), 1e-10, 5000)
        assert st == g.OK
        r["x"] = host(x)
        lam, r["itT"], _, stT = s.solve_transpose(dev(gv), 1e-10, 5000)
        assert stT == g.OK
        r["lam"] = host(lam)
        r["x3"] = host(s.sweep(dev(b), 3))
        L, M = s.get_state()
        r["L"], r["M"] = host(L), host(M)
        rt = torch.empty(A.n, dtype=torch.float64, device="cuda")
        s.residual(dev(b), dev(r["x3"]), rt)  # an O(1) residual (at the solution it is rounding)
        r["res"] = host(rt)
        r["dA"] = host(s.edge_grad(dev(r["lam"]), dev(r["x"])))
        vals = A.data * np.random.default_rng(44).uniform(0.9, 1.1, A.nnz)
        rows = np.repeat(np.arange(A.n), np.diff(A.indptr))
        vals[rows == A.indices] = A.data[rows == A.indices] * 1.5  # keep it dominant
        s.set_values(vals)
        r["xh"] = host(s.solve(dev(b), 1e-10, 5000)[0])
        s.set_values(dev(vals))
        r["xd"] = host(s.solve(dev(b), 1e-10, 5000)[0])
        s.set_schedule("colored")
        r["xc"] = host(s.solve(dev(b), 1e-10, 5000)[0])
        s.set_schedule("flood")
        sm = g.GabpSolver(A, "fp32_ir", layout="csr", check_every=5, reorder=reorder)
        r["xm"] = host(sm.solve(dev(b), 1e-10, 20000)[0])
        out[reorder] = r
    a, c = out[0], out[1]
    assert abs(a["it"] - c["it"]) <= 1 and abs(a["itT"] - c["itT"]) <= 1
    for key in ("x", "lam", "x3", "L", "M", "res", "dA", "xh", "xd", "xc", "xm"):
        assert rel(c[key], a[key]) <= 1e-9, key
    with pytest.raises(g.GabpError):
        ctx[1].set_schedule("lines")


def test_renumbered_context_refused_by_multigrid(g):
    levels, sides, _ = P.config_c2_levels(m_fine=15, m_coarse=7)
    solvers = [g.GabpSolver(levels[0], "fp64", layout="csr", reorder=1),
               g.GabpSolver(levels[1], "fp64")]
    with pytest.raises(g.GabpError):
        g.Multigrid(solvers, sides)
