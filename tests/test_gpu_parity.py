"""GPU parity: the CUDA library through its C ABI against the FP64 CPU oracle.

Tolerances (double precision): one sweep from an identical state <= 1e-12
relative, both normwise (max-norm error over the max-norm of the oracle's
value) and element by element (every output within 1e-12 of the magnitude of
the terms it is computed from, tests/parity_util.py); a 50-sweep trajectory
<= 1e-10, converged solutions <= 1e-10.  Float results state their error
against the oracle in the assertion bounds.
"""
import math

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
    scale = max(np.max(np.abs(b)), 1e-300)
    return float(np.max(np.abs(a - b)) / scale)


def figure_4x4():
    return P.dense_to_csr(np.array([[4.0, -1.0, 1.5, 0.0],
                                    [0.0, 5.0, -2.0, 1.0],
                                    [-1.0, 0.5, 6.0, -2.0],
                                    [0.0, 0.0, 0.0, 3.0]]))


def matrices():
    rng = np.random.default_rng(77)
    return {
        "c1_32": P.config_c1()[0],
        "lognormal_33": P.convdiff_5pt(33, P.lognormal_field(33, 0.5, rng), (1.91, 0.59)),
        "aniso9_31": P.convdiff_9pt_aniso(31, 0.01, (1.91, 0.59)),
        "tridiag_64": P.tridiag(64, 2.0, -1.2, -0.8),
        "random_300": P.random_m_matrix(300, 0.02, 5, nonsym_pattern=True),
        "toy5": P.paper_toy5_pattern(),
        "figure_4x4": figure_4x4(),
        "paper_7x7": P.dense_to_csr(np.loadtxt(__file__.replace("test_gpu_parity.py", "golden/paper_7x7.txt"))),
    }


MATS = matrices()
CONVERGENT = [k for k in MATS if k != "paper_7x7"]


@pytest.fixture(scope="module")
def g():
    import paper_1904_04093_gb300 as g
    g.load()
    assert torch.cuda.is_available()
    return g


def _rhs(n, seed=0):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


@pytest.mark.parametrize("layout", ["auto", "csr"])
@pytest.mark.parametrize("name", list(MATS))
def test_single_sweep_from_injected_state(g, name, layout):
    A = MATS[name]
    b = _rhs(A.n, 1)
    # a realistic precision state (a few sweeps) and random mean messages
    lt, mm = oracle.zero_state(A)
    oracle.sweeps(A, _rhs(A.n, 2), 3, lt, mm)
    edge = (A.data != 0) & (np.repeat(np.arange(A.n), np.diff(A.indptr)) != A.indices)
    mm = np.where(edge, np.random.default_rng(3).uniform(-1, 1, A.nnz), 0.0)
    x_o, beta_o = oracle.beliefs(A, b, lt, mm)
    lt2, mm2, st = oracle.update(A, b, lt, mm)
    assert st == oracle.OK
    lc, lc2 = oracle.diag_contrib(A, lt), oracle.diag_contrib(A, lt2)
    s = g.GabpSolver(A, "fp64", layout=layout)
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


@pytest.mark.parametrize("layout", ["stencil", "csr"])
def test_first_update_within_a_few_ulps(g, layout):
    """Error bound of the library's double reciprocal (approximation + one
    third-order Newton-Raphson step): the first message update from zero
    messages, L = -A_rs A_sr / A_ss and M = -A_rs b_s / A_ss, agrees with the
    oracle's IEEE divisions to a few ulps, element by element."""
    A = MATS["lognormal_33"]
    b = _rhs(A.n, 21)
    lt, mm = oracle.zero_state(A)
    oracle.sweeps(A, b, 1, lt, mm)
    s = g.GabpSolver(A, "fp64", layout=layout)
    s.sweep(dev(b), 1)
    lam, m = s.get_state()
    ref_l = oracle.diag_contrib(A, lt)
    for got, ref in ((host(lam), ref_l), (host(m), mm)):
        nz = ref != 0
        assert np.all(got[~nz] == 0.0)
        assert np.max(np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])) <= 1e-15


@pytest.mark.parametrize("name", CONVERGENT)
def test_trajectory_50_sweeps(g, name):
    A = MATS[name]
    b = _rhs(A.n, 4)
    lt, mm = oracle.zero_state(A)
    x_o, _, _ = oracle.sweeps(A, b, 50, lt, mm)
    s = g.GabpSolver(A, "fp64")
    x = s.sweep(dev(b), 50)
    lam, m = s.get_state()
    assert rel(host(x), x_o) <= 1e-10
    assert rel(host(lam), oracle.diag_contrib(A, lt)) <= 1e-10
    assert rel(host(m), mm) <= 1e-10


@pytest.mark.parametrize("graphs", [True, False])
@pytest.mark.parametrize("name", ["c1_32", "lognormal_33", "aniso9_31", "random_300", "toy5"])
def test_solve_matches_oracle_every_sweep(g, name, graphs):
    A = MATS[name]
    b = _rhs(A.n, 5)
    ref = oracle.solve(A, b, 1e-10, 3000)
    assert ref["status"] == oracle.OK
    s = g.GabpSolver(A, "fp64", check_every=1, use_graphs=graphs)
    x, it, rr, st = s.solve(dev(b), 1e-10, 3000)
    assert st == g.OK
    assert it == ref["iters"]
    assert rr <= 1e-10
    assert rel(host(x), ref["x"]) <= 1e-10


def test_solve_c1_workload(g):
    """Plain FP64 GaBP on the 32x32 convection-diffusion workload: rr <= 1e-10 within 500 sweeps."""
    A, b = P.config_c1()
    ref = oracle.solve(A, b, 1e-10, 500)
    s = g.GabpSolver(A, "fp64", check_every=10)
    x, it, rr, st = s.solve(dev(b), 1e-10, 500)
    assert st == g.OK and rr <= 1e-10
    assert it == int(math.ceil(ref["iters"] / 10.0)) * 10
    xs = np.linalg.solve(A.to_dense(), b)
    assert rel(host(x), xs) <= 1e-9
    # the iterate after the same number of sweeps is the oracle's
    lt, mm = oracle.zero_state(A)
    x_o, _, _ = oracle.sweeps(A, b, it, lt, mm)
    assert rel(host(x), x_o) <= 1e-10


def test_tree_exact_at_diameter_plus_one_gpu(g):
    A = MATS["tridiag_64"]
    b = _rhs(64, 6)
    xs = np.linalg.solve(A.to_dense(), b)
    s = g.GabpSolver(A, "fp64")
    x63 = host(s.sweep(dev(b), 63))
    s.reset()
    x64 = host(s.sweep(dev(b), 64))
    assert rel(x63, xs) > 1e-6
    assert rel(x64, xs) <= 1e-13


def test_lfa_first_sweeps_gpu(g):
    m = 9
    A = P.convdiff_5pt(m, None, (0.0, 0.0))
    b = _rhs(m * m, 7)
    s = g.GabpSolver(A, "fp64")
    x1 = host(s.sweep(dev(b), 1))
    np.testing.assert_allclose(x1, b / 4.0, rtol=1e-15)
    s.reset()
    x2 = host(s.sweep(dev(b), 2)).reshape(m, m)
    B = b.reshape(m, m)
    nb = B[:-2, 1:-1] + B[2:, 1:-1] + B[1:-1, :-2] + B[1:-1, 2:]
    np.testing.assert_allclose(x2[1:-1, 1:-1], (4 * B[1:-1, 1:-1] + nb) / 12.0, rtol=1e-14)


def test_divergence_detected(g):
    A = MATS["paper_7x7"]
    b = _rhs(7, 1)
    assert oracle.solve(A, b, 1e-12, 1000)["status"] == oracle.DIVERGED
    s = g.GabpSolver(A, "fp64")
    _, _, _, st = s.solve(dev(b), 1e-12, 1000)
    assert st == g.DIVERGED


def test_breakdown_detected(g):
    # star: the message from the centre to one leaf has denominator
    # A_00 + tilde-Lambda_20 A_20 = 1 - 1 = 0 at the second sweep
    A = P.dense_to_csr(np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 0.0], [1.0, 0.0, 1.0]]))
    b = np.array([1.0, 2.0, 3.0])
    assert oracle.solve(A, b, 1e-12, 50)["status"] == oracle.BREAKDOWN
    s = g.GabpSolver(A, "fp64", check_every=1)
    _, _, _, st = s.solve(dev(b), 1e-12, 50)
    assert st == g.BREAKDOWN


def test_iteration_cap_returns_last_iterate(g):
    A, b = P.config_c1()
    s = g.GabpSolver(A, "fp64", check_every=10)
    x, it, rr, st = s.solve(dev(b), 1e-14, 27)
    assert st == g.NOT_CONVERGED and it == 27
    lt, mm = oracle.zero_state(A)
    x_o, _, _ = oracle.sweeps(A, b, 27, lt, mm)
    assert rel(host(x), x_o) <= 1e-12
    assert rr == pytest.approx(oracle.residual_inf(A, b, x_o) / np.max(np.abs(b)), rel=1e-6)


def test_degenerate_sizes(g):
    # n = 1: x = b / a after one sweep; zero right-hand side; empty matrix
    A1 = P.dense_to_csr(np.array([[2.5]]))
    s = g.GabpSolver(A1, "fp64", check_every=1)
    x, it, rr, st = s.solve(dev([5.0]), 1e-12, 10)
    assert st == g.OK and host(x)[0] == 2.0 and it == 1
    A, _ = P.config_c1()
    s = g.GabpSolver(A, "fp64")
    x, it, rr, st = s.solve(dev(np.zeros(A.n)), 1e-10, 100)
    assert st == g.OK and it == 0 and np.all(host(x) == 0.0)
    A0 = P.CSR(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    s0 = g.GabpSolver(A0, "fp64")
    x, it, rr, st = s0.solve(torch.zeros(0, dtype=torch.float64, device="cuda"), 1e-10, 10)
    assert st == g.OK and it == 0


def test_structurally_nonsymmetric_layouts_agree(g):
    A = MATS["figure_4x4"]
    b = _rhs(4, 8)
    xs = np.linalg.solve(A.to_dense(), b)
    for layout in ("auto", "csr", "stencil"):
        s = g.GabpSolver(A, "fp64", layout=layout, check_every=1)
        x, it, rr, st = s.solve(dev(b), 1e-14, 500)
        assert st == g.OK
        assert rel(host(x), xs) <= 1e-13


@pytest.mark.parametrize("name", ["c1_32", "lognormal_33", "aniso9_31", "random_300"])
def test_frozen_precision_messages_same_solution(g, name):
    """Precomputed tilde-Lambda (Sec. 4.2): freezing the precision messages once
    they stop changing gives the plain solve's iterates up to rounding."""
    A = MATS[name]
    b = _rhs(A.n, 14)
    ref = oracle.solve(A, b, 1e-10, 5000)
    assert ref["status"] == oracle.OK
    s = g.GabpSolver(A, "fp64", check_every=1, freeze_lambda=1)
    x, it, rr, st = s.solve(dev(b), 1e-10, 5000)
    assert st == g.OK and rr <= 1e-10
    assert abs(it - ref["iters"]) <= 1
    assert rel(host(x), ref["x"]) <= 1e-9
    # the frozen mean-message sweep can be timed; a plain context has none frozen
    assert s.time_sweeps(dev(b), 3, frozen=True) > 0.0
    plain = g.GabpSolver(A, "fp64", check_every=1, freeze_lambda=0)
    with pytest.raises(g.GabpError):
        plain.time_sweeps(dev(b), 3, frozen=True)


def test_frozen_transpose_solve(g):
    A = MATS["lognormal_33"]
    gvec = _rhs(A.n, 15)
    ref = oracle.solve(A.transpose(), gvec, 1e-10, 5000)
    s = g.GabpSolver(A, "fp64", check_every=1, freeze_lambda=1)
    lam, it, rr, st = s.solve_transpose(dev(gvec), 1e-10, 5000)
    assert st == g.OK and abs(it - ref["iters"]) <= 1
    assert rel(host(lam), ref["x"]) <= 1e-9


# --------------------------------------------------------------------------
# coloured schedule (red-black / 4-colour GaBP, Sec. 5.1)
# --------------------------------------------------------------------------
def _greedy_colors(A):
    """Greedy colouring of the symmetrised graph in natural order (test helper)."""
    n = A.n
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    nbrs = [set() for _ in range(n)]
    for r, c in zip(rows, A.indices):
        if r != c:
            nbrs[r].add(int(c))
            nbrs[int(c)].add(int(r))
    col = -np.ones(n, dtype=np.int32)
    for i in range(n):
        used = {col[j] for j in nbrs[i] if col[j] >= 0}
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return col


COLORED = {"c1_32": 2, "lognormal_33": 2, "aniso9_31": 4, "random_300": None, "figure_4x4": None}


@pytest.mark.parametrize("layout", ["auto", "csr"])
@pytest.mark.parametrize("name", list(COLORED))
def test_colored_sweeps_match_oracle(g, name, layout):
    A = MATS[name]
    m = int(round(A.n ** 0.5))
    colors = oracle.grid_colors(m, COLORED[name]) if COLORED[name] else _greedy_colors(A)
    nc = int(colors.max()) + 1
    b = _rhs(A.n, 31)
    # one sweep from an injected state, then a 30-sweep trajectory
    lt, mm = oracle.zero_state(A)
    oracle.sweeps(A, _rhs(A.n, 32), 3, lt, mm)
    edge = (A.data != 0) & (np.repeat(np.arange(A.n), np.diff(A.indptr)) != A.indices)
    mm = np.where(edge, np.random.default_rng(33).uniform(-1, 1, A.nnz), 0.0)
    s = g.GabpSolver(A, "fp64", layout=layout)
    assert s.set_schedule("colored", None if COLORED[name] is None else colors) == nc
    s.set_state(dev(oracle.diag_contrib(A, lt)), dev(mm))
    x_o, _, st = oracle.sweeps_colored(A, b, colors, nc, 1, lt, mm)
    x = s.sweep(dev(b), 1)
    lam, mg_ = s.get_state()
    assert rel(host(x), x_o) <= 1e-12
    assert rel(host(lam), oracle.diag_contrib(A, lt)) <= 1e-12
    assert rel(host(mg_), mm) <= 1e-12
    x_o, _, _ = oracle.sweeps_colored(A, b, colors, nc, 29, lt, mm)
    x = s.sweep(dev(b), 29)
    assert rel(host(x), x_o) <= 1e-10
    # grid colourings run on the parity-class layout, the others on slots
    assert s.info()["parity_layout"] == (1 if (COLORED[name] and layout == "auto") else 0)
    lam, mg_ = s.get_state()
    assert rel(host(lam), oracle.diag_contrib(A, lt)) <= 1e-10
    assert rel(host(mg_), mm) <= 1e-10


def _colored_sweep_reference(A, b, colors, nc, lt, mm):
    """One coloured sweep composed of flood updates, colour by colour (Sec. 5.1):
    the nodes of colour c form their beliefs and replace the messages they send
    from the state left by the colours before them.  Returns the beliefs, the
    new state (as effects on the rows) and the element-wise scales of each
    output, taken from the state its phase read."""
    cols = A.indices.astype(np.int64)
    sender = colors[cols]
    lt_c, mm_c = lt.copy(), mm.copy()
    x_r, sx = np.zeros(A.n), np.zeros(A.n)
    sl, sm = np.zeros(A.nnz), np.zeros(A.nnz)
    for c in range(nc):
        x_c, beta_c = oracle.beliefs(A, b, lt_c, mm_c)
        lt2, mm2, st = oracle.update(A, b, lt_c, mm_c)
        assert st == oracle.OK
        sxc, slc, smc = sweep_scales(A, b, oracle.diag_contrib(A, lt_c), mm_c, x_c, beta_c,
                                     oracle.diag_contrib(A, lt2), mm2)
        sel = sender == c
        lt_c = np.where(sel, lt2, lt_c)
        mm_c = np.where(sel, mm2, mm_c)
        sl[sel], sm[sel] = slc[sel], smc[sel]
        own = colors == c
        x_r[own], sx[own] = x_c[own], sxc[own]
    return x_r, oracle.diag_contrib(A, lt_c), mm_c, sx, sl, sm


@pytest.mark.parametrize("layout", ["auto", "csr"])
@pytest.mark.parametrize("name", list(COLORED))
def test_colored_single_sweep_elementwise(g, name, layout):
    """One coloured sweep from an injected state, element by element: every
    belief and message within 1e-12 of the magnitude of the terms its phase
    computed it from (the composition of flood updates it is checked against
    equals the oracle's coloured sweep)."""
    A = MATS[name]
    m = int(round(A.n ** 0.5))
    colors = oracle.grid_colors(m, COLORED[name]) if COLORED[name] else _greedy_colors(A)
    nc = int(colors.max()) + 1
    b = _rhs(A.n, 43)
    lt, mm = oracle.zero_state(A)
    oracle.sweeps(A, _rhs(A.n, 44), 3, lt, mm)
    edge = (A.data != 0) & (np.repeat(np.arange(A.n), np.diff(A.indptr)) != A.indices)
    mm = np.where(edge, np.random.default_rng(45).uniform(-1, 1, A.nnz), 0.0)
    x_r, lc_r, mm_r, sx, sl, sm = _colored_sweep_reference(A, b, colors, nc, lt, mm)
    lt_o, mm_o = lt.copy(), mm.copy()
    x_o, _, st = oracle.sweeps_colored(A, b, colors, nc, 1, lt_o, mm_o)
    assert st == oracle.OK
    assert rel(x_r, x_o) <= 1e-14 and rel(lc_r, oracle.diag_contrib(A, lt_o)) <= 1e-14
    assert rel(mm_r, mm_o) <= 1e-14
    s = g.GabpSolver(A, "fp64", layout=layout)
    s.set_schedule("colored", None if COLORED[name] is None else colors)
    s.set_state(dev(oracle.diag_contrib(A, lt)), dev(mm))
    x = host(s.sweep(dev(b), 1))
    lam, mg_ = (host(t) for t in s.get_state())
    assert worst_elementwise(x, x_r, sx) <= 1e-12
    assert worst_elementwise(lam, lc_r, sl) <= 1e-12
    assert worst_elementwise(mg_, mm_r, sm) <= 1e-12
    s.close()


@pytest.mark.parametrize("name", ["c1_32", "lognormal_33"])
def test_colored_three_colours_on_slot_layout(g, name):
    """(x + 2y) mod 3 colours a 5-point grid properly but is no union of parity
    classes: it runs on the slot layout, against the oracle."""
    A = MATS[name]
    m = int(round(A.n ** 0.5))
    iy, ix = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    colors = ((ix + 2 * iy) % 3).reshape(-1).astype(np.int32)
    b = _rhs(A.n, 35)
    s = g.GabpSolver(A, "fp64")
    assert s.set_schedule("colored", colors) == 3
    assert s.info()["parity_layout"] == 0
    lt, mm = oracle.zero_state(A)
    x_o, _, _ = oracle.sweeps_colored(A, b, colors, 3, 40, lt, mm)
    x = s.sweep(dev(b), 40)
    assert rel(host(x), x_o) <= 1e-10


@pytest.mark.parametrize("name", ["c1_32", "aniso9_31"])
def test_colored_transpose_on_parity_layout(g, name):
    """The transposed coloured solve (adjoint) on the parity-class layout equals
    the oracle's coloured solve of A^T."""
    A = MATS[name]
    m = int(round(A.n ** 0.5))
    colors = oracle.grid_colors(m, COLORED[name])
    gvec = _rhs(A.n, 36)
    ref = oracle.solve(A.transpose(), gvec, 1e-10, 5000, color=colors, ncolors=COLORED[name])
    assert ref["status"] == oracle.OK
    s = g.GabpSolver(A, "fp64", check_every=1)
    s.set_schedule("colored", colors)
    assert s.info()["parity_layout"] == 1
    lam, it, rr, st = s.solve_transpose(dev(gvec), 1e-10, 5000)
    assert st == g.OK and it == ref["iters"]
    assert rel(host(lam), ref["x"]) <= 1e-10
    # and the forward solve after it still uses A
    ref = oracle.solve(A, gvec, 1e-10, 5000, color=colors, ncolors=COLORED[name])
    x, it, rr, st = s.solve(dev(gvec), 1e-10, 5000)
    assert st == g.OK and it == ref["iters"]
    assert rel(host(x), ref["x"]) <= 1e-10


def _seven_point(m, seed):
    """7-point grid operator ((+-1, 0), (0, +-1), (1, -1), (-1, 1)), nonsymmetric,
    strictly diagonally dominant M-matrix: six stored diagonals."""
    rng = np.random.default_rng(seed)
    off = [(1, -1), (0, -1), (-1, 0), (0, 0), (1, 0), (0, 1), (-1, 1)]
    off.sort(key=lambda o: o[0] + m * o[1])
    c = np.zeros((m, m, 7))
    for k, o in enumerate(off):
        c[:, :, k] = 1.0 if o == (0, 0) else -rng.uniform(0.02, 0.16, (m, m))
    return P.stencil_csr(m, off, c)


@pytest.mark.parametrize("m", [17, 24])
def test_colored_parity_layout_six_diagonals(g, m):
    """Six stored diagonals take the general parity-class kernel (the 5- and
    9-point orders have their own): 4-colour grid colouring, against the oracle."""
    A = _seven_point(m, 40 + m)
    colors = oracle.grid_colors(m, 4)
    b = _rhs(A.n, 38)
    s = g.GabpSolver(A, "fp64")
    assert s.info()["ndiag"] == 6
    s.set_schedule("colored", colors)
    assert s.info()["parity_layout"] == 1
    lt, mm = oracle.zero_state(A)
    x_o, _, _ = oracle.sweeps_colored(A, b, colors, 4, 6, lt, mm)
    x = s.sweep(dev(b), 6)
    assert rel(host(x), x_o) <= 1e-12
    lam, mg_ = s.get_state()
    assert rel(host(lam), oracle.diag_contrib(A, lt)) <= 1e-12
    assert rel(host(mg_), mm) <= 1e-12


def test_colored_float_parity_layout(g):
    """Float messages on the parity-class layout follow the FP64 oracle to float
    accuracy over a 60-sweep trajectory (9-point, 4 colours, odd side)."""
    A = MATS["aniso9_31"]
    colors = oracle.grid_colors(31, 4)
    b = _rhs(A.n, 37)
    s = g.GabpSolver(A, "fp32")
    s.set_schedule("colored")
    assert s.info()["parity_layout"] == 1
    lt, mm = oracle.zero_state(A)
    x_o, _, _ = oracle.sweeps_colored(A, b, colors, 4, 60, lt, mm)
    x = s.sweep(dev(b), 60)
    assert rel(host(x), x_o) <= 2e-5


@pytest.mark.parametrize("name", ["c1_32", "aniso9_31"])
def test_colored_solve_matches_oracle(g, name):
    A = MATS[name]
    m = int(round(A.n ** 0.5))
    colors = oracle.grid_colors(m, COLORED[name])
    b = _rhs(A.n, 34)
    ref = oracle.solve(A, b, 1e-10, 5000, color=colors, ncolors=COLORED[name])
    flood = oracle.solve(A, b, 1e-10, 5000)
    assert ref["status"] == oracle.OK and ref["iters"] < flood["iters"]
    s = g.GabpSolver(A, "fp64", check_every=1)
    s.set_schedule("colored")
    x, it, rr, st = s.solve(dev(b), 1e-10, 5000)
    assert st == g.OK and it == ref["iters"]
    assert rel(host(x), ref["x"]) <= 1e-10
    s.set_schedule("flood")
    x, it, rr, st = s.solve(dev(b), 1e-10, 5000)
    assert it == flood["iters"]


@pytest.mark.parametrize("name", ["c1_32", "aniso9_31"])
def test_colored_frozen_precision_messages(g, name):
    """Frozen precision messages under the coloured schedule (Sec. 4.2 with
    Sec. 5.1) on the parity-class layout: once they stop changing, the gains and
    aggregates are stored and a phase moves only the mean messages.  The FP64
    solve and the transposed solve reach the oracle's coloured solutions (same
    sweeps up to one), the context ends frozen (its frozen sweep can be timed),
    and the mixed-precision solve, which freezes by default, reaches 1e-10 on
    host-checked residuals."""
    A = MATS[name]
    m = int(round(A.n ** 0.5))
    nc = COLORED[name]
    colors = oracle.grid_colors(m, nc)
    b = _rhs(A.n, 39)
    ref = oracle.solve(A, b, 1e-10, 5000, color=colors, ncolors=nc)
    assert ref["status"] == oracle.OK
    s = g.GabpSolver(A, "fp64", check_every=1, freeze_lambda=1)
    s.set_schedule("colored", colors)
    assert s.info()["parity_layout"] == 1
    x, it, rr, st = s.solve(dev(b), 1e-10, 5000)
    assert st == g.OK and rr <= 1e-10
    assert abs(it - ref["iters"]) <= 1
    assert rel(host(x), ref["x"]) <= 1e-9
    assert s.time_sweeps(dev(b), 3, frozen=True) > 0.0
    ref_t = oracle.solve(A.transpose(), b, 1e-10, 5000, color=colors, ncolors=nc)
    lam, it, rr, st = s.solve_transpose(dev(b), 1e-10, 5000)
    assert st == g.OK and abs(it - ref_t["iters"]) <= 1
    assert rel(host(lam), ref_t["x"]) <= 1e-9
    plain = g.GabpSolver(A, "fp64", check_every=1, freeze_lambda=0)
    plain.set_schedule("colored", colors)
    plain.solve(dev(b), 1e-10, 5000)
    with pytest.raises(g.GabpError):
        plain.time_sweeps(dev(b), 3, frozen=True)
    sm = g.GabpSolver(A, "fp32_ir", check_every=5)
    sm.set_schedule("colored", colors)
    x, it, rr, st = sm.solve(dev(b), 1e-10, 20000)
    assert st == g.OK and rr <= 1e-10
    r = b - A.to_dense() @ host(x)
    assert np.max(np.abs(r)) / np.max(np.abs(b)) <= 1.05e-10
    assert rel(host(x), np.linalg.solve(A.to_dense(), b)) <= 1e-8
    assert sm.time_sweeps(dev(b), 3, frozen=True) > 0.0
    for t in (s, plain, sm):
        t.close()


def test_invalid_coloring_rejected(g):
    A = MATS["c1_32"]
    s = g.GabpSolver(A, "fp64")
    with pytest.raises(g.GabpError):
        s.set_schedule("colored", np.zeros(A.n, dtype=np.int32))


@pytest.mark.parametrize("mode", ["cold", "warm"])
def test_colored_vcycle_matches_oracle(g, mode):
    levels, sides, b = _hierarchy()
    mo = oracle.MGOracle(levels, sides, mode=mode, ncolors=4)
    solvers = [g.GabpSolver(A, "fp64") for A in levels]
    mg = g.Multigrid(solvers, sides, mode=mode, schedule="colored")
    xo = np.zeros(levels[0].n)
    xg = torch.zeros(levels[0].n, dtype=torch.float64, device="cuda")
    bd = dev(b)
    for cyc in range(3):
        xo = mo.vcycle(b, xo, 2, 2)
        mg.vcycle(bd, xg, 2, 2)
        assert rel(host(xg), xo) <= 1e-11, f"cycle {cyc}"


def test_colored_mg_solve_converges_faster(g):
    levels, sides, b = _hierarchy()
    ref = oracle.MGOracle(levels, sides, ncolors=4).solve(b, 1e-10, 200, 2, 2)
    assert ref["status"] == oracle.OK
    solvers = [g.GabpSolver(A, "fp64") for A in levels]
    mg = g.Multigrid(solvers, sides, schedule="colored")
    x, c, rr, st = mg.solve(dev(b), 1e-10, 200, 2, 2)
    assert st == g.OK and c == ref["cycles"]
    assert rel(host(x), ref["x"]) <= 1e-9


# --------------------------------------------------------------------------
# float messages and mixed precision
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["c1_32", "lognormal_33", "aniso9_31", "random_300"])
def test_fp32_sweeps_error_against_oracle(g, name):
    """Float messages: 50 sweeps stay within 1e-5 relative of the FP64 oracle."""
    A = MATS[name]
    b = _rhs(A.n, 9)
    lt, mm = oracle.zero_state(A)
    x_o, _, _ = oracle.sweeps(A, b, 50, lt, mm)
    s = g.GabpSolver(A, "fp32")
    x = host(s.sweep(dev(b), 50))
    assert rel(x, x_o) <= 1e-5


@pytest.mark.parametrize("freeze", [-1, 0])
@pytest.mark.parametrize("name", ["c1_32", "lognormal_33", "aniso9_31", "random_300"])
def test_mixed_precision_reaches_1e10(g, name, freeze):
    A = MATS[name]
    b = _rhs(A.n, 10)
    s = g.GabpSolver(A, "fp32_ir", check_every=5, freeze_lambda=freeze)
    x, it, rr, st = s.solve(dev(b), 1e-10, 20000)
    assert st == g.OK and rr <= 1e-10
    xs = np.linalg.solve(A.to_dense(), b)
    r = b - A.to_dense() @ host(x)
    assert np.max(np.abs(r)) / np.max(np.abs(b)) <= 1.05e-10
    assert rel(host(x), xs) <= 1e-8


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["c1_32", "lognormal_33", "random_300", "figure_4x4"])
def test_transpose_solve_matches_oracle(g, name):
    A = MATS[name]
    AT = A.transpose()
    gvec = _rhs(A.n, 11)
    ref = oracle.solve(AT, gvec, 1e-10, 3000)
    assert ref["status"] == oracle.OK
    s = g.GabpSolver(A, "fp64", check_every=1)
    lam, it, rr, st = s.solve_transpose(dev(gvec), 1e-10, 3000)
    assert st == g.OK and it == ref["iters"]
    assert rel(host(lam), ref["x"]) <= 1e-10


def test_edge_grad_matches_definition(g):
    A = MATS["random_300"]
    b, gv = _rhs(300, 12), _rhs(300, 13)
    x, lam, dA = oracle.adjoint(A, b, gv)
    s = g.GabpSolver(A, "fp64")
    out = host(s.edge_grad(dev(lam), dev(x)))
    np.testing.assert_array_equal(out, dA)


# --------------------------------------------------------------------------
# multigrid
# --------------------------------------------------------------------------
def _hierarchy(mf=31, mc=7, seed=5):
    return P.config_c3_levels(m_fine=mf, m_coarse=mc, seed=seed)


@pytest.mark.parametrize("mode", ["cold", "warm", "persist"])
def test_vcycle_matches_oracle(g, mode):
    levels, sides, b = _hierarchy()
    mo = oracle.MGOracle(levels, sides, mode=mode)
    solvers = [g.GabpSolver(A, "fp64") for A in levels]
    mg = g.Multigrid(solvers, sides, mode=mode)
    xo = np.zeros(levels[0].n)
    xg = torch.zeros(levels[0].n, dtype=torch.float64, device="cuda")
    bd = dev(b)
    for cyc in range(3):
        xo = mo.vcycle(b, xo, 2, 2)
        mg.vcycle(bd, xg, 2, 2)
        assert rel(host(xg), xo) <= 1e-11, f"cycle {cyc}"


def test_mg_solve_cold_matches_oracle(g):
    levels, sides, b = _hierarchy()
    ref = oracle.MGOracle(levels, sides).solve(b, 1e-10, 200, 3, 3)
    assert ref["status"] == oracle.OK
    solvers = [g.GabpSolver(A, "fp64") for A in levels]
    mg = g.Multigrid(solvers, sides)
    x, c, rr, st = mg.solve(dev(b), 1e-10, 200, 3, 3)
    assert st == g.OK and c == ref["cycles"]
    assert rel(host(x), ref["x"]) <= 1e-9


def test_mg_float_smoothing_error_stated(g):
    """Float smoothing, double residuals: one cycle within 1e-5 of the FP64 oracle."""
    levels, sides, b = _hierarchy()
    xo = oracle.MGOracle(levels, sides).vcycle(b, np.zeros(levels[0].n), 2, 2)
    solvers = [g.GabpSolver(A, "fp32") for A in levels]
    mg = g.Multigrid(solvers, sides)
    xg = torch.zeros(levels[0].n, dtype=torch.float64, device="cuda")
    mg.vcycle(dev(b), xg, 2, 2)
    assert rel(host(xg), xo) <= 1e-5


# --------------------------------------------------------------------------
# full size (2048 x 2048 convection-diffusion, the bench workload)
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c2():
    return P.config_c2()


def _third_sweep(A, b):
    """Oracle beliefs of sweep 3 and the state after it, with the element-wise
    scales of that sweep (taken from the state after two sweeps)."""
    lt, mm = oracle.zero_state(A)
    oracle.sweeps(A, b, 2, lt, mm)
    x_o, beta_o = oracle.beliefs(A, b, lt, mm)
    lt3, mm3, st = oracle.update(A, b, lt, mm)
    assert st == oracle.OK
    lc, lc3 = oracle.diag_contrib(A, lt), oracle.diag_contrib(A, lt3)
    return x_o, lc3, mm3, sweep_scales(A, b, lc, mm, x_o, beta_o, lc3, mm3)


def test_fullsize_first_sweeps_elementwise(g, c2):
    """Three sweeps of the 2048^2 workload: beliefs, precision and mean messages
    against the oracle, normwise and element by element."""
    A, b = c2
    x_o, lc3, mm3, (sx, sl, sm) = _third_sweep(A, b)
    s = g.GabpSolver(A, "fp64")
    assert s.info()["layout"] == "stencil"
    x = host(s.sweep(dev(b), 3))
    lam, m = (host(t) for t in s.get_state())
    assert rel(x, x_o) <= 1e-12
    assert rel(lam, lc3) <= 1e-12
    assert rel(m, mm3) <= 1e-12
    assert worst_elementwise(x, x_o, sx) <= 1e-12
    assert worst_elementwise(lam, lc3, sl) <= 1e-12
    assert worst_elementwise(m, mm3, sm) <= 1e-12
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_ir"])
def test_fullsize_solve_reaches_1e10(g, c2, precision):
    A, b = c2
    s = g.GabpSolver(A, precision)
    x, it, rr, st = s.solve(dev(b), 1e-10, 20000)
    assert st == g.OK and rr <= 1e-10
    xh = host(x)
    r = b - A.matvec(xh)  # independent residual on the host
    assert np.max(np.abs(r)) / np.max(np.abs(b)) <= 1.05e-10


@pytest.fixture(scope="module")
def c2_fp64(g, c2):
    """FP64 GaBP solution of the full-size system, its residual, and an upper bound
    on ||A^{-1}||_inf from y = A^{-1} 1 (A is an M-matrix, so A^{-1} >= 0 and
    ||A^{-1}||_inf = ||A^{-1} 1||_inf <= ||y||_inf / (1 - ||1 - A y||_inf))."""
    A, b = c2
    s = g.GabpSolver(A, "fp64")
    x, _, _, st = s.solve(dev(b), 1e-10, 20000)
    assert st == g.OK
    y, _, _, st = s.solve(dev(np.ones(A.n)), 1e-10, 20000)
    assert st == g.OK
    y = host(y)
    assert np.min(y) > 0
    ry = np.max(np.abs(1.0 - A.matvec(y)))
    xh = host(x)
    s.close()
    return xh, np.max(np.abs(b - A.matvec(xh))), np.max(y) / (1.0 - ry)


@pytest.mark.parametrize("schedule", ["flood", "lines"])
def test_fullsize_mixed_solution_within_forward_error_bound(g, c2, c2_fp64, schedule):
    """The mixed-precision solution differs from the FP64 one by no more than
    ||A^{-1}||_inf (||r_mixed||_inf + ||r_fp64||_inf), with residuals taken on the host."""
    A, b = c2
    x64, r64, inv_norm = c2_fp64
    s = g.GabpSolver(A, "fp32_ir", check_every=10)
    if schedule == "lines":
        s.set_schedule("lines")
    x, _, rr, st = s.solve(dev(b), 1e-10, 20000)
    assert st == g.OK
    xh = host(x)
    r = np.max(np.abs(b - A.matvec(xh)))
    assert r / np.max(np.abs(b)) <= 1.05e-10
    err = np.max(np.abs(xh - x64))
    assert err <= inv_norm * (r + r64)
    s.close()


# --------------------------------------------------------------------------
# exponent range of the double-precision reciprocal
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec,k", [("fp64", -400), ("fp64", 400), ("fp32", -40), ("fp32", 40)])
@pytest.mark.parametrize("name,layout,schedule", [
    ("lognormal_33", "auto", "flood"), ("lognormal_33", "csr", "flood"),
    ("random_300", "csr", "flood"), ("lognormal_33", "auto", "colored"),
    ("lognormal_33", "auto", "lines")])
def test_power_of_two_scaling_is_exact(g, name, layout, schedule, prec, k):
    """With A, b scaled by s = 2^k the update rules (eq. nonsymmetric_GaBP_rules)
    scale exactly: c by s^2, a, P, B, d and the stored messages by s, the beliefs
    not at all.  Every reciprocal then sees a denominator with the same significand
    and an exponent shifted by k, so in double precision the beliefs are bitwise
    equal and the messages equal after division by s; k = +-400 takes the
    denominators across most of the double exponent range.  In float (k = +-40,
    pivots near 2^52 and 2^-28) the results agree to the float rounding of the
    hardware reciprocal approximation; the line recurrences, whose products of a
    few pivots would leave the float range unscaled, must stay finite."""
    A = MATS[name]
    b = _rhs(A.n, 3)
    s = math.ldexp(1.0, k)
    As = P.CSR(A.n, A.indptr, A.indices, A.data * s)
    outs = []
    for M, rhs in ((A, b), (As, b * s)):
        sv = g.GabpSolver(M, prec, layout=layout)
        if schedule != "flood":
            sv.set_schedule(schedule)
        x = host(sv.sweep(dev(rhs), 20))
        st = None if schedule == "lines" else tuple(host(t) for t in sv.get_state())
        outs.append((x, st))
        sv.close()
    (x0, st0), (x1, st1) = outs
    assert np.all(np.isfinite(x0)) and np.all(np.isfinite(x1)) and np.max(np.abs(x0)) > 0
    if prec == "fp64":
        np.testing.assert_array_equal(x1, x0)
    else:
        assert rel(x1, x0) <= 1e-5
    if st0 is not None:
        for u0, u1 in zip(st0, st1):
            if prec == "fp64":
                np.testing.assert_array_equal(u1 / s, u0)
            else:
                assert rel(u1 / s, u0) <= 1e-5


# --------------------------------------------------------------------------
# the 2-norm residual logged beside the infinity norm
# --------------------------------------------------------------------------
@pytest.mark.parametrize("layout,reorder", [("auto", -1), ("csr", 1)])
def test_residual_2norm(g, layout, reorder):
    """gabp_residual_2norm against the host: ||b - A x||_2 / ||b||_2 of an
    iterate far from convergence (no cancellation, so the two agree to rounding),
    bitwise repeatable, and the same through an internally renumbered context."""
    A = MATS["random_300"] if layout == "csr" else MATS["lognormal_33"]
    b = _rhs(A.n, 8)
    s = g.GabpSolver(A, "fp64", layout=layout, reorder=reorder)
    x = s.sweep(dev(b), 4)
    xh = host(x)
    ref = np.linalg.norm(b - A.matvec(xh)) / np.linalg.norm(b)
    r1 = s.residual_norms(dev(b), x)
    r2 = s.residual_norms(dev(b), x)
    assert r1 == r2
    assert r1["rr_2"] == pytest.approx(ref, rel=1e-12)
    assert r1["rr_inf"] == pytest.approx(np.max(np.abs(b - A.matvec(xh))) / np.max(np.abs(b)), rel=1e-12)
    s.close()


@pytest.mark.parametrize("precision,schedule", [("fp64", "flood"), ("fp32_ir", "colored"), ("fp32_ir", "lines")])
def test_side_stream_matches_default_stream(g, precision, schedule):
    """The library on a stream of its own (eager sweeps launched with
    programmatic dependent launch, graph-replayed solve chunks) gives the bits
    it gives on the default stream."""
    A = MATS["c1_32"]
    b = _rhs(A.n, 50)
    bd = dev(b)
    torch.cuda.synchronize()
    ref = g.GabpSolver(A, precision)
    if schedule != "flood":
        ref.set_schedule(schedule)
    x0 = host(ref.sweep(bd, 7))
    xs0, it0, rr0, st0 = ref.solve(bd, 1e-10, 20000)
    side = torch.cuda.Stream()
    s = g.GabpSolver(A, precision, stream=side)
    if schedule != "flood":
        s.set_schedule(schedule)
    with torch.cuda.stream(side):
        x1 = s.sweep(bd, 7)
        xs1, it1, rr1, st1 = s.solve(bd, 1e-10, 20000)
    side.synchronize()
    assert st0 == st1 == g.OK and it0 == it1
    assert np.array_equal(host(x1), x0)
    assert torch.equal(xs1, xs0)
    ref.close()
    s.close()
