"""Line GaBP (Algorithm 2 with grid lines as large regions) on the GPU against the oracle."""
import numpy as np
import pytest

import oracle
import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def g():
    import paper_1904_04093_gb300 as g
    g.load()
    return g


def _cases():
    rng = np.random.default_rng(41)
    return {
        "c1_32": (P.config_c1()[0], 32),
        "lognormal_33": (P.convdiff_5pt(33, P.lognormal_field(33, 0.5, rng), (1.91, 0.59)), 33),
        "laplace_17": (P.convdiff_5pt(17, None, (0.0, 0.0)), 17),
    }


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_line_sweeps_match_oracle(g, name):
    A, m = CASES[name]
    b = np.random.default_rng(3).uniform(-1, 1, A.n)
    st = oracle.line_zero_state(A.n)
    s = g.GabpSolver(A, "fp64")
    s.set_schedule("lines")
    for nsw, tol in ((1, 1e-12), (19, 1e-10)):
        x_o = oracle.line_sweeps(A, m, b, nsw, st)
        x = host(s.sweep(dev(b), nsw))
        ls = {k: host(v) for k, v in s.get_line_state().items()}
        assert rel(x, x_o) <= tol
        for key in ("LH", "MH", "LV", "MV"):
            assert rel(ls[key], st[key]) <= tol, key


@pytest.mark.parametrize("name", ["c1_32", "lognormal_33"])
def test_line_solve_matches_oracle(g, name):
    A, m = CASES[name]
    b = np.random.default_rng(4).uniform(-1, 1, A.n)
    ref = oracle.line_solve(A, m, b, 1e-10, 2000)
    assert ref["status"] == oracle.OK
    s = g.GabpSolver(A, "fp64", check_every=1)
    s.set_schedule("lines")
    x, it, rr, st = s.solve(dev(b), 1e-10, 2000)
    assert st == g.OK and it == ref["iters"]
    assert rel(host(x), ref["x"]) <= 1e-10


def test_line_schedule_needs_five_point_grid(g):
    A = P.convdiff_9pt_aniso(15, 0.01, (0.5, 0.2))
    s = g.GabpSolver(A, "fp64")
    with pytest.raises(g.GabpError):
        s.set_schedule("lines")
    s2 = g.GabpSolver(P.random_m_matrix(50, 0.1, 3), "fp64")
    with pytest.raises(g.GabpError):
        s2.set_schedule("lines")


def test_line_float_error_stated(g):
    """Float lines: 20 sweeps within 1e-5 of the FP64 oracle."""
    A, m = CASES["lognormal_33"]
    b = np.random.default_rng(5).uniform(-1, 1, A.n)
    st = oracle.line_zero_state(A.n)
    x_o = oracle.line_sweeps(A, m, b, 20, st)
    s = g.GabpSolver(A, "fp32")
    s.set_schedule("lines")
    assert rel(host(s.sweep(dev(b), 20)), x_o) <= 1e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32_ir"])
def test_line_solve_full_size(g, precision):
    A, b = P.config_c2()
    s = g.GabpSolver(A, precision, check_every=10)
    s.set_schedule("lines")
    x, it, rr, st = s.solve(dev(b), 1e-10, 20000)
    assert st == g.OK and rr <= 1e-10
    r = b - A.matvec(host(x))
    assert np.max(np.abs(r)) / np.max(np.abs(b)) <= 1.05e-10


def test_line_float_large_rhs_multiwarp(g):
    """Float lines of 1024 nodes (chunks of eight, four warps per line) with a
    right-hand side of size ~200: the chunk products are rescaled by their
    pivot entries, so the eliminated right-hand side cannot push those to zero
    in the block scan.  The state stays finite and within float rounding of
    the double line sweeps (which the oracle pins at small sizes)."""
    m = 1024
    A, _ = P.config_c2(m=m, seed=77)
    b = np.random.default_rng(6).uniform(-200.0, 200.0, A.n)
    s64 = g.GabpSolver(A, "fp64")
    s64.set_schedule("lines")
    s32 = g.GabpSolver(A, "fp32")
    s32.set_schedule("lines")
    x64 = host(s64.sweep(dev(b), 30))
    x32 = host(s32.sweep(dev(b), 30))
    st64 = {k: host(v) for k, v in s64.get_line_state().items()}
    st32 = {k: host(v) for k, v in s32.get_line_state().items()}
    assert np.all(np.isfinite(x32))
    assert rel(x32, x64) <= 1e-4
    for key in ("LH", "MH", "LV", "MV"):
        assert np.all(np.isfinite(st32[key])), key
        assert rel(st32[key], st64[key]) <= 1e-4, key


@pytest.mark.parametrize("name", ["c1_32", "lognormal_33"])
def test_line_frozen_precision_messages_same_solution(g, name):
    """Precomputed precision messages (Sec. 4.2) under the line schedule:
    once Lambda stops changing, the sweeps move only the mean messages with
    the line's fixed elimination multipliers; the iterates are the plain
    line sweeps' up to rounding, so the solve needs the same sweep count."""
    A, m = CASES[name]
    b = np.random.default_rng(8).uniform(-1, 1, A.n)
    ref = oracle.line_solve(A, m, b, 1e-10, 2000)
    assert ref["status"] == oracle.OK
    s = g.GabpSolver(A, "fp64", check_every=1, freeze_lambda=1)
    s.set_schedule("lines")
    x, it, rr, st = s.solve(dev(b), 1e-10, 2000)
    assert st == g.OK and rr <= 1e-10
    assert abs(it - ref["iters"]) <= 1
    assert rel(host(x), ref["x"]) <= 1e-9
    # the frozen line sweeps can be timed; the messages they leave match the oracle's
    assert s.time_sweeps(dev(b), 3, frozen=True) > 0.0


def test_line_frozen_float_full_size_matches_double(g):
    """Float frozen line sweeps at 2048 x 2048 (the mixed solver's inner
    sweeps): the solve reaches 1e-10 through double refinement, and the frozen
    and unfrozen float line solves agree."""
    A, b = P.config_c2()
    s = g.GabpSolver(A, "fp32_ir", check_every=10, freeze_lambda=1)
    s.set_schedule("lines")
    x, it, rr, st = s.solve(dev(b), 1e-10, 20000)
    assert st == g.OK and rr <= 1e-10
    r = b - A.matvec(host(x))
    assert np.max(np.abs(r)) / np.max(np.abs(b)) <= 1.05e-10
    s0 = g.GabpSolver(A, "fp32_ir", check_every=10, freeze_lambda=0)
    s0.set_schedule("lines")
    x0, it0, rr0, st0 = s0.solve(dev(b), 1e-10, 20000)
    assert st0 == g.OK
    assert rel(host(x), host(x0)) <= 1e-8


@pytest.fixture(scope="module")
def long_lines():
    """A 4700 x 4700 grid: double lines of 4700 nodes exceed shared memory
    (the full phase runs on global memory) and split into chunks longer than
    16 (the frozen phase stages in shared memory)."""
    m = 4700
    A, b = P.config_c2(m=m, seed=4700)
    return A, b, m


def _line_slice(v, m, family, k):
    return v[k * m:(k + 1) * m] if family == "row" else v[k::m]


def test_long_lines_sampled_against_oracle(g, long_lines):
    """One more sweep from a GPU state, checked on sampled rows and columns
    against the oracle's update of those single regions (dense solves)."""
    A, b, m = long_lines
    s = g.GabpSolver(A, "fp64")
    s.set_schedule("lines")
    s.sweep(dev(b), 3)
    s3 = {k: host(v) for k, v in s.get_line_state().items()}
    x = host(s.sweep(dev(b), 1))
    s4 = {k: host(v) for k, v in s.get_line_state().items()}
    for k in (0, 2349, m - 1):
        lam, mu, _ = oracle.line_region_update(A, m, b, "row", k, s3["LV"], s3["MV"])
        assert rel(_line_slice(s4["LH"], m, "row", k), lam) <= 1e-12
        assert rel(_line_slice(s4["MH"], m, "row", k), mu) <= 1e-12
    for k in (1, 4000):
        lam, mu, xl = oracle.line_region_update(A, m, b, "col", k, s4["LH"], s4["MH"])
        assert rel(_line_slice(s4["LV"], m, "col", k), lam) <= 1e-12
        assert rel(_line_slice(s4["MV"], m, "col", k), mu) <= 1e-12
        assert rel(_line_slice(x, m, "col", k), xl) <= 1e-12
    s.close()


def test_long_lines_frozen_sweep_against_oracle(g, long_lines):
    """After the precision messages froze, one frozen sweep (mean messages
    only) agrees with the oracle's full update of sampled regions."""
    A, b, m = long_lines
    s = g.GabpSolver(A, "fp64", check_every=5, freeze_lambda=1)
    s.set_schedule("lines")
    _, it, _, st = s.solve(dev(b), 1e-30, 600)
    assert st == g.NOT_CONVERGED and it == 600
    before = {k: host(v) for k, v in s.get_line_state().items()}
    s.time_sweeps(dev(b), 1, frozen=True)  # raises unless the solve froze Lambda
    after = {k: host(v) for k, v in s.get_line_state().items()}
    for k in (7, 3333):
        lam, mu, _ = oracle.line_region_update(A, m, b, "row", k, before["LV"], before["MV"])
        assert rel(_line_slice(after["MH"], m, "row", k), mu) <= 1e-11
        assert rel(_line_slice(after["LH"], m, "row", k), lam) <= 1e-11
    lam, mu, _ = oracle.line_region_update(A, m, b, "col", 4699, after["LH"], after["MH"])
    assert rel(_line_slice(after["MV"], m, "col", 4699), mu) <= 1e-11
    s.close()


@pytest.mark.parametrize("freeze", [0, 1])
@pytest.mark.parametrize("name", ["c1_32", "lognormal_33"])
def test_line_transposed_solve_matches_oracle(g, name, freeze):
    """The adjoint solve under the line schedule: line GaBP on A^T (the same
    grid lines, couplings shifted to sup_{i-1}, sub_{i+1}) against the
    oracle's line solve of the transposed matrix, with and without frozen
    precision messages."""
    A, m = CASES[name]
    gvec = np.random.default_rng(12).uniform(-1, 1, A.n)
    ref = oracle.line_solve(A.transpose(), m, gvec, 1e-10, 2000)
    assert ref["status"] == oracle.OK
    s = g.GabpSolver(A, "fp64", check_every=1, freeze_lambda=freeze)
    s.set_schedule("lines")
    lam, it, rr, st = s.solve_transpose(dev(gvec), 1e-10, 2000)
    assert st == g.OK and abs(it - ref["iters"]) <= freeze
    assert rel(host(lam), ref["x"]) <= (1e-10 if freeze == 0 else 1e-9)
    # and the forward solve on the same context still is the forward one
    b = np.random.default_rng(13).uniform(-1, 1, A.n)
    fwd = oracle.line_solve(A, m, b, 1e-10, 2000)
    x, it2, _, st2 = s.solve(dev(b), 1e-10, 2000)
    assert st2 == g.OK and abs(it2 - fwd["iters"]) <= freeze
    assert rel(host(x), fwd["x"]) <= (1e-10 if freeze == 0 else 1e-9)


def test_line_differentiable_solve_full_size(g):
    """Forward and adjoint of the mixed solver under the line schedule at
    512 x 512: the gradient matches the flood schedule's."""
    from paper_1904_04093_gb300.autograd import gabp_solve
    import math
    m = 512
    hv = (2.0 * math.cos(0.3), 2.0 * math.sin(0.3))
    theta, b, _ = P.config_c5(m=m)
    xt = torch.zeros(m * m, dtype=torch.float64, device="cuda")
    grads = []
    for schedule in ("flood", "lines"):
        asm = P.ConvDiff5ptTorch(m, hv, device="cuda")
        solver = g.GabpSolver(asm.pattern, "fp32_ir", check_every=10)
        if schedule == "lines":
            solver.set_schedule("lines")
        th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
        x = gabp_solve(asm.values(torch.exp(th)), dev(b), solver, tol=1e-10)
        ((x - xt) ** 2).sum().backward()
        grads.append(host(th.grad))
    assert rel(grads[1], grads[0]) <= 1e-7


@pytest.mark.parametrize("m", [1, 2, 3, 5])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_line_tiny_grids(g, m, precision):
    """Lines shorter than a warp (one CTA of 32 threads, most chunks empty)
    and transposes of a single partial tile: sweeps against the oracle, and
    the solve with frozen precision messages reaches the dense solution."""
    A = P.convdiff_5pt(m, np.exp(np.random.default_rng(m).normal(0, 0.4, (m, m))), (0.7, -0.4))
    b = np.random.default_rng(30 + m).uniform(-1, 1, A.n)
    st = oracle.line_zero_state(A.n)
    x_o = oracle.line_sweeps(A, m, b, 4, st)
    s = g.GabpSolver(A, precision)
    s.set_schedule("lines")
    x = host(s.sweep(dev(b), 4))
    assert rel(x, x_o) <= (1e-12 if precision == "fp64" else 1e-5)
    s2 = g.GabpSolver(A, "fp64" if precision == "fp64" else "fp32_ir", check_every=1, freeze_lambda=1)
    s2.set_schedule("lines")
    xs, it, rr, st2 = s2.solve(dev(b), 1e-10, 500)
    assert st2 == g.OK and rr <= 1e-10
    assert rel(host(xs), np.linalg.solve(A.to_dense(), b)) <= 1e-9


@pytest.mark.parametrize("m", [20, 32, 45, 64, 300, 777, 1024, 1100, 2048, 2601, 4096])
def test_line_frozen_float_natural_columns_against_oracle(g, m):
    """Float frozen sweeps: up to 2048 nodes per line the column family is read
    and written in the natural node order (one CTA per 8 adjacent columns, a
    ragged last group at 20, 45, 777, 1100; every chunk whole, the unguarded
    form, at 32, 64, 1024, 2048; one warp per CTA at 20 and 32), beyond that
    through transposes (2601, 4096).  After the precision messages froze, one
    frozen sweep that writes no beliefs agrees on sampled lines with the
    oracle's full update of those regions from the same state (Algorithm 2;
    float rounding and the freeze threshold bound the difference); its row
    messages, which the natural-order phases hand over as b + m', read back as
    m'.  Then one full sweep (gabp_sweep) agrees too, beliefs included."""
    A, b = P.config_c2(m=m, seed=m)
    s = g.GabpSolver(A, "fp32", check_every=5, freeze_lambda=1)
    s.set_schedule("lines")
    _, it, _, st = s.solve(dev(b), 1e-30, 600)
    assert st == g.NOT_CONVERGED and it == 600
    s.time_sweeps(dev(b), 1, frozen=True)  # raises unless the solve froze Lambda
    prev = {k: host(v) for k, v in s.get_line_state().items()}
    s.time_sweeps(dev(b), 1, frozen=True)  # one frozen sweep, no beliefs written
    before = {k: host(v) for k, v in s.get_line_state().items()}
    cols = (0, m // 2 + 3, m - 1) if m <= 2601 else (5, m - 1)
    k = m // 3
    lam, mu, _ = oracle.line_region_update(A, m, b, "row", k, prev["LV"], prev["MV"])
    assert rel(_line_slice(before["MH"], m, "row", k), mu) <= 1e-4
    for kc in cols:
        lam, mu, _ = oracle.line_region_update(A, m, b, "col", kc, before["LH"], before["MH"])
        assert rel(_line_slice(before["MV"], m, "col", kc), mu) <= 1e-4
    x = host(s.sweep(dev(b), 1))
    after = {k: host(v) for k, v in s.get_line_state().items()}
    for kc in cols:
        lam, mu, xl = oracle.line_region_update(A, m, b, "col", kc, after["LH"], after["MH"])
        assert rel(_line_slice(after["MV"], m, "col", kc), mu) <= 1e-4
        assert rel(_line_slice(x, m, "col", kc), xl) <= 1e-4
    lam, mu, _ = oracle.line_region_update(A, m, b, "row", k, before["LV"], before["MV"])
    assert rel(_line_slice(after["MH"], m, "row", k), mu) <= 1e-4
    s.close()
