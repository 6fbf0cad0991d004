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
