"""Multigrid on the rediscretised 5-point convection-diffusion hierarchy
(log-normal diffusion injected to the coarse nodes, grids of side 2^J - 1)
with red-black and line-GaBP smoothers (Algorithm 3 with the schedules of
Sec. 5.1 and Algorithm 2), against the oracle V-cycle."""
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


SMOOTHERS = {"colored": {"ncolors": 2}, "lines": {"lines": True}}


@pytest.mark.parametrize("nu", [(1, 1), (2, 1)])
@pytest.mark.parametrize("schedule", ["colored", "lines"])
@pytest.mark.parametrize("mode", ["cold", "warm"])
def test_vcycles_match_oracle(g, schedule, mode, nu):
    levels, sides, b = P.config_c2_levels(m_fine=31, m_coarse=7)
    mo = oracle.MGOracle(levels, sides, mode=mode, **SMOOTHERS[schedule])
    solvers = [g.GabpSolver(A, "fp64") for A in levels]
    mg = g.Multigrid(solvers, sides, mode=mode, schedule=schedule)
    xo = np.zeros(levels[0].n)
    xg = torch.zeros(levels[0].n, dtype=torch.float64, device="cuda")
    bd = dev(b)
    for cyc in range(3):
        xo = mo.vcycle(b, xo, *nu)
        mg.vcycle(bd, xg, *nu)
        assert rel(host(xg), xo) <= 1e-11, f"cycle {cyc}"


@pytest.mark.parametrize("schedule", ["colored", "lines"])
def test_mg_solve_matches_oracle(g, schedule):
    levels, sides, b = P.config_c2_levels(m_fine=63, m_coarse=15)
    ref = oracle.MGOracle(levels, sides, **SMOOTHERS[schedule]).solve(b, 1e-10, 100, 1, 1)
    assert ref["status"] == oracle.OK
    solvers = [g.GabpSolver(A, "fp64") for A in levels]
    mg = g.Multigrid(solvers, sides, schedule=schedule)
    x, c, rr, st = mg.solve(dev(b), 1e-10, 100, 1, 1)
    assert st == g.OK and c == ref["cycles"]
    assert rel(host(x), ref["x"]) <= 1e-9


def test_line_smoothed_mg_full_size(g):
    """Float line smoothing, double residuals and transfers at 1023^2: the
    V(1,1) solve reaches 1e-10 (checked on the host) in few cycles."""
    levels, sides, b = P.config_c2_levels(m_fine=1023, m_coarse=31)
    solvers = [g.GabpSolver(A, "fp32") for A in levels]
    mg = g.Multigrid(solvers, sides, schedule="lines")
    x, c, rr, st = mg.solve(dev(b), 1e-10, 100, 1, 1)
    assert st == g.OK and c <= 40
    r = b - levels[0].matvec(host(x))
    assert np.max(np.abs(r)) / np.max(np.abs(b)) <= 1.05e-10


@pytest.mark.parametrize("mode,nu", [("cold", (2, 1)), ("cold", (1, 1)), ("warm", (1, 1)),
                                     ("warm", (2, 1)), ("persist", (1, 2))])
def test_graph_replayed_cycles_match_oracle(g, mode, nu):
    """mg_solve replays its cycles from a captured graph where that is exact
    (cold smoothing, in-place schedules, an even number of sweeps per level)
    and runs them eagerly otherwise; either way four cycles of the solve are
    the oracle's four V-cycles (the warm and persist readings need not
    converge here: the cycles are compared, not the solution), a second solve
    reuses the graphs and continues like the oracle, and the finest level's
    context still solves on its own afterwards."""
    levels, sides, b = P.config_c2_levels(m_fine=31, m_coarse=7)
    mo = oracle.MGOracle(levels, sides, mode=mode)
    xo = np.zeros(levels[0].n)
    for _ in range(4):
        xo = mo.vcycle(b, xo, *nu)
    solvers = [g.GabpSolver(A, "fp64", check_every=1) for A in levels]
    mg = g.Multigrid(solvers, sides, mode=mode)
    x, c, rr, st = mg.solve(dev(b), 1e-30, 4, *nu)
    assert st == g.NOT_CONVERGED and c == 4
    assert rel(host(x), xo) <= 1e-11
    # a second solve reuses the graphs; in the warm and persist readings the
    # messages carry over from the first solve, as in the oracle
    xo2 = np.zeros(levels[0].n)
    for _ in range(4):
        xo2 = mo.vcycle(b, xo2, *nu)
    x2, c2, _, _ = mg.solve(dev(b), 1e-30, 4, *nu)
    assert c2 == 4 and rel(host(x2), xo2) <= 1e-11
    if mode == "cold":
        assert rel(host(x2), host(x)) <= 1e-13
    ref1 = oracle.solve(levels[0], b, 1e-10, 5000)
    x1, it1, _, st1 = solvers[0].solve(dev(b), 1e-10, 5000)
    assert st1 == g.OK and it1 == ref1["iters"]
