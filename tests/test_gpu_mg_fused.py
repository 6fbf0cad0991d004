"""Fused multigrid transfers (mg_set_fused) against one kernel per step.

The fused kernels compute the residual, the full-weighting restriction, the
bilinear prolongation and the corrections of the V-cycle (Sec. 4 with
Algorithm 3 as the smoother) in the order the separate kernels use, so both
paths give the same iterates: equal values after every cycle (a zero may
differ in sign, which compares equal), for every smoother schedule, both
precisions, every smoother mode, cycles without pre- or post-smoothing,
truncated hierarchies and the graph-replayed mg_solve.  The oracle parity of
the cycles themselves is tested in test_gpu_parity.py and test_gpu_mg5.py,
which run the fused path (the default).
"""
import numpy as np
import pytest

import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.fixture(scope="module")
def g():
    import paper_1904_04093_gb300 as g
    g.load()
    return g


def _pair(g, hierarchy, prec, schedule, mode):
    levels, sides, b = hierarchy
    out = []
    for fused in (False, True):
        solvers = [g.GabpSolver(A, prec) for A in levels]
        mg = g.Multigrid(solvers, sides, mode=mode, schedule=schedule)
        mg.set_fused(fused)
        out.append((mg, solvers))
    return out, dev(b)


def _h9():
    return P.config_c3_levels(m_fine=63, m_coarse=7, seed=5)


def _h5():
    return P.config_c2_levels(m_fine=63, m_coarse=7)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("schedule,hier", [("flood", "h9"), ("colored", "h9"), ("colored", "h5"),
                                           ("lines", "h5")])
@pytest.mark.parametrize("mode", ["cold", "warm"])
def test_fused_cycles_equal_separate(g, prec, schedule, hier, mode):
    h = _h9() if hier == "h9" else _h5()
    (pair, bd) = _pair(g, h, prec, schedule, mode)
    xs = [torch.zeros(h[0][0].n, dtype=torch.float64, device="cuda") for _ in pair]
    for nu in [(2, 2), (1, 0), (0, 1), (2, 1)]:
        for (mg, _), x in zip(pair, xs):
            mg.vcycle(bd, x, *nu)
        torch.cuda.synchronize()
        assert torch.equal(xs[0], xs[1]), nu
        assert torch.all(torch.isfinite(xs[1]))
    # a truncated hierarchy (the last used level smooths instead of solving)
    for (mg, _), x in zip(pair, xs):
        mg.vcycle(bd, x, 2, 2, levels=2)
    assert torch.equal(xs[0], xs[1])
    for mg, solvers in pair:
        mg.close()
        for s_ in solvers:
            s_.close()


@pytest.mark.parametrize("schedule,hier", [("colored", "h9"), ("colored", "h5"), ("lines", "h5")])
def test_fused_solve_equals_separate(g, schedule, hier):
    """mg_solve: the first cycle from x = 0, later cycles replayed from graphs
    that start from the convergence check's residual."""
    h = _h9() if hier == "h9" else _h5()
    (pair, bd) = _pair(g, h, "fp32", schedule, "cold")
    res = [mg.solve(bd, 1e-10, 60, 2, 2) for mg, _ in pair]
    (x0, c0, r0, s0), (x1, c1, r1, s1) = res
    assert s0 == s1 and c0 == c1 and r0 == r1
    assert torch.equal(x0, x1)
    for mg, solvers in pair:
        mg.close()


def test_fused_is_the_default_and_refused_when_impossible(g):
    """Grid levels get the fused path by default; a level on the CSR layout
    cannot (it has no grid stencil), so asking for it is refused."""
    levels, sides, b = P.config_c2_levels(m_fine=31, m_coarse=7)
    solvers = [g.GabpSolver(A, "fp64", layout="csr" if i == 1 else "auto")
               for i, A in enumerate(levels)]
    mg = g.Multigrid(solvers, sides)
    with pytest.raises(g.GabpError):
        mg.set_fused(True)
    mg.set_fused(False)
    x = torch.zeros(levels[0].n, dtype=torch.float64, device="cuda")
    mg.vcycle(dev(b), x, 1, 1)
    assert torch.all(torch.isfinite(x))
    mg.close()
