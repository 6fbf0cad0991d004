"""Multigrid at the benchmarked sizes, in the bench's configuration: float GaBP
smoothing with double residuals and transfers, cold smoother, V(2,2).

* 4095 x 4095 anisotropic 9-point hierarchy (eps = 0.01, 8 levels, 4-colour
  smoother, Sec. 5.1 with Algorithm 3);
* 2047 x 2047 5-point convection-diffusion hierarchy (7 levels, red-black
  smoother).

No oracle run fits these sizes, so the checks are properties that hold at any
size: the returned solution's residual recomputed on the host in FP64, and for
the 5-point system agreement with an independent solver (mixed-precision line
GaBP, Algorithm 2) within the forward-error bound of an M-matrix,
||x1 - x2||_inf <= ||A^{-1}||_inf (||r1||_inf + ||r2||_inf), with
||A^{-1}||_inf = ||A^{-1} 1||_inf since A^{-1} >= 0.
"""
import numpy as np
import pytest

import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rinf(A, b, x):
    return float(np.max(np.abs(b - A.matvec(x))))


@pytest.fixture(scope="module")
def g():
    import paper_1904_04093_gb300 as g
    g.load()
    return g


def test_mg_aniso9_4095_four_colour(g):
    levels, sides, b = P.config_c3_levels(m_fine=4095)
    assert sides == [4095, 2047, 1023, 511, 255, 127, 63, 31]
    solvers = [g.GabpSolver(A, "fp32") for A in levels]
    mg = g.Multigrid(solvers, sides, mode="cold", schedule="colored")
    x, cycles, rr, st = mg.solve(dev(b), 1e-10, 400, 2, 2)
    assert st == g.OK and rr <= 1e-10 and cycles <= 100
    assert rinf(levels[0], b, host(x)) / np.max(np.abs(b)) <= 1.05e-10
    mg.close()


def test_mg5_2047_red_black_against_line_gabp(g):
    levels, sides, b = P.config_c2_levels(m_fine=2047, m_coarse=31)
    A = levels[0]
    solvers = [g.GabpSolver(L, "fp32") for L in levels]
    mg = g.Multigrid(solvers, sides, mode="cold", schedule="colored")
    x, cycles, rr, st = mg.solve(dev(b), 1e-10, 200, 2, 2)
    assert st == g.OK and cycles <= 45
    x_mg = host(x)
    r_mg = rinf(A, b, x_mg)
    assert r_mg / np.max(np.abs(b)) <= 1.05e-10
    # ||A^{-1}||_inf from A y = 1, solved by the same cycles
    y, _, _, st = mg.solve(dev(np.ones(A.n)), 1e-10, 200, 2, 2)
    assert st == g.OK
    y = host(y)
    assert np.min(y) > 0
    inv_norm = np.max(y) / (1.0 - rinf(A, np.ones(A.n), y))
    mg.close()
    # an independent solver of the same system: mixed-precision line GaBP
    s = g.GabpSolver(A, "fp32_ir", check_every=10)
    s.set_schedule("lines")
    xl, _, _, st = s.solve(dev(b), 1e-10, 20000)
    assert st == g.OK
    x_ln = host(xl)
    r_ln = rinf(A, b, x_ln)
    assert np.max(np.abs(x_mg - x_ln)) <= inv_norm * (r_mg + r_ln)
    s.close()
