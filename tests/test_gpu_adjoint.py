"""Differentiable solve: the adjoint (GaBP on A^T, dL/dA_ij = -lam_i x_j)
against a dense FP64 reference gradient and central finite differences.

Workload: upwind convection-diffusion with per-node diffusion kappa = exp(theta),
theta ~ N(0, 0.3^2), loss L = ||x - x_target||^2 with x_target the solution
for a second theta field.
"""
import math

import numpy as np
import pytest

import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HV = (2.0 * math.cos(0.3), 2.0 * math.sin(0.3))  # flow angle 0.3, cell Peclet 1


@pytest.fixture(scope="module")
def g():
    import paper_1904_04093_gb300 as g
    g.load()
    return g


def _workload(m, seed=1005):
    theta, b, theta_t = P.config_c5(m=m, seed=seed)
    At = P.convdiff_5pt(m, np.exp(theta_t), HV)
    x_target = np.linalg.solve(At.to_dense(), b) if m <= 48 else None
    return theta, b, theta_t, x_target


def _dense_reference(m, theta, b, x_target):
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    pattern, vals = P.convdiff_5pt_torch(m, torch.exp(th), HV)
    rows = torch.as_tensor(np.repeat(np.arange(pattern.n), np.diff(pattern.indptr)))
    cols = torch.as_tensor(pattern.indices.astype(np.int64))
    A = torch.zeros(pattern.n, pattern.n, dtype=torch.float64).index_put((rows, cols), vals)
    bt = torch.tensor(b, dtype=torch.float64, requires_grad=True)
    x = torch.linalg.solve(A, bt)
    L = ((x - torch.tensor(x_target)) ** 2).sum()
    L.backward()
    return float(L.detach()), th.grad.numpy().copy(), bt.grad.numpy().copy()


def _gabp_loss_grad(g, m, theta, b, x_target, precision, tol):
    from paper_1904_04093_gb300.autograd import gabp_solve
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    pattern, vals = P.convdiff_5pt_torch(m, torch.exp(th), HV)
    solver = g.GabpSolver(pattern, precision, check_every=10, freeze_lambda=1 if precision == "fp64" else -1)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda", requires_grad=True)
    x = gabp_solve(vals, bd, solver, tol=tol)
    L = ((x - torch.as_tensor(x_target, device="cuda")) ** 2).sum()
    L.backward()
    return float(L.detach()), th.grad.numpy().copy(), bd.grad.cpu().numpy().copy()


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-13, 1e-8), ("fp32_ir", 1e-11, 1e-6)])
def test_gradient_matches_dense_fp64_reference(g, precision, tol, bound):
    m = 32
    theta, b, theta_t, xt = _workload(m)
    L_ref, gth_ref, gb_ref = _dense_reference(m, theta, b, xt)
    L, gth, gb = _gabp_loss_grad(g, m, theta, b, xt, precision, tol)
    assert L == pytest.approx(L_ref, rel=bound)
    assert np.max(np.abs(gb - gb_ref)) <= bound * np.max(np.abs(gb_ref))
    assert np.max(np.abs(gth - gth_ref)) <= bound * np.max(np.abs(gth_ref))


def test_gradient_matches_central_differences(g):
    """Central differences of L(theta), step 1e-6, FP64 GaBP forward solves."""
    m = 24
    theta, b, theta_t, xt = _workload(m, seed=2005)
    L0, gth, _ = _gabp_loss_grad(g, m, theta, b, xt, "fp64", 1e-14)
    solver = None
    rng = np.random.default_rng(0)
    picks = [tuple(rng.integers(0, m, 2)) for _ in range(6)]
    step = 1e-6
    for (i, j) in picks:
        vals = []
        for sgn in (+1.0, -1.0):
            tp = theta.copy()
            tp[i, j] += sgn * step
            A = P.convdiff_5pt(m, np.exp(tp), HV)
            solver = g.GabpSolver(A, "fp64", check_every=10, freeze_lambda=1)
            x, it, rr, st = solver.solve(torch.as_tensor(b, device="cuda"), 1e-14, 200000)
            assert st == g.OK
            vals.append(float(((x.cpu().numpy() - xt) ** 2).sum()))
        fd = (vals[0] - vals[1]) / (2 * step)
        assert fd == pytest.approx(gth[i, j], rel=1e-5, abs=1e-7 * np.max(np.abs(gth)))


def test_full_size_workload_forward_backward(g):
    """512 x 512: mixed-precision forward and adjoint; a small step along the
    negative gradient lowers the loss as predicted to first order."""
    from paper_1904_04093_gb300.autograd import gabp_solve
    m = 512
    theta, b, theta_t, _ = _workload(m)
    At = P.convdiff_5pt(m, np.exp(theta_t), HV)
    st_solver = g.GabpSolver(At, "fp32_ir")
    bd = torch.as_tensor(b, device="cuda")
    xt, _, rr, st = st_solver.solve(bd, 1e-10, 200000)
    assert st == g.OK
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    pattern, vals = P.convdiff_5pt_torch(m, torch.exp(th), HV)
    solver = g.GabpSolver(pattern, "fp32_ir")
    x = gabp_solve(vals, bd, solver, tol=1e-10)
    L = ((x - xt) ** 2).sum()
    L.backward()
    grad = th.grad.numpy()
    assert np.all(np.isfinite(grad)) and np.max(np.abs(grad)) > 0
    eta = 1e-3 / np.max(np.abs(grad))
    with torch.no_grad():
        th2 = torch.tensor(theta - eta * grad)
        _, vals2 = P.convdiff_5pt_torch(m, torch.exp(th2), HV)
        x2 = gabp_solve(vals2, bd, solver, tol=1e-10)
        L2 = float(((x2 - xt) ** 2).sum())
    predicted = float(L) - eta * float(np.sum(grad * grad))
    assert L2 < float(L)
    assert abs(L2 - predicted) <= 0.05 * abs(float(L) - predicted)
