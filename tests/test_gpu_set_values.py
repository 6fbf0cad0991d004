"""New matrix values on a fixed pattern: gabp_set_values (host values) and
gabp_set_values_device (device values) give the same contexts, for every
layout, precision and schedule, and the new values reach every derived
coefficient copy (transposed, parity-class, line couplings)."""
import math

import numpy as np
import pytest

import oracle
import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HV = (2.0 * math.cos(0.3), 2.0 * math.sin(0.3))


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


def _pair(m=24, seed=3):
    rng = np.random.default_rng(seed)
    A0 = P.convdiff_5pt(m, P.lognormal_field(m, 0.5, rng), HV)
    A1 = P.convdiff_5pt(m, P.lognormal_field(m, 0.5, rng), HV)
    assert np.array_equal(A0.indices, A1.indices)
    return A0, A1, m


# the coloured and line schedules on grids run on the stencil-derived layouts
@pytest.mark.parametrize("layout,schedule", [("stencil", "flood"), ("csr", "flood"),
                                             ("stencil", "colored"), ("stencil", "lines")])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_device_values_equal_host_values(g, precision, layout, schedule):
    A0, A1, m = _pair()
    b = np.random.default_rng(1).uniform(-1, 1, A0.n)
    outs = []
    for path in ("host", "device"):
        s = g.GabpSolver(A0, precision, layout=layout)
        if schedule != "flood":
            s.set_schedule(schedule)
        s.sweep(dev(b), 2)
        s.set_values(A1.data if path == "host" else dev(A1.data))
        x = host(s.sweep(dev(b), 7))
        lam, mm = s.get_state() if schedule != "lines" else (None, None)
        outs.append((x, None if lam is None else host(lam), None if mm is None else host(mm)))
        s.close()
    for u, v in zip(outs[0], outs[1]):
        if u is not None:
            np.testing.assert_array_equal(u, v)


@pytest.mark.parametrize("path", ["host", "device"])
def test_new_values_reach_the_line_schedule(g, path):
    """After new values the line sweeps are those of the new matrix (the line
    couplings are rebuilt), checked against the oracle."""
    A0, A1, m = _pair(m=17, seed=9)
    b = np.random.default_rng(2).uniform(-1, 1, A0.n)
    s = g.GabpSolver(A0, "fp64")
    s.set_schedule("lines")
    s.sweep(dev(b), 3)
    s.set_values(A1.data if path == "host" else dev(A1.data))
    x = host(s.sweep(dev(b), 5))
    st = oracle.line_zero_state(A1.n)
    x_o = oracle.line_sweeps(A1, m, b, 5, st)
    assert rel(x, x_o) <= 1e-12


@pytest.mark.parametrize("path", ["host", "device"])
def test_new_values_reach_the_transposed_solve(g, path):
    A0, A1, m = _pair(m=20, seed=5)
    gv = np.random.default_rng(4).uniform(-1, 1, A0.n)
    s = g.GabpSolver(A0, "fp64", check_every=1)
    s.solve_transpose(dev(gv), 1e-10, 5000)  # builds the transposed coefficients
    s.set_values(A1.data if path == "host" else dev(A1.data))
    lam, it, rr, st = s.solve_transpose(dev(gv), 1e-10, 5000)
    ref = oracle.solve(A1.transpose(), gv, 1e-10, 5000)
    assert st == g.OK and it == ref["iters"]
    assert rel(host(lam), ref["x"]) <= 1e-10


def test_device_values_are_validated(g):
    A0, _, _ = _pair()
    s = g.GabpSolver(A0, "fp64")
    bad = A0.data.copy()
    rows = np.repeat(np.arange(A0.n), np.diff(A0.indptr))
    bad[np.flatnonzero(rows == A0.indices)[3]] = 0.0  # a zero diagonal
    with pytest.raises(g.GabpError) as e:
        s.set_values(dev(bad))
    assert e.value.status == g.ZERO_DIAG
    bad = A0.data.copy()
    bad[5] = float("nan")
    with pytest.raises(g.GabpError) as e:
        s.set_values(dev(bad))
    assert e.value.status == g.BAD_CSR


def test_differentiable_solve_with_device_assembly(g):
    """A(theta) assembled on the GPU and passed as device values gives the
    gradient of the host-assembled path."""
    from paper_1904_04093_gb300.autograd import gabp_solve
    m = 24
    theta, b, theta_t = P.config_c5(m=m)
    xt = np.linalg.solve(P.convdiff_5pt(m, np.exp(theta_t), HV).to_dense(), b)
    grads = []
    for where in ("cpu", "cuda"):
        asm = P.ConvDiff5ptTorch(m, HV)
        solver = g.GabpSolver(asm.pattern, "fp64", check_every=1)
        th = torch.tensor(theta, dtype=torch.float64, device=where, requires_grad=True)
        x = gabp_solve(asm.values(torch.exp(th)), dev(b), solver, tol=1e-12)
        L = ((x - dev(xt)) ** 2).sum()
        L.backward()
        grads.append(th.grad.detach().cpu().numpy())
        solver.close()
    assert rel(grads[1], grads[0]) <= 1e-12
