"""Batched persistent solver: every system of a batch equals its single solve,
and matches the FP64 oracle."""
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


def _systems(nsys=9, smin=16, smax=41, seed=7):
    # uneven sides (ragged against every block size), as in the batched workload
    return P.config_c4_batch(nsys=nsys, smin=smin, smax=smax, seed=seed)


@pytest.mark.parametrize("shape", [(256, 1), (256, 2), (512, 4), (256, 8)])
@pytest.mark.parametrize("check_every", [1, 7])
def test_batch_equals_single_solves(g, check_every, shape):
    systems = _systems()
    solvers = [g.GabpSolver(A, "fp64", check_every=check_every) for A, _ in systems]
    batch = g.Batch(solvers, check_every=check_every)
    batch.set_shape(*shape)
    bs = [dev(b) for _, b in systems]
    xs, its, rrs, sts = batch.solve(bs, 1e-10, 5000)
    assert all(s == g.OK for s in sts)
    for (A, b), x, it, rr in zip(systems, xs, its, rrs):
        single = g.GabpSolver(A, "fp64", check_every=check_every)
        xs1, it1, rr1, st1 = single.solve(dev(b), 1e-10, 5000)
        assert st1 == g.OK and it == it1
        assert rr == pytest.approx(rr1, rel=1e-12)
        assert rel(host(x), host(xs1)) <= 1e-14


@pytest.mark.parametrize("rows,min_rows", [(2, 4), (2, 2), (1, 8)])
def test_batch_params_keep_single_solve_iterates(g, rows, min_rows):
    """Two rows in flight per thread in the mean-message sweeps, and other
    thresholds for cluster teams, leave each system's iterates those of
    gabp_solve (frozen precision messages on, so the mean sweeps run)."""
    systems = _systems(nsys=7, smin=16, smax=72, seed=23)
    solvers = [g.GabpSolver(A, "fp64", check_every=5, freeze_lambda=1) for A, _ in systems]
    batch = g.Batch(solvers, check_every=5)
    batch.set_shape(256, 2)
    batch.set_params(rows=rows, min_rows=min_rows)
    info = batch.info()
    assert info["rows"] == rows and info["min_rows"] == min_rows and info["check_every"] == 5
    xs, its, rrs, sts = batch.solve([dev(b) for _, b in systems], 1e-10, 5000)
    assert all(s == g.OK for s in sts)
    ref = g.Batch([g.GabpSolver(A, "fp64", check_every=5, freeze_lambda=1) for A, _ in systems],
                  check_every=5)
    ref.set_shape(256, 2)
    x1, it1, rr1, st1 = ref.solve([dev(b) for _, b in systems], 1e-10, 5000)
    assert its == it1
    for a, b_ in zip(xs, x1):
        assert torch.equal(a, b_)


def test_batch_rows_refused_for_other_stencils(g):
    A = P.tridiag(64, 2.0, -1.0, -0.5)  # two diagonals
    batch = g.Batch([g.GabpSolver(A, "fp64", layout="stencil")], check_every=5)
    with pytest.raises(g.GabpError):
        batch.set_params(rows=2)


def test_batch_matches_oracle(g):
    """Tuned on its first solve: an explicit check interval (here 1) is kept."""
    systems = _systems(nsys=5, seed=11)
    solvers = [g.GabpSolver(A, "fp64", check_every=1) for A, _ in systems]
    batch = g.Batch(solvers, check_every=1)
    xs, its, rrs, sts = batch.solve([dev(b) for _, b in systems], 1e-10, 5000)
    for (A, b), x, it, st in zip(systems, xs, its, sts):
        ref = oracle.solve(A, b, 1e-10, 5000)
        assert st == g.OK and it == ref["iters"]
        assert rel(host(x), ref["x"]) <= 1e-10


def test_batch_float_plain(g):
    """Float messages without refinement: the float beliefs bound the attainable
    residual, so the target here is 1e-4."""
    systems = _systems(nsys=6, smin=16, smax=40, seed=17)
    solvers = [g.GabpSolver(A, "fp32") for A, _ in systems]
    batch = g.Batch(solvers, check_every=10)
    xs, its, rrs, sts = batch.solve([dev(b) for _, b in systems], 1e-4, 20000)
    assert all(s == g.OK for s in sts)
    for (A, b), x in zip(systems, xs):
        xh = host(x)
        assert np.max(np.abs(b - A.matvec(xh))) / np.max(np.abs(b)) <= 1.01e-4


def test_batch_float_workload_tolerance(g):
    """Float messages inside double refinement, per-system stop at rr <= 1e-6
    (the batched workload's target)."""
    systems = _systems(nsys=12, smin=16, smax=64, seed=13)
    solvers = [g.GabpSolver(A, "fp32_ir") for A, _ in systems]
    batch = g.Batch(solvers, check_every=0)  # the check interval tuned as well
    blk, cs = batch.tune([dev(b) for _, b in systems], 1e-6, 20000)
    assert blk in (256, 512) and cs in (1, 2, 4, 8, 16)
    info = batch.info()
    assert info["rows"] in (1, 2) and info["min_rows"] in (2, 4, 8) and info["check_every"] in (10, 20)
    xs, its, rrs, sts = batch.solve([dev(b) for _, b in systems], 1e-6, 20000)
    assert all(s == g.OK for s in sts)
    for (A, b), x, rr in zip(systems, xs, rrs):
        assert rr <= 1e-6
        xh = host(x)
        assert np.max(np.abs(b - A.matvec(xh))) / np.max(np.abs(b)) <= 1.01e-6
        xs_ = np.linalg.solve(A.to_dense(), b)
        assert rel(xh, xs_) <= 1e-4


def test_batch_edge_cases(g):
    # a 2x2 grid, a zero right-hand side, and a sweep cap that stops a system
    A1 = P.convdiff_5pt(2, None, (0.3, 0.1))
    b1 = np.array([1.0, -2.0, 0.5, 3.0])
    A2, b2 = P.config_c1(m=17)
    solvers = [g.GabpSolver(A1, "fp64"), g.GabpSolver(A2, "fp64"), g.GabpSolver(A2, "fp64")]
    batch = g.Batch(solvers, check_every=4)
    bs = [dev(b1), dev(np.zeros(A2.n)), dev(b2)]
    xs, its, rrs, sts = batch.solve(bs, 1e-12, 100000)
    assert sts == [g.OK, g.OK, g.OK]
    assert rel(host(xs[0]), np.linalg.solve(A1.to_dense(), b1)) <= 1e-12
    assert its[1] == 0 and np.all(host(xs[1]) == 0.0)
    xs, its, rrs, sts = batch.solve(bs, 1e-12, 6)
    assert sts[2] == g.NOT_CONVERGED and its[2] == 6
    lt, mm = oracle.zero_state(A2)
    x_o, _, _ = oracle.sweeps(A2, b2, 6, lt, mm)
    assert rel(host(xs[2]), x_o) <= 1e-12


def test_batch_frozen_precision_messages_match_single(g):
    """With freeze_lambda the batched systems freeze their precision messages at
    the same check as gabp_solve does and follow the same iterates."""
    systems = _systems(nsys=6, seed=19)
    solvers = [g.GabpSolver(A, "fp64", check_every=5, freeze_lambda=1) for A, _ in systems]
    batch = g.Batch(solvers, check_every=5)
    batch.set_shape(256, 2)
    xs, its, rrs, sts = batch.solve([dev(b) for _, b in systems], 1e-10, 5000)
    assert all(s == g.OK for s in sts)
    for (A, b), x, it in zip(systems, xs, its):
        single = g.GabpSolver(A, "fp64", check_every=5, freeze_lambda=1)
        x1, it1, rr1, st1 = single.solve(dev(b), 1e-10, 5000)
        assert st1 == g.OK and abs(it - it1) <= 5
        assert rel(host(x), host(x1)) <= 1e-9


def _divergent_5pt():
    """A 6 x 6 5-point matrix (unit diagonal, couplings U(-0.8, 0.8), seed 2) on
    which flood GaBP diverges (found with the oracle)."""
    m = 6
    rng = np.random.default_rng(2)
    c = np.empty((m, m, 5))
    c[:, :, 2] = 1.0
    for k in (0, 1, 3, 4):
        c[:, :, k] = rng.uniform(-0.8, 0.8, (m, m))
    A = P.stencil_csr(m, P._OFF5, c)
    b = rng.uniform(-1, 1, m * m)
    return A, b


def test_batch_faults_stay_per_system(g):
    """A breakdown and a divergence in a batch are reported for their own systems;
    the other systems still converge."""
    Ad, bd_ = _divergent_5pt()
    assert oracle.solve(Ad, bd_, 1e-12, 3000)["status"] == oracle.DIVERGED
    Ab = P.dense_to_csr(np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 0.0], [1.0, 0.0, 1.0]]))
    bb = np.array([1.0, 2.0, 3.0])
    assert oracle.solve(Ab, bb, 1e-12, 50)["status"] == oracle.BREAKDOWN
    Ag, bg = P.config_c1(m=20)
    systems = [(Ag, bg), (Ad, bd_), (Ab, bb), (Ag, bg)]
    solvers = [g.GabpSolver(A, "fp64", layout="stencil") for A, _ in systems]
    batch = g.Batch(solvers, check_every=5)
    xs, its, rrs, sts = batch.solve([dev(b) for _, b in systems], 1e-10, 3000)
    assert sts == [g.OK, g.DIVERGED, g.BREAKDOWN, g.OK]
    xs_ = np.linalg.solve(Ag.to_dense(), bg)
    assert rel(host(xs[0]), xs_) <= 1e-8 and rel(host(xs[3]), xs_) <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
@pytest.mark.parametrize("m,shape", [(20, (256, 1)), (96, (256, 2)), (96, (512, 4))])
def test_batch_breakdown_after_passed_checks(g, prec, m, shape):
    """A breakdown that first appears after two passed residual checks.

    problems.late_breakdown_tree is a non-singular matrix whose first zero
    denominator comes at sweep a + 1 = 15 (pinned on the oracle in
    test_oracle_pins); with checks every 5 sweeps the checks after sweeps 5 and
    10 pass and the breakdown is set inside the third chunk.  The system
    returns BREAKDOWN after 15 sweeps, its neighbours in the batch converge to
    their single-solve results.  At m = 96 the system is solved by a whole
    cluster (at least 4 rows per cluster thread), at m = 20 by one CTA."""
    a = 14
    Ab = P.late_breakdown_tree(m, a, a + 2)
    bb = np.random.default_rng(5).uniform(-1, 1, Ab.n)
    ref = oracle.solve(Ab, bb, 1e-12, 100)
    assert ref["status"] == oracle.BREAKDOWN and ref["iters"] == a + 1
    Ag, bg = P.config_c1(m=20)
    systems = [(Ag, bg), (Ab, bb), (Ag, bg)]
    solvers = [g.GabpSolver(A, prec, layout="stencil", check_every=5) for A, _ in systems]
    batch = g.Batch(solvers, check_every=5)
    batch.set_shape(*shape)
    xs, its, rrs, sts = batch.solve([dev(b) for _, b in systems], 1e-10, 3000)
    assert sts == [g.OK, g.BREAKDOWN, g.OK]
    assert its[1] == a + 1
    single = g.GabpSolver(Ab, prec, layout="stencil", check_every=5)
    _, it1, _, st1 = single.solve(dev(bb), 1e-10, 3000)
    assert st1 == g.BREAKDOWN and it1 == a + 1
    for i in (0, 2):
        s1 = g.GabpSolver(Ag, prec, layout="stencil", check_every=5)
        x1, it1, _, st1 = s1.solve(dev(bg), 1e-10, 3000)
        assert st1 == g.OK and its[i] == it1
        assert rel(host(xs[i]), host(x1)) <= 1e-14


@pytest.mark.parametrize("block", [256, 512])
def test_batch_sixteen_cta_clusters(g, block):
    """Clusters of 16 CTAs (the non-portable size): systems with at least 4
    rows per cluster thread (here 128^2 and 136^2 with 256 threads per CTA)
    are solved by a whole 16-CTA cluster, the rest by single CTAs; every
    system equals its single solve."""
    systems = P.config_c4_batch(nsys=3, smin=16, smax=40, seed=11)
    for side in (136, 128):
        A = P.convdiff_5pt(side, P.lognormal_field(side, 0.5, np.random.default_rng(side)), (1.0, 0.6))
        systems.append((A, np.random.default_rng(side + 1).uniform(-1, 1, A.n)))
    solvers = [g.GabpSolver(A, "fp64", check_every=5) for A, _ in systems]
    batch = g.Batch(solvers, check_every=5)
    try:
        batch.set_shape(block, 16)
    except g.GabpError:
        pytest.skip("16-CTA clusters of this block size cannot be resident")
    bs = [dev(b) for _, b in systems]
    xs, its, rrs, sts = batch.solve(bs, 1e-10, 20000)
    assert all(s == g.OK for s in sts)
    for (A, b), x, it in zip(systems, xs, its):
        single = g.GabpSolver(A, "fp64", check_every=5)
        xs1, it1, rr1, st1 = single.solve(dev(b), 1e-10, 20000)
        assert st1 == g.OK and it == it1
        assert rel(host(x), host(xs1)) <= 1e-14


def test_batch_full_workload(g):
    """The batched workload as the bench runs it: 512 systems with sides 16..256,
    float messages inside double refinement, the tuned launch shape, every system
    to rr <= 1e-6.  Every residual is recomputed on the host; on sampled systems
    (the largest, the smallest and three at random) the solution lies within the
    forward-error bound of a sparse direct solve: each system is an M-matrix, so
    ||A^{-1}||_inf = ||A^{-1} 1||_inf and ||x - x_direct||_inf <=
    ||A^{-1}||_inf (||r||_inf + ||r_direct||_inf)."""
    sp = pytest.importorskip("scipy.sparse")
    spla = pytest.importorskip("scipy.sparse.linalg")
    systems = P.config_c4_batch(nsys=512, smax=256)
    solvers = [g.GabpSolver(A, "fp32_ir") for A, _ in systems]
    bs = [dev(b) for _, b in systems]
    batch = g.Batch(solvers, check_every=0)  # as the bench runs it: check interval tuned too
    batch.tune(bs, 1e-6, 20000)
    xs, its, rrs, sts = batch.solve(bs, 1e-6, 20000)
    assert all(s == g.OK for s in sts)
    xh = [host(x) for x in xs]
    for (A, b), x in zip(systems, xh):
        assert np.max(np.abs(b - A.matvec(x))) / np.max(np.abs(b)) <= 1.01e-6
    sizes = [A.n for A, _ in systems]
    pick = {int(np.argmax(sizes)), int(np.argmin(sizes))}
    pick |= set(int(i) for i in np.random.default_rng(3).choice(len(systems), 3, replace=False))
    for i in sorted(pick):
        A, b = systems[i]
        lu = spla.splu(sp.csr_matrix((A.data, A.indices, A.indptr), shape=(A.n, A.n)).tocsc())
        xd, y = lu.solve(b), lu.solve(np.ones(A.n))
        assert np.min(y) > 0
        rb = np.max(np.abs(b - A.matvec(xh[i])))
        rd = np.max(np.abs(b - A.matvec(xd)))
        assert np.max(np.abs(xh[i] - xd)) <= np.max(y) * (rb + rd) * (1 + 1e-6)
