"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module builds sparse matrices and right-hand sides only.  It holds none
of the Gaussian belief propagation (GaBP) arithmetic: no message rule, no
belief, no residual loop.  Both sides of every parity test (the CPU oracle
under ``oracle/`` and the CUDA library) receive the same arrays from here.

Matrices are returned in CSR form with int64 row pointers, int32 column
indices sorted ascending within each row, float64 values, the diagonal always
stored.  Grid unknowns are numbered lexicographically, ``i = ix + m*iy`` with
``ix, iy`` in ``[0, m)``, on the unit square with ``m`` interior points per
side, mesh width ``h = 1/(m+1)`` and homogeneous Dirichlet boundaries.

Discretisation readings (the paper's experiments use second-order finite
differences on uniform grids of the unit square, Sec. 5, but leave the
details open):

* diffusion ``-div(D grad u)`` with a per-node coefficient ``D``; the
  coefficient on the face between two interior nodes is the harmonic mean of
  the two node values, on a face to the boundary it is the node's own value;
* convection ``v . grad u`` by first-order upwind differences;
* every row is multiplied by ``h^2`` so matrix entries are O(1);
* cell Peclet number ``Pe_h = |v| h / 2`` relative to a unit reference
  diffusion, so ``h |v| = 2 Pe_h``.

All such matrices have positive diagonals and non-positive off-diagonals and
are weakly diagonally dominant with strict dominance on boundary rows, hence
non-singular M-matrices, for which GaBP converges (Sec. 2.3, corollary to
Theorem 2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "CSR",
    "stencil_csr",
    "convdiff_5pt",
    "convdiff_9pt_aniso",
    "tridiag",
    "random_m_matrix",
    "paper_toy5_pattern",
    "stand_alone_e1",
    "uniform_rhs",
    "config_c1",
    "config_c2",
    "config_c2_levels",
    "config_c3_levels",
    "config_c4_batch",
    "config_c5",
    "lognormal_field",
    "ConvDiff5ptTorch",
    "convdiff_5pt_torch",
    "sparse_random_m_matrix",
    "permute_symmetric",
    "late_breakdown_tree",
]


@dataclasses.dataclass
class CSR:
    """Compressed sparse row matrix (square)."""

    n: int
    indptr: np.ndarray  # int64, length n+1
    indices: np.ndarray  # int32, length nnz, sorted within each row
    data: np.ndarray  # float64, length nnz

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def to_dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        for r in range(self.n):
            lo, hi = self.indptr[r], self.indptr[r + 1]
            A[r, self.indices[lo:hi]] = self.data[lo:hi]
        return A

    def transpose(self) -> "CSR":
        return dense_to_csr(self.to_dense().T) if self.n <= 4096 else _csr_transpose(self)

    def offdiag_count(self) -> int:
        rows = np.repeat(np.arange(self.n), np.diff(self.indptr))
        return int(np.count_nonzero(rows != self.indices))

    def matvec(self, x: np.ndarray) -> np.ndarray:
        rows = np.repeat(np.arange(self.n), np.diff(self.indptr))
        return np.bincount(rows, weights=self.data * x[self.indices], minlength=self.n)


def _csr_transpose(A: CSR) -> CSR:
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.indptr))
    order = np.lexsort((rows, A.indices.astype(np.int64)))
    new_rows = A.indices.astype(np.int64)[order]
    indptr = np.zeros(A.n + 1, dtype=np.int64)
    np.cumsum(np.bincount(new_rows, minlength=A.n), out=indptr[1:])
    return CSR(A.n, indptr, rows[order].astype(np.int32), A.data[order].copy())


def dense_to_csr(M: np.ndarray, keep_diag: bool = True) -> CSR:
    """CSR of a dense square matrix; exact zeros off the diagonal are dropped."""
    n = M.shape[0]
    indptr = [0]
    indices = []
    data = []
    for r in range(n):
        for c in range(n):
            if M[r, c] != 0.0 or (keep_diag and r == c):
                indices.append(c)
                data.append(float(M[r, c]))
        indptr.append(len(indices))
    return CSR(n, np.asarray(indptr, np.int64), np.asarray(indices, np.int32),
               np.asarray(data, np.float64))


def stencil_csr(m: int, offsets, coeffs: np.ndarray) -> CSR:
    """CSR of a grid operator given per-node stencil coefficients.

    ``offsets`` is a list of ``(dx, dy)`` pairs sorted so that ``dx + m*dy``
    ascends; ``coeffs[iy, ix, k]`` is the coefficient of neighbour ``k``.
    Neighbours outside the grid are dropped (Dirichlet), exact zeros off the
    diagonal are dropped, the diagonal ``(0, 0)`` is always kept.
    """
    offsets = list(offsets)
    K = len(offsets)
    lin = [dx + m * dy for dx, dy in offsets]
    assert lin == sorted(lin), "offsets must ascend in linear index"
    n = m * m
    iy, ix = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    keep = np.empty((m, m, K), dtype=bool)
    for k, (dx, dy) in enumerate(offsets):
        inside = (ix + dx >= 0) & (ix + dx < m) & (iy + dy >= 0) & (iy + dy < m)
        if dx == 0 and dy == 0:
            keep[:, :, k] = True
        else:
            keep[:, :, k] = inside & (coeffs[:, :, k] != 0.0)
    keep = keep.reshape(n, K)
    counts = keep.sum(axis=1)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    rows = np.arange(n, dtype=np.int64)[:, None]
    cols = rows + np.asarray(lin, dtype=np.int64)[None, :]
    indices = cols[keep].astype(np.int32)
    data = np.ascontiguousarray(coeffs.reshape(n, K)[keep], dtype=np.float64)
    return CSR(n, indptr, indices, data)


_OFF5 = [(0, -1), (-1, 0), (0, 0), (1, 0), (0, 1)]
_OFF9 = [(-1, -1), (0, -1), (1, -1), (-1, 0), (0, 0), (1, 0), (-1, 1), (0, 1), (1, 1)]


def convdiff_5pt(m: int, D: np.ndarray | None = None, hv=(0.0, 0.0)) -> CSR:
    """5-point ``-div(D grad u) + v . grad u``, upwind convection, rows times h^2.

    ``D`` is the per-node diffusion field ``D[iy, ix]`` (ones if None) and
    ``hv = h * v`` the dimensionless velocity.
    """
    D = np.ones((m, m)) if D is None else np.asarray(D, dtype=np.float64)
    hvx, hvy = float(hv[0]), float(hv[1])

    def harm(a, b):
        return 2.0 * a * b / (a + b)

    Dw = D.copy(); Dw[:, 1:] = harm(D[:, 1:], D[:, :-1])
    De = D.copy(); De[:, :-1] = harm(D[:, :-1], D[:, 1:])
    Ds = D.copy(); Ds[1:, :] = harm(D[1:, :], D[:-1, :])
    Dn = D.copy(); Dn[:-1, :] = harm(D[:-1, :], D[1:, :])
    coeffs = np.empty((m, m, 5))
    coeffs[:, :, 0] = -Ds - max(hvy, 0.0)
    coeffs[:, :, 1] = -Dw - max(hvx, 0.0)
    coeffs[:, :, 2] = Dw + De + Ds + Dn + abs(hvx) + abs(hvy)
    coeffs[:, :, 3] = -De - max(-hvx, 0.0)
    coeffs[:, :, 4] = -Dn - max(-hvy, 0.0)
    return stencil_csr(m, _OFF5, coeffs)


def convdiff_9pt_aniso(m: int, eps: float, hv=(0.0, 0.0)) -> CSR:
    """9-point anisotropic convection-diffusion, rows times h^2.

    Operator ``(1-eps) [-1 2 -1]_x + eps/6 [[-1,-4,-1],[-4,20,-4],[-1,-4,-1]]``
    (a second-order ``-u_xx - eps u_yy``) plus first-order upwind convection;
    every off-diagonal is non-positive, so the matrix is an M-matrix.
    """
    hvx, hvy = float(hv[0]), float(hv[1])
    c = np.empty((m, m, 9))
    corner = -eps / 6.0
    c[:, :, 0] = corner
    c[:, :, 1] = -4.0 * eps / 6.0 - max(hvy, 0.0)
    c[:, :, 2] = corner
    c[:, :, 3] = -(1.0 - eps) - 4.0 * eps / 6.0 - max(hvx, 0.0)
    c[:, :, 4] = 2.0 * (1.0 - eps) + 20.0 * eps / 6.0 + abs(hvx) + abs(hvy)
    c[:, :, 5] = -(1.0 - eps) - 4.0 * eps / 6.0 - max(-hvx, 0.0)
    c[:, :, 6] = corner
    c[:, :, 7] = -4.0 * eps / 6.0 - max(-hvy, 0.0)
    c[:, :, 8] = corner
    return stencil_csr(m, _OFF9, c)


def tridiag(n: int, d: float, sup: float, sub: float) -> CSR:
    """Constant tridiagonal matrix: ``d`` on the diagonal, ``sup`` above, ``sub`` below."""
    M = np.zeros((n, n))
    idx = np.arange(n)
    M[idx, idx] = d
    M[idx[:-1], idx[:-1] + 1] = sup
    M[idx[1:], idx[1:] - 1] = sub
    return dense_to_csr(M)


def random_m_matrix(n: int, density: float, seed: int, *, nonsym_pattern: bool = True,
                    dominance: float = 1.2) -> CSR:
    """Random sparse non-singular M-matrix.

    Off-diagonals are ``-U(0.1, 1)`` on a random pattern (structurally
    nonsymmetric when ``nonsym_pattern``), the diagonal is ``dominance`` times
    the larger of the absolute row and column sums, so the Jacobi matrix has
    spectral radius below one.
    """
    rng = np.random.default_rng(seed)
    M = np.zeros((n, n))
    mask = rng.random((n, n)) < density
    if not nonsym_pattern:
        mask = mask | mask.T
    np.fill_diagonal(mask, False)
    M[mask] = -rng.uniform(0.1, 1.0, size=int(mask.sum()))
    rs = np.abs(M).sum(axis=1)
    cs = np.abs(M).sum(axis=0)
    np.fill_diagonal(M, dominance * np.maximum(np.maximum(rs, cs), 0.5))
    return dense_to_csr(M)


def _coo_to_csr(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    """CSR from coordinates without duplicates (sorted by row, then column)."""
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=indptr[1:])
    return CSR(n, indptr, cols.astype(np.int32), vals.astype(np.float64))


def sparse_random_m_matrix(n: int, mean_degree: float, seed: int, *, hubs: int = 0,
                           hub_degree: int = 0, isolated: int = 0,
                           dominance: float = 1.2) -> CSR:
    """Sparse random M-matrix with an irregular degree distribution.

    About ``n * mean_degree`` off-diagonal entries ``-U(0.1, 1)`` at uniformly
    random positions (a structurally nonsymmetric pattern), plus ``hubs`` rows
    with ``hub_degree`` entries each (long rows) and their transposed
    entries in part, and ``isolated`` rows and columns left with the diagonal
    only.  The diagonal is ``dominance`` times the larger of the absolute row
    and column sums (at least 0.5), so the Jacobi matrix has spectral radius
    below one.  Built without a dense array, for sizes in the millions.
    """
    rng = np.random.default_rng(seed)
    m = int(round(n * mean_degree))
    rows = rng.integers(0, n, size=m)
    cols = rng.integers(0, n, size=m)
    if hubs > 0 and hub_degree > 0:
        hub_ids = rng.choice(n, size=hubs, replace=False)
        hr = np.repeat(hub_ids, hub_degree)
        hc = rng.integers(0, n, size=hubs * hub_degree)
        back = rng.random(hr.size) < 0.5      # half of them also as (c, hub)
        rows = np.concatenate([rows, hr, hc[back]])
        cols = np.concatenate([cols, hc, hr[back]])
    keep = rows != cols
    if isolated > 0:
        iso = np.zeros(n, dtype=bool)
        iso[rng.choice(n, size=isolated, replace=False)] = True
        keep &= ~iso[rows] & ~iso[cols]
    key = np.unique(rows[keep].astype(np.int64) * n + cols[keep])
    rows, cols = key // n, key % n
    vals = -rng.uniform(0.1, 1.0, size=key.size)
    rs = np.bincount(rows, weights=-vals, minlength=n)
    cs = np.bincount(cols, weights=-vals, minlength=n)
    diag = dominance * np.maximum(np.maximum(rs, cs), 0.5)
    idx = np.arange(n, dtype=np.int64)
    return _coo_to_csr(n, np.concatenate([rows, idx]), np.concatenate([cols, idx]),
                       np.concatenate([vals, diag]))


def permute_symmetric(A: CSR, seed: int):
    """``(Q A Q^T, perm)`` for a seeded random permutation: new node ``k`` is
    old node ``perm[k]``, so ``x_new = x_old[perm]`` and ``b_new = b_old[perm]``."""
    perm = np.random.default_rng(seed).permutation(A.n)
    inv = np.empty(A.n, dtype=np.int64)
    inv[perm] = np.arange(A.n)
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.indptr))
    return _coo_to_csr(A.n, inv[rows], inv[A.indices.astype(np.int64)], A.data.copy()), perm


def late_breakdown_tree(m: int, a: int, x0: int | None = None) -> CSR:
    """A non-singular 5-point grid matrix on which flood GaBP first meets a
    zero denominator at sweep ``a + 1``.

    Node ``j = (x0, a)`` has two arms of ``a`` nodes each: one to its left
    along grid row ``a`` and one above it along grid column ``x0``; a further
    node ``j + m`` hangs below ``j``.  These ``2a + 2`` nodes form a tree and
    are coupled to nothing else; every other grid node belongs to a 5-point
    Laplacian (diagonal 4, couplings -1) among the non-tree nodes.

    Values: arm leaves have diagonal 1, other arm nodes 1.5; along an arm the
    entry towards ``j`` is -1 and the entry towards the leaf -0.5; ``A_jj = 1``
    with -0.5 towards both arms, ``A_{j, j+m} = 1``, ``A_{j+m, j} = -1``,
    ``A_{j+m, j+m} = 2``.  Eliminating an arm from its leaf towards ``j``
    gives pivots of exactly 1 (``1.5 - 0.5 * 1 / 1``), so the Schur complement
    of ``j`` with both arms eliminated is ``1 - 2 * 0.5 = 0``: the principal
    submatrix on the arms and ``j`` is singular, while ``A`` is not.  GaBP on
    a tree is that elimination (Sec. 2.1-2.2), and the message ``j -> j+m``
    divides by this pivot once the leaves' information has reached ``j``.
    Every value and every partial sum of the exact pivots is a short binary
    fraction, so the zero is exact in float and double.  No ball of the tree
    around one node is the singular set, so every belief stays finite.
    """
    if x0 is None:
        x0 = a
    if not (a >= 1 and x0 >= a and x0 < m and a + 1 < m):
        raise ValueError("need 1 <= a <= x0 < m and a + 1 < m")
    y0 = a
    tree = {(x0, y0), (x0, y0 + 1)}
    tree |= {(x0 - i, y0) for i in range(1, a + 1)}
    tree |= {(x0, y0 - i) for i in range(1, a + 1)}
    c = np.zeros((m, m, 5))  # neighbours (0,-1), (-1,0), (0,0), (1,0), (0,1)
    nb = ((0, (0, -1)), (1, (-1, 0)), (3, (1, 0)), (4, (0, 1)))
    for y in range(m):
        for x in range(m):
            if (x, y) in tree:
                continue
            c[y, x, 2] = 4.0
            for k, (dx, dy) in nb:
                if 0 <= x + dx < m and 0 <= y + dy < m and (x + dx, y + dy) not in tree:
                    c[y, x, k] = -1.0
    for i in range(1, a + 1):
        # arm along row y0 (towards j: +x), arm along column x0 (towards j: +y)
        c[y0, x0 - i, 2] = c[y0 - i, x0, 2] = 1.0 if i == a else 1.5
        c[y0, x0 - i, 3] = c[y0 - i, x0, 4] = -1.0
        if i < a:
            c[y0, x0 - i, 1] = c[y0 - i, x0, 0] = -0.5
    c[y0, x0, 2] = 1.0
    c[y0, x0, 1] = c[y0, x0, 0] = -0.5
    c[y0, x0, 4] = 1.0
    c[y0 + 1, x0, 2] = 2.0
    c[y0 + 1, x0, 0] = -1.0
    return stencil_csr(m, _OFF5, c)


def paper_toy5_pattern(seed: int = 7) -> CSR:
    """The 5x5 tree-structured pattern of the paper's elimination example (Sec. 2.1).

    Nonzeros at (1,3), (2,3), (3,1), (3,2), (3,5), (4,5), (5,3), (5,4) and the
    diagonal (1-based), with random nonsymmetric values; diagonally dominant.
    """
    rng = np.random.default_rng(seed)
    M = np.zeros((5, 5))
    pairs = [(1, 3), (2, 3), (3, 1), (3, 2), (3, 5), (4, 5), (5, 3), (5, 4)]
    for i, j in pairs:
        M[i - 1, j - 1] = rng.uniform(-1.5, 1.5)
    for i in range(5):
        M[i, i] = 1.0 + np.abs(M[i]).sum() + rng.uniform(0.0, 1.0)
    return dense_to_csr(M)


def stand_alone_e1(m: int = 63):
    """Stand-alone test problem of Sec. 5.2 (eq. stand_alone), rows times h^2.

    ``a u_xx + b u_yy + alpha u_x + beta u_y = g`` on the unit square with the
    manufactured solution ``cos(pi x) cos(pi y)``; negated so the matrix is an
    M-matrix, second-order central differences for all derivatives, Dirichlet
    values taken from the exact solution.  Returns ``(A, rhs, u_exact)``.
    """
    h = 1.0 / (m + 1)
    xs = (np.arange(m) + 1) * h
    X, Y = np.meshgrid(xs, xs, indexing="xy")  # X[iy, ix] = x
    a = np.exp(-X * (Y + 2.0)) + 10.0
    alpha = np.cos(np.pi * (X + Y / 2.0)) * np.cos(2.0 * np.pi * X) + 4.0
    bb = np.exp(-2.0 * X + 2.0 * Y) * np.cos(2.0 * np.pi * (2.0 * X + Y / 2.0)) ** 2 + 3.0
    beta = np.exp(2.0 * X - 2.0 * Y)

    def ue(x, y):
        return np.cos(np.pi * x) * np.cos(np.pi * y)

    ux = -np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)
    uy = -np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
    uxx = -np.pi ** 2 * ue(X, Y)
    g = a * uxx + bb * uxx + alpha * ux + beta * uy  # u_yy == u_xx for this solution
    # -(a u_xx + b u_yy + alpha u_x + beta u_y) = -g, times h^2
    c = np.empty((m, m, 5))
    c[:, :, 0] = -bb + 0.5 * h * beta       # south (y - h)
    c[:, :, 1] = -a + 0.5 * h * alpha       # west (x - h)
    c[:, :, 2] = 2.0 * a + 2.0 * bb
    c[:, :, 3] = -a - 0.5 * h * alpha       # east
    c[:, :, 4] = -bb - 0.5 * h * beta       # north
    rhs = -(h * h) * g
    # move the known Dirichlet values to the right-hand side
    rhs[0, :] -= c[0, :, 0] * ue(xs, 0.0)
    rhs[:, 0] -= c[:, 0, 1] * ue(0.0, xs)
    rhs[:, -1] -= c[:, -1, 3] * ue(1.0, xs)
    rhs[-1, :] -= c[-1, :, 4] * ue(xs, 1.0)
    A = stencil_csr(m, _OFF5, c)
    return A, rhs.reshape(-1).copy(), ue(X, Y).reshape(-1).copy()


def uniform_rhs(n: int, rng: np.random.Generator, scale: float = 1.0) -> np.ndarray:
    return scale * rng.uniform(-1.0, 1.0, size=n)


def lognormal_field(m: int, sigma: float, rng: np.random.Generator) -> np.ndarray:
    return np.exp(rng.normal(0.0, sigma, size=(m, m)))


def _hv(pe_h: float, theta: float):
    return (2.0 * pe_h * math.cos(theta), 2.0 * pe_h * math.sin(theta))


def config_c1(m: int = 32, seed: int = 1001):
    """Constant-coefficient convection-diffusion, cell Peclet 0.5 along (1, 0.5).

    Returns ``(A, b)`` with ``b = h^2 f`` and ``f ~ U[-1, 1]``.
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / (m + 1)
    d = np.array([1.0, 0.5]) / math.hypot(1.0, 0.5)
    A = convdiff_5pt(m, None, (d[0] * 1.0, d[1] * 1.0))  # h|v| = 2 * 0.5
    b = h * h * uniform_rhs(m * m, rng)
    return A, b


def config_c2(m: int = 2048, seed: int = 1002, sigma: float = 0.5, theta: float = 0.3,
              pe_h: float = 1.0):
    """Log-normal diffusion convection-diffusion (5-point upwind), ``b ~ U[-1, 1]``."""
    rng = np.random.default_rng(seed)
    D = lognormal_field(m, sigma, rng)
    A = convdiff_5pt(m, D, _hv(pe_h, theta))
    b = uniform_rhs(m * m, rng)
    return A, b


def config_c3_levels(m_fine: int = 4095, m_coarse: int = 31, eps: float = 0.01,
                     theta: float = 0.3, pe_h: float = 1.0, seed: int = 1003):
    """Rediscretised 9-point anisotropic hierarchy for the multigrid V-cycle.

    The velocity is fixed in physical units (cell Peclet ``pe_h`` on the
    finest grid), so level ``l`` with mesh ``2^l h`` has ``h_l |v| = 2^(l+1) pe_h``.
    Returns ``(levels, sides, b)`` finest first; ``b ~ U[-1, 1]`` on the finest grid.
    """
    sides = []
    m = m_fine
    while True:
        sides.append(m)
        if m <= m_coarse:
            break
        assert (m - 1) % 2 == 0, "grid sides must be 2^J - 1"
        m = (m - 1) // 2
    levels = []
    for lvl, ms in enumerate(sides):
        hv = _hv(pe_h * (2 ** lvl), theta)
        levels.append(convdiff_9pt_aniso(ms, eps, hv))
    rng = np.random.default_rng(seed)
    b = uniform_rhs(m_fine * m_fine, rng)
    return levels, sides, b


def config_c2_levels(m_fine: int = 2047, m_coarse: int = 31, sigma: float = 0.5,
                     theta: float = 0.3, pe_h: float = 1.0, seed: int = 1002):
    """Rediscretised 5-point hierarchy of the log-normal convection-diffusion
    problem of ``config_c2`` on vertex-centred grids of side 2^J - 1.

    The diffusion field is drawn on the finest grid and injected to the coarse
    nodes (coarse node (I, J) is fine node (2I + 1, 2J + 1)); the velocity is
    fixed in physical units (cell Peclet ``pe_h`` on the finest grid).
    Returns ``(levels, sides, b)`` finest first; ``b ~ U[-1, 1]`` on the finest grid.
    """
    sides = []
    m = m_fine
    while True:
        sides.append(m)
        if m <= m_coarse:
            break
        assert (m - 1) % 2 == 0, "grid sides must be 2^J - 1"
        m = (m - 1) // 2
    rng = np.random.default_rng(seed)
    D = lognormal_field(m_fine, sigma, rng)
    b = uniform_rhs(m_fine * m_fine, rng)
    levels = []
    for lvl, ms in enumerate(sides):
        hv = _hv(pe_h * (2 ** lvl), theta)
        levels.append(convdiff_5pt(ms, D, hv))
        D = D[1::2, 1::2]
    return levels, sides, b


def config_c4_batch(nsys: int = 512, smin: int = 16, smax: int = 256, seed: int = 1004,
                    sigma: float = 0.5):
    """Batch of independent convection-diffusion systems of uneven sizes.

    Per system: side ``s ~ U{smin..smax}``, log-normal diffusion, cell Peclet
    ``~ U[0.1, 2]``, flow angle ``~ U[0, 2 pi)``, ``b ~ U[-1, 1]``.
    Returns a list of ``(A, b)``.
    """
    rng = np.random.default_rng(seed)
    sides = rng.integers(smin, smax + 1, size=nsys)
    out = []
    for s in sides:
        s = int(s)
        D = lognormal_field(s, sigma, rng)
        pe = rng.uniform(0.1, 2.0)
        th = rng.uniform(0.0, 2.0 * math.pi)
        A = convdiff_5pt(s, D, _hv(pe, th))
        b = uniform_rhs(s * s, rng)
        out.append((A, b))
    return out


def config_c5(m: int = 512, seed: int = 1005, sigma: float = 0.3):
    """Differentiable-solve workload: ``kappa = exp(theta)``, ``theta ~ N(0, sigma^2)``.

    Returns ``(theta, b, theta_target)`` where ``theta_target`` is a second
    independent field (used to build ``x_target``).
    """
    rng = np.random.default_rng(seed)
    theta = rng.normal(0.0, sigma, size=(m, m))
    b = uniform_rhs(m * m, rng)
    theta_t = np.random.default_rng(seed + 1).normal(0.0, sigma, size=(m, m))
    return theta, b, theta_t


class ConvDiff5ptTorch:
    """Differentiable assembly of ``convdiff_5pt`` values for one grid and flow.

    The CSR pattern and the map from the ``(m, m, 5)`` stencil coefficients to
    the CSR slots are built once (the pattern is the same for every positive
    diffusion field); ``values(D)`` then assembles the values from a torch
    tensor ``D`` of shape ``(m, m)`` on ``D``'s device, differentiably, with no
    host work.
    """

    def __init__(self, m: int, hv=(0.0, 0.0), device=None):
        import torch

        self.m = m
        self.hv = (float(hv[0]), float(hv[1]))
        self.pattern = convdiff_5pt(m, None, hv)
        iy, ix = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
        keep = np.empty((m, m, 5), dtype=bool)
        for k, (dx, dy) in enumerate(_OFF5):
            keep[:, :, k] = (ix + dx >= 0) & (ix + dx < m) & (iy + dy >= 0) & (iy + dy < m)
        self._flat = np.flatnonzero(keep.reshape(-1))
        self._idx = {}
        if device is not None:
            self._index(torch.device(device))

    def _index(self, device):
        import torch

        key = str(device)
        if key not in self._idx:
            self._idx[key] = torch.as_tensor(self._flat, device=device)
        return self._idx[key]

    def values(self, D):
        import torch

        hvx, hvy = self.hv

        def harm(a, b):
            return 2.0 * a * b / (a + b)

        Dw = torch.cat([D[:, :1], harm(D[:, 1:], D[:, :-1])], dim=1)
        De = torch.cat([harm(D[:, :-1], D[:, 1:]), D[:, -1:]], dim=1)
        Ds = torch.cat([D[:1, :], harm(D[1:, :], D[:-1, :])], dim=0)
        Dn = torch.cat([harm(D[:-1, :], D[1:, :]), D[-1:, :]], dim=0)
        coeffs = torch.stack([
            -Ds - max(hvy, 0.0),
            -Dw - max(hvx, 0.0),
            Dw + De + Ds + Dn + abs(hvx) + abs(hvy),
            -De - max(-hvx, 0.0),
            -Dn - max(-hvy, 0.0),
        ], dim=2)
        return coeffs.reshape(-1)[self._index(D.device)]


def convdiff_5pt_torch(m: int, D, hv=(0.0, 0.0)):
    """Differentiable twin of ``convdiff_5pt``: the CSR values as a torch tensor.

    ``D`` is a torch tensor of shape ``(m, m)`` (positive node diffusion);
    gradients flow from the returned values to ``D``.  Returns ``(pattern,
    values)`` where ``pattern`` is the ``CSR`` of ``convdiff_5pt(m, D, hv)``
    and ``values`` its data in the same slot order, on ``D``'s device.  Used
    for the differentiable-solve workload ``kappa = exp(theta)``; for repeated
    assembly on one grid, ``ConvDiff5ptTorch`` builds the pattern once.
    """
    asm = ConvDiff5ptTorch(m, hv)
    return asm.pattern, asm.values(D)
