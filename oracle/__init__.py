"""Plain, slow, double-precision CPU oracle for GaBP on nonsymmetric systems.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
CUDA library never imports it and shares no code with it.

The per-sweep arithmetic lives in ``gabp_oracle.c`` (plain C loops in the
paper's notation, eq. nonsymmetric_GaBP_rules); this module compiles and loads
it and writes out the drivers in the order the paper gives them:

* ``solve``         Algorithm 1 with the flood schedule of Sec. 2.2, stopping
                    on the infinity-norm residual;
* ``MGOracle``      geometric V-cycle of Sec. 4 with GaBP as the
                    error-correction smoother of Algorithm 3, full-weighting
                    restriction, bilinear prolongation, a direct coarse solve;
* ``adjoint``       implicit differentiation of x = A^{-1} b (plain definition
                    via dense solves; the paper has no counterpart).

Messages are stored per CSR slot: the message j -> i lives at the slot of the
entry (i, j) and holds ``(tilde-Lambda_ji, m_ji)``.

Parity pins for every function are in ``tests/test_oracle_pins.py``; the
V-cycle is pinned through invariants (fixed point, linearity, exact-smoother
limit), the transfer operators through their definitions, and its whole
composition through the nu = 1 cold smoother, which is Jacobi: a V(1,1) cycle
equals an independently written dense Jacobi multigrid recursion.  Its
convergence rates have no printed values to pin ("parity unpinned").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gabp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libgabp_oracle.so")
_lock = threading.Lock()
_lib = None

OK, BREAKDOWN, DIVERGED, NOT_CONVERGED = 0, 4, 5, 6
DIVERGENCE_LIMIT = 1e8  # relative residual above which a run counts as diverged


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP when available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            P = ctypes.c_void_p
            L.oracle_beliefs.argtypes = [i64, P, P, P, P, P, P, P, P]
            L.oracle_beliefs.restype = None
            L.oracle_update.argtypes = [i64, P, P, P, P, P, P, P, P]
            L.oracle_update.restype = i32
            L.oracle_residual_inf.argtypes = [i64, P, P, P, P, P]
            L.oracle_residual_inf.restype = dbl
            L.oracle_residual.argtypes = [i64, P, P, P, P, P, P]
            L.oracle_residual.restype = None
            L.oracle_sweeps.argtypes = [i64, P, P, P, P, i32, P, P, P, P, P, P]
            L.oracle_sweeps.restype = i32
            L.oracle_sweeps_colored.argtypes = [i64, P, P, P, P, P, i32, i32, P, P, P, P]
            L.oracle_sweeps_colored.restype = i32
            L.oracle_set_threads.argtypes = [i32]
            L.oracle_set_threads.restype = None
            L.oracle_max_threads.argtypes = []
            L.oracle_max_threads.restype = i32
            _lib = L
    return _lib


def set_threads(t: int) -> None:
    lib().oracle_set_threads(int(t))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _mat(A):
    ip = np.ascontiguousarray(A.indptr, dtype=np.int64)
    ix = np.ascontiguousarray(A.indices, dtype=np.int32)
    dv = np.ascontiguousarray(A.data, dtype=np.float64)
    return ip, ix, dv


def zero_state(A):
    """Zero messages (the initial state of Algorithm 1)."""
    return np.zeros(A.nnz), np.zeros(A.nnz)


def beliefs(A, b, lt, mm):
    """Beliefs ``mu_i`` and precisions ``beta_i`` (eq. nonsymmetric_GaBP_rules)."""
    ip, ix, dv = _mat(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    mu = np.empty(A.n)
    beta = np.empty(A.n)
    lib().oracle_beliefs(A.n, _p(ip), _p(ix), _p(dv), _p(b), _p(lt), _p(mm), _p(mu), _p(beta))
    return mu, beta


def update(A, b, lt, mm):
    """One flood update of all messages; returns ``(lt_new, mm_new, status)``."""
    ip, ix, dv = _mat(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    lt2 = np.empty(A.nnz)
    mm2 = np.empty(A.nnz)
    st = lib().oracle_update(A.n, _p(ip), _p(ix), _p(dv), _p(b), _p(lt), _p(mm), _p(lt2), _p(mm2))
    return lt2, mm2, int(st)


def sweeps(A, b, nsweeps: int, lt: np.ndarray, mm: np.ndarray):
    """``nsweeps`` sweeps of Algorithm 1 (beliefs, then flood update), in place.

    Returns ``(x, beta, status)``: the beliefs formed in the last sweep.
    """
    ip, ix, dv = _mat(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    assert lt.dtype == np.float64 and mm.dtype == np.float64
    x = np.zeros(A.n)
    beta = np.zeros(A.n)
    lt2 = np.empty(A.nnz)
    mm2 = np.empty(A.nnz)
    st = lib().oracle_sweeps(A.n, _p(ip), _p(ix), _p(dv), _p(b), int(nsweeps), _p(lt), _p(mm),
                             _p(lt2), _p(mm2), _p(x), _p(beta))
    return x, beta, int(st)


def sweeps_colored(A, b, color, ncolors: int, nsweeps: int, lt: np.ndarray, mm: np.ndarray):
    """``nsweeps`` sweeps of Algorithm 1 with a coloured schedule, in place.

    ``color[j]`` in ``[0, ncolors)``, adjacent nodes coloured differently.
    Returns ``(x, beta, status)``: every node's belief from the sweep it was visited in.
    """
    ip, ix, dv = _mat(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    col = np.ascontiguousarray(color, dtype=np.int32)
    x = np.zeros(A.n)
    beta = np.zeros(A.n)
    st = lib().oracle_sweeps_colored(A.n, _p(ip), _p(ix), _p(dv), _p(b), _p(col), int(ncolors),
                                     int(nsweeps), _p(lt), _p(mm), _p(x), _p(beta))
    return x, beta, int(st)


def residual_inf(A, b, x) -> float:
    ip, ix, dv = _mat(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib().oracle_residual_inf(A.n, _p(ip), _p(ix), _p(dv), _p(b), _p(x)))


def residual(A, b, x) -> np.ndarray:
    ip, ix, dv = _mat(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    r = np.empty(A.n)
    lib().oracle_residual(A.n, _p(ip), _p(ix), _p(dv), _p(b), _p(x), _p(r))
    return r


def solve(A, b, tol: float, max_iter: int, lt=None, mm=None, history: bool = False,
          color=None, ncolors: int = 0):
    """Algorithm 1 with the flood schedule, from zero messages unless given.

    Every iteration is one sweep (beliefs from the current messages, then the
    flood update) followed by ``rr = ||b - A x||_inf / ||b||_inf``; the loop
    stops at ``rr <= tol`` (status OK), a breakdown (zero or non-finite
    denominator), ``rr`` non-finite or above ``DIVERGENCE_LIMIT`` (DIVERGED),
    or after ``max_iter`` sweeps (NOT_CONVERGED).
    """
    b = np.ascontiguousarray(b, dtype=np.float64)
    if lt is None or mm is None:
        lt, mm = zero_state(A)
    bn = float(np.max(np.abs(b))) if A.n else 0.0
    hist = []
    x = np.zeros(A.n)
    rr = 0.0 if bn == 0.0 else 1.0
    status = NOT_CONVERGED
    it = 0
    if bn == 0.0:
        return dict(x=x, iters=0, rr=0.0, status=OK, history=hist, lt=lt, mm=mm)
    while it < max_iter:
        if color is None:
            x, beta, st = sweeps(A, b, 1, lt, mm)
        else:
            x, beta, st = sweeps_colored(A, b, color, ncolors, 1, lt, mm)
        it += 1
        rr = residual_inf(A, b, x) / bn
        if history:
            hist.append(rr)
        if st == BREAKDOWN:
            status = BREAKDOWN
            break
        if rr <= tol:
            status = OK
            break
        if not np.isfinite(rr) or rr > DIVERGENCE_LIMIT:
            status = DIVERGED
            break
    return dict(x=x, iters=it, rr=rr, status=status, history=hist, lt=lt, mm=mm)


def dense_solve(A, b) -> np.ndarray:
    """x = A^{-1} b by LAPACK's LU with partial pivoting (Theorem 1's target)."""
    return np.linalg.solve(A.to_dense(), np.asarray(b, dtype=np.float64))


def diag_contrib(A, lt) -> np.ndarray:
    """Per-slot diagonal correction ``tilde-Lambda_ji * A_ji`` of the message j -> i.

    This is the quantity the message carries into the precision of node i
    (eq. nonsymmetric_GaBP_rules, ``beta_i``).
    """
    rows = np.repeat(np.arange(A.n), np.diff(A.indptr))
    cols = A.indices.astype(np.int64)
    Aji = np.zeros(A.nnz)
    for p in range(A.nnz):
        i, j = rows[p], cols[p]
        if i == j:
            continue
        lo, hi = A.indptr[j], A.indptr[j + 1]
        k = np.searchsorted(A.indices[lo:hi], i)
        if k < hi - lo and A.indices[lo + k] == i:
            Aji[p] = A.data[lo + k]
    return lt * Aji


# ---------------------------------------------------------------------------
# Geometric multigrid (Sec. 4).  Grids have m = 2^J - 1 interior points per
# side; the coarse point (I, J) coincides with the fine point (2I+1, 2J+1)
# (0-based).  Values outside the interior are zero (Dirichlet).
# ---------------------------------------------------------------------------

def restrict_full_weighting(r_f: np.ndarray, m_f: int) -> np.ndarray:
    """Full weighting, stencil (1/16)[1 2 1; 2 4 2; 1 2 1] (Trottenberg eq. 2.3.3)."""
    assert (m_f - 1) % 2 == 0
    R = np.asarray(r_f, dtype=np.float64).reshape(m_f, m_f)
    c = R[1::2, 1::2]
    e = R[1::2, 0:-1:2] + R[1::2, 2::2] + R[0:-1:2, 1::2] + R[2::2, 1::2]
    k = R[0:-1:2, 0:-1:2] + R[0:-1:2, 2::2] + R[2::2, 0:-1:2] + R[2::2, 2::2]
    return ((4.0 * c + 2.0 * e + k) / 16.0).reshape(-1)


def prolong_bilinear(e_c: np.ndarray, m_c: int) -> np.ndarray:
    """Bilinear interpolation (Trottenberg eq. 2.3.7) from m_c^2 to (2 m_c + 1)^2 points."""
    m_f = 2 * m_c + 1
    Ep = np.zeros((m_c + 2, m_c + 2))
    Ep[1:-1, 1:-1] = np.asarray(e_c, dtype=np.float64).reshape(m_c, m_c)
    F = np.zeros((m_f, m_f))
    F[1::2, 1::2] = Ep[1:-1, 1:-1]
    F[1::2, 0::2] = 0.5 * (Ep[1:-1, :-1] + Ep[1:-1, 1:])
    F[0::2, 1::2] = 0.5 * (Ep[:-1, 1:-1] + Ep[1:, 1:-1])
    F[0::2, 0::2] = 0.25 * (Ep[:-1, :-1] + Ep[:-1, 1:] + Ep[1:, :-1] + Ep[1:, 1:])
    return F.reshape(-1)


def grid_colors(m: int, ncolors: int) -> np.ndarray:
    """Colouring of the m x m grid (i = ix + m iy) with no two stencil neighbours alike:
    2 colours (red-black, (ix + iy) mod 2) for 5-point operators, 4 colours
    ((ix mod 2) + 2 (iy mod 2)) for 9-point ones."""
    iy, ix = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    if ncolors == 2:
        c = (ix + iy) % 2
    elif ncolors == 4:
        c = (ix % 2) + 2 * (iy % 2)
    else:
        raise ValueError("ncolors must be 2 or 4")
    return c.reshape(-1).astype(np.int32)


class MGOracle:
    """V-cycle with GaBP as the error-correction smoother (Algorithm 3).

    ``levels`` are CSR matrices from fine to coarse on grids of side
    ``sides[l]``; ``transfer_scale`` multiplies every restricted residual (4
    for operators whose rows are scaled by h^2).  The coarsest level is
    solved directly.

    ``mode`` says which messages a smoother call starts from:

    * ``"cold"``  (default) every call runs nu sweeps of Algorithm 1 from zero
      messages, the operator the paper's LFA analyses (Sec. 4.1);
    * ``"warm"``  the tilde-Lambda messages of the level persist across calls
      (they do not depend on the right-hand side, Sec. 2.3), the mean
      messages restart from zero;
    * ``"persist"`` both kinds of messages persist across calls.

    ``ncolors`` = 0 smooths with flood sweeps (Sec. 2.2); 2 or 4 with the
    red-black or 4-colour schedule (Sec. 5.1) on the grid colouring ``grid_colors``.
    ``lines=True`` smooths with line GaBP (Algorithm 2 with the grid's rows and
    columns as regions, ``line_sweeps``; 5-point levels only), the beliefs
    being the column regions' solutions.
    """

    MODES = ("cold", "warm", "persist")

    def __init__(self, levels, sides, transfer_scale: float = 4.0, mode: str = "cold",
                 ncolors: int = 0, lines: bool = False):
        assert len(levels) == len(sides) >= 1
        assert mode in self.MODES
        self.ncolors = ncolors
        self.lines = lines
        self.lstate = [line_zero_state(A.n) for A in levels] if lines else None
        self.colors = [grid_colors(m, ncolors) if ncolors else None for m in sides]
        self.levels = levels
        self.sides = list(sides)
        self.scale = float(transfer_scale)
        self.mode = mode
        self.lt = [np.zeros(A.nnz) for A in levels]
        self.mm = [np.zeros(A.nnz) for A in levels]
        self.coarse = levels[-1].to_dense()

    def smooth(self, lvl: int, b, x, nu: int):
        """Algorithm 3: r = b - A x; nu GaBP sweeps on A e = r; x + e."""
        A = self.levels[lvl]
        r = residual(A, b, x)
        if self.mode == "cold":
            self.lt[lvl][:] = 0.0
        if self.mode in ("cold", "warm"):
            self.mm[lvl][:] = 0.0
        if self.lines:
            stl = self.lstate[lvl]
            for key in ("LH", "LV") if self.mode == "cold" else ():
                stl[key][:] = 0.0
            for key in ("MH", "MV") if self.mode in ("cold", "warm") else ():
                stl[key][:] = 0.0
            e = line_sweeps(A, self.sides[lvl], r, nu, stl)
            st = OK if np.all(np.isfinite(e)) else BREAKDOWN
        elif self.ncolors:
            e, _, st = sweeps_colored(A, r, self.colors[lvl], self.ncolors, nu, self.lt[lvl], self.mm[lvl])
        else:
            e, _, st = sweeps(A, r, nu, self.lt[lvl], self.mm[lvl])
        if st != OK:
            raise FloatingPointError("GaBP breakdown in the smoother")
        return x + e

    def vcycle(self, b, x, nu_pre: int, nu_post: int, lvl: int = 0):
        if lvl == len(self.levels) - 1:
            return np.linalg.solve(self.coarse, b)
        A = self.levels[lvl]
        if nu_pre > 0:
            x = self.smooth(lvl, b, x, nu_pre)
        r = residual(A, b, x)
        bc = self.scale * restrict_full_weighting(r, self.sides[lvl])
        ec = self.vcycle(bc, np.zeros(self.levels[lvl + 1].n), nu_pre, nu_post, lvl + 1)
        x = x + prolong_bilinear(ec, self.sides[lvl + 1])
        if nu_post > 0:
            x = self.smooth(lvl, b, x, nu_post)
        return x

    def solve(self, b, tol: float, max_cycles: int, nu_pre: int, nu_post: int):
        A = self.levels[0]
        b = np.asarray(b, dtype=np.float64)
        bn = float(np.max(np.abs(b)))
        x = np.zeros(A.n)
        hist = []
        for c in range(1, max_cycles + 1):
            x = self.vcycle(b, x, nu_pre, nu_post)
            rr = residual_inf(A, b, x) / bn
            hist.append(rr)
            if rr <= tol:
                return dict(x=x, cycles=c, rr=rr, status=OK, history=hist)
            if not np.isfinite(rr) or rr > DIVERGENCE_LIMIT:
                return dict(x=x, cycles=c, rr=rr, status=DIVERGED, history=hist)
        return dict(x=x, cycles=max_cycles, rr=hist[-1] if hist else 1.0,
                    status=NOT_CONVERGED, history=hist)


# ---------------------------------------------------------------------------
# Implicit differentiation of x = A^{-1} b (no counterpart in the paper).
# ---------------------------------------------------------------------------

def adjoint(A, b, g):
    """Given ``g = dL/dx`` at ``x = A^{-1} b``: ``lam = A^{-T} g = dL/db`` and
    ``dL/dA_ij = -lam_i x_j`` on every stored entry (i, j).

    Returns ``(x, lam, dA)`` with ``dA`` aligned with ``A.data``.
    """
    M = A.to_dense()
    x = np.linalg.solve(M, np.asarray(b, dtype=np.float64))
    lam = np.linalg.solve(M.T, np.asarray(g, dtype=np.float64))
    rows = np.repeat(np.arange(A.n), np.diff(A.indptr))
    dA = -lam[rows] * x[A.indices]
    return x, lam, dA


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))


# ---------------------------------------------------------------------------
# Line GaBP: Algorithm 2 (two-layer generalized GaBP, Sec. 3.2-3.4) with the
# grid lines as large regions and single nodes as small regions (the
# partition the paper calls "line GaBP").  Valid for 5-point grids, where
# every edge lies inside a row or a column.
# ---------------------------------------------------------------------------

def _line_nodes(m: int, family: str, k: int) -> np.ndarray:
    if family == "row":
        return k * m + np.arange(m)
    return np.arange(m) * m + k


def _line_matrix(A, idx: np.ndarray) -> np.ndarray:
    """[A]_L: the entries of A between the nodes of one line (Sec. 3.2 brackets)."""
    pos = {int(v): t for t, v in enumerate(idx)}
    T = np.zeros((len(idx), len(idx)))
    for t, v in enumerate(idx):
        for p in range(A.indptr[v], A.indptr[v + 1]):
            j = int(A.indices[p])
            if j in pos:
                T[t, pos[j]] = A.data[p]
    return T


def line_zero_state(n: int):
    """Messages from every row and every column region to each node: (Lambda, m) pairs."""
    return {"LH": np.zeros(n), "MH": np.zeros(n), "LV": np.zeros(n), "MV": np.zeros(n)}


def line_sweeps(A, m: int, b, nsweeps: int, state):
    """``nsweeps`` sweeps of Algorithm 2 over the region graph of rows and
    columns: first every row region, then every column region (regions of one
    family share no node, so each family is processed at once).  For a region
    L with children l and the other parent L' of each child:

        b0 = [b]_L + sum_l m_{L'l},   Lam0 = [A]_L + sum_l Lambda_{L'l}
        [x]_L = Lam0^{-1} b0
        m_{Ll}      = ([Lam0^{-1}]_l)^{-1} x_l - b_l - m_{L'l}
        Lambda_{Ll} = ([Lam0^{-1}]_l)^{-1} - A_ll - Lambda_{L'l}

    In place on ``state``; returns x as last written (by the column regions).
    """
    b = np.asarray(b, dtype=np.float64)
    n = m * m
    x = np.zeros(n)
    for _ in range(nsweeps):
        for family, (Lown, Mown, Loth, Moth) in (("row", ("LH", "MH", "LV", "MV")),
                                                 ("col", ("LV", "MV", "LH", "MH"))):
            newL = state[Lown].copy()
            newM = state[Mown].copy()
            for k in range(m):
                idx = _line_nodes(m, family, k)
                newL[idx], newM[idx], x[idx] = line_region_update(A, m, b, family, k,
                                                                  state[Loth], state[Moth])
            state[Lown] = newL
            state[Mown] = newM
    return x


def line_region_update(A, m: int, b, family: str, k: int, Loth, Moth):
    """The messages region ``k`` of ``family`` ("row" or "col") sends to its
    nodes, given the other family's messages ``Loth, Moth`` (full-length
    arrays), and the region's solution: one step of Algorithm 2 for one large
    region (see ``line_sweeps``).  Returns ``(Lambda, m, x)`` on the region's
    nodes in line order."""
    b = np.asarray(b, dtype=np.float64)
    idx = _line_nodes(m, family, k)
    rows = np.concatenate([np.full(A.indptr[v + 1] - A.indptr[v], v) for v in idx])
    cols = np.concatenate([A.indices[A.indptr[v]:A.indptr[v + 1]] for v in idx])
    vals = np.concatenate([A.data[A.indptr[v]:A.indptr[v + 1]] for v in idx])
    diag = vals[rows == cols]
    Lam0 = _line_matrix(A, idx) + np.diag(Loth[idx])
    b0 = b[idx] + Moth[idx]
    xl = np.linalg.solve(Lam0, b0)
    S = 1.0 / np.diag(np.linalg.inv(Lam0))
    return S - diag - Loth[idx], S * xl - b[idx] - Moth[idx], xl


def line_solve(A, m: int, b, tol: float, max_iter: int):
    """Line GaBP iterated until ||b - A x||_inf / ||b||_inf <= tol (Algorithm 2's loop)."""
    b = np.asarray(b, dtype=np.float64)
    bn = float(np.max(np.abs(b)))
    st = line_zero_state(A.n)
    x = np.zeros(A.n)
    rr = 1.0
    for it in range(1, max_iter + 1):
        x = line_sweeps(A, m, b, 1, st)
        rr = residual_inf(A, b, x) / bn
        if rr <= tol:
            return dict(x=x, iters=it, rr=rr, status=OK, state=st)
        if not np.isfinite(rr) or rr > DIVERGENCE_LIMIT:
            return dict(x=x, iters=it, rr=rr, status=DIVERGED, state=st)
    return dict(x=x, iters=max_iter, rr=rr, status=NOT_CONVERGED, state=st)
