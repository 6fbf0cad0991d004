"""GB300 Gaussian belief propagation (GaBP) for sparse nonsymmetric ``A x = b``.

Python binding over the C ABI of ``libgabp.so`` (declared in
``include/gabp.h``).  This module only marshals arguments: every step of
every solve runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  The binding fails loudly when the library is missing;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "GabpError", "GabpSolver", "Multigrid", "Batch", "load", "library_path", "STATUS",
    "OK", "BREAKDOWN", "DIVERGED", "NOT_CONVERGED", "fp64_peak",
]

OK, INVALID_ARG, BAD_CSR, ZERO_DIAG, BREAKDOWN, DIVERGED, NOT_CONVERGED, CUDA_ERR, OOM = range(9)
STATUS = {0: "ok", 1: "invalid argument", 2: "malformed CSR matrix",
          3: "missing or zero diagonal entry", 4: "breakdown", 5: "diverged",
          6: "not converged", 7: "CUDA error", 8: "out of memory"}
_PREC = {"fp64": 0, "fp32": 1, "fp32_ir": 2}
_LAYOUT = {"auto": 0, "csr": 1, "stencil": 2}
_MODE = {"cold": 0, "warm": 1, "persist": 2}


class GabpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("layout", ctypes.c_int),
                ("check_every", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("ir_inner_max", ctypes.c_int), ("ir_inner_tol", ctypes.c_double),
                ("block_size", ctypes.c_int), ("freeze_lambda", ctypes.c_int),
                ("reorder", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("edges", ctypes.c_int64),
                ("layout", ctypes.c_int), ("ndiag", ctypes.c_int), ("precision", ctypes.c_int),
                ("slots", ctypes.c_int64), ("sweep_bytes", ctypes.c_double),
                ("mean_sweep_bytes", ctypes.c_double),
                ("residual_bytes", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("parity_layout", ctypes.c_int), ("colored_sweep_bytes", ctypes.c_double),
                ("reordered", ctypes.c_int), ("colored_mean_sweep_bytes", ctypes.c_double)]


class PeakResult(ctypes.Structure):
    _fields_ = [("sms", ctypes.c_int), ("sms_seen", ctypes.c_int), ("blocks", ctypes.c_int),
                ("ms", ctypes.c_float), ("instructions", ctypes.c_double),
                ("per_cycle_per_sm", ctypes.c_double), ("per_cycle_per_sm_min", ctypes.c_double),
                ("per_cycle_per_sm_max", ctypes.c_double), ("per_second", ctypes.c_double),
                ("clock_mhz", ctypes.c_double)]


_lib = None


def library_path() -> str:
    """``libgabp.so``, or the bounds-checked ``libgabp_debug.so`` when the environment
    sets ``GABP_DEBUG=1`` (built by ``build.build(debug=True)``)."""
    return _build.LIB_DEBUG if os.environ.get("GABP_DEBUG") == "1" else _build.LIB


def load() -> ctypes.CDLL:
    """Loads ``libgabp.so``; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"GaBP CUDA library not built ({path} missing); "
                           "run __graft_entry__.build() or python -m paper_1904_04093_gb300.build")
    L = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    PI, PD, PF = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
    sigs = {
        "gabp_default_options": (None, [ctypes.POINTER(Options)]),
        "gabp_status_str": (ctypes.c_char_p, [I]),
        "gabp_last_error": (ctypes.c_char_p, []),
        "gabp_launch_count": (ctypes.c_ulonglong, []),
        "gabp_debug_build": (I, []),
        "gabp_setup": (I, [ctypes.c_int32, I64, P, P, P, ctypes.POINTER(Options), P, ctypes.POINTER(P)]),
        "gabp_set_values": (I, [P, P]),
        "gabp_set_values_device": (I, [P, P]),
        "gabp_destroy": (None, [P]),
        "gabp_reset": (I, [P]),
        "gabp_set_schedule": (I, [P, I, P, PI]),
        "gabp_get_line_state": (I, [P, P, P, P, P]),
        "gabp_sweep": (I, [P, P, I, P]),
        "gabp_solve": (I, [P, P, P, D, I, PI, PD]),
        "gabp_solve_transpose": (I, [P, P, P, D, I, PI, PD]),
        "gabp_edge_grad": (I, [P, P, P, P]),
        "gabp_residual": (I, [P, P, P, P, PD, PD]),
        "gabp_residual_2norm": (I, [P, P, P, PD, PD]),
        "gabp_get_state": (I, [P, P, P]),
        "gabp_set_state": (I, [P, P, P]),
        "gabp_get_info": (I, [P, ctypes.POINTER(Info)]),
        "gabp_time_sweeps": (I, [P, P, I, I, PF]),
        "gabp_fp64_peak": (I, [I, I, ctypes.POINTER(PeakResult)]),
        "mg_setup": (I, [I, ctypes.POINTER(P), ctypes.POINTER(ctypes.c_int32), D, I, P, ctypes.POINTER(P)]),
        "mg_vcycle": (I, [P, I, I, I, P, P]),
        "mg_solve": (I, [P, P, P, D, I, I, I, PI, PD]),
        "mg_destroy": (None, [P]),
        "mg_set_fused": (I, [P, I]),
        "gabp_batch_setup": (I, [I, ctypes.POINTER(P), I, P, ctypes.POINTER(P)]),
        "gabp_batch_tune": (I, [P, ctypes.POINTER(P), ctypes.POINTER(P), D, I, PI, PI]),
        "gabp_batch_set_shape": (I, [P, I, I]),
        "gabp_batch_solve": (I, [P, ctypes.POINTER(P), ctypes.POINTER(P), D, I, PI, PD, PI]),
        "gabp_batch_info": (I, [P, PI, PI, PI]),
        "gabp_batch_set_params": (I, [P, I, I, I]),
        "gabp_batch_params": (I, [P, PI, PI, PI]),
        "gabp_batch_destroy": (None, [P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def launch_count() -> int:
    """Kernel launches the library has enqueued in this process so far."""
    return int(load().gabp_launch_count())


_PEAK_OPS = {"fma": 0, "add": 1, "mul": 2, "rcp": 3}


def fp64_peak(op: str = "fma", iters: int = 1000) -> dict:
    """Measured FP64 instruction throughput of the current device (gabp_fp64_peak):
    instructions per SM cycle (clock-independent), per second, and the implied clock."""
    r = PeakResult()
    _check(load().gabp_fp64_peak(_PEAK_OPS[op], int(iters), ctypes.byref(r)))
    return {f: getattr(r, f) for f, _ in PeakResult._fields_}


def _err(st: int) -> GabpError:
    return GabpError(st, load().gabp_last_error().decode(errors="replace"))


def _check(st: int) -> None:
    if st != OK:
        raise _err(st)


def _torch():
    import torch
    return torch


def _dev_vec(t, n: int, name: str):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous() and t.numel() == n):
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of {n} elements")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream), stream


class GabpSolver:
    """A GaBP context for one sparse matrix (see ``include/gabp.h``).

    ``A`` is any object with ``n``, ``indptr`` (int64), ``indices`` (int32,
    sorted per row) and ``data`` (float64) arrays, e.g. ``problems.CSR``.

    Keyword arguments (the fields of ``gabp_options``):

    * ``precision``: ``"fp64"`` (messages, beliefs, residual in double),
      ``"fp32"`` (float messages, double residual checks) or ``"fp32_ir"``
      (float GaBP inside double iterative refinement; solves only);
    * ``layout``: ``"auto"`` (per-diagonal layout when the matrix has at most
      16 distinct diagonals), ``"stencil"`` or ``"csr"`` (any pattern);
    * ``check_every``: sweeps between residual checks of a solve;
    * ``use_graphs``: replay each chunk of sweeps from a captured CUDA graph;
    * ``ir_inner_max``, ``ir_inner_tol``: float sweeps per refinement step at
      most (0: 150 under the line and coloured schedules, 400 otherwise), and
      the inner relative residual that ends a step (``fp32_ir``);
    * ``block_size``: threads per block of the sweep kernel (0: the default);
    * ``freeze_lambda``: precomputed precision messages (Sec. 4.2): 1 on,
      0 off, -1 on for ``fp32_ir`` and off otherwise;
    * ``reorder``: CSR layout only: reverse Cuthill-McKee renumbering inside
      the library (1), none (0), or when it at least halves the mean index
      distance of coupled unknowns (-1); invisible at the interface;
    * ``stream``: a ``torch.cuda.Stream`` (default: the current stream).

    The product path has no CPU fallback: without the compiled library, or
    without a GPU, construction raises.
    """

    def __init__(self, A, precision: str = "fp64", layout: str = "auto", check_every: int = 10,
                 use_graphs: bool = True, ir_inner_max: int = 0, ir_inner_tol: float = 1e-3,
                 block_size: int = 0, freeze_lambda: int = -1, reorder: int = -1, stream=None):
        L = load()
        torch = _torch()
        self.n = int(A.n)
        self.indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self.indices = np.ascontiguousarray(A.indices, dtype=np.int32)
        data = np.ascontiguousarray(A.data, dtype=np.float64)
        self.nnz = int(self.indptr[-1]) if self.n else 0
        opt = Options()
        L.gabp_default_options(ctypes.byref(opt))
        opt.precision = _PREC[precision]
        opt.layout = _LAYOUT[layout]
        opt.check_every = int(check_every)
        opt.use_graphs = int(bool(use_graphs))
        opt.ir_inner_max = int(ir_inner_max)
        opt.ir_inner_tol = float(ir_inner_tol)
        opt.block_size = int(block_size)
        opt.freeze_lambda = int(freeze_lambda)
        opt.reorder = int(reorder)
        self.precision = precision
        self.device = torch.cuda.current_device()
        self._sh, self.stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(L.gabp_setup(self.n, self.nnz, self.indptr.ctypes.data, self.indices.ctypes.data,
                            data.ctypes.data, ctypes.byref(opt), self._sh, ctypes.byref(h)))
        self._h = h

    # -- lifetime --------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None):
            load().gabp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, t=None):
        torch = _torch()
        if t is None:
            t = torch.empty(self.n, dtype=torch.float64, device=f"cuda:{self.device}")
        return t

    # -- calls -------------------------------------------------------------
    def info(self) -> dict:
        inf = Info()
        _check(load().gabp_get_info(self._h, ctypes.byref(inf)))
        d = {f: getattr(inf, f) for f, _ in Info._fields_}
        d["layout"] = {1: "csr", 2: "stencil"}.get(d["layout"], d["layout"])
        return d

    def reset(self) -> None:
        _check(load().gabp_reset(self._h))

    def set_schedule(self, schedule: str = "flood", colors=None) -> int:
        """``"flood"`` (Sec. 2.2), ``"colored"`` (red-black / 4-colour, Sec. 5.1;
        ``colors`` n ints or greedy colouring) or ``"lines"`` (line GaBP,
        Algorithm 2 on the rows and columns of a square grid).  Returns the
        number of colours (0 unless coloured)."""
        nc = ctypes.c_int()
        cp = None
        if colors is not None:
            self._colors = np.ascontiguousarray(colors, dtype=np.int32)
            cp = self._colors.ctypes.data
        code = {"flood": 0, "colored": 1, "lines": 2}[schedule]
        _check(load().gabp_set_schedule(self._h, code, cp, ctypes.byref(nc)))
        return int(nc.value)

    def get_line_state(self):
        torch = _torch()
        out = [torch.empty(self.n, dtype=torch.float64, device=f"cuda:{self.device}") for _ in range(4)]
        _check(load().gabp_get_line_state(self._h, *[_dev_vec(t, self.n, "state") for t in out]))
        return {"LH": out[0], "MH": out[1], "LV": out[2], "MV": out[3]}

    def set_values(self, data) -> None:
        """New matrix values on the same pattern (setup slot order): a numpy
        array or a host tensor goes through ``gabp_set_values``, a CUDA tensor
        through ``gabp_set_values_device`` (no host assembly)."""
        torch = _torch()
        if isinstance(data, torch.Tensor) and data.is_cuda:
            t = data.detach().to(torch.float64).contiguous()
            assert t.shape == (self.nnz,)
            _check(load().gabp_set_values_device(self._h, _dev_vec(t, self.nnz, "values")))
            return
        if isinstance(data, torch.Tensor):
            data = data.detach().cpu().numpy()
        data = np.ascontiguousarray(data, dtype=np.float64)
        assert data.shape == (self.nnz,)
        _check(load().gabp_set_values(self._h, data.ctypes.data))

    def sweep(self, b, nsweeps: int, x=None):
        x = self._vec(x)
        _check(load().gabp_sweep(self._h, _dev_vec(b, self.n, "b"), int(nsweeps),
                                 _dev_vec(x, self.n, "x")))
        return x

    def time_sweeps(self, b, nsweeps: int, frozen: bool = False) -> float:
        ms = ctypes.c_float()
        _check(load().gabp_time_sweeps(self._h, _dev_vec(b, self.n, "b"), int(nsweeps),
                                       int(bool(frozen)), ctypes.byref(ms)))
        return float(ms.value)

    def _solve(self, fn, b, tol, max_iter, x, raise_on):
        x = self._vec(x)
        it = ctypes.c_int()
        rr = ctypes.c_double()
        st = fn(self._h, _dev_vec(b, self.n, "b"), _dev_vec(x, self.n, "x"), float(tol),
                int(max_iter), ctypes.byref(it), ctypes.byref(rr))
        if st not in (OK, NOT_CONVERGED, BREAKDOWN, DIVERGED) or st in raise_on:
            raise _err(st)
        return x, int(it.value), float(rr.value), int(st)

    def solve(self, b, tol: float = 1e-10, max_iter: int = 10000, x=None, raise_on=()):
        """Returns ``(x, sweeps, relres, status)``."""
        return self._solve(load().gabp_solve, b, tol, max_iter, x, raise_on)

    def solve_transpose(self, g, tol: float = 1e-10, max_iter: int = 10000, lam=None, raise_on=()):
        return self._solve(load().gabp_solve_transpose, g, tol, max_iter, lam, raise_on)

    def edge_grad(self, lam, x, dA=None):
        torch = _torch()
        if dA is None:
            dA = torch.empty(self.nnz, dtype=torch.float64, device=f"cuda:{self.device}")
        _check(load().gabp_edge_grad(self._h, _dev_vec(lam, self.n, "lam"),
                                     _dev_vec(x, self.n, "x"), _dev_vec(dA, self.nnz, "dA")))
        return dA

    def residual(self, b, x, r=None):
        """Returns ``(r or None, ||b - A x||_inf, ||b||_inf)``."""
        rinf, binf = ctypes.c_double(), ctypes.c_double()
        rp = _dev_vec(r, self.n, "r") if r is not None else None
        _check(load().gabp_residual(self._h, _dev_vec(b, self.n, "b"), _dev_vec(x, self.n, "x"),
                                    rp, ctypes.byref(rinf), ctypes.byref(binf)))
        return r, float(rinf.value), float(binf.value)

    def residual_norms(self, b, x) -> dict:
        """Relative residual of ``x`` in the infinity norm (the stopping quantity of
        Algorithm 1) and in the 2-norm: ``{"rr_inf": ..., "rr_2": ...}``."""
        _, rinf, binf = self.residual(b, x)
        r2, b2 = ctypes.c_double(), ctypes.c_double()
        _check(load().gabp_residual_2norm(self._h, _dev_vec(b, self.n, "b"), _dev_vec(x, self.n, "x"),
                                          ctypes.byref(r2), ctypes.byref(b2)))
        return {"rr_inf": rinf / binf if binf > 0 else 0.0,
                "rr_2": r2.value / b2.value if b2.value > 0 else 0.0}

    def get_state(self):
        torch = _torch()
        lam = torch.empty(self.nnz, dtype=torch.float64, device=f"cuda:{self.device}")
        m = torch.empty_like(lam)
        _check(load().gabp_get_state(self._h, _dev_vec(lam, self.nnz, "lam"),
                                     _dev_vec(m, self.nnz, "m")))
        return lam, m

    def set_state(self, lam=None, m=None):
        lp = _dev_vec(lam, self.nnz, "lam") if lam is not None else None
        mp = _dev_vec(m, self.nnz, "m") if m is not None else None
        _check(load().gabp_set_state(self._h, lp, mp))


class Multigrid:
    """V-cycle with GaBP smoothing over level solvers, finest first (Sec. 4)."""

    def __init__(self, levels, sides, transfer_scale: float = 4.0, mode: str = "cold",
                 schedule: str = "flood", stream=None):
        L = load()
        self.levels = list(levels)
        for lv in self.levels:
            lv.set_schedule(schedule)
        self.sides = [int(s) for s in sides]
        self._sh, self.stream = _stream_handle(stream)
        arr = (ctypes.c_void_p * len(self.levels))(*[lv._h for lv in self.levels])
        sides_c = (ctypes.c_int32 * len(self.sides))(*self.sides)
        h = ctypes.c_void_p()
        _check(L.mg_setup(len(self.levels), arr, sides_c, float(transfer_scale), _MODE[mode],
                          self._sh, ctypes.byref(h)))
        self._h = h
        self.n = self.levels[0].n

    def close(self):
        if getattr(self, "_h", None):
            load().mg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fused(self, fused: bool):
        """Fused transfer kernels (default where the levels allow them) or one kernel per
        step; the two compute the same operations in the same order (mg_set_fused)."""
        _check(load().mg_set_fused(self._h, int(bool(fused))))

    def vcycle(self, b, x, nu_pre: int, nu_post: int, levels: int = 0):
        _check(load().mg_vcycle(self._h, int(levels), int(nu_pre), int(nu_post),
                                _dev_vec(b, self.n, "b"), _dev_vec(x, self.n, "x")))
        return x

    def solve(self, b, tol: float, max_cycles: int, nu_pre: int, nu_post: int, x=None):
        torch = _torch()
        if x is None:
            x = torch.empty(self.n, dtype=torch.float64, device=b.device)
        c, rr = ctypes.c_int(), ctypes.c_double()
        st = load().mg_solve(self._h, _dev_vec(b, self.n, "b"), _dev_vec(x, self.n, "x"),
                             float(tol), int(max_cycles), int(nu_pre), int(nu_post),
                             ctypes.byref(c), ctypes.byref(rr))
        if st not in (OK, NOT_CONVERGED, DIVERGED, BREAKDOWN):
            raise _err(st)
        return x, int(c.value), float(rr.value), int(st)


class Batch:
    """Many independent systems solved in one persistent launch (see ``include/gabp.h``)."""

    def __init__(self, solvers, check_every: int = 10, stream=None):
        L = load()
        self.solvers = list(solvers)
        self.nsys = len(self.solvers)
        self._sh, self.stream = _stream_handle(stream)
        arr = (ctypes.c_void_p * self.nsys)(*[s._h for s in self.solvers])
        h = ctypes.c_void_p()
        _check(L.gabp_batch_setup(self.nsys, arr, int(check_every), self._sh, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().gabp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _tables(self, bs, xs):
        torch = _torch()
        if xs is None:
            xs = [torch.empty(s.n, dtype=torch.float64, device=b.device) for s, b in zip(self.solvers, bs)]
        bt = (ctypes.c_void_p * self.nsys)(*[_dev_vec(b, s.n, "b").value for s, b in zip(self.solvers, bs)])
        xt = (ctypes.c_void_p * self.nsys)(*[_dev_vec(x, s.n, "x").value for s, x in zip(self.solvers, xs)])
        return xs, bt, xt

    def tune(self, bs, tol: float, max_iter: int, xs=None):
        xs, bt, xt = self._tables(bs, xs)
        blk, cs = ctypes.c_int(), ctypes.c_int()
        _check(load().gabp_batch_tune(self._h, bt, xt, float(tol), int(max_iter), ctypes.byref(blk),
                                      ctypes.byref(cs)))
        return int(blk.value), int(cs.value)

    def set_shape(self, block: int, cluster: int):
        _check(load().gabp_batch_set_shape(self._h, int(block), int(cluster)))

    def set_params(self, rows: int = 0, min_rows: int = 0, check_every: int = 0):
        """Rows in flight per thread, rows per cluster thread for a cluster team, check
        interval (0 keeps one; gabp_batch_set_params)."""
        _check(load().gabp_batch_set_params(self._h, int(rows), int(min_rows), int(check_every)))

    def info(self):
        blk, cs, grid = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().gabp_batch_info(self._h, ctypes.byref(blk), ctypes.byref(cs), ctypes.byref(grid)))
        r, mr, ce = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().gabp_batch_params(self._h, ctypes.byref(r), ctypes.byref(mr), ctypes.byref(ce)))
        return {"block": blk.value, "cluster": cs.value, "grid": grid.value, "rows": r.value,
                "min_rows": mr.value, "check_every": ce.value}

    def solve(self, bs, tol: float, max_iter: int, xs=None):
        """Returns ``(xs, iters, relres, status)`` (lists over systems)."""
        xs, bt, xt = self._tables(bs, xs)
        it = (ctypes.c_int * self.nsys)()
        rr = (ctypes.c_double * self.nsys)()
        stt = (ctypes.c_int * self.nsys)()
        st = load().gabp_batch_solve(self._h, bt, xt, float(tol), int(max_iter), it, rr, stt)
        if st not in (OK, NOT_CONVERGED, BREAKDOWN, DIVERGED):
            raise _err(st)
        return xs, list(it), list(rr), list(stt)
