"""Element-wise error scales for one flood sweep (test helper, CPU only).

A normwise check (max error over the largest value) lets a small output be
wrong by far more than its own rounding.  The element-wise check below holds
every output of one sweep to a tolerance relative to the magnitude of the
terms it is computed from, which is the natural floor of its rounding error
(a sum that cancels can lose every digit of a small result, but not more than
the size of its terms).  For the slot e = (r, s) (the message s -> r as its
effect on row r: ``Lc = tilde-Lambda_sr A_sr`` and ``m_sr``, eq.
nonsymmetric_GaBP_rules) with ``d_e = A_ss + sum_{k in N(s) \\ r} Lc_ks``:

    scale_L[e] = |Lc'_e| (1 + S_P(s, e) / |d_e|)
    scale_M[e] = (|A_rs| (|b_s| + sum_{k in N(s)} |m_ks| + |m_rs|) + |m'_e| S_P(s, e)) / |d_e|
    S_P(s, e)  = |A_ss| + sum_{k in N(s)} |Lc_ks| + |Lc_rs|
    scale_x[r] = (|b_r| + sum_k |m_kr| + |x_r| (|A_rr| + sum_k |Lc_kr|)) / |beta_r|

computed from the oracle's state before the sweep.  A slot with no message
(diagonal or stored zero) has scale 0 and must be exactly 0.
"""
import numpy as np


def _rows(A):
    return np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.indptr))


def reverse_slots(A):
    """rev[e] = slot of (s, r) for the slot e = (r, s), -1 where it is not stored."""
    rows = _rows(A)
    cols = A.indices.astype(np.int64)
    keys = rows * A.n + cols  # ascending: CSR rows in order, columns sorted
    want = cols * A.n + rows
    pos = np.searchsorted(keys, want)
    pos = np.minimum(pos, len(keys) - 1)
    return np.where(keys[pos] == want, pos, -1)


def sweep_scales(A, b, lc, mm, x, beta, lc2, mm2):
    """Scales of (x, Lc', m') for one sweep from the state (lc, mm): lc = the
    precision messages as effects on their rows (oracle.diag_contrib), x, beta the
    oracle's beliefs and precisions of that state, lc2, mm2 its update."""
    rows = _rows(A)
    cols = A.indices.astype(np.int64)
    isdiag = rows == cols
    msg = (~isdiag) & (A.data != 0.0)
    diag = np.zeros(A.n)
    diag[rows[isdiag]] = A.data[isdiag]
    abs_p = np.abs(diag) + np.bincount(rows, weights=np.abs(lc) * msg, minlength=A.n)
    abs_b = np.abs(b) + np.bincount(rows, weights=np.abs(mm) * msg, minlength=A.n)
    p = diag + np.bincount(rows, weights=lc * msg, minlength=A.n)
    rev = reverse_slots(A)
    has = rev >= 0
    lc_rev = np.where(has, lc[np.maximum(rev, 0)], 0.0)
    mm_rev = np.where(has, mm[np.maximum(rev, 0)], 0.0)
    s = cols
    d = p[s] - lc_rev
    sp = abs_p[s] + np.abs(lc_rev)
    with np.errstate(divide="ignore", invalid="ignore"):
        scale_l = np.where(msg, np.abs(lc2) * (1.0 + sp / np.abs(d)), 0.0)
        scale_m = np.where(msg, (np.abs(A.data) * (abs_b[s] + np.abs(mm_rev)) + np.abs(mm2) * sp)
                           / np.abs(d), 0.0)
        scale_x = (abs_b + np.abs(x) * abs_p) / np.abs(beta)
    return scale_x, scale_l, scale_m


def worst_elementwise(got, ref, scale):
    """max_e |got_e - ref_e| / scale_e (0 where both are exactly equal); inf if an
    element with scale 0 differs."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    err = np.abs(got - ref)
    if np.any(err[scale == 0.0] != 0.0):
        return float("inf")
    nz = scale > 0.0
    return float(np.max(err[nz] / scale[nz])) if np.any(nz) else 0.0
