// Per-row flood update shared by the single-system and batched sweep kernels.
#pragma once

#include <cuda_runtime.h>

#include "gabp_internal.h"

namespace gabp {

// d == 0 or d not finite, decided on the bit pattern (integer pipe): the
// exponent field all ones is inf / NaN, all bits but the sign zero is +-0.
template <typename T>
__device__ __forceinline__ bool bad_den(T d);

template <>
__device__ __forceinline__ bool bad_den<double>(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return ((u >> 52) & 0x7ffull) == 0x7ffull || (u << 1) == 0ull;
}

template <>
__device__ __forceinline__ bool bad_den<float>(float d)
{
    const unsigned u = (unsigned)__float_as_int(d);
    return ((u >> 23) & 0xffu) == 0xffu || (u << 1) == 0u;
}

// x != 0 on the bit pattern (+-0 count as zero).
__device__ __forceinline__ bool nonzero(double x)
{
    return ((unsigned long long)__double_as_longlong(x) << 1) != 0ull;
}

__device__ __forceinline__ bool nonzero(float x)
{
    return ((unsigned)__float_as_int(x) << 1) != 0u;
}

// Reciprocal used by the message update.  Float: the correctly rounded
// reciprocal intrinsic.  Double: the hardware approximation rcp.approx.ftz.f64
// refined by one third-order Newton-Raphson step, y <- y (1 + e + e^2) with
// e = 1 - d y (the truncated series of 1 / (1 - e)); from the approximation's
// ~2^-22 relative error this lands within rounding of 1/d in three FMAs,
// against the longer sequence of an IEEE division.  A zero or non-finite d
// gives a non-finite result and is flagged by the caller.
template <typename T>
__device__ __forceinline__ T fast_rcp(T d);

template <>
__device__ __forceinline__ float fast_rcp<float>(float d)
{
    return __frcp_rn(d);
}

template <>
__device__ __forceinline__ double fast_rcp<double>(double d)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
    const double e = fma(-d, y, 1.0);
    const double e2 = fma(e, e, e);
    return fma(y, e2, y);
}

// Load of message state.  kCoherent (the batched solver, which reads state it
// wrote earlier in the same launch) goes through L2 with ld.global.cg and
// never through the non-coherent read-only path.
template <bool kCoherent, typename T>
__device__ __forceinline__ T ld_state(const T *p)
{
    if (kCoherent) return __ldcg(p);
    return *p;
}

// The loads of one row of the stencil flood update (below), held in registers.
template <typename T, int K>
struct StencilRow {
    T ae[K > 0 ? K : 1], ce[K > 0 ? K : 1], ps[K > 0 ? K : 1], bs[K > 0 ? K : 1],
        lr[K > 0 ? K : 1], mr[K > 0 ? K : 1];
    T dg, bb, bx, px;
    bool oob;  // bounds-checked build: a non-zero coefficient whose neighbour is outside [0, n)
};

template <typename T, int K, bool kCoherent = false>
__device__ __forceinline__ void stencil_row_load(
    int r, int n, const int *off, const int *krev, const T *__restrict__ a,
    const T *__restrict__ c, const T *__restrict__ diag, const T *__restrict__ b,
    const T *__restrict__ Lin, const T *__restrict__ Min, const T *__restrict__ Pin,
    const T *__restrict__ Bin, bool belief, StencilRow<T, K> &R)
{
    const size_t nn = (size_t)n;
    R.oob = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const size_t e = (size_t)k * nn + r;
        R.ae[k] = a[e];
        R.ce[k] = c[e];
        int s = r + off[k];
        if (kIndexChecks && nonzero(R.ae[k]) && (s < 0 || s >= n)) R.oob = true;
        s = s < 0 ? 0 : (s >= n ? n - 1 : s);
        const size_t er = (size_t)krev[k] * nn + s;
        R.ps[k] = ld_state<kCoherent>(Pin + s);
        R.bs[k] = ld_state<kCoherent>(Bin + s);
        R.lr[k] = ld_state<kCoherent>(Lin + er);
        R.mr[k] = ld_state<kCoherent>(Min + er);
    }
    R.dg = diag[r];
    R.bb = ld_state<kCoherent>(b + r);
    if (belief) {
        R.bx = ld_state<kCoherent>(Bin + r);
        R.px = ld_state<kCoherent>(Pin + r);
    }
}

// Returns FLAG_BREAKDOWN on a zero or non-finite denominator (and, in the
// bounds-checked build, FLAG_INDEX for a row whose layout is inconsistent).
template <typename T, int K>
__device__ __forceinline__ unsigned stencil_row_update(int r, int n, const StencilRow<T, K> &R,
                                                       T *__restrict__ Lout, T *__restrict__ Mout,
                                                       T *__restrict__ Pout, T *__restrict__ Bout,
                                                       double *__restrict__ x)
{
    const size_t nn = (size_t)n;
    T pn = R.dg;
    T bn = R.bb;
    if (x) x[r] = (double)(R.bx / R.px);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const size_t e = (size_t)k * nn + r;
        T lam = T(0), mu = T(0);
        if (nonzero(R.ae[k])) {
            const T d = R.ps[k] - R.lr[k];
            bad |= bad_den(d);
            const T q = fast_rcp(d);
            lam = R.ce[k] * q;
            mu = R.ae[k] * (R.bs[k] - R.mr[k]) * q;
        }
        Lout[e] = lam;
        Mout[e] = mu;
        pn += lam;
        bn += mu;
    }
    Pout[r] = pn;
    Bout[r] = bn;
    return (bad ? FLAG_BREAKDOWN : 0u) | (kIndexChecks && R.oob ? FLAG_INDEX : 0u);
}

// Flood update of row r in the stencil (per-diagonal) layout: slot k*n + r
// holds the entry (r, r + off[k]); its reverse edge is slot krev[k]*n + s,
// s = r + off[k].  With a_e = -A_rs, c_e = -A_rs A_sr and the aggregates
// P = diag + sum L, B = b + sum M of the previous state:
//     d = P_s - L[rev],  L' = c / d,  M' = a (B_s - M[rev]) / d,
// and the belief x_r = B_r / P_r of the previous state (Algorithm 1 forms the
// belief before the update).  All loads of the row are issued before any
// arithmetic: the reverse-edge gathers use an index clamped into [0, n), so
// they are always in bounds and need not wait for a_e; a padded slot
// (a_e == 0) discards what it loaded.  Returns the status bits of
// stencil_row_update.
template <typename T, int K, bool kCoherent = false>
__device__ __forceinline__ unsigned sweep_row_stencil(
    int r, int n, const int *off, const int *krev, const T *__restrict__ a,
    const T *__restrict__ c, const T *__restrict__ diag, const T *__restrict__ b,
    const T *__restrict__ Lin, const T *__restrict__ Min, const T *__restrict__ Pin,
    const T *__restrict__ Bin, T *__restrict__ Lout, T *__restrict__ Mout,
    T *__restrict__ Pout, T *__restrict__ Bout, double *__restrict__ x)
{
    StencilRow<T, K> R;
    stencil_row_load<T, K, kCoherent>(r, n, off, krev, a, c, diag, b, Lin, Min, Pin, Bin, x != nullptr, R);
    return stencil_row_update<T, K>(r, n, R, Lout, Mout, Pout, Bout, x);
}

// Mean-message update of row r with frozen precision messages (the fixed
// gains g_e = a_e / d_e): M'[e] = g_e (B_s - M[rev e]), B'_r = b_r + sum M'.
// Returns FLAG_INDEX (bounds-checked build only) for a non-zero gain whose
// neighbour lies outside [0, n), else 0.
template <typename T, int K, bool kCoherent = false>
__device__ __forceinline__ unsigned sweep_row_mean_stencil(
    int r, int n, const int *off, const int *krev, const T *__restrict__ g,
    const T *__restrict__ b, const T *__restrict__ P, const T *__restrict__ Min,
    const T *__restrict__ Bin, T *__restrict__ Mout, T *__restrict__ Bout, double *__restrict__ x)
{
    const size_t nn = (size_t)n;
    T ge[K > 0 ? K : 1], bs[K > 0 ? K : 1], mr[K > 0 ? K : 1];
    bool oob = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const size_t e = (size_t)k * nn + r;
        ge[k] = ld_state<kCoherent>(g + e);
        int s = r + off[k];
        if (kIndexChecks && nonzero(ge[k]) && (s < 0 || s >= n)) oob = true;
        s = s < 0 ? 0 : (s >= n ? n - 1 : s);
        bs[k] = ld_state<kCoherent>(Bin + s);
        mr[k] = ld_state<kCoherent>(Min + (size_t)krev[k] * nn + s);
    }
    T bn = ld_state<kCoherent>(b + r);
    if (x) x[r] = (double)(ld_state<kCoherent>(Bin + r) / ld_state<kCoherent>(P + r));
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const T mu = nonzero(ge[k]) ? ge[k] * (bs[k] - mr[k]) : T(0);
        Mout[(size_t)k * nn + r] = mu;
        bn += mu;
    }
    Bout[r] = bn;
    return kIndexChecks && oob ? FLAG_INDEX : 0u;
}

}  // namespace gabp
