// CUDA kernels of the GaBP library (sm_103a).
//
// Message state: for the directed edge s -> r (matrix entry (r, s), A_rs != 0,
// Sec. 2.3) the library stores
//     L[e] = tilde-Lambda_sr * A_sr   (the message's correction to the diagonal of row r)
//     M[e] = m_sr                      (its correction to the right-hand side of row r)
// and per node the aggregates
//     P_r = A_rr + sum_{e in row r} L[e],   B_r = b_r + sum_{e in row r} M[e].
// With a_e = -A_rs and c_e = -A_rs * A_sr, the flood update of
// eq. nonsymmetric_GaBP_rules becomes, for e = (r, s) and its reverse edge
// rev(e) = (s, r):
//     d_e = P_s - L[rev(e)]                (node s's precision without r's message)
//     L'[e] = c_e / d_e,   M'[e] = a_e (B_s - M[rev(e)]) / d_e
// and the belief of Algorithm 1 is x_r = B_r / P_r, formed from the
// aggregates before the update.  Every thread owns one row r, so the new
// aggregates P'_r, B'_r are summed in registers (no atomics, deterministic).
//
// Two layouts:
//  * stencil (per-diagonal): slot e = k*n + r holds the entry (r, r + off[k]);
//    the reverse edge sits on the diagonal krev[k] (offset -off[k]) at row
//    r + off[k], so every gather is a contiguous, shifted, coalesced stream
//    and no index array is read;
//  * CSR: symmetrised pattern with explicit column and reverse-edge indices.
// Padded or explicit-zero slots have a_e = 0 and carry the zero message.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "gabp_internal.h"
#include "sweep_row.cuh"

namespace gabp {

static std::atomic<unsigned long long> g_launches{0};

// Counts `k` kernel launches enqueued on `s`, unless `s` is being captured
// into a graph (graph replays are counted by the caller when launched).
void count_launches(cudaStream_t s, unsigned long long k)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return;
    g_launches.fetch_add(k, std::memory_order_relaxed);
}

unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

// ---------------------------------------------------------------------------
// Message sweep, stencil layout: one thread per row (sweep_row_stencil in
// sweep_row.cuh, shared with the batched solver).
// ---------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(256) k_sweep_stencil(
    int n, StencilParams sp, const T *__restrict__ a, const T *__restrict__ c,
    const T *__restrict__ diag, const T *__restrict__ b, const T *__restrict__ Lin,
    const T *__restrict__ Min, const T *__restrict__ Pin, const T *__restrict__ Bin,
    T *__restrict__ Lout, T *__restrict__ Mout, T *__restrict__ Pout, T *__restrict__ Bout,
    double *__restrict__ x, unsigned *__restrict__ flags)
{
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const unsigned f = sweep_row_stencil<T, K>(r, n, sp.off, sp.krev, a, c, diag, b, Lin, Min, Pin,
                                               Bin, Lout, Mout, Pout, Bout, x);
    if (f) atomicOr(flags, f);
}

// ---------------------------------------------------------------------------
// Frozen precision messages (the precomputed tilde-Lambda of Sec. 4.2)
//
// tilde-Lambda does not depend on b (Sec. 2.3).  Once it has converged, the
// precision update returns the same values, so a sweep only has to move the
// mean messages: with the fixed g_e = a_e / d_e, d_e = P_s - L[rev e],
//     M'[e] = g_e (B_s - M[rev e]),   B'_r = b_r + sum_{e in row r} M'[e],
// and the beliefs are x_r = B_r / P_r with the fixed P.
// ---------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(256) k_freeze_stencil(int n, StencilParams sp,
                                                        const T *__restrict__ a,
                                                        const T *__restrict__ P,
                                                        const T *__restrict__ Lm,
                                                        T *__restrict__ g,
                                                        unsigned *__restrict__ flags)
{
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const size_t nn = (size_t)n;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const size_t e = (size_t)k * nn + r;
        const T ae = a[e];
        T ge = T(0);
        if (ae != T(0)) {
            const int s = r + sp.off[k];
            const T d = P[s] - Lm[(size_t)sp.krev[k] * nn + s];
            bad |= bad_den(d);
            ge = ae * fast_rcp(d);
        }
        g[e] = ge;
    }
    if (bad) atomicOr(flags, FLAG_BREAKDOWN);
}

template <typename T>
__global__ void k_freeze_csr(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                             const int *__restrict__ rev, const T *__restrict__ a,
                             const T *__restrict__ P, const T *__restrict__ Lm,
                             T *__restrict__ g, unsigned *__restrict__ flags)
{
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    bool bad = false;
    for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        const T ae = a[e];
        T ge = T(0);
        if (ae != T(0)) {
            const T d = P[col[e]] - Lm[rev[e]];
            bad |= bad_den(d);
            ge = ae * fast_rcp(d);
        }
        g[e] = ge;
    }
    if (bad) atomicOr(flags, FLAG_BREAKDOWN);
}

template <typename T, int K>
__global__ void __launch_bounds__(256) k_sweep_mean_stencil(
    int n, StencilParams sp, const T *__restrict__ g, const T *__restrict__ b,
    const T *__restrict__ P, const T *__restrict__ Min, const T *__restrict__ Bin,
    T *__restrict__ Mout, T *__restrict__ Bout, double *__restrict__ x, unsigned *flags)
{
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const size_t nn = (size_t)n;
    T ge[K > 0 ? K : 1], bs[K > 0 ? K : 1], mr[K > 0 ? K : 1];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const size_t e = (size_t)k * nn + r;
        ge[k] = g[e];
        int s = r + sp.off[k];
        if (kIndexChecks && nonzero(ge[k]) && (s < 0 || s >= n)) atomicOr(flags, FLAG_INDEX);
        s = s < 0 ? 0 : (s >= n ? n - 1 : s);
        bs[k] = Bin[s];
        mr[k] = Min[(size_t)sp.krev[k] * nn + s];
    }
    T bn = b[r];
    if (x) x[r] = (double)(Bin[r] / P[r]);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const T mu = nonzero(ge[k]) ? ge[k] * (bs[k] - mr[k]) : T(0);
        Mout[(size_t)k * nn + r] = mu;
        bn += mu;
    }
    Bout[r] = bn;
}

// max |L1 - L0| and max |L1| over all slots (convergence of the precision messages)
template <typename T>
__global__ void __launch_bounds__(256) k_lambda_change(int64_t slots, const T *__restrict__ L0,
                                                       const T *__restrict__ L1, DevStatus *st);

// ---------------------------------------------------------------------------
// Coloured schedule (red-black / 4-colour GaBP, Sec. 5.1): one launch per
// colour class c.  Phase c replaces, in place, every message sent by a node
// of colour c (stored in its recipients' rows) from the current messages,
// and every row not of colour c moves its aggregates by the change of its
// messages.  Race-free in place: phase c reads the aggregates and the
// incoming messages only of colour-c nodes, and writes only slots sent by
// colour-c nodes and aggregates of other colours (adjacent nodes differ in
// colour).
// A row of colour c forms its belief in phase c from the aggregates it has
// then (Algorithm 1: the belief before the node's messages are replaced).
// ---------------------------------------------------------------------------
// Stencil layout without a table: the sender's colour is read per slot.
template <typename T, int K>
__global__ void __launch_bounds__(256) k_sweep_color_stencil_gather(
    int n, StencilParams sp, const unsigned char *__restrict__ color, int cphase,
    const T *__restrict__ a, const T *__restrict__ c, T *Lm, T *Mm, T *P, T *B,
    double *__restrict__ x, unsigned *__restrict__ flags)
{
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const size_t nn = (size_t)n;
    if (color[r] == cphase) {
        if (x) x[r] = (double)(B[r] / P[r]);
        return;
    }
    T dp = T(0), db = T(0);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const size_t e = (size_t)k * nn + r;
        const T ae = a[e];
        if (!nonzero(ae)) continue;
        const int s = r + sp.off[k];
        if (color[s] != cphase) continue;
        const size_t er = (size_t)sp.krev[k] * nn + s;
        const T d = P[s] - Lm[er];
        bad |= bad_den(d);
        const T q = fast_rcp(d);
        const T lam = c[e] * q;
        const T mu = ae * (B[s] - Mm[er]) * q;
        dp += lam - Lm[e];
        db += mu - Mm[e];
        Lm[e] = lam;
        Mm[e] = mu;
    }
    P[r] += dp;
    B[r] += db;
    if (bad) atomicOr(flags, FLAG_BREAKDOWN);
}

// Stencil layout with a colour table: masks[cr][cphase] has bit k set when the
// slot k of a row of colour cr carries a message sent by colour cphase (the
// same for every row of colour cr: checked when the schedule is set).  Only
// those slots are touched, and the row's aggregates move by the change of
// its messages, so every slot is read and written once per sweep.
template <typename T, int K>
__global__ void __launch_bounds__(256) k_sweep_color_stencil(
    int n, StencilParams sp, ColorMasks cm, const unsigned char *__restrict__ color, int cphase,
    const T *__restrict__ a, const T *__restrict__ c, T *Lm, T *Mm, T *P, T *B,
    double *__restrict__ x, unsigned *__restrict__ flags)
{
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const size_t nn = (size_t)n;
    const int cr = color[r];
    if (cr == cphase) {
        if (x) x[r] = (double)(B[r] / P[r]);
        return;
    }
    const unsigned mask = cm.m[cr][cphase];
    if (!mask) return;
    T dp = T(0), db = T(0);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (!(mask & (1u << k))) continue;
        const size_t e = (size_t)k * nn + r;
        const T ae = a[e];
        if (!nonzero(ae)) continue;
        const int s = r + sp.off[k];
        const size_t er = (size_t)sp.krev[k] * nn + s;
        const T d = P[s] - Lm[er];
        bad |= bad_den(d);
        const T q = fast_rcp(d);
        const T lam = c[e] * q;
        const T mu = ae * (B[s] - Mm[er]) * q;
        dp += lam - Lm[e];
        db += mu - Mm[e];
        Lm[e] = lam;
        Mm[e] = mu;
    }
    P[r] += dp;
    B[r] += db;
    if (bad) atomicOr(flags, FLAG_BREAKDOWN);
}

template <typename T>
__global__ void __launch_bounds__(256) k_sweep_color_csr(
    int n, const int *__restrict__ rowptr, const int *__restrict__ col, const int *__restrict__ rev,
    const unsigned char *__restrict__ color, int cphase, const T *__restrict__ a,
    const T *__restrict__ c, T *Lm, T *Mm, T *P, T *B, double *__restrict__ x,
    unsigned *__restrict__ flags)
{
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    if (color[r] == cphase) {
        if (x) x[r] = (double)(B[r] / P[r]);
        return;
    }
    T dp = T(0), db = T(0);
    bool bad = false;
    for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        const int s = col[e];
        if (color[s] != cphase) continue;
        const T ae = a[e];
        if (!nonzero(ae)) continue;
        const int er = rev[e];
        const T d = P[s] - Lm[er];
        bad |= bad_den(d);
        const T q = fast_rcp(d);
        const T lam = c[e] * q;
        const T mu = ae * (B[s] - Mm[er]) * q;
        dp += lam - Lm[e];
        db += mu - Mm[e];
        Lm[e] = lam;
        Mm[e] = mu;
    }
    P[r] += dp;
    B[r] += db;
    if (bad) atomicOr(flags, FLAG_BREAKDOWN);
}

// ---------------------------------------------------------------------------
// Aggregates from a message state: P = diag + sum L, B = b + sum M (per row)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_aggregate_stencil(int n, int K, const T *__restrict__ diag,
                                    const T *__restrict__ b, const T *__restrict__ Lm,
                                    const T *__restrict__ Mm, T *__restrict__ P,
                                    T *__restrict__ B)
{
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    T p = diag[r], q = b[r];
    for (int k = 0; k < K; ++k) {
        p += Lm[(size_t)k * n + r];
        q += Mm[(size_t)k * n + r];
    }
    P[r] = p;
    B[r] = q;
}

template <typename T>
__global__ void k_aggregate_csr(int n, const int *__restrict__ rowptr, const T *__restrict__ diag,
                                const T *__restrict__ b, const T *__restrict__ Lm,
                                const T *__restrict__ Mm, T *__restrict__ P, T *__restrict__ B)
{
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    T p = diag[r], q = b[r];
    for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        p += Lm[e];
        q += Mm[e];
    }
    P[r] = p;
    B[r] = q;
}

// ---------------------------------------------------------------------------
// Residual r = b - A x in double with max |r|, max |b| (block reduction, then
// one atomicMax per block on the bit pattern of a non-negative double).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void reduce_and_publish(double rmax, double bmax, bool nan,
                                                   DevStatus *st)
{
    __shared__ double sr[32], sb[32];
    __shared__ int snan;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) snan = 0;
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) {
        rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
    }
    if (nan) snan = 1;
    if (lane == 0) {
        sr[wid] = rmax;
        sb[wid] = bmax;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        rmax = lane < nw ? sr[lane] : 0.0;
        bmax = lane < nw ? sb[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
            bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
        }
        if (lane == 0) {
            atomicMax(&st->rmax, (unsigned long long)__double_as_longlong(rmax));
            atomicMax(&st->bmax, (unsigned long long)__double_as_longlong(bmax));
            if (snan) atomicOr(&st->flags, FLAG_NAN);
        }
    }
}

// Block maxima of |r| and |b| as bit patterns of non-negative doubles (their
// order is the unsigned integer order), so the comparisons run on the integer
// pipe; one atomicMax per block.
__device__ __forceinline__ void reduce_and_publish_bits(unsigned long long rbits,
                                                        unsigned long long bbits, bool nan,
                                                        DevStatus *st)
{
    __shared__ unsigned long long sr[32], sb[32];
    __shared__ int snan;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) snan = 0;
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) {
        rbits = max(rbits, __shfl_xor_sync(0xffffffffu, rbits, o));
        bbits = max(bbits, __shfl_xor_sync(0xffffffffu, bbits, o));
    }
    if (nan) snan = 1;
    if (lane == 0) {
        sr[wid] = rbits;
        sb[wid] = bbits;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        rbits = lane < nw ? sr[lane] : 0ull;
        bbits = lane < nw ? sb[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
            rbits = max(rbits, __shfl_xor_sync(0xffffffffu, rbits, o));
            bbits = max(bbits, __shfl_xor_sync(0xffffffffu, bbits, o));
        }
        if (lane == 0) {
            atomicMax(&st->rmax, rbits);
            atomicMax(&st->bmax, bbits);
            if (snan) atomicOr(&st->flags, FLAG_NAN);
        }
    }
}

__device__ __forceinline__ unsigned long long abs_bits(double v)
{
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// Two rows per thread per step, grid-strided; every load of both rows (the
// coefficients and the x gathers at clamped, always in-bounds indices) is
// issued before the arithmetic, so no gather waits for its coefficient.  A
// padded slot has a = 0 and contributes 0 * x (x finite).
template <int K>
__global__ void __launch_bounds__(256) k_residual_stencil(
    int n, StencilParams sp, const double *__restrict__ a64, const double *__restrict__ diag64,
    const double *__restrict__ b, const double *__restrict__ x, double *__restrict__ r,
    float *__restrict__ rf, DevStatus *st)
{
    pdl_wait();
    pdl_trigger();
    constexpr int KK = K > 0 ? K : 1;
    unsigned long long rbits = 0ull, bbits = 0ull;
    bool nan = false;
    const size_t nn = (size_t)n;
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 2 * stride) {
        double av[2][KK], xv[2][KK], bi[2], di[2], xi[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = min(i0 + u * stride, n - 1);
            bi[u] = b[i];
            di[u] = diag64[i];
            xi[u] = x[i];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                int s = i + sp.off[k];
                av[u][k] = a64[(size_t)k * nn + i];
                if (kIndexChecks && av[u][k] != 0.0 && (s < 0 || s >= n)) atomicOr(&st->flags, FLAG_INDEX);
                s = s < 0 ? 0 : (s >= n ? n - 1 : s);
                xv[u][k] = x[s];
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = i0 + u * stride;
            if (i >= n) continue;
            double acc = fma(-di[u], xi[u], bi[u]);
#pragma unroll
            for (int k = 0; k < K; ++k) acc = fma(av[u][k], xv[u][k], acc);
            if (r) r[i] = acc;
            if (rf) rf[i] = (float)acc;
            const unsigned long long ab = abs_bits(acc);
            if (ab > 0x7ff0000000000000ull) nan = true;
            else rbits = max(rbits, ab);
            bbits = max(bbits, abs_bits(bi[u]));
        }
    }
    reduce_and_publish_bits(rbits, bbits, nan, st);
}

__global__ void __launch_bounds__(256) k_residual_csr(
    int n, const int *__restrict__ rowptr, const int *__restrict__ col,
    const double *__restrict__ a64, const double *__restrict__ diag64,
    const double *__restrict__ b, const double *__restrict__ x, double *__restrict__ r,
    DevStatus *st)
{
    pdl_wait();
    pdl_trigger();
    double rmax = 0.0, bmax = 0.0;
    bool nan = false;
    const int nslots = kIndexChecks ? rowptr[n] : 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double bi = b[i];
        double acc = bi - diag64[i] * x[i];
        int e0 = rowptr[i], e1 = rowptr[i + 1];
        if (kIndexChecks && !(0 <= e0 && e0 <= e1 && e1 <= nslots)) {
            atomicOr(&st->flags, FLAG_INDEX);
            e0 = e1 = 0;
        }
        for (int e = e0; e < e1; ++e) {
            const double ae = a64[e];
            const int j = col[e];
            if (kIndexChecks && (unsigned)j >= (unsigned)n) {
                atomicOr(&st->flags, FLAG_INDEX);
                continue;
            }
            if (ae != 0.0) acc += ae * x[j];
        }
        if (r) r[i] = acc;
        const double v = fabs(acc);
        if (v != v) nan = true;
        else rmax = fmax(rmax, v);
        bmax = fmax(bmax, fabs(bi));
    }
    reduce_and_publish(rmax, bmax, nan, st);
}

template <typename T>
__global__ void __launch_bounds__(256) k_lambda_change(int64_t slots, const T *__restrict__ L0,
                                                       const T *__restrict__ L1, DevStatus *st)
{
    pdl_wait();
    pdl_trigger();
    double dmax = 0.0, lmax = 0.0;
    bool nan = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < slots;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double l1 = (double)L1[e];
        const double d = fabs(l1 - (double)L0[e]);
        if (d != d) nan = true;
        else dmax = fmax(dmax, d);
        lmax = fmax(lmax, fabs(l1));
    }
    reduce_and_publish(dmax, lmax, nan, st);
}

// ---------------------------------------------------------------------------
// Small vector kernels
// ---------------------------------------------------------------------------
__global__ void k_d2f(const double *__restrict__ in, float *__restrict__ out, int64_t n)
{
    pdl_wait();
    pdl_trigger();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

__global__ void k_f2d(const float *__restrict__ in, double *__restrict__ out, int64_t n)
{
    pdl_wait();
    pdl_trigger();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

__global__ void k_copy(const double *__restrict__ in, double *__restrict__ out, int64_t n)
{
    pdl_wait();
    pdl_trigger();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

template <typename T>
__global__ void k_scale_rhs(const double *__restrict__ in, const DevStatus *st,
                            double *__restrict__ out, T *__restrict__ outT, int64_t n)
{
    pdl_wait();
    pdl_trigger();
    const double s = __longlong_as_double((long long)st->rmax);
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = in[i] * inv;
        out[i] = v;
        if (outT) outT[i] = (T)v;
    }
}

__global__ void k_axpy_status(double *__restrict__ x, const double *__restrict__ e,
                              const DevStatus *st, int64_t n)
{
    pdl_wait();
    pdl_trigger();
    const double s = __longlong_as_double((long long)st->rmax);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] += s * e[i];
}

__global__ void k_axpy(double *__restrict__ x, const double *__restrict__ e, double alpha,
                       int64_t n)
{
    pdl_wait();
    pdl_trigger();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] += alpha * e[i];
}

template <typename T>
__global__ void k_get_state(const int64_t *__restrict__ slotmap, int64_t nnz,
                            const T *__restrict__ Lm, const T *__restrict__ Mm,
                            double *__restrict__ lam, double *__restrict__ m)
{
    pdl_wait();
    pdl_trigger();
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = slotmap[p];
        if (lam) lam[p] = q < 0 ? 0.0 : (double)Lm[q];
        if (m) m[p] = q < 0 ? 0.0 : (double)Mm[q];
    }
}

template <typename T>
__global__ void k_set_state(const int64_t *__restrict__ slotmap, int64_t nnz,
                            const double *__restrict__ lam, const double *__restrict__ m,
                            T *__restrict__ Lm, T *__restrict__ Mm)
{
    pdl_wait();
    pdl_trigger();
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = slotmap[p];
        if (q < 0) continue;
        if (lam) Lm[q] = (T)lam[p];
        if (m) Mm[q] = (T)m[p];
    }
}

__global__ void k_edge_grad(int n, const int64_t *__restrict__ indptr,
                            const int *__restrict__ indices, const double *__restrict__ lam,
                            const double *__restrict__ x, double *__restrict__ dA)
{
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double li = lam[i];
    for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) dA[p] = -li * x[indices[p]];
}

// Full weighting (Trottenberg eq. 2.3.3) onto the coarse point (I, J) = fine (2I+1, 2J+1).
__global__ void k_restrict_fw(const double *__restrict__ rf, int mf, double scale,
                              double *__restrict__ rc)
{
    pdl_wait();
    pdl_trigger();
    const int mc = (mf - 1) / 2;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)mc * mc) return;
    const int I = (int)(idx % mc), J = (int)(idx / mc);
    const int64_t f = (int64_t)(2 * J + 1) * mf + (2 * I + 1);
    const double ctr = rf[f];
    const double edg = rf[f - 1] + rf[f + 1] + rf[f - mf] + rf[f + mf];
    const double crn = rf[f - mf - 1] + rf[f - mf + 1] + rf[f + mf - 1] + rf[f + mf + 1];
    rc[idx] = scale * (4.0 * ctr + 2.0 * edg + crn) * (1.0 / 16.0);
}

__device__ __forceinline__ double coarse_at(const double *__restrict__ ec, int mc, int I, int J)
{
    return (I >= 0 && I < mc && J >= 0 && J < mc) ? ec[(int64_t)J * mc + I] : 0.0;
}

// Bilinear interpolation (Trottenberg eq. 2.3.7) added onto the fine grid.
__global__ void k_prolong_add(const double *__restrict__ ec, int mc, double *__restrict__ xf)
{
    pdl_wait();
    pdl_trigger();
    const int mf = 2 * mc + 1;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)mf * mf) return;
    const int fx = (int)(idx % mf), fy = (int)(idx / mf);
    double v;
    if (fx & 1) {
        const int I = (fx - 1) >> 1;
        if (fy & 1) v = coarse_at(ec, mc, I, (fy - 1) >> 1);
        else v = 0.5 * (coarse_at(ec, mc, I, (fy >> 1) - 1) + coarse_at(ec, mc, I, fy >> 1));
    } else {
        const int I0 = (fx >> 1) - 1, I1 = fx >> 1;
        if (fy & 1) {
            const int J = (fy - 1) >> 1;
            v = 0.5 * (coarse_at(ec, mc, I0, J) + coarse_at(ec, mc, I1, J));
        } else {
            const int J0 = (fy >> 1) - 1, J1 = fy >> 1;
            v = 0.25 * (coarse_at(ec, mc, I0, J0) + coarse_at(ec, mc, I1, J0) +
                        coarse_at(ec, mc, I0, J1) + coarse_at(ec, mc, I1, J1));
        }
    }
    xf[idx] += v;
}

// y = M x, one warp per row of a dense row-major matrix.  A lane keeps four
// partial sums, so four pairs of loads are in flight per step instead of one
// dependent chain through the row.
__global__ void k_dense_gemv(const double *__restrict__ M, const double *__restrict__ x,
                             double *__restrict__ y, int n)
{
    pdl_wait();
    pdl_trigger();
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const double *Mr = M + (int64_t)row * n;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int j = lane;
    for (; j + 96 < n; j += 128) {
        a0 = fma(Mr[j], x[j], a0);
        a1 = fma(Mr[j + 32], x[j + 32], a1);
        a2 = fma(Mr[j + 64], x[j + 64], a2);
        a3 = fma(Mr[j + 96], x[j + 96], a3);
    }
    for (; j < n; j += 32) a0 = fma(Mr[j], x[j], a0);
    double acc = (a0 + a1) + (a2 + a3);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[row] = acc;
}

// Mean-message coefficients of the transposed system: a^T[e] = a[rev(e)].
template <typename T>
__global__ void k_transpose_stencil(int n, StencilParams sp, const T *__restrict__ a,
                                    T *__restrict__ aT)
{
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int k = 0; k < sp.K; ++k) {
        const int s = r + sp.off[k];
        T v = T(0);
        if (s >= 0 && s < n) v = a[(size_t)sp.krev[k] * n + s];
        aT[(size_t)k * n + r] = v;
    }
}

template <typename T>
__global__ void k_transpose_csr(int64_t slots, const int *__restrict__ rev, const T *__restrict__ a,
                                T *__restrict__ aT)
{
    pdl_wait();
    pdl_trigger();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < slots;
         e += (int64_t)gridDim.x * blockDim.x)
        aT[e] = a[rev[e]];
}

// Coefficients from matrix values held on the device (gabp_set_values_device):
// a64[e] = -A_rs for every stored off-diagonal entry p of row r (slotmap[p] =
// e), diag64[r] = A_rr (diagpos[r] = p of the diagonal).  Slots no entry maps
// to (pattern symmetrisation, stencil padding) keep their zero.
__global__ void k_values_scatter(int64_t nnz, int n, const int64_t *__restrict__ slotmap,
                                 const int64_t *__restrict__ diagpos,
                                 const double *__restrict__ data, double *__restrict__ a64,
                                 double *__restrict__ diag64)
{
    pdl_wait();
    pdl_trigger();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += stride) {
        const int64_t e = slotmap[p];
        if (e >= 0) a64[e] = -data[p];
    }
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride)
        diag64[r] = data[diagpos[r]];
}

// c_e = -A_rs A_sr = -a_e a_{rev e} (in double, then in the message precision
// with a and diag).
template <typename T>
__global__ void k_coeffs_c(const DevLayout L, const double *__restrict__ a64,
                           const double *__restrict__ diag64, T *__restrict__ a, T *__restrict__ c,
                           T *__restrict__ diagT)
{
    pdl_wait();
    pdl_trigger();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L.slots; e += stride) {
        double ar = 0.0;
        if (L.kind == GABP_LAYOUT_STENCIL) {
            const int k = (int)(e / L.n), r = (int)(e - (int64_t)k * L.n);
            const int s = r + L.sp.off[k];
            if (s >= 0 && s < L.n) ar = a64[(size_t)L.sp.krev[k] * L.n + s];
        } else {
            ar = a64[L.rev[e]];
        }
        const double ae = a64[e];
        c[e] = (T)(-ae * ar);
        if (a != (const T *)a64) a[e] = (T)ae;
    }
    if (diagT != (const T *)diag64)
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < L.n; r += stride)
            diagT[r] = (T)diag64[r];
}

inline int grid_for(int64_t n, int block, int cap = 152 * 32)
{
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

template <typename T>
cudaError_t sweep_stencil_T(const DevLayout &L, const SweepArgs &a, int block, cudaStream_t s)
{
    if (block > 256) block = 256;  // the stencil kernel holds a whole row's loads in registers
    const int grid = (int)((L.n + block - 1) / block);
    const T *A = (const T *)a.a, *C = (const T *)a.c, *D = (const T *)a.diag, *Bv = (const T *)a.b;
    const T *Li = (const T *)a.Lin, *Mi = (const T *)a.Min, *Pi = (const T *)a.Pin,
            *Bi = (const T *)a.Bin;
    T *Lo = (T *)a.Lout, *Mo = (T *)a.Mout, *Po = (T *)a.Pout, *Bo = (T *)a.Bout;
#define GABP_SWEEP_CASE(KK)                                                                                   \
    case KK:                                                                                                  \
        launch_pdl(k_sweep_stencil<T, KK>, grid, block, 0, s, L.n, L.sp, A, C, D, Bv, Li, Mi, Pi, Bi, Lo, Mo, \
                   Po, Bo, a.x, a.flags);                                                                     \
        break;
    switch (L.sp.K) {
        GABP_SWEEP_CASE(0)
        GABP_SWEEP_CASE(2)
        GABP_SWEEP_CASE(4)
        GABP_SWEEP_CASE(6)
        GABP_SWEEP_CASE(8)
        GABP_SWEEP_CASE(10)
        GABP_SWEEP_CASE(12)
        GABP_SWEEP_CASE(14)
        GABP_SWEEP_CASE(16)
        default:
            return cudaErrorInvalidValue;
    }
#undef GABP_SWEEP_CASE
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep(const DevLayout &L, int prec, const SweepArgs &a, int block,
                         cudaStream_t s)
{
    if (L.n == 0) return cudaSuccess;
    count_launches(s, 1);
    if (L.kind == GABP_LAYOUT_STENCIL)
        return prec == 0 ? sweep_stencil_T<double>(L, a, block, s)
                         : sweep_stencil_T<float>(L, a, block, s);
    return launch_sweep_csr_edge(L, prec, a, s);
}

cudaError_t launch_aggregate(const DevLayout &L, int prec, const void *diag, const void *b,
                             const void *Lm, const void *Mm, void *P, void *B, cudaStream_t s)
{
    if (L.n == 0) return cudaSuccess;
    const int block = 256, grid = (L.n + block - 1) / block;
    if (L.kind == GABP_LAYOUT_STENCIL) {
        if (prec == 0)
            launch_pdl(k_aggregate_stencil<double>, grid, block, 0, s, L.n, L.sp.K, (const double *)diag,
                       (const double *)b, (const double *)Lm, (const double *)Mm, (double *)P, (double *)B);
        else
            launch_pdl(k_aggregate_stencil<float>, grid, block, 0, s, L.n, L.sp.K, (const float *)diag,
                       (const float *)b, (const float *)Lm, (const float *)Mm, (float *)P, (float *)B);
    } else {
        if (prec == 0)
            launch_pdl(k_aggregate_csr<double>, grid, block, 0, s, L.n, L.rowptr, (const double *)diag,
                       (const double *)b, (const double *)Lm, (const double *)Mm, (double *)P, (double *)B);
        else
            launch_pdl(k_aggregate_csr<float>, grid, block, 0, s, L.n, L.rowptr, (const float *)diag,
                       (const float *)b, (const float *)Lm, (const float *)Mm, (float *)P, (float *)B);
    }
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_residual(const DevLayout &L, const double *a64, const double *diag64,
                            const double *b, const double *x, double *r, DevStatus *st,
                            cudaStream_t s)
{
    return launch_residual2(L, a64, diag64, b, x, r, nullptr, st, s);
}

cudaError_t launch_residual2(const DevLayout &L, const double *a64, const double *diag64,
                             const double *b, const double *x, double *r, float *rf,
                             DevStatus *st, cudaStream_t s)
{
    if (L.n == 0) return cudaSuccess;
    if (rf && L.kind != GABP_LAYOUT_STENCIL) return cudaErrorInvalidValue;
    const int block = 256, grid = grid_for(L.n, block, 152 * 16);
    if (L.kind == GABP_LAYOUT_STENCIL) {
#define GABP_RES_CASE(KK)                                                                               \
    case KK:                                                                                            \
        launch_pdl(k_residual_stencil<KK>, grid, block, 0, s, L.n, L.sp, a64, diag64, b, x, r, rf, st); \
        break;
        switch (L.sp.K) {
            GABP_RES_CASE(0)
            GABP_RES_CASE(2)
            GABP_RES_CASE(4)
            GABP_RES_CASE(6)
            GABP_RES_CASE(8)
            GABP_RES_CASE(10)
            GABP_RES_CASE(12)
            GABP_RES_CASE(14)
            GABP_RES_CASE(16)
            default:
                return cudaErrorInvalidValue;
        }
#undef GABP_RES_CASE
    } else {
        launch_pdl(k_residual_csr, grid, block, 0, s, L.n, L.rowptr, L.col, a64, diag64, b, x, r, st);
    }
    count_launches(s, 1);
    return cudaGetLastError();
}

// Per-block partial sums of u^2 and v^2 over a fixed grid-stride partition:
// part[2 * block] = sum u_i^2, part[2 * block + 1] = sum v_i^2, each in the
// same order on every call (thread sums, then a fixed tree in shared memory).
__global__ void __launch_bounds__(256) k_sumsq2(const double *__restrict__ u,
                                                const double *__restrict__ v, int64_t n,
                                                double *__restrict__ part)
{
    pdl_wait();
    pdl_trigger();
    __shared__ double su[256], sv[256];
    double a = 0.0, c = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        a = fma(u[i], u[i], a);
        c = fma(v[i], v[i], c);
    }
    su[threadIdx.x] = a;
    sv[threadIdx.x] = c;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            su[threadIdx.x] += su[threadIdx.x + w];
            sv[threadIdx.x] += sv[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = su[0];
        part[2 * blockIdx.x + 1] = sv[0];
    }
}

cudaError_t launch_sumsq2(const double *u, const double *v, int64_t n, double *part, int nblocks,
                          cudaStream_t s)
{
    launch_pdl(k_sumsq2, nblocks, 256, 0, s, u, v, n, part);
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_convert_d2f(const double *in, float *out, int64_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    launch_pdl(k_d2f, grid_for(n, 256), 256, 0, s, in, out, n);
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_to_double(int prec, const void *in, double *out, int64_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    if (prec == 0) {
        launch_pdl(k_copy, grid_for(n, 256), 256, 0, s, (const double *)in, out, n);
    } else {
        launch_pdl(k_f2d, grid_for(n, 256), 256, 0, s, (const float *)in, out, n);
    }
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_copy_vec(const double *in, double *out, int64_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    launch_pdl(k_copy, grid_for(n, 256), 256, 0, s, in, out, n);
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_scale_rhs(const double *in, const DevStatus *st, double *out, void *outT,
                             int prec, int64_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    if (prec == 0 || outT == nullptr)
        launch_pdl(k_scale_rhs<double>, grid_for(n, 256), 256, 0, s, in, st, out, nullptr, n);
    else
        launch_pdl(k_scale_rhs<float>, grid_for(n, 256), 256, 0, s, in, st, out, (float *)outT, n);
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_axpy_status(double *x, const double *e, const DevStatus *st, int64_t n,
                               cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    launch_pdl(k_axpy_status, grid_for(n, 256), 256, 0, s, x, e, st, n);
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_axpy(double *x, const double *e, double alpha, int64_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    launch_pdl(k_axpy, grid_for(n, 256), 256, 0, s, x, e, alpha, n);
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_get_state(const int64_t *slotmap, int64_t nnz, int prec, const void *Lm,
                             const void *Mm, double *lam, double *m, cudaStream_t s)
{
    if (nnz == 0) return cudaSuccess;
    if (prec == 0)
        launch_pdl(k_get_state<double>, grid_for(nnz, 256), 256, 0, s, slotmap, nnz, (const double *)Lm,
                   (const double *)Mm, lam, m);
    else
        launch_pdl(k_get_state<float>, grid_for(nnz, 256), 256, 0, s, slotmap, nnz, (const float *)Lm,
                   (const float *)Mm, lam, m);
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_set_state(const int64_t *slotmap, int64_t nnz, int prec, const double *lam,
                             const double *m, void *Lm, void *Mm, cudaStream_t s)
{
    if (nnz == 0) return cudaSuccess;
    if (prec == 0)
        launch_pdl(k_set_state<double>, grid_for(nnz, 256), 256, 0, s, slotmap, nnz, lam, m, (double *)Lm,
                   (double *)Mm);
    else
        launch_pdl(k_set_state<float>, grid_for(nnz, 256), 256, 0, s, slotmap, nnz, lam, m, (float *)Lm,
                   (float *)Mm);
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_edge_grad(int n, const int64_t *indptr, const int *indices, const double *lam,
                             const double *x, double *dA, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    launch_pdl(k_edge_grad, (n + 255) / 256, 256, 0, s, n, indptr, indices, lam, x, dA);
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_restrict_fw(const double *rf, int mf, double scale, double *rc, cudaStream_t s)
{
    const int mc = (mf - 1) / 2;
    const int64_t nc = (int64_t)mc * mc;
    if (nc == 0) return cudaSuccess;
    launch_pdl(k_restrict_fw, (int)((nc + 255) / 256), 256, 0, s, rf, mf, scale, rc);
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_prolong_add(const double *ec, int mc, double *xf, cudaStream_t s)
{
    const int64_t nf = (int64_t)(2 * mc + 1) * (2 * mc + 1);
    launch_pdl(k_prolong_add, (int)((nf + 255) / 256), 256, 0, s, ec, mc, xf);
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_dense_gemv(const double *M, const double *x, double *y, int n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int rows_per_block = 4;
    launch_pdl(k_dense_gemv, (n + rows_per_block - 1) / rows_per_block, 32 * rows_per_block, 0, s, M, x, y, n);
    count_launches(s, 1);
    return cudaGetLastError();
}

// out[i] = in[idx[i]] (gather) or out[idx[i]] = in[i] (scatter), n doubles.
__global__ void k_permute(int n, const int *__restrict__ idx, const double *__restrict__ in,
                          double *__restrict__ out, int scatter)
{
    pdl_wait();
    pdl_trigger();
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (scatter) out[idx[i]] = in[i];
        else out[i] = in[idx[i]];
    }
}

cudaError_t launch_permute(int n, const int *idx, const double *in, double *out, int scatter,
                           cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    launch_pdl(k_permute, grid_for(n, 256), 256, 0, s, n, idx, in, out, scatter);
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_coeffs_from_values(const DevLayout &L, int prec, int64_t nnz,
                                      const int64_t *slotmap, const int64_t *diagpos,
                                      const double *data, double *a64, double *diag64, void *a,
                                      void *c, void *diagT, cudaStream_t s)
{
    if (L.n == 0) return cudaSuccess;
    launch_pdl(k_values_scatter, grid_for(std::max<int64_t>(nnz, L.n), 256), 256, 0, s, nnz, L.n, slotmap,
               diagpos, data, a64, diag64);
    const int grid = grid_for(std::max<int64_t>(L.slots, L.n), 256);
    if (prec == 0)
        launch_pdl(k_coeffs_c<double>, grid, 256, 0, s, L, a64, diag64, (double *)a, (double *)c,
                   (double *)diagT);
    else
        launch_pdl(k_coeffs_c<float>, grid, 256, 0, s, L, a64, diag64, (float *)a, (float *)c, (float *)diagT);
    count_launches(s, 2);
    return cudaGetLastError();
}

cudaError_t launch_transpose_coeffs(const DevLayout &L, int prec, const void *a, void *aT,
                                    cudaStream_t s)
{
    if (L.n == 0) return cudaSuccess;
    if (L.kind == GABP_LAYOUT_STENCIL) {
        const int grid = (L.n + 255) / 256;
        if (prec == 0)
            launch_pdl(k_transpose_stencil<double>, grid, 256, 0, s, L.n, L.sp, (const double *)a,
                       (double *)aT);
        else
            launch_pdl(k_transpose_stencil<float>, grid, 256, 0, s, L.n, L.sp, (const float *)a, (float *)aT);
    } else {
        if (L.slots == 0) return cudaSuccess;
        if (prec == 0)
            launch_pdl(k_transpose_csr<double>, grid_for(L.slots, 256), 256, 0, s, L.slots, L.rev,
                       (const double *)a, (double *)aT);
        else
            launch_pdl(k_transpose_csr<float>, grid_for(L.slots, 256), 256, 0, s, L.slots, L.rev,
                       (const float *)a, (float *)aT);
    }
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_freeze(const DevLayout &L, int prec, const void *a, const void *P, const void *Lm,
                          void *g, unsigned *flags, cudaStream_t s)
{
    if (L.n == 0) return cudaSuccess;
    const int grid = (L.n + 255) / 256;
    count_launches(s, 1);
    if (L.kind == GABP_LAYOUT_STENCIL) {
#define GABP_FRZ_CASE(KK)                                                                           \
    case KK:                                                                                        \
        if (prec == 0)                                                                              \
            launch_pdl(k_freeze_stencil<double, KK>, grid, 256, 0, s, L.n, L.sp, (const double *)a, \
                       (const double *)P, (const double *)Lm, (double *)g, flags);                  \
        else                                                                                        \
            launch_pdl(k_freeze_stencil<float, KK>, grid, 256, 0, s, L.n, L.sp, (const float *)a,   \
                       (const float *)P, (const float *)Lm, (float *)g, flags);                     \
        break;
        switch (L.sp.K) {
            GABP_FRZ_CASE(0)
            GABP_FRZ_CASE(2)
            GABP_FRZ_CASE(4)
            GABP_FRZ_CASE(6)
            GABP_FRZ_CASE(8)
            GABP_FRZ_CASE(10)
            GABP_FRZ_CASE(12)
            GABP_FRZ_CASE(14)
            GABP_FRZ_CASE(16)
            default:
                return cudaErrorInvalidValue;
        }
#undef GABP_FRZ_CASE
    } else {
        if (prec == 0)
            launch_pdl(k_freeze_csr<double>, grid, 256, 0, s, L.n, L.rowptr, L.col, L.rev, (const double *)a,
                       (const double *)P, (const double *)Lm, (double *)g, flags);
        else
            launch_pdl(k_freeze_csr<float>, grid, 256, 0, s, L.n, L.rowptr, L.col, L.rev, (const float *)a,
                       (const float *)P, (const float *)Lm, (float *)g, flags);
    }
    return cudaGetLastError();
}

cudaError_t launch_sweep_mean(const DevLayout &L, int prec, const void *g, const void *b,
                              const void *P, const void *Min, const void *Bin, void *Mout,
                              void *Bout, double *x, int block, unsigned *flags, cudaStream_t s)
{
    if (L.n == 0) return cudaSuccess;
    count_launches(s, 1);
    if (L.kind == GABP_LAYOUT_STENCIL) {
        if (block > 256) block = 256;
        const int grid = (L.n + block - 1) / block;
#define GABP_MEAN_CASE(KK)                                                                                \
    case KK:                                                                                              \
        if (prec == 0)                                                                                    \
            launch_pdl(k_sweep_mean_stencil<double, KK>, grid, block, 0, s, L.n, L.sp, (const double *)g, \
                       (const double *)b, (const double *)P, (const double *)Min, (const double *)Bin,    \
                       (double *)Mout, (double *)Bout, x, flags);                                         \
        else                                                                                              \
            launch_pdl(k_sweep_mean_stencil<float, KK>, grid, block, 0, s, L.n, L.sp, (const float *)g,   \
                       (const float *)b, (const float *)P, (const float *)Min, (const float *)Bin,        \
                       (float *)Mout, (float *)Bout, x, flags);                                           \
        break;
        switch (L.sp.K) {
            GABP_MEAN_CASE(0)
            GABP_MEAN_CASE(2)
            GABP_MEAN_CASE(4)
            GABP_MEAN_CASE(6)
            GABP_MEAN_CASE(8)
            GABP_MEAN_CASE(10)
            GABP_MEAN_CASE(12)
            GABP_MEAN_CASE(14)
            GABP_MEAN_CASE(16)
            default:
                return cudaErrorInvalidValue;
        }
#undef GABP_MEAN_CASE
    } else {
        return launch_sweep_mean_csr_edge(L, prec, g, b, P, Min, Bin, Mout, Bout, x, flags, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_lambda_change(int64_t slots, int prec, const void *L0, const void *L1,
                                 DevStatus *st, cudaStream_t s)
{
    if (slots == 0) return cudaSuccess;
    count_launches(s, 1);
    const int grid = grid_for(slots, 256, 152 * 8);
    if (prec == 0)
        launch_pdl(k_lambda_change<double>, grid, 256, 0, s, slots, (const double *)L0, (const double *)L1, st);
    else
        launch_pdl(k_lambda_change<float>, grid, 256, 0, s, slots, (const float *)L0, (const float *)L1, st);
    return cudaGetLastError();
}

cudaError_t launch_sweep_color(const DevLayout &L, int prec, const unsigned char *color, int cphase,
                               const ColorMasks *cm, const void *a, const void *c, void *Lm,
                               void *Mm, void *P, void *B, double *x, unsigned *flags,
                               cudaStream_t s)
{
    if (L.n == 0) return cudaSuccess;
    count_launches(s, 1);
    const int grid = (L.n + 255) / 256;
    if (L.kind == GABP_LAYOUT_STENCIL) {
#define GABP_COL_CASE(KK)                                                                                      \
    case KK:                                                                                                   \
        if (cm) {                                                                                              \
            if (prec == 0)                                                                                     \
                launch_pdl(k_sweep_color_stencil<double, KK>, grid, 256, 0, s, L.n, L.sp, *cm, color, cphase,  \
                           (const double *)a, (const double *)c, (double *)Lm, (double *)Mm, (double *)P,      \
                           (double *)B, x, flags);                                                             \
            else                                                                                               \
                launch_pdl(k_sweep_color_stencil<float, KK>, grid, 256, 0, s, L.n, L.sp, *cm, color, cphase,   \
                           (const float *)a, (const float *)c, (float *)Lm, (float *)Mm, (float *)P,           \
                           (float *)B, x, flags);                                                              \
        } else {                                                                                               \
            if (prec == 0)                                                                                     \
                launch_pdl(k_sweep_color_stencil_gather<double, KK>, grid, 256, 0, s, L.n, L.sp, color,        \
                           cphase, (const double *)a, (const double *)c, (double *)Lm, (double *)Mm,           \
                           (double *)P, (double *)B, x, flags);                                                \
            else                                                                                               \
                launch_pdl(k_sweep_color_stencil_gather<float, KK>, grid, 256, 0, s, L.n, L.sp, color, cphase, \
                           (const float *)a, (const float *)c, (float *)Lm, (float *)Mm, (float *)P,           \
                           (float *)B, x, flags);                                                              \
        }                                                                                                      \
        break;
        switch (L.sp.K) {
            GABP_COL_CASE(0)
            GABP_COL_CASE(2)
            GABP_COL_CASE(4)
            GABP_COL_CASE(6)
            GABP_COL_CASE(8)
            GABP_COL_CASE(10)
            GABP_COL_CASE(12)
            GABP_COL_CASE(14)
            GABP_COL_CASE(16)
            default:
                return cudaErrorInvalidValue;
        }
#undef GABP_COL_CASE
    } else {
        if (prec == 0)
            launch_pdl(k_sweep_color_csr<double>, grid, 256, 0, s, L.n, L.rowptr, L.col, L.rev, color, cphase,
                       (const double *)a, (const double *)c, (double *)Lm, (double *)Mm, (double *)P,
                       (double *)B, x, flags);
        else
            launch_pdl(k_sweep_color_csr<float>, grid, 256, 0, s, L.n, L.rowptr, L.col, L.rev, color, cphase,
                       (const float *)a, (const float *)c, (float *)Lm, (float *)Mm, (float *)P, (float *)B,
                       x, flags);
    }
    return cudaGetLastError();
}

}  // namespace gabp
