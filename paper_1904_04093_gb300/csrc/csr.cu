// Edge-parallel message sweep on the CSR layout (sm_103a).
//
// The flood update of eq. nonsymmetric_GaBP_rules for the CSR entry e = (r, s)
// with reverse edge rev(e) = (s, r) (Sec. 2.3):
//     d_e = P_s - L[rev e],   L'[e] = c_e / d_e,   M'[e] = a_e (B_s - M[rev e]) / d_e,
// followed by the row aggregation of Algorithm 1,
//     P'_r = A_rr + sum_{e in row r} L'[e],   B'_r = b_r + sum_{e in row r} M'[e],
// and the belief x_r = B_r / P_r of the previous state.  With frozen
// precision messages (the precomputed tilde-Lambda of Sec. 4.2) only the mean
// messages move: M'[e] = g_e (B_s - M[rev e]), B'_r as above.
//
// Work split.  Each warp owns 32 consecutive rows r0 .. r0 + 31 and therefore
// the contiguous slot range [rowptr[r0], rowptr[r0 + 32]).  The slots are
// processed in tiles of 32 * EPT: lane l takes the slots t0 + 32 j + l
// (j < EPT), so every load of col, rev, a, c and every store of L', M' is a
// coalesced warp-contiguous stream whatever the row lengths are.  A lane issues
// all loads of its EPT slots (the index arrays, then the gathers at col and
// rev) before any arithmetic, which keeps several DRAM round trips in flight.
// The new messages are staged in the warp's own slice of shared memory; after
// __syncwarp lane l adds the staged values of its row r0 + l in slot order, so
// a row's sums are formed in the order of a sequential loop over the row
// (deterministic, no atomics) and a row of any length is handled, tile by
// tile.  Warps never wait for one another (no block barrier).
#include <cuda_runtime.h>

#include "gabp_internal.h"
#include "sweep_row.cuh"

namespace gabp {

namespace {

constexpr int kCsrBlock = 128;  // four warps, each on its own 32 rows
constexpr int kEptMax = 8;

// Blocks per SM the register allocation aims at: the sweep is latency-bound
// (each slot's gathers wait for its index loads), so occupancy pays: 40 warps
// per SM (<= 51 registers) for float, 32 (<= 64) for double, fewer for the
// eight-slot width, which holds twice the loads in flight per thread.
constexpr int csr_min_blocks(bool dbl, int ept)
{
    return ept <= 4 ? (dbl ? 8 : 10) : (dbl ? 4 : 6);
}

// kFull: full update (L', M', P', B'); otherwise the mean-only update with
// gains g passed in `a` (c, Lin, Lout, Pout unused; P = Pin fixed).
template <typename T, int EPT, bool kFull>
__global__ void __launch_bounds__(kCsrBlock, csr_min_blocks(sizeof(T) == 8, EPT)) k_sweep_csr(
    int n, const int *__restrict__ rowptr, const int *__restrict__ col,
    const int *__restrict__ rev, const T *__restrict__ a, const T *__restrict__ c,
    const T *__restrict__ diag, const T *__restrict__ b, const T *__restrict__ Lin,
    const T *__restrict__ Min, const T *__restrict__ Pin, const T *__restrict__ Bin,
    T *__restrict__ Lout, T *__restrict__ Mout, T *__restrict__ Pout, T *__restrict__ Bout,
    double *__restrict__ x, unsigned *__restrict__ flags, int nslots)
{
    pdl_wait();
    pdl_trigger();
    constexpr int WT = 32 * EPT;
    constexpr int NW = kCsrBlock / 32;
    __shared__ T sL[kFull ? NW * WT : 1];
    __shared__ T sM[NW * WT];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = (blockIdx.x * NW + w) * 32;
    if (r0 >= n) return;
    const int nrows = min(32, n - r0);
    const bool own = lane < nrows;
    const int r = r0 + lane;
    int lo = 0, hi = 0;
    T pn = T(0), bn = T(0);
    bool oob = false;  // bounds-checked build: an index outside its array (access skipped)
    if (own) {
        lo = rowptr[r];
        hi = rowptr[r + 1];
        if (kIndexChecks && !(0 <= lo && lo <= hi && hi <= nslots)) {
            oob = true;
            lo = hi = 0;
        }
        if (kFull) pn = diag[r];
        bn = b[r];
        if (x) x[r] = (double)(Bin[r] / Pin[r]);
    }
    int e0 = __shfl_sync(0xffffffffu, lo, 0);
    int e1 = __shfl_sync(0xffffffffu, hi, nrows - 1);
    if (kIndexChecks && __any_sync(0xffffffffu, oob)) e0 = e1 = 0;  // no slot range to walk
    T *wL = sL + (kFull ? w * WT : 0);
    T *wM = sM + w * WT;
    bool bad = false;
    for (int t0 = e0; t0 < e1; t0 += WT) {
        int cs[EPT], rs[EPT];
        T ae[EPT], ce[EPT], ps[EPT], bs[EPT], lr[EPT], mr[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            int e = t0 + j * 32 + lane;
            e = e < e1 ? e : e1 - 1;
            cs[j] = col[e];
            rs[j] = rev[e];
            ae[j] = a[e];
            if (kFull) ce[j] = c[e];
            if (kIndexChecks && !((unsigned)cs[j] < (unsigned)n && (unsigned)rs[j] < (unsigned)nslots)) {
                oob = true;
                cs[j] = rs[j] = 0;
                ae[j] = T(0);
            }
        }
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            if (kFull) {
                ps[j] = Pin[cs[j]];
                lr[j] = Lin[rs[j]];
            }
            bs[j] = Bin[cs[j]];
            mr[j] = Min[rs[j]];
        }
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const int e = t0 + j * 32 + lane;
            T lam = T(0), mu = T(0);
            if (nonzero(ae[j])) {
                if (kFull) {
                    const T d = ps[j] - lr[j];
                    bad |= e < e1 && bad_den(d);
                    const T q = fast_rcp(d);
                    lam = ce[j] * q;
                    mu = ae[j] * (bs[j] - mr[j]) * q;
                } else {
                    mu = ae[j] * (bs[j] - mr[j]);
                }
            }
            if (e < e1) {
                if (kFull) {
                    Lout[e] = lam;
                    wL[j * 32 + lane] = lam;
                }
                Mout[e] = mu;
                wM[j * 32 + lane] = mu;
            }
        }
        __syncwarp();
        if (own) {
            const int j0 = max(lo, t0), j1 = min(hi, t0 + WT);
            for (int j = j0; j < j1; ++j) {
                if (kFull) pn += wL[j - t0];
                bn += wM[j - t0];
            }
        }
        __syncwarp();
    }
    if (own) {
        if (kFull) Pout[r] = pn;
        Bout[r] = bn;
    }
    if (bad) atomicOr(flags, FLAG_BREAKDOWN);
    if (kIndexChecks && oob && flags) atomicOr(flags, FLAG_INDEX);
}

// Slots handled per thread and tile: the smallest power of two at least the
// mean row length (at most 8; longer rows take several tiles).
int ept_for(const DevLayout &L)
{
    const double mean = L.n > 0 ? (double)L.slots / (double)L.n : 0.0;
    int ept = 1;
    while (ept < kEptMax && ept < mean) ept *= 2;
    return ept;
}

template <typename T, bool kFull>
cudaError_t launch_T(const DevLayout &L, const void *a, const void *c, const void *diag,
                     const void *b, const void *Lin, const void *Min, const void *Pin,
                     const void *Bin, void *Lout, void *Mout, void *Pout, void *Bout, double *x,
                     unsigned *flags, cudaStream_t s)
{
    const int grid = (L.n + kCsrBlock - 1) / kCsrBlock;
    if (grid == 0) return cudaSuccess;
#define GABP_CSR_CASE(E)                                                                                       \
    case E:                                                                                                    \
        launch_pdl(k_sweep_csr<T, E, kFull>, grid, kCsrBlock, 0, s, L.n, L.rowptr, L.col, L.rev, (const T *)a, \
                   (const T *)c, (const T *)diag, (const T *)b, (const T *)Lin, (const T *)Min,                \
                   (const T *)Pin, (const T *)Bin, (T *)Lout, (T *)Mout, (T *)Pout, (T *)Bout, x, flags,       \
                   (int)L.slots);                                                                              \
        break;
    switch (ept_for(L)) {
        GABP_CSR_CASE(1)
        GABP_CSR_CASE(2)
        GABP_CSR_CASE(4)
        GABP_CSR_CASE(8)
        default:
            return cudaErrorInvalidValue;
    }
#undef GABP_CSR_CASE
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep_csr_edge(const DevLayout &L, int prec, const SweepArgs &a, cudaStream_t s)
{
    if (prec == 0)
        return launch_T<double, true>(L, a.a, a.c, a.diag, a.b, a.Lin, a.Min, a.Pin, a.Bin, a.Lout,
                                      a.Mout, a.Pout, a.Bout, a.x, a.flags, s);
    return launch_T<float, true>(L, a.a, a.c, a.diag, a.b, a.Lin, a.Min, a.Pin, a.Bin, a.Lout,
                                 a.Mout, a.Pout, a.Bout, a.x, a.flags, s);
}

cudaError_t launch_sweep_mean_csr_edge(const DevLayout &L, int prec, const void *g, const void *b,
                                       const void *P, const void *Min, const void *Bin, void *Mout,
                                       void *Bout, double *x, unsigned *flags, cudaStream_t s)
{
    if (prec == 0)
        return launch_T<double, false>(L, g, nullptr, nullptr, b, nullptr, Min, P, Bin, nullptr,
                                       Mout, nullptr, Bout, x, flags, s);
    return launch_T<float, false>(L, g, nullptr, nullptr, b, nullptr, Min, P, Bin, nullptr, Mout,
                                  nullptr, Bout, x, flags, s);
}

}  // namespace gabp
