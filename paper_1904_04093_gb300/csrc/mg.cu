// Multigrid transfers fused with the double residual (Algorithm 3 inside the
// V-cycle of Sec. 4, full weighting and bilinear interpolation as in
// k_restrict_fw / k_prolong_add).
//
// Two tiled kernels replace the separate correction, residual, restriction,
// prolongation and conversion passes of a level:
//
//  k_mg_restrict_residual: x1 = X + E (the level's iterate plus the
//    pre-smoothing correction, either may be absent) on a tile with a halo,
//    r = b - A x1 on the fine points the tile's coarse points need, and the
//    full-weighting restriction of r onto those coarse points (the coarse
//    right-hand side, in double and in the coarse smoother's precision); x1
//    is written out for the tile's own points when a later step needs it.
//  k_mg_prolong_residual: the coarse solution x_c (+ its post-smoothing
//    correction e_c, when the coarse level left the sum to this kernel) on
//    the tile's coarse patch, x2 = x1 + P x_c (bilinear interpolation) on a
//    tile with a halo, written out for the tile's own points, and
//    r = b - A x2 there, in double and / or float (the post-smoothing
//    right-hand side).
//
// The fine residual and the interpolated correction stay in shared memory, so
// a level's transfers read the matrix once per residual and write no
// intermediate vector.  Every operation is done in the order the separate
// kernels use (x + e, the residual's fma chain in slot order, the
// restriction's sums, the interpolation's sums), so the results are theirs.
// A tile recomputes the residual on one line of fine points beyond its own in
// each direction.  Each level takes the large tiles when they give the GPU
// enough CTAs, else small ones: a CTA walks its tile in a few dependent rounds
// of loads, and on a coarse level with few tiles those rounds are the
// kernel's whole duration.  Grids are lexicographic, m_f = 2 m_c + 1, the
// stencil inside the 3 x 3 neighbourhood.
#include <cuda_runtime.h>

#include "gabp_internal.h"

#ifndef GABP_MG_BIG_TILES_MIN
#define GABP_MG_BIG_TILES_MIN 608
#endif

namespace gabp {
namespace {

// coarse points per restriction tile, fine points per prolongation tile
constexpr int RX = 32, RY = 16, RXS = 8, RYS = 8;
constexpr int PX = 64, PY = 16, PXS = 16, PYS = 16;
// fewer large tiles than this (4 per SM) and a level takes the small ones
constexpr int kBigTilesMin = GABP_MG_BIG_TILES_MIN;
constexpr int kMgThreads = 256;  // threads per CTA of both kernels
// at most this many small restriction tiles (two per SM) and they prefetch
constexpr int kPrefetchTilesMax = 304;

struct Dirs {
    int dx[8], dy[8];
};

__device__ __forceinline__ double sum_or_zero(const double *__restrict__ X,
                                              const double *__restrict__ E, int64_t i)
{
    return X ? (E ? X[i] + E[i] : X[i]) : (E ? E[i] : 0.0);
}

template <int K, int TX, int TY, bool kPre>
__global__ void __launch_bounds__(kMgThreads) k_mg_restrict_residual(
    int mf, Dirs dir, const double *__restrict__ a64, const double *__restrict__ diag64,
    const double *__restrict__ b, const double *__restrict__ X, const double *__restrict__ E,
    double *__restrict__ T, double scale, double *__restrict__ rc, float *__restrict__ rcf,
    double *__restrict__ rcd, unsigned *flags)
{
    pdl_wait();
    pdl_trigger();
    constexpr int XW = 2 * TX + 3, XH = 2 * TY + 3, RW = 2 * TX + 1, RH = 2 * TY + 1;
    __shared__ double xs[XH][XW];
    __shared__ double rs[RH][RW];
    const int mc = (mf - 1) / 2;
    const int64_t n = (int64_t)mf * mf;
    const int I0 = blockIdx.x * TX, J0 = blockIdx.y * TY;
    const int nI = min(TX, mc - I0), nJ = min(TY, mc - J0);
    // own fine points [2 I0, ox1) x [2 J0, oy1); the last tile of a row or column
    // also owns the grid's last fine line
    const int ox1 = I0 + TX >= mc ? mf : 2 * (I0 + TX);
    const int oy1 = J0 + TY >= mc ? mf : 2 * (J0 + TY);
    const int fx0 = 2 * I0 - 1, fy0 = 2 * J0 - 1;
    const int rw = 2 * nI + 1, rh = 2 * nJ + 1;
    // kPre (small tiles on a level that fills one wave at most): a thread's
    // residual points, two at most, have their matrix entries loaded first, so
    // those loads are in flight while x1 is staged; on larger levels the
    // registers this takes cost more occupancy than the overlap gains
    constexpr int NR = (RW * RH + kMgThreads - 1) / kMgThreads;
    static_assert(!kPre || NR <= 2, "prefetch holds two residual points per thread");
    constexpr int NP = kPre ? NR : 1;
    double pd[NP], pb[NP], pa[NP][K > 0 ? K : 1];
    if constexpr (kPre) {
#pragma unroll
        for (int u = 0; u < NR; ++u) {
            const int t = threadIdx.x + u * kMgThreads;
            const int ly = t / rw, lx = t - ly * rw;
            const int64_t i = (int64_t)(2 * J0 + ly) * mf + (2 * I0 + lx);
            const bool ok = t < rw * rh && !(kIndexChecks && (i < 0 || i >= n));
            pd[u] = ok ? diag64[i] : 0.0;
            pb[u] = ok ? b[i] : 0.0;
#pragma unroll
            for (int k = 0; k < K; ++k) pa[u][k] = ok ? a64[k * n + i] : 0.0;
        }
    }
    for (int t = threadIdx.x; t < XW * XH; t += blockDim.x) {
        const int ly = t / XW, lx = t - ly * XW;
        const int fx = fx0 + lx, fy = fy0 + ly;
        double v = 0.0;
        if (fx >= 0 && fx < mf && fy >= 0 && fy < mf) {
            const int64_t i = (int64_t)fy * mf + fx;
            v = sum_or_zero(X, E, i);
            if (T && fx >= 2 * I0 && fx < ox1 && fy >= 2 * J0 && fy < oy1) T[i] = v;
        }
        xs[ly][lx] = v;
    }
    __syncthreads();
    if constexpr (kPre) {
#pragma unroll
        for (int u = 0; u < NR; ++u) {
            const int t = threadIdx.x + u * kMgThreads;
            if (t >= rw * rh) break;
            const int ly = t / rw, lx = t - ly * rw;
            const int64_t i = (int64_t)(2 * J0 + ly) * mf + (2 * I0 + lx);
            if (kIndexChecks && (i < 0 || i >= n)) {
                atomicOr(flags, FLAG_INDEX);
                rs[ly][lx] = 0.0;
                continue;
            }
            double acc = fma(-pd[u], xs[ly + 1][lx + 1], pb[u]);
#pragma unroll
            for (int k = 0; k < K; ++k) acc = fma(pa[u][k], xs[ly + 1 + dir.dy[k]][lx + 1 + dir.dx[k]], acc);
            rs[ly][lx] = acc;
        }
    } else {
        for (int t = threadIdx.x; t < rw * rh; t += blockDim.x) {
            const int ly = t / rw, lx = t - ly * rw;
            const int64_t i = (int64_t)(2 * J0 + ly) * mf + (2 * I0 + lx);
            if (kIndexChecks && (i < 0 || i >= n)) {
                atomicOr(flags, FLAG_INDEX);
                rs[ly][lx] = 0.0;
                continue;
            }
            double acc = fma(-diag64[i], xs[ly + 1][lx + 1], b[i]);
#pragma unroll
            for (int k = 0; k < K; ++k) acc = fma(a64[k * n + i], xs[ly + 1 + dir.dy[k]][lx + 1 + dir.dx[k]], acc);
            rs[ly][lx] = acc;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nI * nJ; t += blockDim.x) {
        const int cj = t / nI, ci = t - cj * nI;
        const int lx = 2 * ci + 1, ly = 2 * cj + 1;
        const double ctr = rs[ly][lx];
        const double edg = rs[ly][lx - 1] + rs[ly][lx + 1] + rs[ly - 1][lx] + rs[ly + 1][lx];
        const double crn = rs[ly - 1][lx - 1] + rs[ly - 1][lx + 1] + rs[ly + 1][lx - 1] + rs[ly + 1][lx + 1];
        const double v = scale * (4.0 * ctr + 2.0 * edg + crn) * (1.0 / 16.0);
        const int64_t ic = (int64_t)(J0 + cj) * mc + (I0 + ci);
        if (kIndexChecks && (ic < 0 || ic >= (int64_t)mc * mc)) {
            atomicOr(flags, FLAG_INDEX);
            continue;
        }
        rc[ic] = v;
        if (rcf) rcf[ic] = (float)v;
        if (rcd) rcd[ic] = v;
    }
}

// Bilinear interpolation at fine point (fx, fy) (the rule of k_prolong_add)
// from the coarse patch cs, whose entry [j][i] is the coarse point
// (cx0 + i, cy0 + j) (zero outside the coarse grid).
template <int CW>
__device__ __forceinline__ double prolong_at(const double (*cs)[CW], int cx0, int cy0, int fx, int fy)
{
    if (fx & 1) {
        const int i = ((fx - 1) >> 1) - cx0;
        if (fy & 1) return cs[((fy - 1) >> 1) - cy0][i];
        const int j1 = (fy >> 1) - cy0;
        return 0.5 * (cs[j1 - 1][i] + cs[j1][i]);
    }
    const int i1 = (fx >> 1) - cx0;
    if (fy & 1) {
        const int j = ((fy - 1) >> 1) - cy0;
        return 0.5 * (cs[j][i1 - 1] + cs[j][i1]);
    }
    const int j1 = (fy >> 1) - cy0;
    return 0.25 * (cs[j1 - 1][i1 - 1] + cs[j1 - 1][i1] + cs[j1][i1 - 1] + cs[j1][i1]);
}

template <int K, int TX, int TY>
__global__ void __launch_bounds__(kMgThreads) k_mg_prolong_residual(
    int mf, Dirs dir, const double *__restrict__ a64, const double *__restrict__ diag64,
    const double *__restrict__ b, const double *__restrict__ Xin, const double *__restrict__ Ein,
    const double *__restrict__ ec, const double *__restrict__ ec2, double *__restrict__ Xout,
    double *__restrict__ r, float *__restrict__ rf, unsigned *flags)
{
    pdl_wait();
    pdl_trigger();
    // fine points x0 - 1 .. x0 + TX interpolate from coarse points
    // x0 / 2 - 1 .. x0 / 2 + TX / 2 (TX even), likewise in y
    constexpr int XW = TX + 2, XH = TY + 2, CW = TX / 2 + 2, CH = TY / 2 + 2;
    static_assert(TX % 2 == 0 && TY % 2 == 0, "tiles start on even fine points");
    __shared__ double cs[CH][CW];
    __shared__ double xs[XH][XW];
    const int mc = (mf - 1) / 2;
    const int64_t n = (int64_t)mf * mf;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int cx0 = x0 / 2 - 1, cy0 = y0 / 2 - 1;
    // the tile's x1 = Xin + Ein is loaded first, so its loads are in flight
    // while the coarse patch is staged
    constexpr int NXS = XW * XH, NU = (NXS + kMgThreads - 1) / kMgThreads;
    double x1[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        const int t = threadIdx.x + u * kMgThreads;
        const int ly = t / XW, lx = t - ly * XW;
        const int fx = x0 - 1 + lx, fy = y0 - 1 + ly;
        x1[u] = t < NXS && fx >= 0 && fx < mf && fy >= 0 && fy < mf
                    ? sum_or_zero(Xin, Ein, (int64_t)fy * mf + fx) : 0.0;
    }
    for (int t = threadIdx.x; t < CW * CH; t += kMgThreads) {
        const int ly = t / CW, lx = t - ly * CW;
        const int I = cx0 + lx, J = cy0 + ly;
        double v = 0.0;
        if (I >= 0 && I < mc && J >= 0 && J < mc) {
            const int64_t i = (int64_t)J * mc + I;
            v = ec2 ? ec[i] + ec2[i] : ec[i];
        }
        cs[ly][lx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        const int t = threadIdx.x + u * kMgThreads;
        if (t >= NXS) break;
        const int ly = t / XW, lx = t - ly * XW;
        const int fx = x0 - 1 + lx, fy = y0 - 1 + ly;
        double v = 0.0;
        if (fx >= 0 && fx < mf && fy >= 0 && fy < mf) {
            v = x1[u] + prolong_at<CW>(cs, cx0, cy0, fx, fy);
            if (lx >= 1 && lx <= TX && ly >= 1 && ly <= TY) Xout[(int64_t)fy * mf + fx] = v;
        }
        xs[ly][lx] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < TX * TY; t += kMgThreads) {
        const int ly = t / TX, lx = t - ly * TX;
        const int fx = x0 + lx, fy = y0 + ly;
        if (fx >= mf || fy >= mf) continue;
        const int64_t i = (int64_t)fy * mf + fx;
        if (kIndexChecks && (i < 0 || i >= n)) {
            atomicOr(flags, FLAG_INDEX);
            continue;
        }
        double acc = fma(-diag64[i], xs[ly + 1][lx + 1], b[i]);
#pragma unroll
        for (int k = 0; k < K; ++k) acc = fma(a64[k * n + i], xs[ly + 1 + dir.dy[k]][lx + 1 + dir.dx[k]], acc);
        if (r) r[i] = acc;
        if (rf) rf[i] = (float)acc;
    }
}

// Stored diagonals as grid directions; false unless every one lies in the
// 3 x 3 neighbourhood of an m x m grid.
bool grid_dirs(const StencilParams &sp, int m, Dirs &d)
{
    if (m < 3 || sp.K > 8) return false;
    for (int k = 0; k < sp.K; ++k) {
        const int o = sp.off[k];
        const int dy = (o + (o >= 0 ? m / 2 : -(m / 2))) / m;
        const int dx = o - dy * m;
        if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || (dx == 0 && dy == 0)) return false;
        d.dx[k] = dx;
        d.dy[k] = dy;
    }
    return true;
}

template <int K>
cudaError_t restrict_k(int mf, const Dirs &d, const double *a64, const double *diag64, const double *b,
                       const double *X, const double *E, double *T, double scale, double *rc, float *rcf,
                       double *rcd, unsigned *flags, cudaStream_t s)
{
    const int mc = (mf - 1) / 2;
    const unsigned gx = (unsigned)((mc + RX - 1) / RX), gy = (unsigned)((mc + RY - 1) / RY);
    if ((int64_t)gx * gy >= kBigTilesMin)
        return launch_pdl(k_mg_restrict_residual<K, RX, RY, false>, dim3(gx, gy), kMgThreads, 0, s, mf, d, a64,
                          diag64, b, X, E, T, scale, rc, rcf, rcd, flags);
    const dim3 gs((unsigned)((mc + RXS - 1) / RXS), (unsigned)((mc + RYS - 1) / RYS));
    if ((int64_t)gs.x * gs.y > kPrefetchTilesMax)
        return launch_pdl(k_mg_restrict_residual<K, RXS, RYS, false>, gs, kMgThreads, 0, s, mf, d, a64, diag64, b, X,
                          E, T, scale, rc, rcf, rcd, flags);
    return launch_pdl(k_mg_restrict_residual<K, RXS, RYS, true>, gs, kMgThreads, 0, s, mf, d, a64, diag64, b, X, E,
                      T, scale, rc, rcf, rcd, flags);
}

template <int K>
cudaError_t prolong_k(int mf, const Dirs &d, const double *a64, const double *diag64, const double *b,
                      const double *Xin, const double *Ein, const double *ec, const double *ec2, double *Xout,
                      double *r, float *rf, unsigned *flags, cudaStream_t s)
{
    const unsigned gx = (unsigned)((mf + PX - 1) / PX), gy = (unsigned)((mf + PY - 1) / PY);
    if ((int64_t)gx * gy >= kBigTilesMin)
        return launch_pdl(k_mg_prolong_residual<K, PX, PY>, dim3(gx, gy), kMgThreads, 0, s, mf, d, a64, diag64, b, Xin,
                          Ein, ec, ec2, Xout, r, rf, flags);
    return launch_pdl(k_mg_prolong_residual<K, PXS, PYS>,
                      dim3((unsigned)((mf + PXS - 1) / PXS), (unsigned)((mf + PYS - 1) / PYS)), kMgThreads, 0, s, mf, d,
                      a64, diag64, b, Xin, Ein, ec, ec2, Xout, r, rf, flags);
}

}  // namespace

bool mg_fusable(const StencilParams &sp, int m)
{
    Dirs d;
    return (sp.K == 4 || sp.K == 8) && grid_dirs(sp, m, d);
}

cudaError_t launch_mg_restrict_residual(const StencilParams &sp, int mf, const double *a64,
                                        const double *diag64, const double *b, const double *X,
                                        const double *E, double *T, double scale, double *rc,
                                        float *rcf, double *rcd, unsigned *flags, cudaStream_t s)
{
    Dirs d;
    if (!grid_dirs(sp, mf, d) || mf % 2 == 0) return cudaErrorInvalidValue;
    if ((mf - 1) / 2 < 1) return cudaErrorInvalidValue;
    cudaError_t e;
    if (sp.K == 4) e = restrict_k<4>(mf, d, a64, diag64, b, X, E, T, scale, rc, rcf, rcd, flags, s);
    else if (sp.K == 8) e = restrict_k<8>(mf, d, a64, diag64, b, X, E, T, scale, rc, rcf, rcd, flags, s);
    else return cudaErrorInvalidValue;
    count_launches(s, 1);
    return e;
}

cudaError_t launch_mg_prolong_residual(const StencilParams &sp, int mf, const double *a64,
                                       const double *diag64, const double *b, const double *Xin,
                                       const double *Ein, const double *ec, const double *ec2,
                                       double *Xout, double *r, float *rf, unsigned *flags, cudaStream_t s)
{
    Dirs d;
    if (!grid_dirs(sp, mf, d) || mf % 2 == 0) return cudaErrorInvalidValue;
    cudaError_t e;
    if (sp.K == 4) e = prolong_k<4>(mf, d, a64, diag64, b, Xin, Ein, ec, ec2, Xout, r, rf, flags, s);
    else if (sp.K == 8) e = prolong_k<8>(mf, d, a64, diag64, b, Xin, Ein, ec, ec2, Xout, r, rf, flags, s);
    else return cudaErrorInvalidValue;
    count_launches(s, 1);
    return e;
}

}  // namespace gabp
