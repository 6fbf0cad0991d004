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
//  k_mg_prolong_residual: x2 = x1 + P e_c (bilinear interpolation of the
//    coarse solution) on a tile with a halo, written out for the tile's own
//    points, and r = b - A x2 there, in double and / or float (the
//    post-smoothing right-hand side).
//
// The fine residual and the interpolated correction stay in shared memory, so
// a level's transfers read the matrix once per residual and write no
// intermediate vector.  Every operation is done in the order the separate
// kernels use (x + e, the residual's fma chain in slot order, the
// restriction's sums), so the results are theirs.  A tile recomputes the
// residual on one line of fine points beyond its own in each direction (about
// 5 % extra at 32 x 16 coarse points per tile).  Grids are lexicographic,
// m_f = 2 m_c + 1, the stencil inside the 3 x 3 neighbourhood.
#include <cuda_runtime.h>

#include "gabp_internal.h"

namespace gabp {
namespace {

constexpr int RX = 32, RY = 16;  // coarse points per restriction tile
constexpr int PX = 64, PY = 16;  // fine points per prolongation tile

struct Dirs {
    int dx[8], dy[8];
};

__device__ __forceinline__ double coarse_v(const double *__restrict__ ec, int mc, int I, int J)
{
    return (I >= 0 && I < mc && J >= 0 && J < mc) ? ec[(int64_t)J * mc + I] : 0.0;
}

// Bilinear interpolation at fine point (fx, fy) (the rule of k_prolong_add).
__device__ __forceinline__ double prolong_at(const double *__restrict__ ec, int mc, int fx, int fy)
{
    if (fx & 1) {
        const int I = (fx - 1) >> 1;
        if (fy & 1) return coarse_v(ec, mc, I, (fy - 1) >> 1);
        return 0.5 * (coarse_v(ec, mc, I, (fy >> 1) - 1) + coarse_v(ec, mc, I, fy >> 1));
    }
    const int I0 = (fx >> 1) - 1, I1 = fx >> 1;
    if (fy & 1) {
        const int J = (fy - 1) >> 1;
        return 0.5 * (coarse_v(ec, mc, I0, J) + coarse_v(ec, mc, I1, J));
    }
    const int J0 = (fy >> 1) - 1, J1 = fy >> 1;
    return 0.25 * (coarse_v(ec, mc, I0, J0) + coarse_v(ec, mc, I1, J0) + coarse_v(ec, mc, I0, J1) +
                   coarse_v(ec, mc, I1, J1));
}

__device__ __forceinline__ double sum_or_zero(const double *__restrict__ X,
                                              const double *__restrict__ E, int64_t i)
{
    return X ? (E ? X[i] + E[i] : X[i]) : (E ? E[i] : 0.0);
}

template <int K>
__global__ void __launch_bounds__(256) k_mg_restrict_residual(
    int mf, Dirs dir, const double *__restrict__ a64, const double *__restrict__ diag64,
    const double *__restrict__ b, const double *__restrict__ X, const double *__restrict__ E,
    double *__restrict__ T, double scale, double *__restrict__ rc, float *__restrict__ rcf,
    double *__restrict__ rcd, unsigned *flags)
{
    constexpr int XW = 2 * RX + 3, XH = 2 * RY + 3, RW = 2 * RX + 1, RH = 2 * RY + 1;
    __shared__ double xs[XH][XW];
    __shared__ double rs[RH][RW];
    const int mc = (mf - 1) / 2;
    const int64_t n = (int64_t)mf * mf;
    const int I0 = blockIdx.x * RX, J0 = blockIdx.y * RY;
    const int nI = min(RX, mc - I0), nJ = min(RY, mc - J0);
    // own fine points [2 I0, ox1) x [2 J0, oy1); the last tile of a row or column
    // also owns the grid's last fine line
    const int ox1 = I0 + RX >= mc ? mf : 2 * (I0 + RX);
    const int oy1 = J0 + RY >= mc ? mf : 2 * (J0 + RY);
    const int fx0 = 2 * I0 - 1, fy0 = 2 * J0 - 1;
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
    const int rw = 2 * nI + 1, rh = 2 * nJ + 1;
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

template <int K>
__global__ void __launch_bounds__(256) k_mg_prolong_residual(
    int mf, Dirs dir, const double *__restrict__ a64, const double *__restrict__ diag64,
    const double *__restrict__ b, const double *__restrict__ Xin, const double *__restrict__ Ein,
    const double *__restrict__ ec, double *__restrict__ Xout, double *__restrict__ r,
    float *__restrict__ rf, unsigned *flags)
{
    constexpr int XW = PX + 2, XH = PY + 2;
    __shared__ double xs[XH][XW];
    const int mc = (mf - 1) / 2;
    const int64_t n = (int64_t)mf * mf;
    const int x0 = blockIdx.x * PX, y0 = blockIdx.y * PY;
    for (int t = threadIdx.x; t < XW * XH; t += blockDim.x) {
        const int ly = t / XW, lx = t - ly * XW;
        const int fx = x0 - 1 + lx, fy = y0 - 1 + ly;
        double v = 0.0;
        if (fx >= 0 && fx < mf && fy >= 0 && fy < mf) {
            const int64_t i = (int64_t)fy * mf + fx;
            v = sum_or_zero(Xin, Ein, i) + prolong_at(ec, mc, fx, fy);
            if (lx >= 1 && lx <= PX && ly >= 1 && ly <= PY) Xout[i] = v;
        }
        xs[ly][lx] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < PX * PY; t += blockDim.x) {
        const int ly = t / PX, lx = t - ly * PX;
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
    const int mc = (mf - 1) / 2;
    if (mc < 1) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((mc + RX - 1) / RX), (unsigned)((mc + RY - 1) / RY));
    if (sp.K == 4)
        k_mg_restrict_residual<4><<<grid, 256, 0, s>>>(mf, d, a64, diag64, b, X, E, T, scale, rc, rcf, rcd, flags);
    else if (sp.K == 8)
        k_mg_restrict_residual<8><<<grid, 256, 0, s>>>(mf, d, a64, diag64, b, X, E, T, scale, rc, rcf, rcd, flags);
    else
        return cudaErrorInvalidValue;
    count_launches(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_mg_prolong_residual(const StencilParams &sp, int mf, const double *a64,
                                       const double *diag64, const double *b, const double *Xin,
                                       const double *Ein, const double *ec, double *Xout,
                                       double *r, float *rf, unsigned *flags, cudaStream_t s)
{
    Dirs d;
    if (!grid_dirs(sp, mf, d) || mf % 2 == 0) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((mf + PX - 1) / PX), (unsigned)((mf + PY - 1) / PY));
    if (sp.K == 4)
        k_mg_prolong_residual<4><<<grid, 256, 0, s>>>(mf, d, a64, diag64, b, Xin, Ein, ec, Xout, r, rf, flags);
    else if (sp.K == 8)
        k_mg_prolong_residual<8><<<grid, 256, 0, s>>>(mf, d, a64, diag64, b, Xin, Ein, ec, Xout, r, rf, flags);
    else
        return cudaErrorInvalidValue;
    count_launches(s, 1);
    return cudaGetLastError();
}

}  // namespace gabp
