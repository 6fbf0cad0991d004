// Line GaBP: the two-layer generalized GaBP of Algorithm 2 (Sec. 3) with the
// grid lines as large regions and single nodes as small regions, on 5-point
// grids (every edge lies inside a row or a column).
//
// Each node l receives one message from its row region and one from its
// column region, (Lambda, m) pairs.  Updating the messages of one line L with
// the other family's messages (Lambda', m') fixed:
//     d_i = A_ii + Lambda'_i,  r_i = b_i + m'_i
//     T   = tridiagonal(sub_i, d_i, sup_i)     ([A]_L plus the diagonal corrections)
//     x   = T^{-1} r                           (the region's solution)
//     S_i = 1 / (T^{-1})_ii = f_i + g_i - d_i  (f, g: forward and backward pivots)
//     Lambda_i = S_i - d_i,   m_i = S_i x_i - r_i
// which is the message rule of Algorithm 2 written for a tridiagonal block.
// One thread walks one line (Thomas elimination; the loads of a step do not
// depend on the recurrence, so unrolling keeps several steps' loads in
// flight); lines are laid out so that consecutive threads touch consecutive
// addresses: element i of line c sits at i * m + c.  Columns are lines in the natural (row-major) order; rows are
// lines in the transposed order, so the messages cross between the two
// orders through tiled transposes.
#include <cuda_runtime.h>

#include "gabp_internal.h"
#include "sweep_row.cuh"

namespace gabp {
namespace {

template <typename T>
__global__ void __launch_bounds__(32) k_line_phase(int m, const T *__restrict__ sub,
                                                   const T *__restrict__ sup,
                                                   const T *__restrict__ diag,
                                                   const T *__restrict__ b,
                                                   const T *__restrict__ Loth,
                                                   const T *__restrict__ Moth, T *__restrict__ Lown,
                                                   T *__restrict__ Mown, T *__restrict__ f,
                                                   T *__restrict__ y, double *__restrict__ x,
                                                   unsigned *__restrict__ flags)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    const size_t mm = (size_t)m;
    bool bad = false;
    // forward elimination: f_i = d_i - sub_i sup_{i-1} / f_{i-1},  y_i = r_i - (sub_i / f_{i-1}) y_{i-1}
    T fp = T(0), yp = T(0), supp = T(0);
#pragma unroll 8
    for (int i = 0; i < m; ++i) {
        const size_t p = (size_t)i * mm + c;
        const T d = diag[p] + Loth[p];
        const T r = b[p] + Moth[p];
        T fi, yi;
        if (i == 0) {
            fi = d;
            yi = r;
        } else {
            const T w = sub[p] * fast_rcp(fp);
            fi = d - w * supp;
            yi = r - w * yp;
        }
        bad |= bad_den(fi);
        f[p] = fi;
        y[p] = yi;
        fp = fi;
        yp = yi;
        supp = sup[p];
    }
    // back substitution with the backward pivots g_i = d_i - sup_i sub_{i+1} / g_{i+1}
    T xn = T(0), gn = T(0), subn = T(0);
#pragma unroll 8
    for (int i = m - 1; i >= 0; --i) {
        const size_t p = (size_t)i * mm + c;
        const T d = diag[p] + Loth[p];
        const T r = b[p] + Moth[p];
        const T fi = f[p];
        const T su = sup[p];
        T xi, gi;
        if (i == m - 1) {
            xi = y[p] * fast_rcp(fi);
            gi = d;
        } else {
            xi = (y[p] - su * xn) * fast_rcp(fi);
            gi = d - su * subn * fast_rcp(gn);
        }
        bad |= bad_den(gi);
        const T S = fi + gi - d;
        Lown[p] = S - d;
        Mown[p] = S * xi - r;
        if (x) x[p] = (double)xi;
        xn = xi;
        gn = gi;
        subn = sub[p];
    }
    if (bad) atomicOr(flags, FLAG_BREAKDOWN);
}

// out[c * m + r] = in[r * m + c] through 32 x 32 shared-memory tiles.
template <typename T>
__global__ void k_transpose(int m, const T *__restrict__ in, T *__restrict__ out)
{
    __shared__ T tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = by + j, c = bx + threadIdx.x;
        if (r < m && c < m) tile[j][threadIdx.x] = in[(size_t)r * m + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = bx + j, c = by + threadIdx.x;  // output row = input column
        if (r < m && c < m) out[(size_t)r * m + c] = tile[threadIdx.x][j];
    }
}

}  // namespace

cudaError_t launch_line_phase(int prec, int m, const void *sub, const void *sup, const void *diag,
                              const void *b, const void *Loth, const void *Moth, void *Lown,
                              void *Mown, void *f, void *y, double *x, unsigned *flags,
                              cudaStream_t s)
{
    if (m == 0) return cudaSuccess;
    count_launches(s, 1);
    // few threads exist (one per line): small blocks spread them over more SMs
    const int block = 32, grid = (m + block - 1) / block;
    if (prec == 0)
        k_line_phase<double><<<grid, block, 0, s>>>(
            m, (const double *)sub, (const double *)sup, (const double *)diag, (const double *)b,
            (const double *)Loth, (const double *)Moth, (double *)Lown, (double *)Mown,
            (double *)f, (double *)y, x, flags);
    else
        k_line_phase<float><<<grid, block, 0, s>>>(
            m, (const float *)sub, (const float *)sup, (const float *)diag, (const float *)b,
            (const float *)Loth, (const float *)Moth, (float *)Lown, (float *)Mown, (float *)f,
            (float *)y, x, flags);
    return cudaGetLastError();
}

cudaError_t launch_transpose(int prec, int m, const void *in, void *out, cudaStream_t s)
{
    if (m == 0) return cudaSuccess;
    count_launches(s, 1);
    const dim3 block(32, 8), grid((m + 31) / 32, (m + 31) / 32);
    if (prec == 0)
        k_transpose<double><<<grid, block, 0, s>>>(m, (const double *)in, (double *)out);
    else
        k_transpose<float><<<grid, block, 0, s>>>(m, (const float *)in, (float *)out);
    return cudaGetLastError();
}

}  // namespace gabp
