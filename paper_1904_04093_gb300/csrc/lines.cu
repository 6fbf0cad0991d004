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
//     S_i = 1 / (T^{-1})_ii
//     Lambda_i = S_i - d_i,   m_i = S_i x_i - r_i
// which is the message rule of Algorithm 2 written for a tridiagonal block.
//
// Both quantities come from the forward and the backward elimination of T:
//     f_i = d_i - sub_i sup_{i-1} / f_{i-1},   yF_i = r_i - sub_i yF_{i-1} / f_{i-1}
//     g_i = d_i - sup_i sub_{i+1} / g_{i+1},   yB_i = r_i - sup_i yB_{i+1} / g_{i+1}
// Adding the two eliminated forms of row i (f_i x_i + sup_i x_{i+1} = yF_i and
// sub_i x_{i-1} + g_i x_i = yB_i) and subtracting row i itself gives
//     (f_i + g_i - d_i) x_i = yF_i + yB_i - r_i,
// so S_i = f_i + g_i - d_i (the twisted-factorisation pivot, the inverse of
// the diagonal of T^{-1}) and
//     Lambda_i = (f_i - d_i) + (g_i - d_i),   m_i = (yF_i - r_i) + (yB_i - r_i).
//
// Parallel form.  One CTA per line; thread t owns the contiguous chunk
// [t C, t C + C) of the line.  In homogeneous coordinates (N, D, Y) with
// f = N / D and yF = Y / D the forward elimination is linear:
//     (N, D, Y)_i = [[d_i, -p_i, 0], [1, 0, 0], [r_i, 0, -sub_i]] (N, D, Y)_{i-1},
// p_i = sub_i sup_{i-1}, starting from (1, 0, 0); the backward one likewise
// with sup_i, q_i = sup_i sub_{i+1}.  Each thread forms the product of its
// chunk's matrices, a block scan of the products (warp shuffles, then the
// warp totals) gives every chunk its exact entry state, and each thread then
// runs the ordinary recurrences over its chunk from that state.  Products and
// states are rescaled by powers of two (exact; the ratios N/D, Y/D are what
// matter).  The line's data are staged in shared memory and the results leave
// through coalesced copies; lines too long for shared memory run the same
// algorithm on global memory.
//
// Layout: element i of line c sits at c * m + i (rows: natural order;
// columns: transposed order), so a line is contiguous.
#include <cuda_runtime.h>

#include <algorithm>

#include "gabp_internal.h"
#include "sweep_row.cuh"

namespace gabp {
namespace {

constexpr int kLineMaxThreads = 256;
constexpr int kLineMaxWarps = kLineMaxThreads / 32;
constexpr size_t kLineSmemMax = 220 * 1024;  // dynamic part; the scan's own arrays are static

// [[a, b, 0], [c, e, 0], [g, h, k]]
template <typename T>
struct Xf {
    T a, b, c, e, g, h, k;
};

template <typename T>
__device__ __forceinline__ Xf<T> xf_identity()
{
    return {T(1), T(0), T(0), T(1), T(0), T(0), T(1)};
}

// t2 * t1 (t1 applied first)
template <typename T>
__device__ __forceinline__ Xf<T> xf_mul(const Xf<T> &t2, const Xf<T> &t1)
{
    Xf<T> r;
    r.a = t2.a * t1.a + t2.b * t1.c;
    r.b = t2.a * t1.b + t2.b * t1.e;
    r.c = t2.c * t1.a + t2.e * t1.c;
    r.e = t2.c * t1.b + t2.e * t1.e;
    r.g = t2.g * t1.a + t2.h * t1.c + t2.k * t1.g;
    r.h = t2.g * t1.b + t2.h * t1.e + t2.k * t1.h;
    r.k = t2.k * t1.k;
    return r;
}

template <typename T>
__device__ __forceinline__ Xf<T> xf_shfl_up(const Xf<T> &v, int off)
{
    const unsigned F = 0xffffffffu;
    return {__shfl_up_sync(F, v.a, off), __shfl_up_sync(F, v.b, off), __shfl_up_sync(F, v.c, off),
            __shfl_up_sync(F, v.e, off), __shfl_up_sync(F, v.g, off), __shfl_up_sync(F, v.h, off),
            __shfl_up_sync(F, v.k, off)};
}

template <typename T>
__device__ __forceinline__ Xf<T> xf_shfl_down(const Xf<T> &v, int off)
{
    const unsigned F = 0xffffffffu;
    return {__shfl_down_sync(F, v.a, off), __shfl_down_sync(F, v.b, off),
            __shfl_down_sync(F, v.c, off), __shfl_down_sync(F, v.e, off),
            __shfl_down_sync(F, v.g, off), __shfl_down_sync(F, v.h, off),
            __shfl_down_sync(F, v.k, off)};
}

// Biased exponent field and the power of two 2^(bias - e) that scales a
// number with exponent field e to about 1 (exact).
__device__ __forceinline__ int expo(double v)
{
    return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ffull);
}
__device__ __forceinline__ int expo(float v) { return (int)(((unsigned)__float_as_int(v) >> 23) & 0xffu); }
__device__ __forceinline__ bool expo_scalable(int e, double) { return e > 0 && e < 0x7ff; }
__device__ __forceinline__ bool expo_scalable(int e, float) { return e > 0 && e < 0xff; }
__device__ __forceinline__ double pow2_inv(int e, double)
{
    int f = 2046 - e;
    f = f < 1 ? 1 : f;
    return __longlong_as_double((long long)f << 52);
}
__device__ __forceinline__ float pow2_inv(int e, float)
{
    int f = 254 - e;
    f = f < 1 ? 1 : f;
    return __int_as_float(f << 23);
}

// Exact power-of-two prescale of a line.  Between two rescalings the chunk
// product of kRescaleMask + 1 steps grows like |d|^(kRescaleMask + 1), which
// leaves the exponent range once |d| passes about 2^31 (float) or 2^127
// (double).  A line whose first pivot d0 lies outside 2^(+-kScaleSlack) is
// therefore brought to |d0| in [1, 2): returns sc = 2^-k and sets isc = 2^k,
// with the shift k clamped so that sc^2 stays representable; otherwise 1.
template <typename T>
constexpr int kScaleSlack = sizeof(T) == 8 ? 64 : 12;

__device__ __forceinline__ double line_scale(double d0, double &isc)
{
    const int k = expo(d0) - 1023;
    if (expo(d0) == 0 || expo(d0) == 0x7ff || abs(k) <= kScaleSlack<double>) {
        isc = 1.0;
        return 1.0;
    }
    const int c = max(-500, min(500, k));
    isc = __longlong_as_double((long long)(1023 + c) << 52);
    return __longlong_as_double((long long)(1023 - c) << 52);
}
__device__ __forceinline__ float line_scale(float d0, float &isc)
{
    const int k = expo(d0) - 127;
    if (expo(d0) == 0 || expo(d0) == 0xff || abs(k) <= kScaleSlack<float>) {
        isc = 1.0f;
        return 1.0f;
    }
    const int c = max(-62, min(62, k));
    isc = __int_as_float((127 + c) << 23);
    return __int_as_float((127 - c) << 23);
}

// Rescales a product by the exponent of its larger pivot entry (a or b, the
// N components of the images of (1, 0, 0) and (0, 1, 0)).  These carry the
// growth of the pivots; the Y row then holds ratios Y / N = yF / f, bounded by
// the data, while c, e trail a, b by one step and k only shrinks.  Scaling by
// a larger Y entry instead would leave a, b tiny, and the squaring in the
// block scan would flush them to zero.
template <typename T>
__device__ __forceinline__ void xf_normalize(Xf<T> &t)
{
    const int e = max(expo(t.a), expo(t.b));
    if (!expo_scalable(e, T(0))) return;
    const T s = pow2_inv(e, T(0));
    t.a *= s; t.b *= s; t.c *= s; t.e *= s; t.g *= s; t.h *= s; t.k *= s;
}

// Same for a state (N, D, Y): by the exponent of N or D (f = N / D, yF = Y / D).
template <typename T>
__device__ __forceinline__ void st_normalize(T &N, T &D, T &Y)
{
    const int e = max(expo(N), expo(D));
    if (!expo_scalable(e, T(0))) return;
    const T s = pow2_inv(e, T(0));
    N *= s; D *= s; Y *= s;
}

// One elimination step (forward or backward) applied on the left of t:
// t <- [[d, -p, 0], [1, 0, 0], [r, 0, -s]] t
template <typename T>
__device__ __forceinline__ void xf_step(Xf<T> &t, T d, T p, T r, T s)
{
    const T na = d * t.a - p * t.c, nb = d * t.b - p * t.e;
    const T ng = r * t.a - s * t.g, nh = r * t.b - s * t.h;
    t.c = t.a;
    t.e = t.b;
    t.a = na;
    t.b = nb;
    t.g = ng;
    t.h = nh;
    t.k = -s * t.k;
}

// Steps between rescalings of a chunk product: the entries grow by about the
// pivot per step, so float rescales more often.
template <typename T>
constexpr int kRescaleMask = sizeof(T) == 8 ? 7 : 3;

// Reciprocal of the line recurrences: the double one of the sweep; for float
// the hardware approximation and one Newton-Raphson step (within an ulp or
// so, enough for float messages; the IEEE-rounded intrinsic costs more).
template <typename T>
__device__ __forceinline__ T line_rcp(T d)
{
    return fast_rcp(d);
}
template <>
__device__ __forceinline__ float line_rcp<float>(float d)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(d));
    return fmaf(y, fmaf(-d, y, 1.0f), y);
}

template <typename T>
constexpr int kPadShift = sizeof(T) == 8 ? 4 : 5;

// Length of a padded shared array of m elements (pad shift sh).
__host__ __device__ __forceinline__ int line_padded(int m, int sh) { return m + (m >> sh) + 1; }

// kFreeze: instead of the messages, write the frozen-state coefficients of
// the line (precision messages converged): aF_i = -sub_i / f_{i-1},
// aB_i = -sup_i / g_{i+1} and sinv_i = 1 / (f_i + g_i - d_i).
template <typename T, bool kSmem, bool kFreeze>
__global__ void __launch_bounds__(kLineMaxThreads) k_line_scan(
    int m, const T *__restrict__ sub, const T *__restrict__ sup, const T *__restrict__ diag,
    const T *__restrict__ b, const T *__restrict__ Loth, const T *__restrict__ Moth,
    T *__restrict__ Lown, T *__restrict__ Mown, T *__restrict__ fws, T *__restrict__ yws,
    double *__restrict__ x, int x_transposed, unsigned *__restrict__ flags,
    T *__restrict__ aF, T *__restrict__ aB, T *__restrict__ sinv)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char line_smem[];
    __shared__ Xf<T> wF[kLineMaxWarps], wB[kLineMaxWarps];
    __shared__ T stF[kLineMaxWarps][3], stB[kLineMaxWarps][3];

    const int line = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
    if (kIndexChecks && line >= m) {  // the grid is m lines by construction
        if (tid == 0) atomicOr(flags, FLAG_INDEX);
        return;
    }
    const int lane = tid & 31, w = tid >> 5, NW = NT >> 5;
    const size_t base = (size_t)line * m;
    const T *gd = diag + base, *gLo = Loth + base, *gb = b + base, *gMo = Moth + base;
    // per element: d, r, the couplings sub, sup and their products
    // p_i = sub_i sup_{i-1} (forward) and q_i = sup_i sub_{i+1} (backward);
    // the forward results f, yF later take the places of p and sub, which the
    // backward recurrences no longer read
    const T *su, *sq;
    const T *sp, *sl;
    T *sd = nullptr, *sr = nullptr, *sf, *sy;
    // shared arrays hold element i at i + (i >> kPadShift): one pad word per
    // 32 floats (16 doubles), so that the threads' chunk walks (stride C)
    // fall in distinct banks; global arrays use plain indices
    const int sh = kSmem ? kPadShift<T> : 31;
    auto ix = [&](int i) -> int { return i + (i >> sh); };
    // the line's prescale (line_scale): d, the couplings and their products are
    // taken times sc, the right-hand sides r are not.  The pivots f, g then come
    // out times sc, while yF, yB, the mean messages and the multipliers aF, aB
    // are unchanged; every product is exact, so the results are those of the
    // unscaled recurrences wherever these stay in range.
    T isc;
    const T sc = line_scale(m > 0 ? gd[0] + gLo[0] : T(1), isc);
    const bool scaled = sc != T(1);
    const T sc2 = sc * sc;
    if (kSmem) {
        const int mp = line_padded(m, kPadShift<T>);
        T *sm = reinterpret_cast<T *>(line_smem);
        sd = sm;
        sr = sm + mp;
        T *wl = sm + 2 * (size_t)mp, *wu = sm + 3 * (size_t)mp;
        T *wp = sm + 4 * (size_t)mp, *wq = sm + 5 * (size_t)mp;
        const T *gl = sub + base, *gu = sup + base;
        // an unscaled double line (the usual case) takes a loop without the
        // multiplies, which would cost FP64-pipe issue; float always multiplies
        // (sc = 1 when unscaled)
        if (sizeof(T) == 8 && !scaled) {
            for (int i = tid; i < m; i += NT) {
                const T li = gl[i], ui = gu[i];
                const int j = ix(i);
                sd[j] = gd[i] + gLo[i];
                sr[j] = gb[i] + gMo[i];
                wl[j] = li;
                wu[j] = ui;
                wp[j] = i > 0 ? li * gu[i - 1] : T(0);
                wq[j] = i + 1 < m ? ui * gl[i + 1] : T(0);
            }
        } else {
            for (int i = tid; i < m; i += NT) {
                const T li = gl[i], ui = gu[i];
                const int j = ix(i);
                sd[j] = (gd[i] + gLo[i]) * sc;
                sr[j] = gb[i] + gMo[i];
                wl[j] = li * sc;
                wu[j] = ui * sc;
                wp[j] = i > 0 ? (li * gu[i - 1]) * sc2 : T(0);
                wq[j] = i + 1 < m ? (ui * gl[i + 1]) * sc2 : T(0);
            }
        }
        sl = wl;
        su = wu;
        sp = wp;
        sq = wq;
        sf = wp;
        sy = wl;
        __syncthreads();
    } else {
        sl = sub + base;
        su = sup + base;
        sp = nullptr;
        sq = nullptr;
        sf = fws + base;
        sy = yws + base;
    }
    // staged values carry the prescale already; values read from global memory
    // (lines too long for shared memory) take it here
    auto G = [&](T v, T f) -> T { return (!kSmem && scaled) ? v * f : v; };
    auto Dv = [&](int i) -> T { return kSmem ? sd[ix(i)] : G(gd[i] + gLo[i], sc); };
    auto Rv = [&](int i) -> T { return kSmem ? sr[ix(i)] : gb[i] + gMo[i]; };
    auto Lv = [&](int i) -> T { return G(sl[ix(i)], sc); };
    auto Uv = [&](int i) -> T { return G(su[ix(i)], sc); };
    auto Pv = [&](int i) -> T { return kSmem ? sp[ix(i)] : G(i > 0 ? sl[i] * su[i - 1] : T(0), sc2); };
    auto Qv = [&](int i) -> T { return kSmem ? sq[ix(i)] : G(i + 1 < m ? su[i] * sl[i + 1] : T(0), sc2); };

    const int C = (m + NT - 1) / NT;
    const int lo = min(m, tid * C), hi = min(m, lo + C);

    // chunk products, forward (ascending i) and backward (descending i)
    Xf<T> pf = xf_identity<T>(), pb = xf_identity<T>();
    for (int i = lo, k = 0; i < hi; ++i, ++k) {
        xf_step(pf, Dv(i), Pv(i), Rv(i), Lv(i));
        if ((k & kRescaleMask<T>) == kRescaleMask<T>) xf_normalize(pf);
    }
    xf_normalize(pf);
    for (int i = hi - 1, k = 0; i >= lo; --i, ++k) {
        xf_step(pb, Dv(i), Qv(i), Rv(i), Uv(i));
        if ((k & kRescaleMask<T>) == kRescaleMask<T>) xf_normalize(pb);
    }
    xf_normalize(pb);

    // inclusive prefix (forward) and suffix (backward) products within the warp
    for (int off = 1; off < 32; off <<= 1) {
        const Xf<T> o = xf_shfl_up(pf, off);
        if (lane >= off) {
            pf = xf_mul(pf, o);
            xf_normalize(pf);
        }
    }
    for (int off = 1; off < 32; off <<= 1) {
        const Xf<T> o = xf_shfl_down(pb, off);
        if (lane + off < 32) {
            pb = xf_mul(pb, o);
            xf_normalize(pb);
        }
    }
    if (lane == 31) wF[w] = pf;
    if (lane == 0) wB[w] = pb;
    __syncthreads();
    if (tid == 0) {
        // entry state of every warp, forward from (1, 0, 0) at the line start
        T N = T(1), D = T(0), Y = T(0);
        for (int v = 0; v < NW; ++v) {
            stF[v][0] = N;
            stF[v][1] = D;
            stF[v][2] = Y;
            const Xf<T> &t = wF[v];
            const T n2 = t.a * N + t.b * D, d2 = t.c * N + t.e * D, y2 = t.g * N + t.h * D + t.k * Y;
            N = n2;
            D = d2;
            Y = y2;
            st_normalize(N, D, Y);
        }
        // and backward from (1, 0, 0) past the line end
        N = T(1);
        D = T(0);
        Y = T(0);
        for (int v = NW - 1; v >= 0; --v) {
            stB[v][0] = N;
            stB[v][1] = D;
            stB[v][2] = Y;
            const Xf<T> &t = wB[v];
            const T n2 = t.a * N + t.b * D, d2 = t.c * N + t.e * D, y2 = t.g * N + t.h * D + t.k * Y;
            N = n2;
            D = d2;
            Y = y2;
            st_normalize(N, D, Y);
        }
    }
    __syncthreads();
    Xf<T> ef = xf_shfl_up(pf, 1), eb = xf_shfl_down(pb, 1);
    if (lane == 0) ef = xf_identity<T>();
    if (lane == 31) eb = xf_identity<T>();

    bool bad = false;
    // forward recurrences over the chunk from its entry state
    {
        const T N0 = stF[w][0], D0 = stF[w][1], Y0 = stF[w][2];
        const T N = ef.a * N0 + ef.b * D0, D = ef.c * N0 + ef.e * D0,
                Y = ef.g * N0 + ef.h * D0 + ef.k * Y0;
        const T rn = line_rcp(N);
        T inv = D * rn, wv = Y * rn;  // 1 / f_{i-1}, yF_{i-1} / f_{i-1}
        for (int i = lo; i < hi; ++i) {
            const T s = Lv(i);
            if (kFreeze) aF[base + i] = -s * inv;
            const T f = Dv(i) - Pv(i) * inv;
            const T y = Rv(i) - s * wv;
            bad |= bad_den(f);
            inv = line_rcp(f);
            wv = y * inv;
            sf[ix(i)] = f;
            sy[ix(i)] = y;
        }
    }
    // backward recurrences and the outputs
    {
        const T N0 = stB[w][0], D0 = stB[w][1], Y0 = stB[w][2];
        const T N = eb.a * N0 + eb.b * D0, D = eb.c * N0 + eb.e * D0,
                Y = eb.g * N0 + eb.h * D0 + eb.k * Y0;
        const T rn = line_rcp(N);
        T inv = D * rn, wv = Y * rn;  // 1 / g_{i+1}, yB_{i+1} / g_{i+1}
        for (int i = hi - 1; i >= lo; --i) {
            const T u = Uv(i);
            const T d = Dv(i), r = Rv(i);
            if (kFreeze) aB[base + i] = -u * inv;
            const T g = d - Qv(i) * inv;
            const T yb = r - u * wv;
            bad |= bad_den(g);
            inv = line_rcp(g);
            wv = yb * inv;
            const T f = sf[ix(i)], y = sy[ix(i)];
            if (kFreeze) {
                const T si = T(1) / ((f - d) + g);
                sinv[base + i] = scaled ? si * sc : si;
                continue;
            }
            // times sc when the line is prescaled: undone where it is written
            const T lam = (f - d) + (g - d);
            const T mu = (y - r) + (yb - r);
            if (x) {
                T xs = ((y - r) + yb) / ((f - d) + g);
                if (scaled) xs *= sc;
                const double xi = (double)xs;
                x[x_transposed ? (size_t)i * m + line : base + i] = xi;
            }
            if (kSmem) {
                sf[ix(i)] = lam;
                sy[ix(i)] = mu;
            } else {
                Lown[base + i] = scaled ? lam * isc : lam;
                Mown[base + i] = mu;
            }
        }
    }
    if (kSmem && !kFreeze) {
        __syncthreads();
        if (scaled) {
            for (int i = tid; i < m; i += NT) {
                Lown[base + i] = sf[ix(i)] * isc;
                Mown[base + i] = sy[ix(i)];
            }
        } else {
            for (int i = tid; i < m; i += NT) {
                Lown[base + i] = sf[ix(i)];
                Mown[base + i] = sy[ix(i)];
            }
        }
    }
    if (bad) atomicOr(flags, FLAG_BREAKDOWN);
}

// Line phase with frozen precision messages: only the mean messages move.
// With the fixed multipliers aF, aB and 1 / S of the line,
//     yF_i = r_i + aF_i yF_{i-1},   yB_i = r_i + aB_i yB_{i+1},   r_i = b_i + m'_i,
//     m_i = (yF_i - r_i) + (yB_i - r_i),   x_i = (yF_i + yB_i - r_i) / S_i,
// the same update as the full phase up to rounding.  The recurrences are
// affine, so a chunk is the map y -> A y + B and the block scan composes
// pairs (A, B); no rescaling is needed.
template <typename T, bool kSmem>
__global__ void __launch_bounds__(kLineMaxThreads) k_line_mean(
    int m, const T *__restrict__ aF, const T *__restrict__ aB, const T *__restrict__ sinv,
    const T *__restrict__ b, const T *__restrict__ Moth, T *__restrict__ Mown,
    T *__restrict__ yws, double *__restrict__ x, int x_transposed, unsigned *__restrict__ flags)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char line_smem[];
    __shared__ T wF[kLineMaxWarps][2], wB[kLineMaxWarps][2], yinF[kLineMaxWarps],
        yinB[kLineMaxWarps];

    const int line = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
    if (kIndexChecks && line >= m) {  // the grid is m lines by construction
        if (tid == 0) atomicOr(flags, FLAG_INDEX);
        return;
    }
    const int lane = tid & 31, w = tid >> 5, NW = NT >> 5;
    const size_t base = (size_t)line * m;
    const T *gb = b + base, *gMo = Moth + base;
    const int sh = kSmem ? kPadShift<T> : 31;
    auto ix = [&](int i) -> int { return i + (i >> sh); };
    T *sr = nullptr, *sa = nullptr, *sb = nullptr, *sy;
    if (kSmem) {
        const int mp = line_padded(m, kPadShift<T>);
        T *sm = reinterpret_cast<T *>(line_smem);
        sr = sm;
        sa = sm + mp;
        sb = sm + 2 * (size_t)mp;
        sy = sm + 3 * (size_t)mp;
        for (int i = tid; i < m; i += NT) {
            const int j = ix(i);
            sr[j] = gb[i] + gMo[i];
            sa[j] = aF[base + i];
            sb[j] = aB[base + i];
        }
        __syncthreads();
    } else {
        sy = yws + base;
    }
    auto Rv = [&](int i) -> T { return kSmem ? sr[ix(i)] : gb[i] + gMo[i]; };
    auto Av = [&](int i) -> T { return kSmem ? sa[ix(i)] : aF[base + i]; };
    auto Bv = [&](int i) -> T { return kSmem ? sb[ix(i)] : aB[base + i]; };

    const int C = (m + NT - 1) / NT;
    const int lo = min(m, tid * C), hi = min(m, lo + C);
    // the chunk's maps: forward y_{hi-1} = fa y_{lo-1} + fb, backward y_lo = ba y_hi + bb
    T fa = T(1), fb = T(0), ba = T(1), bb = T(0);
    for (int i = lo; i < hi; ++i) {
        const T a = Av(i);
        fb = a * fb + Rv(i);
        fa = a * fa;
    }
    for (int i = hi - 1; i >= lo; --i) {
        const T a = Bv(i);
        bb = a * bb + Rv(i);
        ba = a * ba;
    }
    const unsigned F = 0xffffffffu;
    for (int off = 1; off < 32; off <<= 1) {
        const T oa = __shfl_up_sync(F, fa, off), ob = __shfl_up_sync(F, fb, off);
        if (lane >= off) {
            fb = fa * ob + fb;
            fa = fa * oa;
        }
    }
    for (int off = 1; off < 32; off <<= 1) {
        const T oa = __shfl_down_sync(F, ba, off), ob = __shfl_down_sync(F, bb, off);
        if (lane + off < 32) {
            bb = ba * ob + bb;
            ba = ba * oa;
        }
    }
    if (lane == 31) {
        wF[w][0] = fa;
        wF[w][1] = fb;
    }
    if (lane == 0) {
        wB[w][0] = ba;
        wB[w][1] = bb;
    }
    __syncthreads();
    if (tid == 0) {
        T y = T(0);
        for (int v = 0; v < NW; ++v) {
            yinF[v] = y;
            y = wF[v][0] * y + wF[v][1];
        }
    } else if (tid == (NW > 1 ? 32 : 1)) {  // the backward scan on warp 1 when there is one
        T y = T(0);
        for (int v = NW - 1; v >= 0; --v) {
            yinB[v] = y;
            y = wB[v][0] * y + wB[v][1];
        }
    }
    __syncthreads();
    T efa = __shfl_up_sync(F, fa, 1), efb = __shfl_up_sync(F, fb, 1);
    T eba = __shfl_down_sync(F, ba, 1), ebb = __shfl_down_sync(F, bb, 1);
    if (lane == 0) {
        efa = T(1);
        efb = T(0);
    }
    if (lane == 31) {
        eba = T(1);
        ebb = T(0);
    }
    T y = efa * yinF[w] + efb;  // yF_{lo-1}
    for (int i = lo; i < hi; ++i) {
        y = Av(i) * y + Rv(i);
        sy[ix(i)] = y;
    }
    T yb = eba * yinB[w] + ebb;  // yB_hi
    for (int i = hi - 1; i >= lo; --i) {
        const T r = Rv(i);
        yb = Bv(i) * yb + r;
        const T yf = sy[ix(i)];
        const T mu = (yf - r) + (yb - r);
        if (x) x[x_transposed ? (size_t)i * m + line : base + i] = (double)(((yf - r) + yb) * sinv[base + i]);
        if (kSmem)
            sy[ix(i)] = mu;
        else
            Mown[base + i] = mu;
    }
    if (kSmem) {
        __syncthreads();
        for (int i = tid; i < m; i += NT) Mown[base + i] = sy[ix(i)];
    }
}

// Loads n <= C consecutive elements p[0..n) into v (v[j] = fill for j >= n),
// with 16-byte vector loads when the whole chunk is present and aligned.
template <typename T, int C>
__device__ __forceinline__ void load_chunk(T (&v)[C], const T *__restrict__ p, int n, bool vec, T fill)
{
    constexpr int V = 16 / sizeof(T);
    if (C % V == 0 && vec && n == C) {
#pragma unroll
        for (int j = 0; j < C; j += V) {
            if (sizeof(T) == 4) {
                const float4 q = *reinterpret_cast<const float4 *>(p + j);
                v[j] = (T)q.x; v[j + 1] = (T)q.y; v[j + 2] = (T)q.z; v[j + 3] = (T)q.w;
            } else {
                const double2 q = *reinterpret_cast<const double2 *>(p + j);
                v[j] = (T)q.x; v[j + 1] = (T)q.y;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < C; ++j) v[j] = j < n ? p[j] : fill;
    }
}

// The frozen line phase with each thread's chunk of C elements held in
// registers (no shared-memory staging): the loads are issued up front as
// vectors, the chunk maps, the block scan and the recurrences then run on
// registers.  Used when the line splits into at most 256 chunks of C <= 16.
// kSumOut: Mown receives b + m' (the sum the column phase on the natural
// order starts from) instead of m'.
template <typename T, int C, bool kSumOut = false>
__global__ void __launch_bounds__(kLineMaxThreads) k_line_mean_reg(
    int m, const T *__restrict__ aF, const T *__restrict__ aB, const T *__restrict__ sinv,
    const T *__restrict__ b, const T *__restrict__ Moth, T *__restrict__ Mown,
    double *__restrict__ x, int x_transposed, int vec, unsigned *__restrict__ flags)
{
    pdl_wait();
    pdl_trigger();
    __shared__ T wF[kLineMaxWarps][2], wB[kLineMaxWarps][2], yinF[kLineMaxWarps],
        yinB[kLineMaxWarps];
    const int line = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
    if (kIndexChecks && (line >= m || (long long)NT * C < m)) {  // m lines of at most NT chunks
        if (tid == 0) atomicOr(flags, FLAG_INDEX);
        return;
    }
    const int lane = tid & 31, w = tid >> 5, NW = NT >> 5;
    const size_t base = (size_t)line * m;
    const int lo = tid * C;
    const int n = max(0, min(C, m - lo));
    const size_t p0 = base + (n > 0 ? lo : 0);
    T r[C], a[C], c[C], mo[C];
    // past the line end: identity steps (a = c = 1, r = 0)
    load_chunk<T, C>(r, b + p0, n, vec != 0, T(0));
    load_chunk<T, C>(mo, Moth + p0, n, vec != 0, T(0));
    load_chunk<T, C>(a, aF + p0, n, vec != 0, T(1));
    load_chunk<T, C>(c, aB + p0, n, vec != 0, T(1));
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const T bj = r[j];
        r[j] += mo[j];
        if (kSumOut) mo[j] = bj;  // b kept for the output sum
    }

    T fa = T(1), fb = T(0), ba = T(1), bb = T(0);
#pragma unroll
    for (int j = 0; j < C; ++j) {
        fb = a[j] * fb + r[j];
        fa = a[j] * fa;
    }
#pragma unroll
    for (int j = C - 1; j >= 0; --j) {
        bb = c[j] * bb + r[j];
        ba = c[j] * ba;
    }
    const unsigned F = 0xffffffffu;
    for (int off = 1; off < 32; off <<= 1) {
        const T oa = __shfl_up_sync(F, fa, off), ob = __shfl_up_sync(F, fb, off);
        const T qa = __shfl_down_sync(F, ba, off), qb = __shfl_down_sync(F, bb, off);
        if (lane >= off) {
            fb = fa * ob + fb;
            fa = fa * oa;
        }
        if (lane + off < 32) {
            bb = ba * qb + bb;
            ba = ba * qa;
        }
    }
    if (lane == 31) {
        wF[w][0] = fa;
        wF[w][1] = fb;
    }
    if (lane == 0) {
        wB[w][0] = ba;
        wB[w][1] = bb;
    }
    __syncthreads();
    if (tid == 0) {
        T y = T(0);
        for (int v = 0; v < NW; ++v) {
            yinF[v] = y;
            y = wF[v][0] * y + wF[v][1];
        }
    } else if (tid == (NW > 1 ? 32 : 1)) {  // the backward scan on warp 1 when there is one
        T y = T(0);
        for (int v = NW - 1; v >= 0; --v) {
            yinB[v] = y;
            y = wB[v][0] * y + wB[v][1];
        }
    }
    __syncthreads();
    T efa = __shfl_up_sync(F, fa, 1), efb = __shfl_up_sync(F, fb, 1);
    T eba = __shfl_down_sync(F, ba, 1), ebb = __shfl_down_sync(F, bb, 1);
    if (lane == 0) {
        efa = T(1);
        efb = T(0);
    }
    if (lane == 31) {
        eba = T(1);
        ebb = T(0);
    }
    T yf[C];
    T y = efa * yinF[w] + efb;
#pragma unroll
    for (int j = 0; j < C; ++j) {
        y = a[j] * y + r[j];
        yf[j] = y;
    }
    T yb = eba * yinB[w] + ebb;
    T mu[C];
#pragma unroll
    for (int j = C - 1; j >= 0; --j) {
        yb = c[j] * yb + r[j];
        mu[j] = (yf[j] - r[j]) + (yb - r[j]);
        if (x && j < n)
            x[x_transposed ? (size_t)(lo + j) * m + line : base + lo + j] =
                (double)(((yf[j] - r[j]) + yb) * sinv[base + lo + j]);
    }
    if (kSumOut) {
#pragma unroll
        for (int j = 0; j < C; ++j) mu[j] = mo[j] + mu[j];  // the same rounding as the reader's b + m'
    }
    constexpr int V = 16 / sizeof(T);
    if (C % V == 0 && vec && n == C) {
#pragma unroll
        for (int j = 0; j < C; j += V) {
            if (sizeof(T) == 4) {
                *reinterpret_cast<float4 *>(Mown + p0 + j) =
                    make_float4((float)mu[j], (float)mu[j + 1], (float)mu[j + 2], (float)mu[j + 3]);
            } else {
                *reinterpret_cast<double2 *>(Mown + p0 + j) = make_double2((double)mu[j], (double)mu[j + 1]);
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < C; ++j)
            if (j < n) Mown[p0 + j] = mu[j];
    }
}

// Frozen column phase read and written in the natural node order (no
// transposes).  A CTA owns kColLines adjacent column lines; thread (warp w,
// lane l) takes line x0 + l % kColLines and chunk k = (32 / kColLines) w +
// l / kColLines of C consecutive rows y (node y m + x).  A warp instruction
// then touches row segments of kColLines adjacent columns.  The chunk maps of
// a line are scanned across its lanes (shuffles by multiples of kColLines),
// then across the warps (one thread per line and direction, the two
// directions on two warps).  Float messages, lines of at most 128 C rows.
// The row family's messages arrive folded into the right-hand side, S = b +
// m'_row (written so by the row phase), which is the r the recurrences start
// from: one array fewer to read.  A sweep that writes the beliefs x also reads
// b and leaves the row messages themselves, S - b, in S's place (kX: the
// form of the sweeps that write x).
// kFull: every chunk of the grid is a whole chunk inside the matrix (m a
// multiple of 32 / kColLines chunks of C), so the loads and stores go
// unguarded; the guarded form of the same kernel measured 25.6 against
// 18.5 us at 2048 x 2048.
constexpr int kColLines = 8;  // 8 adjacent columns: 32-byte row segments (4 lines measured slower)
template <typename T, int C, bool kFull, bool kX>
__global__ void __launch_bounds__(1024, 1) k_line_mean_cols(
    int m, const T *__restrict__ aF, const T *__restrict__ aB, const T *__restrict__ sinv,
    const T *__restrict__ b, T *S, T *__restrict__ Mown, double *__restrict__ x,
    unsigned *__restrict__ flags)
{
    pdl_wait();
    pdl_trigger();
    constexpr int QW = 32 / kColLines;  // chunks of each line per warp
    __shared__ T wF[32][kColLines][2], wB[32][kColLines][2], yinF[32][kColLines],
        yinB[32][kColLines];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, NW = blockDim.x >> 5;
    const int li = lane % kColLines, q = lane / kColLines;
    if (kIndexChecks && (int)blockIdx.x * kColLines >= m) {  // the grid covers the m columns
        if (tid == 0) atomicOr(flags, FLAG_INDEX);
        return;
    }
    const int xc = blockIdx.x * kColLines + li;
    const int lo = (QW * w + q) * C;
    const int n = xc < m ? max(0, min(C, m - lo)) : 0;
    T r[C], a[C], c[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        if (kFull || j < n) {
            const size_t idx = (size_t)(lo + j) * m + xc;
            r[j] = S[idx];
            a[j] = aF[idx];
            c[j] = aB[idx];
        } else {  // identity steps
            r[j] = T(0);
            a[j] = T(1);
            c[j] = T(1);
        }
    }
    // forward map y_{hi-1} = fa y_{lo-1} + fb; backward map y_lo = ba y_hi + bb,
    // composed in ascending order on the right
    T fa = T(1), fb = T(0), ba = T(1), bb = T(0);
#pragma unroll
    for (int j = 0; j < C; ++j) {
        fb = a[j] * fb + r[j];
        fa = a[j] * fa;
        bb = ba * r[j] + bb;
        ba = ba * c[j];
    }
    const unsigned F = 0xffffffffu;
    for (int off = kColLines; off < 32; off <<= 1) {
        const T oa = __shfl_up_sync(F, fa, off), ob = __shfl_up_sync(F, fb, off);
        const T pa = __shfl_down_sync(F, ba, off), pb = __shfl_down_sync(F, bb, off);
        if (lane >= off) {
            fb = fa * ob + fb;
            fa = fa * oa;
        }
        if (lane + off < 32) {
            bb = ba * pb + bb;
            ba = ba * pa;
        }
    }
    if (q == QW - 1) {
        wF[w][li][0] = fa;
        wF[w][li][1] = fb;
    }
    if (q == 0) {
        wB[w][li][0] = ba;
        wB[w][li][1] = bb;
    }
    __syncthreads();
    const int bw = NW > 1 ? 32 : kColLines;  // the backward scan's first thread: warp 1 when there is one
    if (tid < kColLines) {
        T y = T(0);
        for (int v = 0; v < NW; ++v) {
            yinF[v][tid] = y;
            y = wF[v][tid][0] * y + wF[v][tid][1];
        }
    } else if (tid >= bw && tid < bw + kColLines) {
        const int l2 = tid - bw;
        T y = T(0);
        for (int v = NW - 1; v >= 0; --v) {
            yinB[v][l2] = y;
            y = wB[v][l2][0] * y + wB[v][l2][1];
        }
    }
    __syncthreads();
    T efa = __shfl_up_sync(F, fa, kColLines), efb = __shfl_up_sync(F, fb, kColLines);
    T eba = __shfl_down_sync(F, ba, kColLines), ebb = __shfl_down_sync(F, bb, kColLines);
    if (q == 0) {
        efa = T(1);
        efb = T(0);
    }
    if (q == QW - 1) {
        eba = T(1);
        ebb = T(0);
    }
    // the backward recurrence first, its values in place of the multipliers c
    // (no longer needed), then the forward one and the outputs
    T yb = eba * yinB[w][li] + ebb;
#pragma unroll
    for (int j = C - 1; j >= 0; --j) {
        yb = c[j] * yb + r[j];
        c[j] = yb;
    }
    T y = efa * yinF[w][li] + efb;
#pragma unroll
    for (int j = 0; j < C; ++j) {
        y = a[j] * y + r[j];
        if (kFull || j < n) {
            const size_t idx = (size_t)(lo + j) * m + xc;
            Mown[idx] = (y - r[j]) + (c[j] - r[j]);
            if (kX) {
                x[idx] = (double)(((y - r[j]) + c[j]) * sinv[idx]);
                S[idx] = r[j] - b[idx];  // read by this thread only, above
            }
        }
    }
}

// out[c * m + r] = in[r * m + c] through 64 x 64 shared-memory tiles: a
// 32 x 8 block moves 16 elements per thread, enough loads in flight to run
// near the copy bandwidth.
constexpr int kTile = 64;
template <typename T>
__global__ void __launch_bounds__(256) k_transpose(int m, const T *__restrict__ in, T *__restrict__ out)
{
    pdl_wait();
    pdl_trigger();
    __shared__ T tile[kTile][kTile + 1];
    const int bx = blockIdx.x * kTile, by = blockIdx.y * kTile;
#pragma unroll
    for (int j = threadIdx.y; j < kTile; j += 8)
#pragma unroll
        for (int k = 0; k < kTile; k += 32) {
            const int r = by + j, c = bx + threadIdx.x + k;
            if (r < m && c < m) tile[j][threadIdx.x + k] = in[(size_t)r * m + c];
        }
    __syncthreads();
#pragma unroll
    for (int j = threadIdx.y; j < kTile; j += 8)
#pragma unroll
        for (int k = 0; k < kTile; k += 32) {
            const int r = bx + j, c = by + threadIdx.x + k;  // output row = input column
            if (r < m && c < m) out[(size_t)r * m + c] = tile[threadIdx.x + k][j];
        }
}

// Couplings of the transposed system along contiguous lines of length m:
// (A^T)_{i,i-1} = A_{i-1,i}, so subT_i = sup_{i-1} and supT_i = sub_{i+1}
// (zero past the line ends).
template <typename T>
__global__ void k_line_couplings_transpose(int m, int64_t total, const T *__restrict__ sub,
                                           const T *__restrict__ sup, T *__restrict__ subT,
                                           T *__restrict__ supT)
{
    pdl_wait();
    pdl_trigger();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += stride) {
        const int i = (int)(p % m);
        subT[p] = i > 0 ? sup[p - 1] : T(0);
        supT[p] = i + 1 < m ? sub[p + 1] : T(0);
    }
}

// Line couplings from the stencil layout's coefficients (a_e = -A_rs at
// slot k * n + r, offset off[k]): along the rows (natural order) the west and
// east entries, along the columns (transposed order) the south and north ones
// and the diagonal.  The matrix is a 5-point grid (checked at setup), so a
// missing offset or a slot past a line end holds zero.
template <typename T>
__global__ void k_line_couplings_from_stencil(int n, int m, StencilParams sp,
                                              const double *__restrict__ a64,
                                              const double *__restrict__ diag64,
                                              T *__restrict__ subH, T *__restrict__ supH,
                                              T *__restrict__ subV, T *__restrict__ supV,
                                              T *__restrict__ diagV)
{
    pdl_wait();
    pdl_trigger();
    int kw = -1, ke = -1, ks = -1, kn = -1;
    for (int k = 0; k < sp.K; ++k) {
        if (sp.off[k] == -1) kw = k;
        if (sp.off[k] == 1) ke = k;
        if (sp.off[k] == -m) ks = k;
        if (sp.off[k] == m) kn = k;
    }
    const size_t nn = (size_t)n;
    const int stride = gridDim.x * blockDim.x;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const int x = r % m, y = r / m;
        const size_t t = (size_t)x * m + y;
        subH[r] = (T)(x > 0 && kw >= 0 ? -a64[kw * nn + r] : 0.0);
        supH[r] = (T)(x + 1 < m && ke >= 0 ? -a64[ke * nn + r] : 0.0);
        subV[t] = (T)(y > 0 && ks >= 0 ? -a64[ks * nn + r] : 0.0);
        supV[t] = (T)(y + 1 < m && kn >= 0 ? -a64[kn * nn + r] : 0.0);
        diagV[t] = (T)diag64[r];
    }
}

// Threads per line: at most 128 (double) or 256 (float), chunks of at least
// m / 128 or m / 256 elements, rounded up to whole warps.  Long chunks keep the
// scan's share of the work small; double is bound by the FP64 pipe, not by
// occupancy.  At 2048 nodes fewer threads per line ran slower (the chunk
// recurrences are latency-bound) and more added scan work.
constexpr int kLineThreadsF64 = 128;
constexpr int kLineThreadsF32 = 256;
int line_threads(int prec, int m)
{
    const int ntmax = prec == 0 ? kLineThreadsF64 : kLineThreadsF32;
    const int C = (m + ntmax - 1) / ntmax;
    const int nt = (m + C - 1) / C;
    return ((nt + 31) / 32) * 32;
}

size_t line_smem_bytes(int prec, int m)
{
    return prec == 0 ? 6 * (size_t)line_padded(m, kPadShift<double>) * 8
                     : 6 * (size_t)line_padded(m, kPadShift<float>) * 4;
}

size_t line_mean_smem_bytes(int prec, int m)
{
    return prec == 0 ? 4 * (size_t)line_padded(m, kPadShift<double>) * 8
                     : 4 * (size_t)line_padded(m, kPadShift<float>) * 4;
}

template <typename T, bool kFreeze>
cudaError_t launch_T(int m, const void *sub, const void *sup, const void *diag, const void *b,
                     const void *Loth, const void *Moth, void *Lown, void *Mown, void *f, void *y,
                     double *x, int x_transposed, unsigned *flags, void *aF, void *aB, void *sinv,
                     cudaStream_t s)
{
    const int prec = sizeof(T) == 8 ? 0 : 1;
    const int nt = line_threads(prec, m);
    const size_t smem = line_smem_bytes(prec, m);
    if (smem <= kLineSmemMax) {
        launch_pdl(k_line_scan<T, true, kFreeze>, m, nt, smem, s, m, (const T *)sub, (const T *)sup,
                   (const T *)diag, (const T *)b, (const T *)Loth, (const T *)Moth, (T *)Lown, (T *)Mown,
                   nullptr, nullptr, x, x_transposed, flags, (T *)aF, (T *)aB, (T *)sinv);
    } else {
        if (!f || !y) return cudaErrorInvalidValue;
        launch_pdl(k_line_scan<T, false, kFreeze>, m, nt, 0, s, m, (const T *)sub, (const T *)sup,
                   (const T *)diag, (const T *)b, (const T *)Loth, (const T *)Moth, (T *)Lown, (T *)Mown,
                   (T *)f, (T *)y, x, x_transposed, flags, (T *)aF, (T *)aB, (T *)sinv);
    }
    return cudaGetLastError();
}

// The register form, with the folded output (float only) when sum_out.
template <typename T, int CC>
void launch_mean_reg(bool sum_out, int m, int nt, const void *aF, const void *aB, const void *sinv,
                     const void *b, const void *Moth, void *Mown, double *x, int x_transposed, int vec,
                     unsigned *flags, cudaStream_t s)
{
    if constexpr (sizeof(T) == 4) {
        if (sum_out) {
            launch_pdl(k_line_mean_reg<T, CC, true>, m, nt, 0, s, m, (const T *)aF, (const T *)aB,
                       (const T *)sinv, (const T *)b, (const T *)Moth, (T *)Mown, x, x_transposed, vec, flags);
            return;
        }
    }
    launch_pdl(k_line_mean_reg<T, CC, false>, m, nt, 0, s, m, (const T *)aF, (const T *)aB, (const T *)sinv,
               (const T *)b, (const T *)Moth, (T *)Mown, x, x_transposed, vec, flags);
}

template <typename T>
cudaError_t launch_mean_T(int m, const void *aF, const void *aB, const void *sinv, const void *b,
                          const void *Moth, void *Mown, void *y, double *x, int x_transposed,
                          bool sum_out, unsigned *flags, cudaStream_t s)
{
    if (sum_out && sizeof(T) != 4) return cudaErrorInvalidValue;
    // register form: chunks of a power-of-two length C <= 16 over at most 256 threads
    int C = 1;
    while (C < 16 && (long long)C * kLineMaxThreads < m) C *= 2;
    if ((long long)C * kLineMaxThreads >= m) {
        const int nt = ((m + C - 1) / C + 31) / 32 * 32;
        const int vec = m % (16 / (int)sizeof(T)) == 0;
#define GABP_MEAN_REG(CC)                                                                                   \
    case CC:                                                                                                \
        launch_mean_reg<T, CC>(sum_out, m, nt, aF, aB, sinv, b, Moth, Mown, x, x_transposed, vec, flags, s); \
        break;
        switch (C) {
            GABP_MEAN_REG(1)
            GABP_MEAN_REG(2)
            GABP_MEAN_REG(4)
            GABP_MEAN_REG(8)
            GABP_MEAN_REG(16)
            default:
                return cudaErrorInvalidValue;
        }
#undef GABP_MEAN_REG
        return cudaGetLastError();
    }
    if (sum_out) return cudaErrorInvalidValue;  // the folded output has the register form only
    const int prec = sizeof(T) == 8 ? 0 : 1;
    const int nt = line_threads(1, m);  // little arithmetic per element: the wider split
    const size_t smem = line_mean_smem_bytes(prec, m);
    if (smem <= kLineSmemMax) {
        launch_pdl(k_line_mean<T, true>, m, nt, smem, s, m, (const T *)aF, (const T *)aB, (const T *)sinv,
                   (const T *)b, (const T *)Moth, (T *)Mown, nullptr, x, x_transposed, flags);
    } else {
        if (!y) return cudaErrorInvalidValue;
        launch_pdl(k_line_mean<T, false>, m, nt, 0, s, m, (const T *)aF, (const T *)aB, (const T *)sinv,
                   (const T *)b, (const T *)Moth, (T *)Mown, (T *)y, x, x_transposed, flags);
    }
    return cudaGetLastError();
}

}  // namespace

bool line_needs_scratch(int prec, int m) { return line_smem_bytes(prec, m) > kLineSmemMax; }

// The dynamic shared-memory limit of the staged line kernels is a property of
// the kernel, shared by every context in the process: it is raised to the
// largest size the launches may request (not to this context's), so contexts
// of different line lengths can coexist.
cudaError_t prepare_line_kernels(int prec, int m)
{
    (void)m;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int cap = (int)kLineSmemMax;
    cudaError_t e;
    if (prec == 0) {
        if ((e = cudaFuncSetAttribute(k_line_scan<double, true, false>, A, cap)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_line_scan<double, true, true>, A, cap)) != cudaSuccess) return e;
        return cudaFuncSetAttribute(k_line_mean<double, true>, A, cap);
    }
    if ((e = cudaFuncSetAttribute(k_line_scan<float, true, false>, A, cap)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_line_scan<float, true, true>, A, cap)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_line_mean<float, true>, A, cap);
}

cudaError_t launch_line_phase(int prec, int m, const void *sub, const void *sup, const void *diag,
                              const void *b, const void *Loth, const void *Moth, void *Lown,
                              void *Mown, void *f, void *y, double *x, int x_transposed,
                              unsigned *flags, cudaStream_t s)
{
    if (m == 0) return cudaSuccess;
    count_launches(s, 1);
    if (prec == 0)
        return launch_T<double, false>(m, sub, sup, diag, b, Loth, Moth, Lown, Mown, f, y, x,
                                       x_transposed, flags, nullptr, nullptr, nullptr, s);
    return launch_T<float, false>(m, sub, sup, diag, b, Loth, Moth, Lown, Mown, f, y, x,
                                  x_transposed, flags, nullptr, nullptr, nullptr, s);
}

cudaError_t launch_line_freeze(int prec, int m, const void *sub, const void *sup,
                               const void *diag, const void *Loth, void *f, void *y, void *aF,
                               void *aB, void *sinv, unsigned *flags, cudaStream_t s)
{
    if (m == 0) return cudaSuccess;
    count_launches(s, 1);
    // the right-hand side does not enter the coefficients: b and m' are read as the diagonal
    if (prec == 0)
        return launch_T<double, true>(m, sub, sup, diag, diag, Loth, Loth, nullptr, nullptr, f, y,
                                      nullptr, 0, flags, aF, aB, sinv, s);
    return launch_T<float, true>(m, sub, sup, diag, diag, Loth, Loth, nullptr, nullptr, f, y,
                                 nullptr, 0, flags, aF, aB, sinv, s);
}

bool line_cols_natural(int prec, int m) { return prec == 1 && m >= 1 && m <= 128 * 16; }

cudaError_t launch_line_mean_cols(int prec, int m, const void *aF, const void *aB,
                                  const void *sinv, const void *b, void *S, void *Mown,
                                  double *x, unsigned *flags, cudaStream_t s)
{
    if (m == 0) return cudaSuccess;
    if (!line_cols_natural(prec, m)) return cudaErrorInvalidValue;
    count_launches(s, 1);
    const int C = m <= 128 * 8 ? 8 : 16;
    const int nch = (m + C - 1) / C;              // chunks per line
    const int qw = 32 / kColLines;                 // chunks of each line per warp
    const int nt = ((nch + qw - 1) / qw) * 32;
    const int grid = (m + kColLines - 1) / kColLines;
    // every thread's chunk whole and inside the matrix (the grid's columns too: C qw is a multiple of kColLines)
    const bool full = m % (C * qw) == 0;
#define GABP_MEAN_COLS(CC, FULL)                                                                           \
    if (x)                                                                                                 \
        launch_pdl(k_line_mean_cols<float, CC, FULL, true>, grid, nt, 0, s, m, (const float *)aF,            \
                   (const float *)aB, (const float *)sinv, (const float *)b, (float *)S, (float *)Mown, x, \
                   flags);                                                                                 \
    else                                                                                                   \
        launch_pdl(k_line_mean_cols<float, CC, FULL, false>, grid, nt, 0, s, m, (const float *)aF,           \
                   (const float *)aB, (const float *)sinv, (const float *)b, (float *)S, (float *)Mown, x, \
                   flags)
    if (C == 8) {
        if (full) GABP_MEAN_COLS(8, true);
        else GABP_MEAN_COLS(8, false);
    } else {
        if (full) GABP_MEAN_COLS(16, true);
        else GABP_MEAN_COLS(16, false);
    }
#undef GABP_MEAN_COLS
    return cudaGetLastError();
}

cudaError_t launch_line_mean(int prec, int m, const void *aF, const void *aB, const void *sinv,
                             const void *b, const void *Moth, void *Mown, void *y, double *x,
                             int x_transposed, int sum_out, unsigned *flags, cudaStream_t s)
{
    if (m == 0) return cudaSuccess;
    count_launches(s, 1);
    if (prec == 0)
        return launch_mean_T<double>(m, aF, aB, sinv, b, Moth, Mown, y, x, x_transposed, sum_out != 0,
                                     flags, s);
    return launch_mean_T<float>(m, aF, aB, sinv, b, Moth, Mown, y, x, x_transposed, sum_out != 0, flags, s);
}

// out_i = S_i - b_i in double (exact for two floats of nearby magnitude)
__global__ void k_line_unfold(int64_t n, const float *__restrict__ S, const float *__restrict__ b,
                              double *__restrict__ out)
{
    pdl_wait();
    pdl_trigger();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)S[i] - (double)b[i];
}

cudaError_t launch_line_unfold(int64_t n, const void *S, const void *b, double *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    count_launches(s, 1);
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    launch_pdl(k_line_unfold, grid, 256, 0, s, n, (const float *)S, (const float *)b, out);
    return cudaGetLastError();
}

cudaError_t launch_line_couplings_from_stencil(int prec, int m, const StencilParams &sp,
                                               const double *a64, const double *diag64,
                                               void *subH, void *supH, void *subV, void *supV,
                                               void *diagV, cudaStream_t s)
{
    const int n = m * m;
    if (n == 0) return cudaSuccess;
    count_launches(s, 1);
    const int grid = std::min((n + 255) / 256, 152 * 16);
    if (prec == 0)
        launch_pdl(k_line_couplings_from_stencil<double>, grid, 256, 0, s, n, m, sp, a64, diag64,
                   (double *)subH, (double *)supH, (double *)subV, (double *)supV, (double *)diagV);
    else
        launch_pdl(k_line_couplings_from_stencil<float>, grid, 256, 0, s, n, m, sp, a64, diag64,
                   (float *)subH, (float *)supH, (float *)subV, (float *)supV, (float *)diagV);
    return cudaGetLastError();
}

cudaError_t launch_line_couplings_transpose(int prec, int m, const void *sub, const void *sup,
                                            void *subT, void *supT, cudaStream_t s)
{
    if (m == 0) return cudaSuccess;
    count_launches(s, 1);
    const int64_t total = (int64_t)m * m;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    if (prec == 0)
        launch_pdl(k_line_couplings_transpose<double>, grid, 256, 0, s, m, total, (const double *)sub,
                   (const double *)sup, (double *)subT, (double *)supT);
    else
        launch_pdl(k_line_couplings_transpose<float>, grid, 256, 0, s, m, total, (const float *)sub,
                   (const float *)sup, (float *)subT, (float *)supT);
    return cudaGetLastError();
}

cudaError_t launch_transpose(int prec, int m, const void *in, void *out, cudaStream_t s)
{
    if (m == 0) return cudaSuccess;
    count_launches(s, 1);
    const dim3 block(32, 8), grid((m + kTile - 1) / kTile, (m + kTile - 1) / kTile);
    if (prec == 0)
        launch_pdl(k_transpose<double>, grid, block, 0, s, m, (const double *)in, (double *)out);
    else
        launch_pdl(k_transpose<float>, grid, block, 0, s, m, (const float *)in, (float *)out);
    return cudaGetLastError();
}

}  // namespace gabp
