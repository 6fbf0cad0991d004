// Coloured schedule (red-black / 4-colour GaBP, Sec. 5.1) on grids whose
// colours are unions of the four parity classes (x mod 2, y mod 2): red-black
// on 5-point grids is classes {0, 3} then {1, 2}; 4-colour on 9-point grids is
// one class per colour.
//
// The messages are stored by their sender, class by class (ParityGrid).  A
// node s of the current colour pulls its incoming messages from the slots of
// its neighbours (other classes), forms its aggregates and belief (the second
// line of eq. nonsymmetric_GaBP_rules) and writes the messages it sends (the
// first line) to its own slots.  Consecutive threads take consecutive nodes of
// one class, so every load and store of a slot array is contiguous, every slot
// is read once and written once per sweep, and no aggregate arrays are kept.
#include <cuda_runtime.h>

#include "gabp_internal.h"
#include "sweep_row.cuh"

namespace gabp {
namespace {

// v[q] by selects (a runtime index into a kernel parameter array would copy
// the array to local memory).
template <typename V>
__device__ __forceinline__ V pick4(const V (&v)[4], int q)
{
    return q == 0 ? v[0] : q == 1 ? v[1] : q == 2 ? v[2] : v[3];
}

// Node of the class position p (base[q] <= p < base[q] + |class q|).
__device__ __forceinline__ void class_node(const ParityGrid &g, long long p, int &q, int &x,
                                           int &y)
{
    q = p >= g.base[3] ? 3 : p >= g.base[2] ? 2 : p >= g.base[1] ? 1 : 0;
    const int i = (int)(p - pick4(g.base, q));
    const int w = pick4(g.w, q);
    const int cy = i / w;
    x = 2 * (i - cy * w) + (q & 1);
    y = 2 * cy + (q >> 1);
}

__device__ __forceinline__ long long class_pos(const ParityGrid &g, int x, int y)
{
    const int q = (x & 1) | ((y & 1) << 1);
    return pick4(g.base, q) + (long long)(y >> 1) * pick4(g.w, q) + (x >> 1);
}

__device__ __forceinline__ bool in_grid(const ParityGrid &g, int x, int y)
{
    return (unsigned)x < (unsigned)g.m && (unsigned)y < (unsigned)g.m;
}

// Class layout <-> slot layout (slot k * n + r holds the entry (r, r + off[k]),
// i.e. the message r + off[k] -> r).  Every destination element is written.
template <typename T>
__global__ void k_parity_convert(ParityGrid g, int to_class, const T *__restrict__ src,
                                 T *__restrict__ dst)
{
    pdl_wait();
    pdl_trigger();
    const long long n = (long long)g.m * g.m;
    const long long total = n * g.K;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t / n);
        const long long p = t - (long long)k * n;
        int x, y;
        if (to_class) {
            int q;
            class_node(g, p, q, x, y);  // sender s; recipient r = s + off[k]
            const int rx = x + g.dx[k], ry = y + g.dy[k];
            dst[t] = in_grid(g, rx, ry) ? src[(long long)g.krev[k] * n + (long long)ry * g.m + rx]
                                        : T(0);
        } else {
            x = (int)(p % g.m);  // recipient r; sender s = r + off[k]
            y = (int)(p / g.m);
            const int sx = x + g.dx[k], sy = y + g.dy[k];
            dst[t] = in_grid(g, sx, sy) ? src[(long long)g.krev[k] * n + class_pos(g, sx, sy)]
                                        : T(0);
        }
    }
}

// zl, zm: classes whose precision / mean messages read as zero (bit q for
// class q): after a reset of the messages the first sweep reads the classes
// that have not sent yet as zero instead of clearing the arrays first.
// kMean (frozen precision messages, Sec. 4.2): a holds the gains g = a / d of
// the node's outgoing slots, diag the frozen aggregate P (natural order, read
// only for the belief), and only the mean messages move,
// M' = g (B - M[rev]); c, Lo and zl are unused.
template <typename T, int K, bool kMean>
__global__ void __launch_bounds__(256) k_sweep_parity(ParityGrid g, PhaseClasses ph,
                                                      const T *__restrict__ a,
                                                      const T *__restrict__ c,
                                                      const T *__restrict__ diag,
                                                      const T *__restrict__ b, T *Lo, T *Mo,
                                                      double *__restrict__ x,
                                                      unsigned *__restrict__ flags, unsigned zl,
                                                      unsigned zm)
{
    pdl_wait();
    pdl_trigger();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long end = ph.nq >= 4 ? ph.start[4] : ph.nq == 3 ? ph.start[3] : ph.nq == 2 ? ph.start[2] : ph.start[1];
    if (t >= end) return;
    int q = ph.q[0];
    long long t0 = 0;
#pragma unroll
    for (int j = 1; j < 4; ++j)
        if (j < ph.nq && t >= ph.start[j]) {
            q = ph.q[j];
            t0 = ph.start[j];
        }
    const int i = (int)(t - t0);
    const int w = pick4(g.w, q);
    const int cy = i / w;
    const int sx = 2 * (i - cy * w) + (q & 1), sy = 2 * cy + (q >> 1);
    const long long n = (long long)g.m * g.m;
    const long long pos = pick4(g.base, q) + i;
    const long long s = (long long)sy * g.m + sx;
    // every load of the node first: incoming messages (the neighbour's slot
    // krev[k] is its message to s), the coefficients of the outgoing ones
    T lin[K], min_[K], av[K], cv[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int nx = sx + g.dx[k], ny = sy + g.dy[k];
        const bool in = in_grid(g, nx, ny);
        const unsigned qn = (unsigned)((nx & 1) | ((ny & 1) << 1));
        long long src = in ? (long long)g.krev[k] * n + class_pos(g, nx, ny)
                           : (long long)k * n + pos;  // any valid address
        if (kIndexChecks && (src < 0 || src >= (long long)K * n)) {
            atomicOr(flags, FLAG_INDEX);
            src = 0;
        }
        if (!kMean) lin[k] = in && !((zl >> qn) & 1u) ? Lo[src] : T(0);
        min_[k] = in && !((zm >> qn) & 1u) ? Mo[src] : T(0);
        av[k] = a[(long long)k * n + pos];
        if (!kMean) cv[k] = c[(long long)k * n + pos];
    }
    T B = b[s];
#pragma unroll
    for (int k = 0; k < K; ++k) B += min_[k];
    if (kMean) {
        if (x) x[s] = (double)(B / diag[s]);
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (nonzero(av[k])) Mo[(long long)k * n + pos] = av[k] * (B - min_[k]);
        return;
    }
    T P = diag[s];
#pragma unroll
    for (int k = 0; k < K; ++k) P += lin[k];
    if (x) x[s] = (double)(B / P);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (!nonzero(av[k])) continue;  // no recipient: the slot stays zero
        const T d = P - lin[k];
        bad |= bad_den(d);
        const T qd = fast_rcp(d);
        Lo[(long long)k * n + pos] = cv[k] * qd;
        Mo[(long long)k * n + pos] = av[k] * (B - min_[k]) * qd;
    }
    if (bad) atomicOr(flags, FLAG_BREAKDOWN);
}

// Freezing of the precision messages on the class layout (every node of every
// class): P_s = diag_s + sum of its incoming L into Pf (natural order), and for
// each outgoing slot the gain g = a / (P_s - L[rev]) (zero where a = 0).
template <typename T, int K>
__global__ void __launch_bounds__(256) k_freeze_parity(ParityGrid g, const T *__restrict__ a,
                                                       const T *__restrict__ diag,
                                                       const T *__restrict__ Lo,
                                                       T *__restrict__ gains, T *__restrict__ Pf,
                                                       unsigned *__restrict__ flags)
{
    pdl_wait();
    pdl_trigger();
    const long long n = (long long)g.m * g.m;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int q, sx, sy;
    class_node(g, p, q, sx, sy);
    T lin[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int nx = sx + g.dx[k], ny = sy + g.dy[k];
        const bool in = in_grid(g, nx, ny);
        long long src = in ? (long long)g.krev[k] * n + class_pos(g, nx, ny) : 0;
        if (kIndexChecks && (src < 0 || src >= (long long)K * n)) {
            atomicOr(flags, FLAG_INDEX);
            src = 0;
        }
        lin[k] = in ? Lo[src] : T(0);
    }
    const long long s = (long long)sy * g.m + sx;
    T P = diag[s];
#pragma unroll
    for (int k = 0; k < K; ++k) P += lin[k];
    Pf[s] = P;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const T ak = a[(long long)k * n + p];
        T ge = T(0);
        if (nonzero(ak)) {
            const T d = P - lin[k];
            bad |= bad_den(d);
            ge = ak * fast_rcp(d);
        }
        gains[(long long)k * n + p] = ge;
    }
    if (bad) atomicOr(flags, FLAG_BREAKDOWN);
}

// Compile-time neighbourhood of the standard diagonal orders: offsets
// ascending, 5-point (K = 4) or 9-point (K = 8); krev[k] = K - 1 - k.
template <int K>
__device__ constexpr int std_dx(int k)
{
    return K == 4 ? (k == 1 ? -1 : k == 2 ? 1 : 0) : ((k == 0 || k == 3 || k == 5) ? -1 : (k == 1 || k == 6) ? 0 : 1);
}
template <int K>
__device__ constexpr int std_dy(int k)
{
    return K == 4 ? (k == 0 ? -1 : k == 3 ? 1 : 0) : (k < 3 ? -1 : k < 5 ? 0 : 1);
}
__device__ constexpr int floor_half(int v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); }

// One node (cx, cy) of the class (PX, PY): the neighbour in direction k lies
// in the class QT at class row cy + DY2 and column cx + DX2, all known at
// compile time; only the grid edge is tested at run time.  kMean as in
// k_sweep_parity.  parity_load issues every load of the node (the belief's P
// up front as well), parity_store does its arithmetic and writes.
template <typename T, int K>
struct ParityNode {
    T lin[K], min_[K], av[K], cv[K];
    T B, P;
    unsigned pos, s;
    bool valid;
};

template <typename T, int K, int PX, int PY, bool kMean>
__device__ __forceinline__ void parity_load(const ParityGrid &g, unsigned cx, unsigned cy,
                                            const T *__restrict__ a, const T *__restrict__ c,
                                            const T *__restrict__ diag, const T *__restrict__ b,
                                            const T *Lo, const T *Mo, bool want_p, unsigned zl, unsigned zm,
                                            bool &bad_index, ParityNode<T, K> &N)
{
    constexpr int Q = PX | (PY << 1);
    const unsigned m = (unsigned)g.m, n = m * m;
    N.valid = cx < (unsigned)g.w[Q] && cy < (unsigned)g.h[Q];
    if (!N.valid) return;
    const unsigned pos = (unsigned)g.base[Q] + cy * (unsigned)g.w[Q] + cx;
    if (kIndexChecks && pos >= n) {  // nothing of this node is touched
        bad_index = true;
        N.valid = false;
        return;
    }
    const unsigned sx = 2u * cx + PX, sy = 2u * cy + PY;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int dx = std_dx<K>(k), dy = std_dy<K>(k);
        const int qt = ((PX + dx) & 1) | (((PY + dy) & 1) << 1);
        const int dx2 = floor_half(PX + dx), dy2 = floor_half(PY + dy);
        const bool in = (sx + dx < m) && (sy + dy < m);  // unsigned: -1 wraps high
        unsigned src =
            in ? (unsigned)(K - 1 - k) * n + (unsigned)g.base[qt] +
                     (cy + dy2) * (unsigned)g.w[qt] + (cx + dx2)
               : (unsigned)k * n + pos;  // any valid address
        if (kIndexChecks && src >= (unsigned)K * n) {
            bad_index = true;
            src = 0;
        }
        if (!kMean) N.lin[k] = in && !((zl >> qt) & 1u) ? Lo[src] : T(0);
        N.min_[k] = in && !((zm >> qt) & 1u) ? Mo[src] : T(0);
        N.av[k] = a[(unsigned)k * n + pos];
        if (!kMean) N.cv[k] = c[(unsigned)k * n + pos];
    }
    N.pos = pos;
    N.s = sy * m + sx;
    N.B = b[N.s];
    N.P = (!kMean || want_p) ? diag[N.s] : T(1);
}

template <typename T, int K, bool kMean>
__device__ __forceinline__ void parity_store(const ParityGrid &g, ParityNode<T, K> &N, T *Lo, T *Mo,
                                             double *__restrict__ x, bool &bad)
{
    if (!N.valid) return;
    const unsigned n = (unsigned)g.m * (unsigned)g.m;
    T B = N.B;
#pragma unroll
    for (int k = 0; k < K; ++k) B += N.min_[k];
    if (kMean) {
        if (x) x[N.s] = (double)(B / N.P);
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (nonzero(N.av[k])) Mo[(unsigned)k * n + N.pos] = N.av[k] * (B - N.min_[k]);
        return;
    }
    T P = N.P;
#pragma unroll
    for (int k = 0; k < K; ++k) P += N.lin[k];
    if (x) x[N.s] = (double)(B / P);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (!nonzero(N.av[k])) continue;  // no recipient: the slot stays zero
        const T d = P - N.lin[k];
        bad |= bad_den(d);
        const T qd = fast_rcp(d);
        Lo[(unsigned)k * n + N.pos] = N.cv[k] * qd;
        Mo[(unsigned)k * n + N.pos] = N.av[k] * (B - N.min_[k]) * qd;
    }
}

template <typename T, int K, int PX, int PY, bool kMean>
__device__ __forceinline__ void parity_node(const ParityGrid &g, unsigned cx, unsigned cy,
                                            const T *__restrict__ a, const T *__restrict__ c,
                                            const T *__restrict__ diag, const T *__restrict__ b, T *Lo,
                                            T *Mo, double *__restrict__ x, bool &bad, unsigned zl,
                                            unsigned zm, bool &bad_index)
{
    ParityNode<T, K> N;
    parity_load<T, K, PX, PY, kMean>(g, cx, cy, a, c, diag, b, Lo, Mo, x != nullptr, zl, zm, bad_index, N);
    parity_store<T, K, kMean>(g, N, Lo, Mo, x, bad);
}

// Standard orders: block (x, y, z) = (class columns, class row, class of the
// phase), so a thread finds its node without division.
template <typename T, int K, bool kMean>
__global__ void __launch_bounds__(256) k_sweep_parity_std(ParityGrid g, PhaseClasses ph,
                                                          const T *__restrict__ a,
                                                          const T *__restrict__ c,
                                                          const T *__restrict__ diag,
                                                          const T *__restrict__ b, T *Lo, T *Mo,
                                                          double *__restrict__ x,
                                                          unsigned *__restrict__ flags,
                                                          unsigned zl, unsigned zm)
{
    pdl_wait();
    pdl_trigger();
    const int z = blockIdx.z;
    const int q = z == 0 ? ph.q[0] : z == 1 ? ph.q[1] : z == 2 ? ph.q[2] : ph.q[3];
    const unsigned cx = blockIdx.x * blockDim.x + threadIdx.x, cy = blockIdx.y;
    bool bad = false, bad_index = false;
    switch (q) {
        case 0: parity_node<T, K, 0, 0, kMean>(g, cx, cy, a, c, diag, b, Lo, Mo, x, bad, zl, zm, bad_index); break;
        case 1: parity_node<T, K, 1, 0, kMean>(g, cx, cy, a, c, diag, b, Lo, Mo, x, bad, zl, zm, bad_index); break;
        case 2: parity_node<T, K, 0, 1, kMean>(g, cx, cy, a, c, diag, b, Lo, Mo, x, bad, zl, zm, bad_index); break;
        default: parity_node<T, K, 1, 1, kMean>(g, cx, cy, a, c, diag, b, Lo, Mo, x, bad, zl, zm, bad_index); break;
    }
    if (bad) atomicOr(flags, FLAG_BREAKDOWN);
    if (kIndexChecks && bad_index) atomicOr(flags, FLAG_INDEX);
}

}  // namespace

cudaError_t launch_parity_convert(const ParityGrid &g, int prec, int to_class, const void *src,
                                  void *dst, cudaStream_t s)
{
    const long long total = (long long)g.m * g.m * g.K;
    if (total == 0) return cudaSuccess;
    count_launches(s, 1);
    const long long want = (total + 255) / 256;
    const int grid = (int)(want < 152 * 32 ? want : 152 * 32);
    if (prec == 0)
        launch_pdl(k_parity_convert<double>, grid, 256, 0, s, g, to_class, (const double *)src, (double *)dst);
    else
        launch_pdl(k_parity_convert<float>, grid, 256, 0, s, g, to_class, (const float *)src, (float *)dst);
    return cudaGetLastError();
}

namespace {

template <typename T, bool kMean>
cudaError_t sweep_parity_T(const ParityGrid &g, const PhaseClasses &ph, const T *a, const T *c,
                           const T *diag, const T *b, T *Lo, T *Mo, double *x, unsigned *flags,
                           unsigned zl, unsigned zm, cudaStream_t s)
{
    const long long nodes = ph.start[ph.nq];
    if (g.std_order) {
        int wmax = 0, hmax = 0;
        for (int j = 0; j < ph.nq; ++j) {
            wmax = wmax > g.w[ph.q[j]] ? wmax : g.w[ph.q[j]];
            hmax = hmax > g.h[ph.q[j]] ? hmax : g.h[ph.q[j]];
        }
        const int block = wmax >= 256 ? 256 : ((wmax + 31) / 32) * 32;
        const dim3 grid3((unsigned)((wmax + block - 1) / block), (unsigned)hmax, (unsigned)ph.nq);
        if (hmax > 65535) return cudaErrorInvalidValue;
        if (g.K == 4)
            return launch_pdl(k_sweep_parity_std<T, 4, kMean>, grid3, block, 0, s, g, ph, a, c, diag, b, Lo, Mo,
                              x, flags, zl, zm);
        return launch_pdl(k_sweep_parity_std<T, 8, kMean>, grid3, block, 0, s, g, ph, a, c, diag, b, Lo, Mo, x,
                          flags, zl, zm);
    }
    const int grid = (int)((nodes + 255) / 256);
    switch (g.K) {
        case 2: return launch_pdl(k_sweep_parity<T, 2, kMean>, grid, 256, 0, s, g, ph, a, c, diag, b, Lo, Mo, x, flags, zl, zm);
        case 4: return launch_pdl(k_sweep_parity<T, 4, kMean>, grid, 256, 0, s, g, ph, a, c, diag, b, Lo, Mo, x, flags, zl, zm);
        case 6: return launch_pdl(k_sweep_parity<T, 6, kMean>, grid, 256, 0, s, g, ph, a, c, diag, b, Lo, Mo, x, flags, zl, zm);
        case 8: return launch_pdl(k_sweep_parity<T, 8, kMean>, grid, 256, 0, s, g, ph, a, c, diag, b, Lo, Mo, x, flags, zl, zm);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t freeze_parity_T(const ParityGrid &g, const T *a, const T *diag, const T *Lo, T *gains, T *Pf,
                            unsigned *flags, cudaStream_t s)
{
    const long long n = (long long)g.m * g.m;
    const int grid = (int)((n + 255) / 256);
    switch (g.K) {
        case 2: return launch_pdl(k_freeze_parity<T, 2>, grid, 256, 0, s, g, a, diag, Lo, gains, Pf, flags);
        case 4: return launch_pdl(k_freeze_parity<T, 4>, grid, 256, 0, s, g, a, diag, Lo, gains, Pf, flags);
        case 6: return launch_pdl(k_freeze_parity<T, 6>, grid, 256, 0, s, g, a, diag, Lo, gains, Pf, flags);
        case 8: return launch_pdl(k_freeze_parity<T, 8>, grid, 256, 0, s, g, a, diag, Lo, gains, Pf, flags);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_sweep_parity(const ParityGrid &g, const PhaseClasses &ph, int prec,
                                const void *a, const void *c, const void *diag, const void *b,
                                void *Lo, void *Mo, double *x, unsigned *flags, unsigned zl,
                                unsigned zm, int mean, cudaStream_t s)
{
    if (ph.start[ph.nq] == 0) return cudaSuccess;
    count_launches(s, 1);
    if (prec == 0) {
        if (mean)
            return sweep_parity_T<double, true>(g, ph, (const double *)a, (const double *)c, (const double *)diag,
                                                (const double *)b, (double *)Lo, (double *)Mo, x, flags, zl, zm, s);
        return sweep_parity_T<double, false>(g, ph, (const double *)a, (const double *)c, (const double *)diag,
                                             (const double *)b, (double *)Lo, (double *)Mo, x, flags, zl, zm, s);
    }
    if (mean)
        return sweep_parity_T<float, true>(g, ph, (const float *)a, (const float *)c, (const float *)diag,
                                           (const float *)b, (float *)Lo, (float *)Mo, x, flags, zl, zm, s);
    return sweep_parity_T<float, false>(g, ph, (const float *)a, (const float *)c, (const float *)diag,
                                        (const float *)b, (float *)Lo, (float *)Mo, x, flags, zl, zm, s);
}

cudaError_t launch_freeze_parity(const ParityGrid &g, int prec, const void *a, const void *diag,
                                 const void *Lo, void *gains, void *Pf, unsigned *flags, cudaStream_t s)
{
    if (g.m == 0) return cudaSuccess;
    count_launches(s, 1);
    if (prec == 0)
        return freeze_parity_T<double>(g, (const double *)a, (const double *)diag, (const double *)Lo,
                                       (double *)gains, (double *)Pf, flags, s);
    return freeze_parity_T<float>(g, (const float *)a, (const float *)diag, (const float *)Lo, (float *)gains,
                                  (float *)Pf, flags, s);
}

}  // namespace gabp
