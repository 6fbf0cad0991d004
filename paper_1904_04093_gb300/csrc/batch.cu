// Batched GaBP: many independent systems solved in one persistent launch.
//
// Each thread-block cluster (1 to 16 CTAs, one SM each) takes the next system
// from a global queue (largest first), runs every flood sweep of that system
// with all its threads (one thread per row, strided over the cluster),
// checks its own double residual every `check_every` sweeps and stops it on
// convergence, breakdown, divergence or the sweep cap; then it takes the next
// system.  Sweeps are separated by the hardware cluster barrier and the
// reductions combine the CTAs' partial results through distributed shared
// memory.  Clusters never wait on one another: the only cross-cluster
// operation is one atomicAdd on the queue, so every cluster finishes in
// bounded time.  The per-row update is the
// single-system kernel's (sweep_row_stencil), so a system solved in a batch
// follows the same iterates as gabp_solve with the same check interval.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <string>
#include <vector>

#include "gabp_internal.h"
#include "sweep_row.cuh"

namespace gabp {

template <typename T>
struct BatchSys {
    int n;
    int pad_;
    int off[KMAX];
    int krev[KMAX];
    const T *a, *c, *diag;
    const double *a64, *diag64;
    T *L0, *L1, *M0, *M1, *P0, *P1, *B0, *B1, *bT;
    double *e, *r;  // refinement: correction (beliefs of the inner solve), residual
    T *g;           // frozen gains a_e / d_e (precision messages frozen once converged)
};

struct BatchResult {
    int iters;
    int status;
    double rr;
};

namespace {

namespace cg = cooperative_groups;

// Shared per-CTA state of the batched kernel.
struct BatchShared {
    int idx;             // system index taken from a queue
    unsigned flags;      // 1 breakdown, 2 non-finite residual, 4 failed index check
    double red[33];      // reduction scratch; red[32] = this CTA's partial result
    int off[8], krev[8]; // diagonals of the current system
};

__device__ __forceinline__ double cta_max_partial(double v, BatchShared &sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sh.red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? sh.red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sh.red[32] = v;
    }
    return v;
}

// A whole thread-block cluster works on one system: rows strided over all
// its threads, sweeps separated by the hardware cluster barrier, reductions
// combined through distributed shared memory, error flags in rank 0's copy.
struct ClusterTeam {
    cg::cluster_group cl;
    BatchShared *sh, *root;
    int t0, nt;
    __device__ ClusterTeam(BatchShared *s) : cl(cg::this_cluster()), sh(s)
    {
        root = cl.map_shared_rank(s, 0);
        t0 = (int)cl.block_rank() * blockDim.x + threadIdx.x;
        nt = (int)cl.num_blocks() * blockDim.x;
    }
    __device__ void sync() { cl.sync(); }
    __device__ unsigned *flags() { return &root->flags; }
    // Team maximum of v.  With fl != nullptr also the team's error flags:
    // read after the first cluster barrier (every flag set before the call is
    // visible) and before the second (no thread can set one in between), so
    // every thread of the team gets the same value.
    __device__ double max(double v, unsigned *fl = nullptr)
    {
        cta_max_partial(v, *sh);
        cl.sync();
        double m = 0.0;
        const unsigned nb = cl.num_blocks();
        for (unsigned r = 0; r < nb; ++r) m = fmax(m, cl.map_shared_rank(sh, r)->red[32]);
        if (fl) *fl = *(volatile unsigned *)&root->flags;
        cl.sync();  // every CTA has read the partials and the flags before they change
        return m;
    }
};

// One CTA works on one system on its own.
struct CtaTeam {
    BatchShared *sh;
    int t0, nt;
    __device__ CtaTeam(BatchShared *s) : sh(s), t0(threadIdx.x), nt(blockDim.x) {}
    __device__ void sync() { __syncthreads(); }
    __device__ unsigned *flags() { return &sh->flags; }
    // As ClusterTeam::max: the flags are read between two block barriers.
    __device__ double max(double v, unsigned *fl = nullptr)
    {
        cta_max_partial(v, *sh);
        __syncthreads();
        const double m = sh->red[32];
        if (fl) *fl = *(volatile unsigned *)&sh->flags;
        __syncthreads();
        return m;
    }
};

// Residual max_r |rhs_r - (A y)_r| in double, rhs_r = src[r] * scale, over this
// thread's rows; writes rhs - A y into `out` when not null.  src and y are
// read coherently (written earlier in this launch).
// R rows of a thread are in flight at once: rows r0 + u nt, u < R, all loads
// issued before the arithmetic (the neighbour loads at a clamped, always valid
// index; a padded slot has a = 0 and drops its value).
template <typename T, int K, int R>
__device__ double batch_residual(const BatchSys<T> &S, int n, const int *off, const double *src,
                                 double scale, const double *y, double *out, int t0, int nt,
                                 bool &nan)
{
    constexpr int KK = K > 0 ? K : 1;
    double rm = 0.0;
    for (int r0 = t0; r0 < n; r0 += R * nt) {
        double sv[R], dv[R], yv[R], av[R][KK], ys[R][KK];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int r = min(r0 + u * nt, n - 1);
            sv[u] = __ldcg(src + r);
            dv[u] = S.diag64[r];
            yv[u] = __ldcg(y + r);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                av[u][k] = S.a64[(size_t)k * n + r];
                int q = r + off[k];
                q = q < 0 ? 0 : (q >= n ? n - 1 : q);
                ys[u][k] = __ldcg(y + q);
            }
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int r = r0 + u * nt;
            if (r >= n) continue;
            double acc = sv[u] * scale - dv[u] * yv[u];
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (av[u][k] != 0.0) acc += av[u][k] * ys[u][k];
            if (out) out[r] = acc;
            const double v = fabs(acc);
            if (v != v) nan = true;
            else rm = fmax(rm, v);
        }
    }
    return rm;
}

// The loads of one row of the mean-message update with frozen precision
// messages, and the update itself: the arithmetic of sweep_row_mean_stencil,
// split so that several rows' loads can be in flight before any update.
template <typename T, int K>
struct MeanRow {
    T ge[K > 0 ? K : 1], bs[K > 0 ? K : 1], mr[K > 0 ? K : 1];
    T bb, bx, px;
    bool oob;  // bounds-checked build: a non-zero gain whose neighbour is outside [0, n)
};

template <typename T, int K>
__device__ __forceinline__ void mean_row_load(int r, int n, const int *off, const int *krev,
                                              const T *g, const T *b, const T *P, const T *Min,
                                              const T *Bin, bool belief, MeanRow<T, K> &M)
{
    const size_t nn = (size_t)n;
    M.oob = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        M.ge[k] = __ldcg(g + (size_t)k * nn + r);
        int s = r + off[k];
        if (kIndexChecks && nonzero(M.ge[k]) && (s < 0 || s >= n)) M.oob = true;
        s = s < 0 ? 0 : (s >= n ? n - 1 : s);
        M.bs[k] = __ldcg(Bin + s);
        M.mr[k] = __ldcg(Min + (size_t)krev[k] * nn + s);
    }
    M.bb = __ldcg(b + r);
    if (belief) {
        M.bx = __ldcg(Bin + r);
        M.px = __ldcg(P + r);
    }
}

template <typename T, int K>
__device__ __forceinline__ unsigned mean_row_update(int r, int n, const MeanRow<T, K> &M, T *Mout,
                                                    T *Bout, double *x)
{
    const size_t nn = (size_t)n;
    T bn = M.bb;
    if (x) x[r] = (double)(M.bx / M.px);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const T mu = nonzero(M.ge[k]) ? M.ge[k] * (M.bs[k] - M.mr[k]) : T(0);
        Mout[(size_t)k * nn + r] = mu;
        bn += mu;
    }
    Bout[r] = bn;
    return kIndexChecks && M.oob ? 4u : 0u;
}

// `kk` flood sweeps of system S from state `cur` (beliefs of the last go to y);
// with frozen precision messages only the mean messages move.
// With frozen precision messages (where a batched solve spends most of its
// sweeps) R rows of a thread are in flight at once (rows r0 + u nt, u < R):
// every load of the R rows, then their updates, with the per-row arithmetic
// of the single-system mean sweep.  Full sweeps take one row at a time (the
// row state of two would not fit the registers).
template <typename T, int K, int R, typename Team>
__device__ void batch_sweeps(const BatchSys<T> &S, int n, const int *off, const int *krev, int kk,
                             int &cur, double *y, Team &tm, bool frozen)
{
    if (frozen) {
        for (int j = 0; j < kk; ++j) {
            T *Min = cur ? S.M1 : S.M0, *Mout = cur ? S.M0 : S.M1;
            T *Bin = cur ? S.B1 : S.B0, *Bout = cur ? S.B0 : S.B1;
            T *Pc = cur ? S.P1 : S.P0;
            double *yo = j == kk - 1 ? y : nullptr;
            unsigned bad = 0u;
            for (int r0 = tm.t0; r0 < n; r0 += R * tm.nt) {
                MeanRow<T, K> rows[R];
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    const int r = r0 + u * tm.nt;
                    if (r < n) mean_row_load<T, K>(r, n, off, krev, S.g, S.bT, Pc, Min, Bin, yo != nullptr, rows[u]);
                }
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    const int r = r0 + u * tm.nt;
                    if (r < n) bad |= mean_row_update<T, K>(r, n, rows[u], Mout, Bout, yo);
                }
            }
            if (kIndexChecks && bad) atomicOr(tm.flags(), bad);
            tm.sync();
            cur ^= 1;
        }
        return;
    }
    for (int j = 0; j < kk; ++j) {
        T *Lin = cur ? S.L1 : S.L0, *Lout = cur ? S.L0 : S.L1;
        T *Min = cur ? S.M1 : S.M0, *Mout = cur ? S.M0 : S.M1;
        T *Pin = cur ? S.P1 : S.P0, *Pout = cur ? S.P0 : S.P1;
        T *Bin = cur ? S.B1 : S.B0, *Bout = cur ? S.B0 : S.B1;
        double *yo = j == kk - 1 ? y : nullptr;
        unsigned bad = 0u;  // FLAG_BREAKDOWN (1), and FLAG_INDEX (4) in the bounds-checked build
        for (int r = tm.t0; r < n; r += tm.nt)
            bad |= sweep_row_stencil<T, K, true>(r, n, off, krev, S.a, S.c, S.diag, S.bT, Lin, Min,
                                                 Pin, Bin, Lout, Mout, Pout, Bout, yo);
        if (bad) atomicOr(tm.flags(), bad);
        tm.sync();
        cur ^= 1;
    }
}

// Freezes the precision messages of S once the last sweep changed none of them
// by more than `rel` times the largest and no error flag is set (returns the
// new frozen state): gains g = a / (P_s - L[rev]) from the current state, both
// L and both P buffers set to the current ones.
template <typename T, int K, typename Team>
__device__ bool batch_maybe_freeze(const BatchSys<T> &S, int n, const int *off, const int *krev,
                                   int cur, double rel, Team &tm)
{
    const T *Lc = cur ? S.L1 : S.L0, *Lp = cur ? S.L0 : S.L1;
    double dm = 0.0, lm = 0.0;
    for (int r = tm.t0; r < n; r += tm.nt)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const double l1 = (double)__ldcg(Lc + (size_t)k * n + r);
            dm = fmax(dm, fabs(l1 - (double)__ldcg(Lp + (size_t)k * n + r)));
            lm = fmax(lm, fabs(l1));
        }
    unsigned fl = 0u;
    dm = tm.max(dm, &fl);
    lm = tm.max(lm);
    if (fl || !(dm <= rel * lm)) return false;
    T *Lo = cur ? S.L0 : S.L1, *Pc = cur ? S.P1 : S.P0, *Po = cur ? S.P0 : S.P1;
    for (int r = tm.t0; r < n; r += tm.nt) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const size_t e = (size_t)k * n + r;
            const T ae = S.a[e];
            T ge = T(0);
            if (nonzero(ae)) {
                const int s = r + off[k];
                ge = ae * fast_rcp(__ldcg(Pc + s) - __ldcg(Lc + (size_t)krev[k] * n + s));
            }
            S.g[e] = ge;
            Lo[e] = __ldcg(Lc + e);
        }
        Po[r] = __ldcg(Pc + r);
    }
    tm.sync();
    return true;
}

// Solves system `id` with team `tm` (every thread of the team calls this with
// the same arguments; all control flow below is uniform across the team).
//
// Invariant that keeps it uniform: no branch reads the shared error word
// `flags` directly.  Threads set bits in it at any time (a breakdown in a
// sweep, a non-finite residual), and a fast thread may already be sweeping
// the next chunk while a slow one finishes the previous check; every decision
// is taken on the snapshot `fl` that tm.max() returns, read between two team
// barriers and therefore the same in every thread.
//
// refine = 0: plain GaBP on A x = b (Algorithm 1).
// refine = 1: GaBP in the message precision inside double iterative
// refinement: x accumulates in double, every refinement step solves
// A e = r / ||r||_inf from zero mean messages (precision messages kept warm:
// they do not depend on the right-hand side) for at most inner_max sweeps or
// until its own relative residual <= inner_tol, then x += ||r|| e and
// r = b - A x in double; max_iter caps the total sweeps.
template <typename T, int K, int R, typename Team>
__device__ void solve_system(const BatchSys<T> &S, int id, const double *b, double *x, Team &tm,
                             double tol, int max_iter, int check_every, int refine,
                             double inner_tol, int inner_max, int freeze, BatchResult *res,
                             bool leader)
{
    bool frozen = false;
    const double frz_rel = sizeof(T) == 8 ? 1e-14 : 1e-6;
    const int n = S.n, t0 = tm.t0, nt = tm.nt;
    const int *off = tm.sh->off, *krev = tm.sh->krev;
    unsigned *flags = tm.flags();
    unsigned fl = 0u;  // team-uniform snapshot of *flags (see above)
    // zero messages: P = diag, B = b (plain) or the first refinement rhs b / ||b||
    double bm = 0.0;
    for (int r = t0; r < n; r += nt) bm = fmax(bm, fabs(b[r]));
    const double bnorm = tm.max(bm);
    const double inv0 = bnorm > 0.0 ? 1.0 / bnorm : 0.0;
    for (int r = t0; r < n; r += nt) {
        const double bv = b[r];
        const T bt = (T)(refine ? bv * inv0 : bv);
        S.bT[r] = bt;
        S.P0[r] = S.diag[r];
        S.B0[r] = bt;
        if (refine) {
            x[r] = 0.0;
            S.r[r] = bv;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            S.L0[(size_t)k * n + r] = T(0);
            S.M0[(size_t)k * n + r] = T(0);
        }
    }
    if (bnorm == 0.0)
        for (int r = t0; r < n; r += nt) x[r] = 0.0;
    tm.sync();
    int it = 0, cur = 0, status = bnorm == 0.0 ? GABP_OK : GABP_E_NOT_CONVERGED;
    double rr = 0.0;
    if (!refine) {
        while (status == GABP_E_NOT_CONVERGED && it < max_iter) {
            const int kk = min(check_every, max_iter - it);
            batch_sweeps<T, K, R>(S, n, off, krev, kk, cur, x, tm, frozen);
            it += kk;
            if (freeze && !frozen) frozen = batch_maybe_freeze<T, K>(S, n, off, krev, cur, frz_rel, tm);
            bool nan = false;
            double rm = batch_residual<T, K, 1>(S, n, off, b, 1.0, x, nullptr, t0, nt, nan);
            if (nan) atomicOr(flags, 2u);
            rm = tm.max(rm, &fl);
            rr = rm / bnorm;
            if (fl & 4u) status = GABP_E_CUDA;  // bounds-checked build: an index check failed
            else if (fl & 1u) status = GABP_E_BREAKDOWN;
            else if ((fl & 2u) || !(rr <= 1e8)) status = GABP_E_DIVERGED;
            else if (rr <= tol) status = GABP_OK;
        }
    } else {
        double scale = bnorm;  // ||r||_inf of the current refinement step
        bool first = true;
        while (status == GABP_E_NOT_CONVERGED && it < max_iter) {
            if (!first) {
                // new inner problem A e = r / ||r||: zero mean messages, warm precision messages
                const double inv = 1.0 / scale;
                T *Lc = cur ? S.L1 : S.L0, *Mc = cur ? S.M1 : S.M0;
                T *Pc = cur ? S.P1 : S.P0, *Bc = cur ? S.B1 : S.B0;
                for (int r = t0; r < n; r += nt) {
                    const T bt = (T)(__ldcg(S.r + r) * inv);
                    S.bT[r] = bt;
                    T p = S.diag[r];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        p += __ldcg(Lc + (size_t)k * n + r);
                        Mc[(size_t)k * n + r] = T(0);
                    }
                    Pc[r] = p;
                    Bc[r] = bt;
                }
                tm.sync();
            }
            first = false;
            int inner = 0;
            while (inner < inner_max && it < max_iter) {
                const int kk = min(min(check_every, inner_max - inner), max_iter - it);
                batch_sweeps<T, K, R>(S, n, off, krev, kk, cur, S.e, tm, frozen);
                inner += kk;
                it += kk;
                if (freeze && !frozen)
                    frozen = batch_maybe_freeze<T, K>(S, n, off, krev, cur, frz_rel, tm);
                bool nan = false;
                double rin = batch_residual<T, K, 1>(S, n, off, S.r, 1.0 / scale, S.e, nullptr, t0,
                                                  nt, nan);
                if (nan) atomicOr(flags, 2u);
                rin = tm.max(rin, &fl);
                if (fl) break;
                if (rin <= inner_tol) break;
            }
            if (fl & 5u) {
                status = (fl & 4u) ? GABP_E_CUDA : GABP_E_BREAKDOWN;
                break;
            }
            // x += ||r|| e ;  r = b - A x
            for (int r = t0; r < n; r += nt) x[r] = __ldcg(x + r) + scale * __ldcg(S.e + r);
            tm.sync();
            bool nan = false;
            double rm = batch_residual<T, K, 1>(S, n, off, b, 1.0, x, S.r, t0, nt, nan);
            if (nan) atomicOr(flags, 2u);
            rm = tm.max(rm, &fl);
            rr = rm / bnorm;
            scale = rm;
            if ((fl & 2u) || !(rr <= 1e8)) status = GABP_E_DIVERGED;
            else if (rr <= tol) status = GABP_OK;
        }
    }
    if (leader) {
        res[id].iters = it;
        res[id].status = status;
        res[id].rr = rr;
    }
    tm.sync();
}

// Persistent kernel.  Phase 1: each cluster takes the next of the first
// `nbig` systems (largest first) from queue[0] and solves it with all its
// CTAs.  Phase 2: once those are taken, every CTA on its own takes the next
// remaining system from queue[1].  Message state written earlier in this
// launch is read back with coherent loads (sweep_row_stencil<..., true>,
// __ldcg), never through the non-coherent read-only path; the barriers order
// it across the team.
template <typename T, int K, int R>
__global__ void __launch_bounds__(512) k_batch_solve(
    const BatchSys<T> *__restrict__ sys, const int *__restrict__ order, int nsys, int nbig,
    const double *const *__restrict__ bptr, double *const *__restrict__ xptr, int *queue,
    double tol, int max_iter, int check_every, int refine, double inner_tol, int inner_max,
    int freeze, BatchResult *__restrict__ res)
{
    __shared__ BatchShared sh;
    const int tid = threadIdx.x;
    {
        ClusterTeam tm(&sh);
        const bool rank0 = tm.cl.block_rank() == 0;
        for (;;) {
            if (rank0 && tid == 0) {
                sh.idx = atomicAdd(&queue[0], 1);
                sh.flags = 0u;
            }
            tm.cl.sync();
            const int q = tm.root->idx;
            tm.cl.sync();  // every CTA has read rank 0's shared memory before it changes
            if (q >= nbig) break;
            const int id = order[q];
            if (tid < K) {
                sh.off[tid] = sys[id].off[tid];
                sh.krev[tid] = sys[id].krev[tid];
            }
            solve_system<T, K, R>(sys[id], id, bptr[id], xptr[id], tm, tol, max_iter, check_every,
                               refine, inner_tol, inner_max, freeze, res, rank0 && tid == 0);
        }
    }
    // phase 2: no distributed shared memory from here on
    CtaTeam tm(&sh);
    for (;;) {
        if (tid == 0) {
            sh.idx = nbig + atomicAdd(&queue[1], 1);
            sh.flags = 0u;
        }
        __syncthreads();
        const int q = sh.idx;
        if (q >= nsys) break;
        const int id = order[q];
        if (tid < K) {
            sh.off[tid] = sys[id].off[tid];
            sh.krev[tid] = sys[id].krev[tid];
        }
        solve_system<T, K, R>(sys[id], id, bptr[id], xptr[id], tm, tol, max_iter, check_every, refine,
                           inner_tol, inner_max, freeze, res, tid == 0);
    }
}

}  // namespace

// Clusters above the portable 8 CTAs (16 on this GPU) need the kernel's
// non-portable attribute; set before every occupancy query and launch.
template <typename T, int K, int R>
void allow_big_clusters()
{
    if (cudaFuncSetAttribute(k_batch_solve<T, K, R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
}

template <typename T, int K, int R>
cudaError_t launch_batch_k(int cs, int grid, int block, const void *sys, const int *order, int nsys,
                           int nbig, const double *const *bptr, double *const *xptr, int *queue, double tol,
                           int max_iter, int check_every, int refine, double inner_tol,
                           int inner_max, int freeze, void *res, cudaStream_t s)
{
    if (cs > 8) allow_big_clusters<T, K, R>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(block, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_solve<T, K, R>, (const BatchSys<T> *)sys, order, nsys, nbig, bptr,
                              xptr, queue, tol, max_iter, check_every, refine, inner_tol, inner_max,
                              freeze, (BatchResult *)res);
}

// Rows in flight per thread: 1 for every diagonal count, 2 also for the 5- and
// 9-point orders (K = 4, 8).
bool batch_rows_supported(int K, int rows) { return rows == 1 || (rows == 2 && (K == 4 || K == 8)); }

template <typename T>
cudaError_t launch_batch(int K, int rows, int cs, int grid, int block, const void *sys, const int *order,
                         int nsys, int nbig, const double *const *bptr, double *const *xptr, int *queue,
                         double tol, int max_iter, int check_every, int refine, double inner_tol,
                         int inner_max, int freeze, void *res, cudaStream_t s)
{
#define GABP_BATCH_CASE(KK, RR)                                                                       \
    if (K == KK && rows == RR)                                                                        \
        return launch_batch_k<T, KK, RR>(cs, grid, block, sys, order, nsys, nbig, bptr, xptr, queue, tol, \
                                         max_iter, check_every, refine, inner_tol, inner_max, freeze, \
                                         res, s);
    GABP_BATCH_CASE(0, 1)
    GABP_BATCH_CASE(2, 1)
    GABP_BATCH_CASE(4, 1)
    GABP_BATCH_CASE(6, 1)
    GABP_BATCH_CASE(8, 1)
    GABP_BATCH_CASE(4, 2)
    GABP_BATCH_CASE(8, 2)
#undef GABP_BATCH_CASE
    return cudaErrorInvalidValue;
}

// Clusters of `cs` CTAs of `block` threads that can be resident at once (0 = none).
template <typename T, int K, int R>
int batch_max_clusters_k(int cs, int block)
{
    if (cs > 8) allow_big_clusters<T, K, R>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(block, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_batch_solve<T, K, R>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc;
}

template <typename T>
int batch_max_clusters(int K, int rows, int cs, int block)
{
    if (!batch_rows_supported(K, rows)) return 0;
    if (rows == 2) return K == 4 ? batch_max_clusters_k<T, 4, 2>(cs, block) : batch_max_clusters_k<T, 8, 2>(cs, block);
    switch (K) {
        case 0: return batch_max_clusters_k<T, 0, 1>(cs, block);
        case 2: return batch_max_clusters_k<T, 2, 1>(cs, block);
        case 4: return batch_max_clusters_k<T, 4, 1>(cs, block);
        case 6: return batch_max_clusters_k<T, 6, 1>(cs, block);
        case 8: return batch_max_clusters_k<T, 8, 1>(cs, block);
        default: return 0;
    }
}

template cudaError_t launch_batch<float>(int, int, int, int, int, const void *, const int *, int, int,
                                         const double *const *, double *const *, int *, double,
                                         int, int, int, double, int, int, void *, cudaStream_t);
template cudaError_t launch_batch<double>(int, int, int, int, int, const void *, const int *, int, int,
                                          const double *const *, double *const *, int *, double,
                                          int, int, int, double, int, int, void *, cudaStream_t);
template int batch_max_clusters<float>(int, int, int, int);
template int batch_max_clusters<double>(int, int, int, int);

void fill_batch_sys(int prec, void *dst, int n, const StencilParams &sp, const void *a, const void *c,
                    const void *diag, const double *a64, const double *diag64, void *const L[2],
                    void *const M[2], void *const P[2], void *const B[2], void *bT, double *e,
                    double *r, void *g)
{
    auto fill = [&](auto *S, auto *tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        std::memset(S, 0, sizeof(*S));
        S->n = n;
        for (int k = 0; k < KMAX; ++k) {
            S->off[k] = sp.off[k];
            S->krev[k] = sp.krev[k];
        }
        S->a = (const T *)a;
        S->c = (const T *)c;
        S->diag = (const T *)diag;
        S->a64 = a64;
        S->diag64 = diag64;
        S->L0 = (T *)L[0];
        S->L1 = (T *)L[1];
        S->M0 = (T *)M[0];
        S->M1 = (T *)M[1];
        S->P0 = (T *)P[0];
        S->P1 = (T *)P[1];
        S->B0 = (T *)B[0];
        S->B1 = (T *)B[1];
        S->bT = (T *)bT;
        S->e = e;
        S->r = r;
        S->g = (T *)g;
    };
    if (prec == 0) fill((BatchSys<double> *)dst, (double *)nullptr);
    else fill((BatchSys<float> *)dst, (float *)nullptr);
}

size_t batch_sys_bytes(int prec) { return prec == 0 ? sizeof(BatchSys<double>) : sizeof(BatchSys<float>); }
size_t batch_result_bytes() { return sizeof(BatchResult); }

}  // namespace gabp
