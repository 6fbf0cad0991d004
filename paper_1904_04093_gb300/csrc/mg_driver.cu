// Multigrid with GaBP smoothing (Sec. 4, Algorithm 3): the hierarchy, the
// V-cycle (with fused or separate transfers), its CUDA-graph replay and the
// solve loop.
#include "host.h"

// ---------------------------------------------------------------------------
// Multigrid
// ---------------------------------------------------------------------------
static gabp_status coarse_inverse(const gabp_ctx *c, std::vector<double> &inv)
{
    const int n = c->n;
    std::vector<double> A((size_t)n * n, 0.0);
    for (int r = 0; r < n; ++r)
        for (int64_t p = c->h_indptr[r]; p < c->h_indptr[r + 1]; ++p)
            A[(size_t)r * n + c->h_indices[p]] = c->h_data[p];
    // LU with partial pivoting, P A = L U (in place)
    std::vector<int> piv(n);
    for (int k = 0; k < n; ++k) {
        int pr = k;
        double best = std::fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(A[(size_t)i * n + k]) > best) {
                best = std::fabs(A[(size_t)i * n + k]);
                pr = i;
            }
        if (best == 0.0) return fail(GABP_E_INVALID_ARG, "singular coarsest-level matrix");
        piv[k] = pr;
        if (pr != k)
            for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)pr * n + j]);
        const double d = A[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            double &l = A[(size_t)i * n + k];
            if (l == 0.0) continue;
            l /= d;
            const double *uk = &A[(size_t)k * n];
            double *ai = &A[(size_t)i * n];
            for (int j = k + 1; j < n; ++j) ai[j] -= l * uk[j];
        }
    }
    // columns of the inverse: solve L U x = P e_j
    inv.assign((size_t)n * n, 0.0);
    std::vector<double> y(n);
    for (int j = 0; j < n; ++j) {
        std::fill(y.begin(), y.end(), 0.0);
        y[j] = 1.0;
        for (int k = 0; k < n; ++k) std::swap(y[k], y[piv[k]]);
        for (int i = 0; i < n; ++i) {
            double s = y[i];
            for (int k = 0; k < i; ++k) s -= A[(size_t)i * n + k] * y[k];
            y[i] = s;
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = y[i];
            for (int k = i + 1; k < n; ++k) s -= A[(size_t)i * n + k] * y[k];
            y[i] = s / A[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i) inv[(size_t)i * n + j] = y[i];
    }
    return GABP_OK;
}

gabp_status mg_setup(int levels, gabp_ctx *const *level_ctx, const int32_t *grid_side,
                     double transfer_scale, int mode, void *stream, mg_ctx **out)
{
    if (!out) return fail(GABP_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (levels < 1 || !level_ctx || !grid_side || mode < 0 || mode > 2 || !std::isfinite(transfer_scale))
        return fail(GABP_E_INVALID_ARG, "bad argument");
    for (int l = 0; l < levels; ++l) {
        if (!level_ctx[l]) return fail(GABP_E_INVALID_ARG, "null level context");
        const int m = grid_side[l];
        if (m < 1 || (int64_t)m * m != level_ctx[l]->n) return fail(GABP_E_INVALID_ARG, "grid side does not match level size");
        if (l > 0 && grid_side[l - 1] != 2 * m + 1) return fail(GABP_E_INVALID_ARG, "sides must satisfy m_fine = 2 m_coarse + 1");
        if (level_ctx[l]->dev != level_ctx[0]->dev) return fail(GABP_E_INVALID_ARG, "levels on different devices");
    }
    if (level_ctx[levels - 1]->n > 4096) return fail(GABP_E_INVALID_ARG, "coarsest level above 4096 unknowns");
    for (int l = 0; l < levels; ++l)
        if (level_ctx[l]->reordered)
            return fail(GABP_E_INVALID_ARG, "multigrid levels need the grid numbering (reorder = 0)");
    mg_ctx *mg = new (std::nothrow) mg_ctx;
    if (!mg) return fail(GABP_E_OOM, "host allocation");
    auto bail = [&](gabp_status s) {
        mg_destroy(mg);
        return s;
    };
    mg->dev = level_ctx[0]->dev;
    gabp_status s;
    if ((s = set_dev(mg->dev)) != GABP_OK) return bail(s);
    mg->stream = (cudaStream_t)stream;
    mg->levels = levels;
    mg->lv.assign(level_ctx, level_ctx + levels);
    mg->side.assign(grid_side, grid_side + levels);
    mg->scale = transfer_scale;
    mg->mode = mode;
    mg->b.assign(levels, nullptr);
    mg->x.assign(levels, nullptr);
    for (int l = 1; l < levels; ++l) {
        const size_t nb = (size_t)mg->lv[l]->n * sizeof(double);
        if ((s = dalloc(mg, (void **)&mg->b[l], nb)) != GABP_OK) return bail(s);
        if ((s = dalloc(mg, (void **)&mg->x[l], nb)) != GABP_OK) return bail(s);
    }
    std::vector<double> inv;
    if ((s = coarse_inverse(mg->lv[levels - 1], inv)) != GABP_OK) return bail(s);
    mg->nc = mg->lv[levels - 1]->n;
    if ((s = dalloc(mg, (void **)&mg->coarse_inv, inv.size() * sizeof(double))) != GABP_OK) return bail(s);
    cudaError_t e = cudaMemcpy(mg->coarse_inv, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(fail_cuda(e, "cudaMemcpy"));
    if ((s = dalloc(mg, (void **)&mg->dstat, sizeof(DevStatus))) != GABP_OK) return bail(s);
    if ((e = cudaMallocHost((void **)&mg->hstat, sizeof(DevStatus))) != cudaSuccess) return bail(fail_cuda(e, "cudaMallocHost"));
    if ((e = cudaMallocHost((void **)&mg->hflags, (size_t)levels * sizeof(unsigned))) != cudaSuccess)
        return bail(fail_cuda(e, "cudaMallocHost"));
    if ((e = cudaStreamCreateWithFlags(&mg->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(fail_cuda(e, "cudaStreamCreate"));
    // every level works on the multigrid stream
    for (auto *c : mg->lv) c->stream = mg->stream;
    mg->fusable = true;
    for (int l = 0; l < levels; ++l) {
        const gabp_ctx *c = mg->lv[l];
        if (c->L.kind != GABP_LAYOUT_STENCIL || !mg_fusable(c->L.sp, mg->side[l])) mg->fusable = false;
    }
    if (mg->fusable && levels > 1) {
        if ((s = dalloc(mg, (void **)&mg->tbuf, (size_t)mg->lv[0]->n * sizeof(double))) != GABP_OK) return bail(s);
    }
    mg->fused = mg->fusable;
    *out = mg;
    return GABP_OK;
}

gabp_status mg_set_fused(mg_ctx *mg, int fused)
{
    if (!mg) return fail(GABP_E_INVALID_ARG, "null multigrid context");
    if (fused && !mg->fusable) return fail(GABP_E_INVALID_ARG, "levels are not 3 x 3 grid stencils: no fused transfers");
    CKS(set_dev(mg->dev));
    if (mg->stream) CK(cudaStreamSynchronize(mg->stream));
    if (mg->fused != (fused != 0)) {
        for (auto &g : mg->graphs) cudaGraphExecDestroy(g.exec);
        mg->graphs.clear();
    }
    mg->fused = fused != 0;
    return GABP_OK;
}

void mg_destroy(mg_ctx *mg)
{
    if (!mg) return;
    cudaSetDevice(mg->dev);
    if (mg->stream) cudaStreamSynchronize(mg->stream);
    for (auto &g : mg->graphs) cudaGraphExecDestroy(g.exec);
    free_all(mg->allocs);
    if (mg->hstat) cudaFreeHost(mg->hstat);
    if (mg->hflags) cudaFreeHost(mg->hflags);
    if (mg->cap_stream) cudaStreamDestroy(mg->cap_stream);
    delete mg;
}

namespace {

// Where the smoother's right-hand side r = b - A x comes from: computed, equal
// to b because x is zero (every level below the finest starts from zero), or
// already in the level's residual buffer (the finest level's convergence check
// computed it for the same x).
enum MgRes { MG_RES_COMPUTE, MG_RES_XZERO, MG_RES_READY, MG_RES_BT };

// Algorithm 3 on level l: r = b - A x; nu GaBP sweeps on A e = r; x += e.
gabp_status mg_smooth(mg_ctx *mg, int l, const double *b, double *x, int nu, MgRes res)
{
    gabp_ctx *c = mg->lv[l];
    cudaStream_t s = mg->stream;
    const double *r = c->bres;
    if (res == MG_RES_COMPUTE)
        CK(launch_residual(c->L, c->a64, c->diag64, b, x, c->bres, &c->dstat[1], s));
    else if (res == MG_RES_XZERO)
        r = b;
    if (c->prec == 1) {
        CK(launch_convert_d2f(r, (float *)c->bT, c->n, s));
    } else if (r != c->bres) {
        CK(cudaMemcpyAsync(c->bres, r, (size_t)c->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    // the line schedule's column phase reads the right-hand side in transposed order
    if (c->lines_m > 0) CK(launch_transpose(c->prec, c->lines_m, c->bT, c->lbT, s));
    if (mg->mode == MG_SMOOTH_COLD) CKS(zero_messages(c, true, true));
    else if (mg->mode == MG_SMOOTH_WARM) CKS(zero_messages(c, false, true));
    CKS(aggregate(c));
    for (int i = 0; i < nu; ++i) CK(sweep_once(c, false, i == nu - 1 ? c->xbuf : nullptr, s));
    CK(launch_axpy(x, c->xbuf, 1.0, c->n, s));
    return GABP_OK;
}

// One V-cycle from level l; `top` says where level l's first residual comes
// from (levels below start from x = 0).
gabp_status mg_cycle(mg_ctx *mg, int l, int last, int nu_pre, int nu_post, const double *b, double *x,
                     MgRes top)
{
    cudaStream_t s = mg->stream;
    gabp_ctx *c = mg->lv[l];
    if (l == last) {
        if (l == mg->levels - 1) {
            CK(launch_dense_gemv(mg->coarse_inv, b, x, mg->nc, s));
        } else {
            // truncated hierarchy: smooth on the last used level instead of a direct solve
            CKS(mg_smooth(mg, l, b, x, std::max(1, nu_pre + nu_post), top));
        }
        return GABP_OK;
    }
    if (nu_pre > 0) CKS(mg_smooth(mg, l, b, x, nu_pre, top));
    CK(launch_residual(c->L, c->a64, c->diag64, b, x, c->bres, &c->dstat[1], s));
    CK(launch_restrict_fw(c->bres, mg->side[l], mg->scale, mg->b[l + 1], s));
    CK(cudaMemsetAsync(mg->x[l + 1], 0, (size_t)mg->lv[l + 1]->n * sizeof(double), s));
    CKS(mg_cycle(mg, l + 1, last, nu_pre, nu_post, mg->b[l + 1], mg->x[l + 1], MG_RES_XZERO));
    CK(launch_prolong_add(mg->x[l + 1], mg->side[l + 1], x, s));
    if (nu_post > 0) CKS(mg_smooth(mg, l, b, x, nu_post, MG_RES_COMPUTE));
    return GABP_OK;
}

// ---- fused transfers (mg.cu) ----
//
// The same cycle with the right-hand side of every smoother call produced by
// the kernel before it, in the smoother's precision: the restriction kernel
// writes the coarse level's (as its rhs b and its sweep input bT), the
// prolongation kernel the post-smoothing one, the convergence check of
// mg_solve the next pre-smoothing one (MG_RES_READY).  Levels below the
// finest start from x = 0, so their x is first written by the prolongation
// (no clearing pass) and their pre-smoothing correction e is read directly.

// The smoother's right-hand side in bT for the cases no kernel has written.
gabp_status mg_fused_rhs(mg_ctx *mg, int l, const double *b, const double *x, MgRes res)
{
    gabp_ctx *c = mg->lv[l];
    cudaStream_t s = mg->stream;
    if (res == MG_RES_XZERO) {
        if (c->prec == 1) CK(launch_convert_d2f(b, (float *)c->bT, c->n, s));
        else if (b != c->bres) CK(cudaMemcpyAsync(c->bres, b, (size_t)c->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else if (res == MG_RES_COMPUTE) {
        CK(launch_residual2(c->L, c->a64, c->diag64, b, x, c->bres, c->prec == 1 ? (float *)c->bT : nullptr,
                            &c->dstat[1], s));
    }
    return GABP_OK;
}

// Algorithm 3's nu sweeps on A e = r with r already in bT; e in the level's xbuf.
gabp_status mg_fused_sweeps(mg_ctx *mg, int l, int nu)
{
    gabp_ctx *c = mg->lv[l];
    cudaStream_t s = mg->stream;
    if (c->lines_m > 0) CK(launch_transpose(c->prec, c->lines_m, c->bT, c->lbT, s));
    const bool lam = mg->mode == MG_SMOOTH_COLD, mean = mg->mode != MG_SMOOTH_PERSIST;
    if (c->parity && nu > 0) {
        // no clearing pass: the first sweep reads the classes that have not sent yet as zero
        if (lam) c->frozen = false;
        c->zero_pending |= (lam ? 1u : 0u) | (mean ? 2u : 0u);
    } else if (lam || mean) {
        CKS(zero_messages(c, lam, mean));
    }
    CKS(aggregate(c));
    for (int i = 0; i < nu; ++i) CK(sweep_once(c, false, i == nu - 1 ? c->xbuf : nullptr, s));
    return GABP_OK;
}

// With post_e (a level below the finest), the level's final x + e is left to
// the caller's prolongation: *post_e = e (or nullptr when x is already final).
gabp_status mg_cycle_fused(mg_ctx *mg, int l, int last, int nu_pre, int nu_post, const double *b,
                           double *x, MgRes top, const double **post_e = nullptr)
{
    if (post_e) *post_e = nullptr;
    cudaStream_t s = mg->stream;
    gabp_ctx *c = mg->lv[l];
    const size_t nb = (size_t)c->n * sizeof(double);
    const bool xzero = top == MG_RES_XZERO || top == MG_RES_BT;
    if (l == last) {
        if (l == mg->levels - 1) {
            CK(launch_dense_gemv(mg->coarse_inv, b, x, mg->nc, s));
        } else {
            // truncated hierarchy: smooth on the last used level instead of a direct solve
            CKS(mg_fused_rhs(mg, l, b, x, top));
            CKS(mg_fused_sweeps(mg, l, std::max(1, nu_pre + nu_post)));
            if (xzero) CK(cudaMemcpyAsync(x, c->xbuf, nb, cudaMemcpyDeviceToDevice, s));
            else CK(launch_axpy(x, c->xbuf, 1.0, c->n, s));
        }
        return GABP_OK;
    }
    if (nu_pre > 0) {
        CKS(mg_fused_rhs(mg, l, b, x, top));
        CKS(mg_fused_sweeps(mg, l, nu_pre));
    }
    const double *E = nu_pre > 0 ? c->xbuf : nullptr;
    const double *X = xzero ? nullptr : x;
    // x1 = x + e is kept in tbuf for the prolongation when x is not zero (finest level)
    double *T = nullptr;
    if (X && E) T = mg->tbuf;
    else if (X) CK(cudaMemcpyAsync(mg->tbuf, X, nb, cudaMemcpyDeviceToDevice, s));
    gabp_ctx *cc = mg->lv[l + 1];
    CK(launch_mg_restrict_residual(c->L.sp, mg->side[l], c->a64, c->diag64, b, X, E, T, mg->scale,
                                   mg->b[l + 1], cc->prec == 1 ? (float *)cc->bT : nullptr,
                                   cc->prec == 0 ? cc->bres : nullptr, &c->dstat[0].flags, s));
    const double *ec2 = nullptr;
    CKS(mg_cycle_fused(mg, l + 1, last, nu_pre, nu_post, mg->b[l + 1], mg->x[l + 1], MG_RES_BT, &ec2));
    // x2 = x1 + P (x_c + e_c) into x, and the post-smoothing right-hand side b - A x2
    const double *Xin = X ? mg->tbuf : nullptr;
    const double *Ein = X ? nullptr : E;
    CK(launch_mg_prolong_residual(c->L.sp, mg->side[l], c->a64, c->diag64, b, Xin, Ein,
                                  mg->x[l + 1], ec2, x, c->prec == 0 ? c->bres : nullptr,
                                  c->prec == 1 ? (float *)c->bT : nullptr, &c->dstat[0].flags, s));
    if (nu_post > 0) {
        CKS(mg_fused_sweeps(mg, l, nu_post));
        if (post_e) *post_e = c->xbuf;
        else CK(launch_axpy(x, c->xbuf, 1.0, c->n, s));
    }
    return GABP_OK;
}

gabp_status mg_cycle_any(mg_ctx *mg, int l, int last, int nu_pre, int nu_post, const double *b,
                         double *x, MgRes top)
{
    if (mg->fused) return mg_cycle_fused(mg, l, last, nu_pre, nu_post, b, x, top);
    return mg_cycle(mg, l, last, nu_pre, nu_post, b, x, top);
}

// After a cycle of mg_solve: the convergence residual b - A x of the finest
// level (left in its residual buffer for the next cycle, and with fused
// transfers also in its sweep input), its maxima and every level's breakdown
// flags copied to pinned host memory.
gabp_status mg_cycle_tail(mg_ctx *mg, const double *b, double *x, cudaStream_t s)
{
    gabp_ctx *f = mg->lv[0];
    CK(cudaMemsetAsync(mg->dstat, 0, sizeof(DevStatus), s));
    CK(launch_residual2(f->L, f->a64, f->diag64, b, x, f->bres,
                        mg->fused && f->prec == 1 ? (float *)f->bT : nullptr, mg->dstat, s));
    CK(cudaMemcpyAsync(mg->hstat, mg->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    for (int l = 0; l < mg->levels; ++l)
        CK(cudaMemcpyAsync(&mg->hflags[l], &mg->lv[l]->dstat[0].flags, sizeof(unsigned),
                           cudaMemcpyDeviceToHost, s));
    return GABP_OK;
}

// A replayed cycle starts from the message buffers it was captured with.
// That is right when the smoother restarts from zero messages (cold), when
// every level updates its messages in place (coloured and line schedules),
// or when a cycle does an even number of double-buffered sweeps per level.
bool mg_graph_safe(const mg_ctx *mg, int nu_pre, int nu_post)
{
    if (mg->mode == MG_SMOOTH_COLD || (nu_pre + nu_post) % 2 == 0) return true;
    for (const gabp_ctx *c : mg->lv)
        if (!(c->ncolors > 0 || c->lines_m > 0)) return false;
    return true;
}

// One cycle of mg_solve after the first (pre-smoothing residual known) and
// its tail, replayed from a graph captured on the first use of (b, x, nu).
gabp_status mg_cycle_graph(mg_ctx *mg, const double *b, double *x, int nu_pre, int nu_post)
{
    cudaGraphExec_t exec = nullptr;
    unsigned long long kernels = 0;
    for (auto &g : mg->graphs)
        if (g.b == b && g.x == x && g.nu_pre == nu_pre && g.nu_post == nu_post) {
            exec = g.exec;
            kernels = g.kernels;
        }
    if (!exec) {
        // enqueue everything on the capture stream: the multigrid and every level
        cudaStream_t home = mg->stream;
        mg->stream = mg->cap_stream;
        for (auto *c : mg->lv) c->stream = mg->cap_stream;
        cudaGraph_t graph = nullptr;
        gabp_status st = GABP_OK;
        cudaError_t e = cudaStreamBeginCapture(mg->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = mg_cycle_any(mg, 0, mg->levels - 1, nu_pre, nu_post, b, x, MG_RES_READY);
            if (st == GABP_OK) st = mg_cycle_tail(mg, b, x, mg->cap_stream);
            e = cudaStreamEndCapture(mg->cap_stream, &graph);
        }
        mg->stream = home;
        for (auto *c : mg->lv) c->stream = home;
        if (st != GABP_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return fail_cuda(e, "multigrid cycle capture");
        size_t nn = 0;
        cudaGraphGetNodes(graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
        for (auto &nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail_cuda(e, "cudaGraphInstantiate");
        mg->graphs.push_back({b, x, nu_pre, nu_post, exec, kernels});
    }
    CK(cudaGraphLaunch(exec, mg->stream));
    count_launches(mg->stream, kernels);
    return GABP_OK;
}

gabp_status mg_check_flags(mg_ctx *mg)
{
    for (auto *c : mg->lv) {
        CK(cudaMemcpyAsync(&c->hstat[0].flags, &c->dstat[0].flags, sizeof(unsigned), cudaMemcpyDeviceToHost, mg->stream));
    }
    CK(cudaStreamSynchronize(mg->stream));
    for (auto *c : mg->lv) {
        CKS(index_error(c->hstat[0].flags));
        if (c->hstat[0].flags & FLAG_BREAKDOWN) return fail(GABP_E_BREAKDOWN, "zero or non-finite message denominator in a smoother");
    }
    return GABP_OK;
}

}  // namespace

gabp_status mg_vcycle(mg_ctx *mg, int levels, int nu_pre, int nu_post, const double *b, double *x)
{
    if (!mg || levels < 0 || levels > mg->levels || nu_pre < 0 || nu_post < 0 || !b || !x)
        return fail(GABP_E_INVALID_ARG, "bad argument");
    CKS(set_dev(mg->dev));
    const int last = (levels == 0 ? mg->levels : levels) - 1;
    for (auto *c : mg->lv) CK(cudaMemsetAsync(&c->dstat[0].flags, 0, sizeof(unsigned), mg->stream));
    CKS(mg_cycle_any(mg, 0, last, nu_pre, nu_post, b, x, MG_RES_COMPUTE));
    return mg_check_flags(mg);
}

gabp_status mg_solve(mg_ctx *mg, const double *b, double *x, double tol, int max_cycles, int nu_pre,
                     int nu_post, int *cycles, double *relres)
{
    if (!mg || !b || !x || max_cycles < 0 || !(tol >= 0.0) || nu_pre < 0 || nu_post < 0)
        return fail(GABP_E_INVALID_ARG, "bad argument");
    CKS(set_dev(mg->dev));
    gabp_ctx *f = mg->lv[0];
    cudaStream_t s = mg->stream;
    CK(cudaMemsetAsync(x, 0, (size_t)f->n * sizeof(double), s));
    CK(cudaMemsetAsync(mg->dstat, 0, sizeof(DevStatus), s));
    CK(launch_residual(f->L, f->a64, f->diag64, b, x, nullptr, mg->dstat, s));
    CK(cudaMemcpyAsync(mg->hstat, mg->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double bn = bits_to_double(mg->hstat->bmax);
    double rr = bn == 0.0 ? 0.0 : 1.0;
    int c = 0;
    gabp_status st = bn == 0.0 ? GABP_OK : GABP_E_NOT_CONVERGED;
    for (auto *lc : mg->lv) CK(cudaMemsetAsync(&lc->dstat[0].flags, 0, sizeof(unsigned), s));
    while (st == GABP_E_NOT_CONVERGED && c < max_cycles) {
        if (c == 0) {
            // the first cycle starts from x = 0
            CKS(mg_cycle_any(mg, 0, mg->levels - 1, nu_pre, nu_post, b, x, MG_RES_XZERO));
            CKS(mg_cycle_tail(mg, b, x, s));
        } else if (mg_graph_safe(mg, nu_pre, nu_post)) {
            // later cycles reuse the check's residual of the same x: one graph replay each
            CKS(mg_cycle_graph(mg, b, x, nu_pre, nu_post));
        } else {
            CKS(mg_cycle_any(mg, 0, mg->levels - 1, nu_pre, nu_post, b, x, MG_RES_READY));
            CKS(mg_cycle_tail(mg, b, x, s));
        }
        ++c;
        CK(cudaStreamSynchronize(s));
        rr = bits_to_double(mg->hstat->rmax) / bn;
        gabp_status fs = GABP_OK;
        for (int l = 0; l < mg->levels; ++l) {
            if (mg->hflags[l] & FLAG_BREAKDOWN)
                fs = fail(GABP_E_BREAKDOWN, "zero or non-finite message denominator in a smoother");
            if (mg->hflags[l] & FLAG_INDEX) fs = index_error(mg->hflags[l]);
        }
        if (fs == GABP_OK) fs = index_error(mg->hstat->flags);
        if (fs != GABP_OK) { st = fs; break; }
        if ((mg->hstat->flags & FLAG_NAN) || !std::isfinite(rr) || rr > kDivergence) { st = fail(GABP_E_DIVERGED, "residual diverged"); break; }
        if (rr <= tol) st = GABP_OK;
    }
    if (st == GABP_E_NOT_CONVERGED) fail(st, "cycle cap reached");
    if (cycles) *cycles = c;
    if (relres) *relres = rr;
    return st;
}
