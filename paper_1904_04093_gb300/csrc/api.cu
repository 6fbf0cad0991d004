// C ABI of the GaBP library: context set-up, values, schedules, sweeps,
// solves, residuals, state and information.  The declarations and their
// contracts are in include/gabp.h; layouts and set-up helpers are in
// layout.cu, the solve drivers in solve.cu, multigrid in mg_driver.cu, the
// batched solver's front end in batch_driver.cu.
#include "host.h"

namespace {

thread_local std::string g_last_error;

}  // namespace

namespace gabp {

void set_last_error(const std::string &msg) { g_last_error = msg; }

gabp_status fail(gabp_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

gabp_status fail_cuda(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();  // clear a non-sticky error
    return e == cudaErrorMemoryAllocation ? GABP_E_OOM : GABP_E_CUDA;
}

double bits_to_double(unsigned long long u)
{
    double d;
    std::memcpy(&d, &u, sizeof d);
    return d;
}

// The bounds-checked build's index flag as an error (never set in release builds).
gabp_status index_error(unsigned fl)
{
    if (fl & FLAG_INDEX) return fail(GABP_E_CUDA, "a device index check failed (bounds-checked build)");
    return GABP_OK;
}

}  // namespace gabp

extern "C" {

void gabp_default_options(gabp_options *opt)
{
    if (!opt) return;
    opt->precision = GABP_FP64;
    opt->layout = GABP_LAYOUT_AUTO;
    opt->check_every = 10;
    opt->use_graphs = 1;
    opt->ir_inner_max = 0;  // by schedule: 400 flood / coloured, 150 lines
    opt->ir_inner_tol = 1e-3;
    opt->block_size = 0;
    opt->freeze_lambda = -1;
    opt->reorder = -1;
}


const char *gabp_status_str(gabp_status s)
{
    switch (s) {
        case GABP_OK: return "ok";
        case GABP_E_INVALID_ARG: return "invalid argument";
        case GABP_E_BAD_CSR: return "malformed CSR matrix";
        case GABP_E_ZERO_DIAG: return "missing or zero diagonal entry";
        case GABP_E_BREAKDOWN: return "zero or non-finite message denominator";
        case GABP_E_DIVERGED: return "diverged";
        case GABP_E_NOT_CONVERGED: return "not converged";
        case GABP_E_CUDA: return "CUDA error";
        case GABP_E_OOM: return "out of memory";
    }
    return "unknown status";
}

const char *gabp_last_error(void) { return g_last_error.c_str(); }

unsigned long long gabp_launch_count(void) { return launch_count(); }

int gabp_debug_build(void) { return kIndexChecks ? 1 : 0; }

gabp_status gabp_setup(int32_t n, int64_t nnz, const int64_t *indptr, const int32_t *indices,
                       const double *data, const gabp_options *opt, void *stream, gabp_ctx **out)
{
    if (!out) return fail(GABP_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    gabp_options o;
    gabp_default_options(&o);
    if (opt) o = *opt;
    if (o.precision < 0 || o.precision > 2 || o.layout < 0 || o.layout > 2 || o.check_every < 0 ||
        o.block_size < 0 || o.block_size > 1024 || (o.block_size % 32) != 0 ||
        o.freeze_lambda < -1 || o.freeze_lambda > 1 || o.reorder < -1 || o.reorder > 1)
        return fail(GABP_E_INVALID_ARG, "bad option");
    CKS(validate_csr(n, nnz, indptr, indices, data));
    int64_t nonzero_off = 0;
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p)
            if (indices[p] != r && data[p] != 0.0) ++nonzero_off;

    HostLayout H;
    StencilParams sp{};
    bool can_stencil = o.layout != GABP_LAYOUT_CSR && stencil_offsets(n, indptr, indices, sp);
    if (o.layout == GABP_LAYOUT_STENCIL && !can_stencil)
        return fail(GABP_E_INVALID_ARG, "stencil layout needs at most 16 off-diagonal diagonals");
    const int64_t offd = nnz - n;
    bool use_stencil = can_stencil &&
                       (o.layout == GABP_LAYOUT_STENCIL || (int64_t)sp.K * n <= 3 * offd + 4096);
    std::vector<int32_t> perm;
    std::vector<int64_t> pindptr, pmap;
    std::vector<int32_t> pindices;
    bool reordered = false;
    if (use_stencil) {
        build_stencil(n, indptr, indices, data, sp, H);
    } else if (o.reorder != 0 && n > 2 && rcm_order(n, indptr, indices, o.reorder == 1, perm)) {
        // the layout is built on P A P^T; the caller's entries map through pmap
        permute_csr(n, indptr, indices, perm, pindptr, pindices, pmap);
        const std::vector<double> pdata = permute_values(pmap, data);
        build_csr(n, pindptr.data(), pindices.data(), pdata.data(), H);
        std::vector<int64_t> sm((size_t)nnz);
        for (int64_t p = 0; p < nnz; ++p) sm[p] = H.slotmap[pmap[p]];
        H.slotmap.swap(sm);
        reordered = true;
    } else {
        build_csr(n, indptr, indices, data, H);
    }
    if (H.kind == GABP_LAYOUT_CSR && H.slots >= (int64_t)1 << 31)
        return fail(GABP_E_INVALID_ARG, "too many edges for the CSR layout");

    gabp_ctx *ctx = new (std::nothrow) gabp_ctx;
    if (!ctx) return fail(GABP_E_OOM, "host allocation");
    auto bail = [&](gabp_status s) {
        gabp_destroy(ctx);
        return s;
    };
    cudaError_t e = cudaGetDevice(&ctx->dev);
    if (e != cudaSuccess) return bail(fail_cuda(e, "cudaGetDevice"));
    ctx->stream = (cudaStream_t)stream;
    ctx->opt = o;
    ctx->prec = o.precision == GABP_FP64 ? 0 : 1;
    ctx->n = n;
    ctx->nnz = nnz;
    ctx->edges = nonzero_off;
    ctx->h_indptr.assign(indptr, indptr + n + 1);
    ctx->h_indices.assign(indices, indices + nnz);
    ctx->h_data.assign(data, data + nnz);
    e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(fail_cuda(e, "cudaStreamCreate"));
    if ((e = cudaEventCreate(&ctx->ev0)) != cudaSuccess || (e = cudaEventCreate(&ctx->ev1)) != cudaSuccess)
        return bail(fail_cuda(e, "cudaEventCreate"));

    DevLayout &L = ctx->L;
    L.kind = H.kind;
    L.n = n;
    L.slots = H.slots;
    L.sp = H.sp;
    gabp_status s;
    if (H.kind == GABP_LAYOUT_CSR) {
        if ((s = upload(ctx, (void **)&L.rowptr, H.rowptr.data(), H.rowptr.size() * sizeof(int))) != GABP_OK) return bail(s);
        if ((s = upload(ctx, (void **)&L.col, H.col.data(), H.col.size() * sizeof(int))) != GABP_OK) return bail(s);
        if ((s = upload(ctx, (void **)&L.rev, H.rev.data(), H.rev.size() * sizeof(int))) != GABP_OK) return bail(s);
    }
    if ((s = upload_coeffs(ctx, H, true)) != GABP_OK) return bail(s);
    if ((s = upload(ctx, (void **)&ctx->slotmap, H.slotmap.data(), H.slotmap.size() * sizeof(int64_t))) != GABP_OK) return bail(s);
    if (reordered) {
        ctx->reordered = true;
        if ((s = upload(ctx, (void **)&ctx->d_perm, perm.data(), perm.size() * sizeof(int32_t))) != GABP_OK) return bail(s);
        ctx->h_perm.swap(perm);
        ctx->h_pindptr.swap(pindptr);
        ctx->h_pindices.swap(pindices);
        ctx->h_pmap.swap(pmap);
    }
    const size_t S = (size_t)H.slots * esz(ctx->prec), NB = (size_t)n * esz(ctx->prec);
    for (int i = 0; i < 2; ++i) {
        if ((s = dalloc(ctx, &ctx->Lm[i], S)) != GABP_OK) return bail(s);
        if ((s = dalloc(ctx, &ctx->Mm[i], S)) != GABP_OK) return bail(s);
        if ((s = dalloc(ctx, &ctx->P[i], NB)) != GABP_OK) return bail(s);
        if ((s = dalloc(ctx, &ctx->B[i], NB)) != GABP_OK) return bail(s);
    }
    if ((s = dalloc(ctx, (void **)&ctx->bres, (size_t)n * sizeof(double))) != GABP_OK) return bail(s);
    if (ctx->prec == 0) ctx->bT = ctx->bres;
    else if ((s = dalloc(ctx, &ctx->bT, NB)) != GABP_OK) return bail(s);
    if ((s = dalloc(ctx, (void **)&ctx->xbuf, (size_t)n * sizeof(double))) != GABP_OK) return bail(s);
    if ((s = dalloc(ctx, (void **)&ctx->dstat, 3 * sizeof(DevStatus))) != GABP_OK) return bail(s);
    e = cudaMallocHost((void **)&ctx->hstat, 3 * sizeof(DevStatus));
    if (e != cudaSuccess) return bail(fail_cuda(e, "cudaMallocHost"));
    std::memset(ctx->hstat, 0, 3 * sizeof(DevStatus));
    for (int i = 0; i < 2; ++i) {
        if ((e = cudaMemset(ctx->Lm[i], 0, S)) != cudaSuccess) return bail(fail_cuda(e, "cudaMemset"));
        if ((e = cudaMemset(ctx->Mm[i], 0, S)) != cudaSuccess) return bail(fail_cuda(e, "cudaMemset"));
    }
    if ((e = cudaMemset(ctx->dstat, 0, 3 * sizeof(DevStatus))) != cudaSuccess) return bail(fail_cuda(e, "cudaMemset"));
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(fail_cuda(e, "setup"));
    *out = ctx;
    return GABP_OK;
}

namespace {

// After new matrix values: the edge count, the derived coefficient copies
// (transposed, parity-class, line schedule) and zero messages.
gabp_status after_new_values(gabp_ctx *ctx)
{
    const double *data = ctx->h_data.data();
    int64_t nz = 0;
    for (int32_t r = 0; r < ctx->n; ++r)
        for (int64_t p = ctx->h_indptr[r]; p < ctx->h_indptr[r + 1]; ++p)
            if (ctx->h_indices[p] != r && data[p] != 0.0) ++nz;
    ctx->edges = nz;
    if (ctx->aT) {
        CK(launch_transpose_coeffs(ctx->L, 0, ctx->a64, ctx->aT64, ctx->stream));
        if (ctx->prec == 1) CK(launch_transpose_coeffs(ctx->L, 1, ctx->a, ctx->aT, ctx->stream));
    }
    if (ctx->parity) {
        CK(launch_parity_convert(ctx->pg, ctx->prec, 1, ctx->a, ctx->pa, ctx->stream));
        CK(launch_parity_convert(ctx->pg, ctx->prec, 1, ctx->c, ctx->pc, ctx->stream));
        if (ctx->paT) CKS(ensure_parity_transpose(ctx));
    }
    if (ctx->lines_m > 0) {
        // couplings of the line regions: from the stencil layout on the device, else on the host
        if (ctx->L.kind == GABP_LAYOUT_STENCIL)
            CK(launch_line_couplings_from_stencil(ctx->prec, ctx->lines_m, ctx->L.sp, ctx->a64,
                                                  ctx->diag64, ctx->lsubH, ctx->lsupH, ctx->lsubV,
                                                  ctx->lsupV, ctx->ldiagT, ctx->stream));
        else
            CKS(setup_lines(ctx));
    }
    CKS(zero_messages(ctx, true, true));
    CK(cudaStreamSynchronize(ctx->stream));
    return GABP_OK;
}

}  // namespace

gabp_status gabp_set_values(gabp_ctx *ctx, const double *data)
{
    if (!ctx || (!data && ctx->nnz > 0)) return fail(GABP_E_INVALID_ARG, "null argument");
    CKS(set_dev(ctx->dev));
    CKS(validate_csr(ctx->n, ctx->nnz, ctx->h_indptr.data(), ctx->h_indices.data(), data));
    HostLayout H;
    if (ctx->L.kind == GABP_LAYOUT_STENCIL) {
        build_stencil(ctx->n, ctx->h_indptr.data(), ctx->h_indices.data(), data, ctx->L.sp, H);
    } else if (ctx->reordered) {
        const std::vector<double> pdata = permute_values(ctx->h_pmap, data);
        build_csr(ctx->n, ctx->h_pindptr.data(), ctx->h_pindices.data(), pdata.data(), H);
    } else {
        build_csr(ctx->n, ctx->h_indptr.data(), ctx->h_indices.data(), data, H);
    }
    CK(cudaStreamSynchronize(ctx->stream));
    CKS(upload_coeffs(ctx, H, false));
    ctx->h_data.assign(data, data + ctx->nnz);
    return after_new_values(ctx);
}

gabp_status gabp_set_values_device(gabp_ctx *ctx, const double *data)
{
    if (!ctx || (!data && ctx->nnz > 0)) return fail(GABP_E_INVALID_ARG, "null argument");
    CKS(set_dev(ctx->dev));
    // the host copy keeps the host-side consumers (line couplings, multigrid
    // coarse solve, validation) in step with the device values
    std::vector<double> h((size_t)ctx->nnz);
    if (ctx->nnz) {
        CK(cudaMemcpyAsync(h.data(), data, (size_t)ctx->nnz * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    CKS(validate_csr(ctx->n, ctx->nnz, ctx->h_indptr.data(), ctx->h_indices.data(), h.data()));
    if (!ctx->diagpos) {
        std::vector<int64_t> dp((size_t)ctx->n, 0);  // by internal row
        for (int32_t i = 0; i < ctx->n; ++i) {
            const int32_t r = ctx->reordered ? ctx->h_perm[i] : i;
            for (int64_t p = ctx->h_indptr[r]; p < ctx->h_indptr[r + 1]; ++p)
                if (ctx->h_indices[p] == r) dp[i] = p;
        }
        CKS(upload(ctx, (void **)&ctx->diagpos, dp.data(), dp.size() * sizeof(int64_t)));
    }
    CK(launch_coeffs_from_values(ctx->L, ctx->prec, ctx->nnz, ctx->slotmap, ctx->diagpos, data,
                                 ctx->a64, ctx->diag64, ctx->a, ctx->c, ctx->diagT, ctx->stream));
    ctx->h_data.swap(h);
    return after_new_values(ctx);
}

void gabp_destroy(gabp_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->dev);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    free_all(ctx->allocs);
    if (ctx->hstat) cudaFreeHost(ctx->hstat);
    if (ctx->h_sq_part) cudaFreeHost(ctx->h_sq_part);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
}

gabp_status gabp_set_schedule(gabp_ctx *ctx, int schedule, const int32_t *color, int *ncolors)
{
    if (!ctx || schedule < 0 || schedule > 2) return fail(GABP_E_INVALID_ARG, "bad argument");
    CKS(set_dev(ctx->dev));
    CK(cudaStreamSynchronize(ctx->stream));
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
    ctx->frozen = false;
    ctx->parity = false;
    CKS(zero_messages(ctx, true, true));
    CKS(aggregate(ctx));
    if (schedule != 1) {
        ctx->ncolors = 0;
        if (ncolors) *ncolors = 0;
    }
    if (schedule == 0) {
        ctx->lines_m = 0;
        CK(cudaStreamSynchronize(ctx->stream));
        return GABP_OK;
    }
    if (schedule == 2) {
        ctx->lines_m = 0;
        return setup_lines(ctx);
    }
    ctx->lines_m = 0;
    const int n = ctx->n;
    const int64_t *ip = ctx->h_indptr.data();
    const int32_t *ix = ctx->h_indices.data();
    std::vector<int> col(n, -1);
    if (color) {
        for (int i = 0; i < n; ++i) {
            if (color[i] < 0 || color[i] > 254) return fail(GABP_E_INVALID_ARG, "colours must lie in [0, 254]");
            col[i] = color[i];
        }
    } else {
        // greedy colouring of the symmetrised graph in natural order
        std::vector<int64_t> tp(n + 1, 0);
        for (int64_t p = 0; p < ip[n]; ++p) tp[ix[p] + 1]++;
        for (int i = 0; i < n; ++i) tp[i + 1] += tp[i];
        std::vector<int> trow(ip[n]);
        std::vector<int64_t> fill(tp.begin(), tp.end() - 1);
        for (int i = 0; i < n; ++i)
            for (int64_t p = ip[i]; p < ip[i + 1]; ++p) trow[fill[ix[p]]++] = i;
        std::vector<int> mark(256, -1);
        for (int i = 0; i < n; ++i) {
            for (int64_t p = ip[i]; p < ip[i + 1]; ++p)
                if (ix[p] != i && col[ix[p]] >= 0) mark[col[ix[p]]] = i;
            for (int64_t p = tp[i]; p < tp[i + 1]; ++p)
                if (trow[p] != i && col[trow[p]] >= 0) mark[col[trow[p]]] = i;
            int c = 0;
            while (c < 255 && mark[c] == i) ++c;
            if (c >= 255) return fail(GABP_E_INVALID_ARG, "graph needs more than 255 colours");
            col[i] = c;
        }
    }
    int nc = 0;
    for (int i = 0; i < n; ++i) nc = std::max(nc, col[i] + 1);
    for (int i = 0; i < n; ++i)
        for (int64_t p = ip[i]; p < ip[i + 1]; ++p)
            if (ix[p] != i && col[ix[p]] == col[i])
                return fail(GABP_E_INVALID_ARG, "adjacent nodes share a colour");
    std::vector<unsigned char> c8(n);
    for (int i = 0; i < n; ++i) c8[i] = (unsigned char)col[ctx->reordered ? ctx->h_perm[i] : i];
    // stencil layout: one sender colour per (row colour, diagonal) -> slot masks
    ctx->has_masks = false;
    if (ctx->L.kind == GABP_LAYOUT_STENCIL && nc <= KMAXCOLOR) {
        const int K = ctx->L.sp.K;
        std::vector<int> tab((size_t)nc * KMAX, -1);
        bool ok = true;
        for (int r = 0; r < n && ok; ++r)
            for (int64_t p = ip[r]; p < ip[r + 1]; ++p) {
                const int j = ix[p];
                if (j == r) continue;
                int k = 0;
                while (k < K && ctx->L.sp.off[k] != j - r) ++k;
                if (k == K) { ok = false; break; }
                int &t = tab[(size_t)col[r] * KMAX + k];
                if (t < 0) t = col[j];
                else if (t != col[j]) { ok = false; break; }
            }
        if (ok) {
            std::memset(&ctx->masks, 0, sizeof ctx->masks);
            for (int cr = 0; cr < nc; ++cr)
                for (int k = 0; k < K; ++k) {
                    const int t = tab[(size_t)cr * KMAX + k];
                    if (t >= 0) ctx->masks.m[cr][t] |= (unsigned short)(1u << k);
                }
            ctx->has_masks = true;
        }
    }
    if (!ctx->color) CKS(dalloc(ctx, (void **)&ctx->color, (size_t)std::max(n, 1)));
    if (n) CK(cudaMemcpy(ctx->color, c8.data(), (size_t)n, cudaMemcpyHostToDevice));
    ctx->ncolors = nc;
    ctx->frozen = false;
    CKS(setup_parity(ctx, col, nc));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ncolors) *ncolors = nc;
    return GABP_OK;
}

gabp_status gabp_reset(gabp_ctx *ctx)
{
    if (!ctx) return fail(GABP_E_INVALID_ARG, "null context");
    CKS(set_dev(ctx->dev));
    CKS(zero_messages(ctx, true, true));
    return GABP_OK;
}

gabp_status gabp_sweep(gabp_ctx *ctx, const double *b, int nsweeps, double *x)
{
    if (!ctx || nsweeps < 0 || (!b && ctx->n > 0)) return fail(GABP_E_INVALID_ARG, "bad argument");
    CKS(set_dev(ctx->dev));
    ctx->frozen = false;  // full sweeps; a frozen state is held in both buffers
    CKS(load_rhs(ctx, b));
    CKS(aggregate(ctx));
    CK(cudaMemsetAsync(&ctx->dstat[0].flags, 0, sizeof(unsigned), ctx->stream));
    double *xo = ctx->reordered && x ? ctx->xbuf : x;  // beliefs in internal order first
    for (int i = 0; i < nsweeps; ++i) CK(sweep_once(ctx, false, i == nsweeps - 1 ? xo : nullptr, ctx->stream));
    if (xo != x && nsweeps > 0) CKS(store_vector(ctx, xo, x, ctx->stream));
    unsigned fl = 0;
    CKS(read_status(ctx, 0, nullptr, nullptr, &fl));
    CKS(index_error(fl));
    if (fl & FLAG_BREAKDOWN) return fail(GABP_E_BREAKDOWN, "zero or non-finite message denominator");
    return GABP_OK;
}

gabp_status gabp_time_sweeps(gabp_ctx *ctx, const double *b, int nsweeps, int frozen, float *ms)
{
    if (!ctx || nsweeps < 1 || !ms || (!b && ctx->n > 0) || frozen < 0 || frozen > 1)
        return fail(GABP_E_INVALID_ARG, "bad argument");
    if (frozen && !ctx->frozen) return fail(GABP_E_INVALID_ARG, "no frozen precision messages in this context");
    CKS(set_dev(ctx->dev));
    CKS(load_rhs(ctx, b));
    CKS(aggregate(ctx));
    if (frozen) {
        // the frozen L sits in both buffers; restore the frozen-sweep mode
        ctx->frozen = true;
    } else {
        ctx->frozen = false;
    }
    CK(cudaMemsetAsync(&ctx->dstat[0].flags, 0, sizeof(unsigned), ctx->stream));
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    for (int i = 0; i < nsweeps; ++i) CK(sweep_once(ctx, false, nullptr, ctx->stream));
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    CK(cudaEventSynchronize(ctx->ev1));
    CK(cudaEventElapsedTime(ms, ctx->ev0, ctx->ev1));
    unsigned fl = 0;
    CKS(read_status(ctx, 0, nullptr, nullptr, &fl));
    CKS(index_error(fl));
    if (fl & FLAG_BREAKDOWN) return fail(GABP_E_BREAKDOWN, "zero or non-finite message denominator");
    return GABP_OK;
}

gabp_status gabp_solve(gabp_ctx *ctx, const double *b, double *x, double tol, int max_iter,
                       int *iters, double *relres)
{
    if (!ctx || max_iter < 0 || !(tol >= 0.0) || ((!b || !x) && ctx->n > 0))
        return fail(GABP_E_INVALID_ARG, "bad argument");
    CKS(set_dev(ctx->dev));
    if (ctx->opt.precision == GABP_FP32_IR) return solve_ir(ctx, b, x, tol, max_iter, iters, relres);
    return solve_plain(ctx, b, x, tol, max_iter, iters, relres, false);
}

gabp_status gabp_solve_transpose(gabp_ctx *ctx, const double *g, double *lam, double tol,
                                  int max_iter, int *iters, double *relres)
{
    if (!ctx || max_iter < 0 || !(tol >= 0.0) || ((!g || !lam) && ctx->n > 0))
        return fail(GABP_E_INVALID_ARG, "bad argument");
    CKS(set_dev(ctx->dev));
    CKS(ensure_transpose(ctx));
    if (ctx->lines_m > 0) {
        // line couplings of A^T (rebuilt every call: they follow the current values)
        const size_t nb = (size_t)ctx->n * esz(ctx->prec);
        void **bufs[] = {&ctx->lsubHT, &ctx->lsupHT, &ctx->lsubVT, &ctx->lsupVT};
        for (void **bp : bufs)
            if (!*bp) CKS(dalloc(ctx, bp, nb));
        CK(launch_line_couplings_transpose(ctx->prec, ctx->lines_m, ctx->lsubH, ctx->lsupH,
                                           ctx->lsubHT, ctx->lsupHT, ctx->stream));
        CK(launch_line_couplings_transpose(ctx->prec, ctx->lines_m, ctx->lsubV, ctx->lsupV,
                                           ctx->lsubVT, ctx->lsupVT, ctx->stream));
    }
    if (ctx->opt.precision == GABP_FP32_IR) return solve_ir(ctx, g, lam, tol, max_iter, iters, relres, true);
    return solve_plain(ctx, g, lam, tol, max_iter, iters, relres, true);
}

gabp_status gabp_edge_grad(gabp_ctx *ctx, const double *lam, const double *x, double *dA)
{
    if (!ctx || ((!lam || !x || !dA) && ctx->n > 0)) return fail(GABP_E_INVALID_ARG, "null argument");
    CKS(set_dev(ctx->dev));
    if (!ctx->d_indptr) {
        CKS(upload(ctx, (void **)&ctx->d_indptr, ctx->h_indptr.data(), ctx->h_indptr.size() * sizeof(int64_t)));
        CKS(upload(ctx, (void **)&ctx->d_indices, ctx->h_indices.data(), ctx->h_indices.size() * sizeof(int)));
    }
    CK(launch_edge_grad(ctx->n, ctx->d_indptr, ctx->d_indices, lam, x, dA, ctx->stream));
    return GABP_OK;
}

gabp_status gabp_residual(gabp_ctx *ctx, const double *b, const double *x, double *r, double *rinf,
                          double *binf)
{
    if (!ctx || ((!b || !x) && ctx->n > 0)) return fail(GABP_E_INVALID_ARG, "null argument");
    CKS(set_dev(ctx->dev));
    CK(cudaMemsetAsync(&ctx->dstat[1], 0, sizeof(DevStatus), ctx->stream));
    if (ctx->reordered) {
        // through the refinement vectors: caller order in, caller order out
        CKS(ensure_ir(ctx));
        CK(launch_permute(ctx->n, ctx->d_perm, b, ctx->b0, 0, ctx->stream));
        CK(launch_permute(ctx->n, ctx->d_perm, x, ctx->xacc, 0, ctx->stream));
        CK(launch_residual(ctx->L, ctx->a64, ctx->diag64, ctx->b0, ctx->xacc, r ? ctx->rbuf : nullptr,
                           &ctx->dstat[1], ctx->stream));
        if (r) CKS(store_vector(ctx, ctx->rbuf, r, ctx->stream));
    } else {
        CK(launch_residual(ctx->L, ctx->a64, ctx->diag64, b, x, r, &ctx->dstat[1], ctx->stream));
    }
    if (rinf || binf || kIndexChecks) {
        unsigned fl = 0;
        CKS(read_status(ctx, 1, rinf, binf, &fl));
        CKS(index_error(fl));
    }
    return GABP_OK;
}

gabp_status gabp_residual_2norm(gabp_ctx *ctx, const double *b, const double *x, double *r2,
                                double *b2)
{
    if (!ctx || ((!b || !x) && ctx->n > 0) || !r2 || !b2) return fail(GABP_E_INVALID_ARG, "null argument");
    CKS(set_dev(ctx->dev));
    *r2 = *b2 = 0.0;
    if (ctx->n == 0) return GABP_OK;
    CKS(ensure_ir(ctx));
    const size_t pbytes = 2 * (size_t)kSumsqBlocks * sizeof(double);
    if (!ctx->sq_part) CKS(dalloc(ctx, (void **)&ctx->sq_part, pbytes));
    if (!ctx->h_sq_part) {
        cudaError_t e = cudaMallocHost(&ctx->h_sq_part, pbytes);
        if (e != cudaSuccess) {
            ctx->h_sq_part = nullptr;
            return fail_cuda(e, "cudaMallocHost");
        }
    }
    // r = b - A x in the internal order (rbuf); b in the same order (b0)
    CK(cudaMemsetAsync(&ctx->dstat[1], 0, sizeof(DevStatus), ctx->stream));
    const double *bi = b, *xi = x;
    if (ctx->reordered) {
        CK(launch_permute(ctx->n, ctx->d_perm, b, ctx->b0, 0, ctx->stream));
        CK(launch_permute(ctx->n, ctx->d_perm, x, ctx->xacc, 0, ctx->stream));
        bi = ctx->b0;
        xi = ctx->xacc;
    }
    CK(launch_residual(ctx->L, ctx->a64, ctx->diag64, bi, xi, ctx->rbuf, &ctx->dstat[1], ctx->stream));
    CK(launch_sumsq2(ctx->rbuf, bi, ctx->n, ctx->sq_part, kSumsqBlocks, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_sq_part, ctx->sq_part, pbytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double sr = 0.0, sb = 0.0;
    for (int i = 0; i < kSumsqBlocks; ++i) {
        sr += ctx->h_sq_part[2 * i];
        sb += ctx->h_sq_part[2 * i + 1];
    }
    *r2 = std::sqrt(sr);
    *b2 = std::sqrt(sb);
    return GABP_OK;
}

gabp_status gabp_get_state(gabp_ctx *ctx, double *lam, double *m)
{
    if (!ctx) return fail(GABP_E_INVALID_ARG, "null context");
    CKS(set_dev(ctx->dev));
    const void *Ls = ctx->Lm[ctx->cur], *Ms = ctx->Mm[ctx->cur];
    if (ctx->parity) {  // class layout -> slot layout in the idle buffers
        const int o = ctx->cur ^ 1;
        CK(launch_parity_convert(ctx->pg, ctx->prec, 0, ctx->Lm[ctx->cur], ctx->Lm[o], ctx->stream));
        CK(launch_parity_convert(ctx->pg, ctx->prec, 0, ctx->Mm[ctx->cur], ctx->Mm[o], ctx->stream));
        Ls = ctx->Lm[o];
        Ms = ctx->Mm[o];
    }
    CK(launch_get_state(ctx->slotmap, ctx->nnz, ctx->prec, Ls, Ms, lam, m, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return GABP_OK;
}

gabp_status gabp_set_state(gabp_ctx *ctx, const double *lam, const double *m)
{
    if (!ctx) return fail(GABP_E_INVALID_ARG, "null context");
    CKS(set_dev(ctx->dev));
    CKS(zero_messages(ctx, lam != nullptr, m != nullptr));
    if (ctx->parity) {  // through the slot layout in the idle buffers
        const int o = ctx->cur ^ 1;
        CK(launch_parity_convert(ctx->pg, ctx->prec, 0, ctx->Lm[ctx->cur], ctx->Lm[o], ctx->stream));
        CK(launch_parity_convert(ctx->pg, ctx->prec, 0, ctx->Mm[ctx->cur], ctx->Mm[o], ctx->stream));
        CK(launch_set_state(ctx->slotmap, ctx->nnz, ctx->prec, lam, m, ctx->Lm[o], ctx->Mm[o], ctx->stream));
        CK(launch_parity_convert(ctx->pg, ctx->prec, 1, ctx->Lm[o], ctx->Lm[ctx->cur], ctx->stream));
        CK(launch_parity_convert(ctx->pg, ctx->prec, 1, ctx->Mm[o], ctx->Mm[ctx->cur], ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return GABP_OK;
    }
    CK(launch_set_state(ctx->slotmap, ctx->nnz, ctx->prec, lam, m, ctx->Lm[ctx->cur], ctx->Mm[ctx->cur], ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return GABP_OK;
}

gabp_status gabp_get_line_state(gabp_ctx *ctx, double *LH, double *MH, double *LV, double *MV)
{
    if (!ctx) return fail(GABP_E_INVALID_ARG, "null context");
    if (ctx->lines_m == 0) return fail(GABP_E_INVALID_ARG, "the line schedule is not selected");
    CKS(set_dev(ctx->dev));
    const int64_t n = ctx->n;
    if (LH) CK(launch_to_double(ctx->prec, ctx->LH, LH, n, ctx->stream));
    if (MH && ctx->mh_sum)  // folded by the last sweep: b + m' back to m' with the current b
        CK(launch_line_unfold(n, ctx->MH, ctx->bT, MH, ctx->stream));
    else if (MH)
        CK(launch_to_double(ctx->prec, ctx->MH, MH, n, ctx->stream));
    if (LV) CK(launch_to_double(ctx->prec, ctx->LV, LV, n, ctx->stream));
    if (MV) CK(launch_to_double(ctx->prec, ctx->MV, MV, n, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return GABP_OK;
}

gabp_status gabp_get_info(gabp_ctx *ctx, gabp_info *info)
{
    if (!ctx || !info) return fail(GABP_E_INVALID_ARG, "null argument");
    const double p = (double)esz(ctx->prec);
    const double S = (double)ctx->L.slots, n = (double)ctx->n;
    info->n = ctx->n;
    info->nnz = ctx->nnz;
    info->edges = ctx->edges;
    info->layout = ctx->L.kind;
    info->ndiag = ctx->L.kind == GABP_LAYOUT_STENCIL ? ctx->L.sp.K : 0;
    info->precision = ctx->opt.precision;
    info->slots = ctx->L.slots;
    // per slot: a, c, L[rev], M[rev] read, L', M' written; per row: diag, b, P, B
    // read, P', B' written; CSR adds col, rev (per slot) and the row pointer.
    double sweep = 6.0 * p * S + 6.0 * p * n;
    double resid = 8.0 * S + 8.0 * 4.0 * n;  // a64 per slot; diag, b, x read, r written
    if (ctx->L.kind == GABP_LAYOUT_CSR) {
        sweep += 8.0 * S + 4.0 * n;
        resid += 4.0 * S + 4.0 * n;
    }
    // frozen precision messages: per slot g, M[rev] read, M' written; per row b, B read, B' written
    double mean = 3.0 * p * S + 3.0 * p * n;
    if (ctx->L.kind == GABP_LAYOUT_CSR) mean += 8.0 * S + 4.0 * n;
    info->sweep_bytes = sweep;
    info->mean_sweep_bytes = mean;
    info->residual_bytes = resid;
    info->device_bytes = ctx->dev_bytes;
    info->parity_layout = ctx->parity ? 1 : 0;
    info->reordered = ctx->reordered ? 1 : 0;
    // parity-class coloured sweep: per slot a, c, incoming L, M read and L', M'
    // written; per node diag and b read (no aggregates)
    info->colored_sweep_bytes = 6.0 * p * S + 2.0 * p * n;
    // with frozen precision messages: per slot the gain and the incoming M read, M'
    // written; per node b read (the frozen P only on sweeps that form the beliefs)
    info->colored_mean_sweep_bytes = 3.0 * p * S + 1.0 * p * n;
    return GABP_OK;
}

}  // extern "C"
