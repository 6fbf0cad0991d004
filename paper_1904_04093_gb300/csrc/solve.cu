// The solve drivers behind the C ABI: message resets, right-hand-side
// loading, one sweep under each schedule, chunks of sweeps with their
// residual check replayed as CUDA graphs, freezing of the precision messages
// (Sec. 4.2), the plain solve (Algorithm 1) and the float solve inside double
// iterative refinement.
#include "host.h"

namespace gabp {

// ---------------------------------------------------------------------------
// Drivers
// ---------------------------------------------------------------------------
gabp_status zero_messages(gabp_ctx *ctx, bool lam, bool mean)
{
    const size_t bytes = (size_t)ctx->L.slots * esz(ctx->prec);
    if (lam) {
        ctx->frozen = false;
        ctx->lprev_valid = false;
    }
    if (ctx->lines_m > 0) {
        const size_t nb = (size_t)ctx->n * esz(ctx->prec);
        if (lam) CK(cudaMemsetAsync(ctx->LH, 0, nb, ctx->stream));
        if (lam) CK(cudaMemsetAsync(ctx->LV, 0, nb, ctx->stream));
        if (mean) CK(cudaMemsetAsync(ctx->MH, 0, nb, ctx->stream));
        if (mean) CK(cudaMemsetAsync(ctx->MV, 0, nb, ctx->stream));
        if (mean) ctx->mh_sum = false;
    }
    if (lam) CK(cudaMemsetAsync(ctx->Lm[ctx->cur], 0, bytes, ctx->stream));
    if (mean) CK(cudaMemsetAsync(ctx->Mm[ctx->cur], 0, bytes, ctx->stream));
    return GABP_OK;
}

// bres = b (double) and bT = b in message precision.
gabp_status load_rhs(gabp_ctx *ctx, const double *b)
{
    const int64_t n = ctx->n;
    if (b != ctx->bres) {
        if (ctx->reordered)  // caller order -> internal order
            CK(launch_permute((int)n, ctx->d_perm, b, ctx->bres, 0, ctx->stream));
        else
            CK(cudaMemcpyAsync(ctx->bres, b, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (ctx->prec == 1) CK(launch_convert_d2f(ctx->bres, (float *)ctx->bT, n, ctx->stream));
    if (ctx->lines_m > 0) CK(launch_transpose(ctx->prec, ctx->lines_m, ctx->bT, ctx->lbT, ctx->stream));
    return GABP_OK;
}

// An internal-order vector out to the caller's order.
gabp_status store_vector(gabp_ctx *ctx, const double *in, double *out, cudaStream_t s)
{
    if (ctx->n == 0) return GABP_OK;
    if (ctx->reordered) CK(launch_permute(ctx->n, ctx->d_perm, in, out, 1, s));
    else CK(cudaMemcpyAsync(out, in, (size_t)ctx->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return GABP_OK;
}

gabp_status aggregate(gabp_ctx *ctx)
{
    // the parity-class and line sweeps keep no aggregates
    if (ctx->parity || ctx->lines_m > 0) return GABP_OK;
    CK(launch_aggregate(ctx->L, ctx->prec, ctx->diagT, ctx->bT, ctx->Lm[ctx->cur],
                        ctx->Mm[ctx->cur], ctx->P[ctx->cur], ctx->B[ctx->cur], ctx->stream));
    return GABP_OK;
}

int block_of(const gabp_ctx *ctx)
{ return ctx->opt.block_size > 0 ? ctx->opt.block_size : 256; }

// One sweep from state cur into 1 - cur (mean messages only while frozen);
// with a coloured schedule, one in-place phase per colour class.
cudaError_t sweep_once(gabp_ctx *ctx, bool transposed, double *x, cudaStream_t s)
{
    const int c0 = ctx->cur, c1 = c0 ^ 1;
    // line couplings of A, or of A^T for the transposed solve
    void *lsH = transposed ? ctx->lsubHT : ctx->lsubH, *luH = transposed ? ctx->lsupHT : ctx->lsupH;
    void *lsV = transposed ? ctx->lsubVT : ctx->lsubV, *luV = transposed ? ctx->lsupVT : ctx->lsupV;
    if (ctx->lines_m > 0 && ctx->frozen && line_cols_natural(ctx->prec, ctx->lines_m)) {
        // frozen precision messages, both families in the natural order: no transposes; the
        // row phase hands b + m'_row to the column phase, which restores m'_row when it writes x
        const int m = ctx->lines_m, pr = ctx->prec;
        cudaError_t e;
        if ((e = launch_line_mean(pr, m, ctx->laFH, ctx->laBH, ctx->lSH, ctx->bT, ctx->MV, ctx->MH,
                                  ctx->ly, nullptr, 0, 1, &ctx->dstat[0].flags, s)) != cudaSuccess)
            return e;
        ctx->mh_sum = x == nullptr;
        return launch_line_mean_cols(pr, m, ctx->laFVn, ctx->laBVn, ctx->lSVn, ctx->bT, ctx->MH,
                                     ctx->MV, x, &ctx->dstat[0].flags, s);
    }
    if (ctx->lines_m > 0 && ctx->frozen) {
        // frozen precision messages: the mean messages move, rows then columns
        const int m = ctx->lines_m, pr = ctx->prec;
        cudaError_t e;
        ctx->mh_sum = false;
        if ((e = launch_line_mean(pr, m, ctx->laFH, ctx->laBH, ctx->lSH, ctx->bT, ctx->MV, ctx->MH,
                                  ctx->ly, nullptr, 0, 0, &ctx->dstat[0].flags, s)) != cudaSuccess)
            return e;
        if ((e = launch_transpose(pr, m, ctx->MH, ctx->MHt, s)) != cudaSuccess) return e;
        if ((e = launch_line_mean(pr, m, ctx->laFV, ctx->laBV, ctx->lSV, ctx->lbT, ctx->MHt,
                                  ctx->MVt, ctx->ly, x, 1, 0, &ctx->dstat[0].flags, s)) != cudaSuccess)
            return e;
        return launch_transpose(pr, m, ctx->MVt, ctx->MV, s);
    }
    if (ctx->lines_m > 0) {
        // Algorithm 2 over the rows (natural order), then the columns (transposed order)
        const int m = ctx->lines_m, pr = ctx->prec;
        ctx->mh_sum = false;
        unsigned *fl = &ctx->dstat[0].flags;
        cudaError_t e;
        if ((e = launch_line_phase(pr, m, lsH, luH, ctx->diagT, ctx->bT, ctx->LV,
                                   ctx->MV, ctx->LH, ctx->MH, ctx->lf, ctx->ly, nullptr, 0, fl, s)) != cudaSuccess)
            return e;
        if ((e = launch_transpose(pr, m, ctx->LH, ctx->LHt, s)) != cudaSuccess) return e;
        if ((e = launch_transpose(pr, m, ctx->MH, ctx->MHt, s)) != cudaSuccess) return e;
        if ((e = launch_line_phase(pr, m, lsV, luV, ctx->ldiagT, ctx->lbT, ctx->LHt,
                                   ctx->MHt, ctx->LVt, ctx->MVt, ctx->lf, ctx->ly, x, 1, fl, s)) != cudaSuccess)
            return e;
        if ((e = launch_transpose(pr, m, ctx->LVt, ctx->LV, s)) != cudaSuccess) return e;
        return launch_transpose(pr, m, ctx->MVt, ctx->MV, s);
    }
    if (ctx->parity) {
        const unsigned zp = ctx->zero_pending;
        ctx->zero_pending = 0;
        for (size_t j = 0; j < ctx->phases.size(); ++j) {
            const PhaseClasses &ph = ctx->phases[j];
            if (ph.nq == 0) continue;
            // classes of the colours after this phase: they have not sent in this sweep
            unsigned later = 0;
            for (size_t k = j + 1; k < ctx->phases.size(); ++k)
                for (int t = 0; t < ctx->phases[k].nq; ++t) later |= 1u << ctx->phases[k].q[t];
            // frozen precision messages: the gains and the frozen aggregates P
            // (in P[0]) stand for the coefficients and the diagonal
            const bool fz = ctx->frozen;
            cudaError_t e = launch_sweep_parity(
                ctx->pg, ph, ctx->prec, fz ? ctx->g : (transposed ? ctx->paT : ctx->pa), fz ? nullptr : ctx->pc,
                fz ? ctx->P[0] : ctx->diagT, ctx->bT, ctx->Lm[c0], ctx->Mm[c0], x, &ctx->dstat[0].flags,
                (zp & 1u) ? later : 0u, (zp & 2u) ? later : 0u, fz ? 1 : 0, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (ctx->ncolors > 0) {
        for (int c = 0; c < ctx->ncolors; ++c) {
            cudaError_t e = launch_sweep_color(ctx->L, ctx->prec, ctx->color, c,
                                               ctx->has_masks ? &ctx->masks : nullptr,
                                               transposed ? ctx->aT : ctx->a, ctx->c, ctx->Lm[c0],
                                               ctx->Mm[c0], ctx->P[c0], ctx->B[c0], x,
                                               &ctx->dstat[0].flags, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (ctx->frozen) {
        ctx->cur = c1;
        return launch_sweep_mean(ctx->L, ctx->prec, ctx->g, ctx->bT, ctx->P[c0], ctx->Mm[c0],
                                 ctx->B[c0], ctx->Mm[c1], ctx->B[c1], x, block_of(ctx),
                                 &ctx->dstat[0].flags, s);
    }
    SweepArgs a;
    a.n = ctx->n;
    a.a = transposed ? ctx->aT : ctx->a;
    a.c = ctx->c;
    a.diag = ctx->diagT;
    a.b = ctx->bT;
    a.Lin = ctx->Lm[c0];
    a.Min = ctx->Mm[c0];
    a.Pin = ctx->P[c0];
    a.Bin = ctx->B[c0];
    a.Lout = ctx->Lm[c1];
    a.Mout = ctx->Mm[c1];
    a.Pout = ctx->P[c1];
    a.Bout = ctx->B[c1];
    a.x = x;
    a.flags = &ctx->dstat[0].flags;
    ctx->cur = c1;
    return launch_sweep(ctx->L, ctx->prec, a, block_of(ctx), s);
}

// k sweeps (beliefs of the last into xbuf), residual of (bres, xbuf) into
// dstat[0], status copy to the pinned host mirror.
cudaError_t enqueue_chunk(gabp_ctx *ctx, int k, bool transposed, cudaStream_t s)
{
    cudaError_t e;
    for (int i = 0; i < k; ++i)
        if ((e = sweep_once(ctx, transposed, i == k - 1 ? ctx->xbuf : nullptr, s)) != cudaSuccess)
            return e;
    if ((e = cudaMemsetAsync(ctx->dstat, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if ((e = launch_residual(ctx->L, transposed ? ctx->aT64 : ctx->a64, ctx->diag64, ctx->bres,
                             ctx->xbuf, nullptr, &ctx->dstat[0], s)) != cudaSuccess)
        return e;
    return cudaMemcpyAsync(ctx->hstat, ctx->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
}

gabp_status run_chunk(gabp_ctx *ctx, int k, bool transposed)
{
    if (!ctx->opt.use_graphs) {
        CK(enqueue_chunk(ctx, k, transposed, ctx->stream));
    } else {
        const int parity = ctx->cur, frozen = ctx->frozen ? 1 : 0;
        cudaGraphExec_t exec = nullptr;
        for (auto &g : ctx->graphs)
            if (g.k == k && g.parity == parity && g.transposed == (int)transposed && g.frozen == frozen)
                exec = g.exec;
        if (!exec) {
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = enqueue_chunk(ctx, k, transposed, ctx->cap_stream);
            cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &graph);
            ctx->cur = parity;
            if (e != cudaSuccess) return fail_cuda(e, "chunk capture");
            if (e2 != cudaSuccess) return fail_cuda(e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return fail_cuda(e, "cudaGraphInstantiate");
            ctx->graphs.push_back({k, parity, (int)transposed, frozen, exec});
        }
        CK(cudaGraphLaunch(exec, ctx->stream));
        ctx->mh_sum = false;  // a chunk's last sweep writes the beliefs
        int per_sweep = ctx->ncolors > 0 ? ctx->ncolors : 1;
        if (ctx->lines_m > 0)
            per_sweep = !ctx->frozen ? 6 : (line_cols_natural(ctx->prec, ctx->lines_m) ? 2 : 4);
        if (ctx->parity) {
            per_sweep = 0;
            for (const PhaseClasses &ph : ctx->phases) per_sweep += ph.nq > 0 ? 1 : 0;
        }
        count_launches(ctx->stream, (unsigned long long)k * per_sweep + 1);  // sweeps + residual
        const bool in_place = ctx->ncolors > 0 || ctx->lines_m > 0;
        ctx->cur = in_place ? parity : parity ^ (k & 1);
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return GABP_OK;
}

gabp_status read_status(gabp_ctx *ctx, int which, double *rinf, double *binf, unsigned *flags)
{
    CK(cudaMemcpyAsync(ctx->hstat + which, ctx->dstat + which, sizeof(DevStatus),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (rinf) *rinf = bits_to_double(ctx->hstat[which].rmax);
    if (binf) *binf = bits_to_double(ctx->hstat[which].bmax);
    if (flags) *flags = ctx->hstat[which].flags;
    return GABP_OK;
}

gabp_status ensure_parity_transpose(gabp_ctx *ctx)
{
    if (!ctx->parity || !ctx->aT) return GABP_OK;
    if (!ctx->paT) CKS(dalloc(ctx, &ctx->paT, (size_t)ctx->L.slots * esz(ctx->prec)));
    CK(launch_parity_convert(ctx->pg, ctx->prec, 1, ctx->aT, ctx->paT, ctx->stream));
    return GABP_OK;
}

gabp_status ensure_transpose(gabp_ctx *ctx)
{
    if (ctx->aT) {
        if (ctx->parity && !ctx->paT) CKS(ensure_parity_transpose(ctx));
        return GABP_OK;
    }
    const size_t S = (size_t)ctx->L.slots;
    CKS(dalloc(ctx, (void **)&ctx->aT64, S * sizeof(double)));
    CK(launch_transpose_coeffs(ctx->L, 0, ctx->a64, ctx->aT64, ctx->stream));
    if (ctx->prec == 0) {
        ctx->aT = ctx->aT64;
    } else {
        CKS(dalloc(ctx, &ctx->aT, S * sizeof(float)));
        CK(launch_transpose_coeffs(ctx->L, 1, ctx->a, ctx->aT, ctx->stream));
    }
    return ensure_parity_transpose(ctx);
}

gabp_status ensure_ir(gabp_ctx *ctx)
{
    if (ctx->b0) return GABP_OK;
    const size_t nb = (size_t)ctx->n * sizeof(double);
    CKS(dalloc(ctx, (void **)&ctx->b0, nb));
    CKS(dalloc(ctx, (void **)&ctx->xacc, nb));
    CKS(dalloc(ctx, (void **)&ctx->rbuf, nb));
    return GABP_OK;
}

// Freezes the precision messages at the current state: g = a / (P_s - L[rev]),
// both L buffers and both P buffers set to the current ones.
gabp_status freeze(gabp_ctx *ctx, bool transposed)
{
    const size_t S = (size_t)ctx->L.slots * esz(ctx->prec), NB = (size_t)ctx->n * esz(ctx->prec);
    if (!ctx->g) CKS(dalloc(ctx, &ctx->g, S));
    const int c0 = ctx->cur, c1 = c0 ^ 1;
    CK(launch_freeze(ctx->L, ctx->prec, transposed ? ctx->aT : ctx->a, ctx->P[c0], ctx->Lm[c0],
                     ctx->g, &ctx->dstat[0].flags, ctx->stream));
    CK(cudaMemcpyAsync(ctx->Lm[c1], ctx->Lm[c0], S, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->P[c1], ctx->P[c0], NB, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->frozen = true;
    ctx->frozen_transposed = transposed;
    return GABP_OK;
}

// Line schedule: the multipliers of both families from the current
// precision messages (the row family sees LV, the column family LH).
gabp_status freeze_lines(gabp_ctx *ctx, bool transposed)
{
    const int m = ctx->lines_m, pr = ctx->prec;
    const size_t nb = (size_t)ctx->n * esz(pr);
    void **bufs[] = {&ctx->laFH, &ctx->laBH, &ctx->lSH, &ctx->laFV, &ctx->laBV, &ctx->lSV};
    for (void **bp : bufs)
        if (!*bp) CKS(dalloc(ctx, bp, nb));
    cudaStream_t s = ctx->stream;
    unsigned *fl = &ctx->dstat[0].flags;
    CK(launch_line_freeze(pr, m, transposed ? ctx->lsubHT : ctx->lsubH,
                          transposed ? ctx->lsupHT : ctx->lsupH, ctx->diagT, ctx->LV, ctx->lf,
                          ctx->ly, ctx->laFH, ctx->laBH, ctx->lSH, fl, s));
    CK(launch_transpose(pr, m, ctx->LH, ctx->LHt, s));
    CK(launch_line_freeze(pr, m, transposed ? ctx->lsubVT : ctx->lsubV,
                          transposed ? ctx->lsupVT : ctx->lsupV, ctx->ldiagT, ctx->LHt, ctx->lf,
                          ctx->ly, ctx->laFV, ctx->laBV, ctx->lSV, fl, s));
    if (line_cols_natural(pr, m)) {
        // the column family's coefficients in natural order, for the transpose-free frozen sweep
        void **nbufs[] = {&ctx->laFVn, &ctx->laBVn, &ctx->lSVn};
        for (void **bp : nbufs)
            if (!*bp) CKS(dalloc(ctx, bp, nb));
        CK(launch_transpose(pr, m, ctx->laFV, ctx->laFVn, s));
        CK(launch_transpose(pr, m, ctx->laBV, ctx->laBVn, s));
        CK(launch_transpose(pr, m, ctx->lSV, ctx->lSVn, s));
    }
    ctx->frozen = true;
    return GABP_OK;
}

// Line schedule: freezes once the precision messages of both families moved
// by at most `rel` times their largest value since the previous check.
gabp_status maybe_freeze_lines(gabp_ctx *ctx, double rel, bool transposed)
{
    const int64_t n = ctx->n;
    const size_t nb = (size_t)n * esz(ctx->prec);
    if (!ctx->lprevH) CKS(dalloc(ctx, &ctx->lprevH, nb));
    if (!ctx->lprevV) CKS(dalloc(ctx, &ctx->lprevV, nb));
    if (ctx->lprev_valid) {
        CK(cudaMemsetAsync(&ctx->dstat[2], 0, sizeof(DevStatus), ctx->stream));
        CK(launch_lambda_change(n, ctx->prec, ctx->lprevH, ctx->LH, &ctx->dstat[2], ctx->stream));
        CK(launch_lambda_change(n, ctx->prec, ctx->lprevV, ctx->LV, &ctx->dstat[2], ctx->stream));
        double dmax = 0.0, lmax = 0.0;
        unsigned fl = 0;
        CKS(read_status(ctx, 2, &dmax, &lmax, &fl));
        if (!(fl & FLAG_NAN) && dmax <= rel * lmax) return freeze_lines(ctx, transposed);
    }
    CK(cudaMemcpyAsync(ctx->lprevH, ctx->LH, nb, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->lprevV, ctx->LV, nb, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->lprev_valid = true;
    return GABP_OK;
}

// Parity-class layout (coloured schedule in place): the gains of every
// outgoing slot and the aggregates P from the current precision messages.
gabp_status freeze_parity(gabp_ctx *ctx, bool transposed)
{
    if (!ctx->g) CKS(dalloc(ctx, &ctx->g, (size_t)ctx->L.slots * esz(ctx->prec)));
    CK(launch_freeze_parity(ctx->pg, ctx->prec, transposed ? ctx->paT : ctx->pa, ctx->diagT, ctx->Lm[ctx->cur],
                            ctx->g, ctx->P[0], &ctx->dstat[0].flags, ctx->stream));
    ctx->frozen = true;
    return GABP_OK;
}

// Parity-class layout: freezes once the precision messages moved by at most
// `rel` times their largest value since the previous check (the update is in
// place, so the previous state is a copy taken at that check).
gabp_status maybe_freeze_parity(gabp_ctx *ctx, double rel, bool transposed)
{
    const size_t S = (size_t)ctx->L.slots * esz(ctx->prec);
    if (!ctx->pprevL) CKS(dalloc(ctx, &ctx->pprevL, S));
    if (ctx->lprev_valid) {
        CK(cudaMemsetAsync(&ctx->dstat[2], 0, sizeof(DevStatus), ctx->stream));
        CK(launch_lambda_change(ctx->L.slots, ctx->prec, ctx->pprevL, ctx->Lm[ctx->cur], &ctx->dstat[2],
                                ctx->stream));
        double dmax = 0.0, lmax = 0.0;
        unsigned fl = 0;
        CKS(read_status(ctx, 2, &dmax, &lmax, &fl));
        if (!(fl & FLAG_NAN) && dmax <= rel * lmax) return freeze_parity(ctx, transposed);
    }
    CK(cudaMemcpyAsync(ctx->pprevL, ctx->Lm[ctx->cur], S, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->lprev_valid = true;
    return GABP_OK;
}

// Freezes once the last sweep changed no precision message by more than
// `rel` times the largest one (rounding level).
gabp_status maybe_freeze(gabp_ctx *ctx, bool transposed)
{
    if (ctx->frozen) return GABP_OK;
    if (ctx->lines_m > 0) return maybe_freeze_lines(ctx, ctx->prec == 0 ? 1e-14 : 1e-6, transposed);
    if (ctx->parity) return maybe_freeze_parity(ctx, ctx->prec == 0 ? 1e-14 : 1e-6, transposed);
    const double rel = ctx->prec == 0 ? 1e-14 : 1e-6;
    CK(cudaMemsetAsync(&ctx->dstat[2], 0, sizeof(DevStatus), ctx->stream));
    CK(launch_lambda_change(ctx->L.slots, ctx->prec, ctx->Lm[ctx->cur ^ 1], ctx->Lm[ctx->cur],
                            &ctx->dstat[2], ctx->stream));
    double dmax = 0.0, lmax = 0.0;
    unsigned fl = 0;
    CKS(read_status(ctx, 2, &dmax, &lmax, &fl));
    if (!(fl & FLAG_NAN) && dmax <= rel * lmax) CKS(freeze(ctx, transposed));
    return GABP_OK;
}

#ifndef GABP_FREEZE_PROBE
#define GABP_FREEZE_PROBE 5
#endif
// Sweeps per chunk while the precision messages may still freeze: a freeze is
// decided at the end of a chunk, so shorter chunks stop the full sweeps sooner
// after the messages have converged (0: the check interval throughout).
int chunk_before_freeze(const gabp_ctx *ctx, int every)
{
    if (GABP_FREEZE_PROBE <= 0 || ctx->frozen || !freeze_enabled(ctx)) return every;
    return std::min(every, GABP_FREEZE_PROBE);
}

bool freeze_enabled(const gabp_ctx *ctx)
{
    // frozen sweeps: flood, line and coloured (parity-class layout) schedules
    if (ctx->ncolors > 0 && !ctx->parity) return false;
    if (ctx->opt.freeze_lambda < 0) return ctx->opt.precision == GABP_FP32_IR;
    return ctx->opt.freeze_lambda > 0;
}

// Plain GaBP solve (Algorithm 1, flood schedule) on A or A^T.
gabp_status solve_plain(gabp_ctx *ctx, const double *b, double *x, double tol, int max_iter,
                        int *iters, double *relres, bool transposed)
{
    const int64_t n = ctx->n;
    CKS(load_rhs(ctx, b));
    CKS(zero_messages(ctx, true, true));
    CKS(aggregate(ctx));
    CK(cudaMemsetAsync(ctx->dstat, 0, sizeof(DevStatus), ctx->stream));
    // ||b||_inf (residual of x = 0)
    CK(cudaMemsetAsync(ctx->xbuf, 0, n * sizeof(double), ctx->stream));
    CK(launch_residual(ctx->L, ctx->a64, ctx->diag64, ctx->bres, ctx->xbuf, nullptr, &ctx->dstat[0], ctx->stream));
    double binf = 0.0;
    CKS(read_status(ctx, 0, nullptr, &binf, nullptr));
    int it = 0;
    double rr = 0.0;
    gabp_status st = GABP_E_NOT_CONVERGED;
    if (binf == 0.0) {
        st = GABP_OK;
    } else {
        const int every = std::max(1, ctx->opt.check_every);
        while (it < max_iter) {
            const int k = std::min(chunk_before_freeze(ctx, every), max_iter - it);
            CKS(run_chunk(ctx, k, transposed));
            it += k;
            const DevStatus h = ctx->hstat[0];
            if (h.flags & FLAG_INDEX) { st = index_error(h.flags); break; }
            if (freeze_enabled(ctx) && !(h.flags & FLAG_BREAKDOWN)) CKS(maybe_freeze(ctx, transposed));
            rr = bits_to_double(h.rmax) / binf;
            if (h.flags & FLAG_BREAKDOWN) { st = fail(GABP_E_BREAKDOWN, "zero or non-finite message denominator"); break; }
            if ((h.flags & FLAG_NAN) || !std::isfinite(rr) || rr > kDivergence) { st = fail(GABP_E_DIVERGED, "residual diverged"); break; }
            if (rr <= tol) { st = GABP_OK; break; }
        }
        if (st == GABP_E_NOT_CONVERGED) fail(st, "iteration cap reached");
    }
    CKS(store_vector(ctx, ctx->xbuf, x, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (iters) *iters = it;
    if (relres) *relres = rr;
    return st;
}

// Float GaBP inside double iterative refinement (on A, or on A^T).
gabp_status solve_ir(gabp_ctx *ctx, const double *b, double *x, double tol, int max_iter,
                     int *iters, double *relres, bool transposed)
{
    const double *A64 = transposed ? ctx->aT64 : ctx->a64;
    const int64_t n = ctx->n;
    const size_t nb = n * sizeof(double);
    CKS(ensure_ir(ctx));
    cudaStream_t s = ctx->stream;
    if (ctx->reordered) CK(launch_permute((int)n, ctx->d_perm, b, ctx->b0, 0, s));
    else CK(cudaMemcpyAsync(ctx->b0, b, nb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(ctx->xacc, 0, nb, s));
    CK(cudaMemsetAsync(ctx->dstat, 0, 2 * sizeof(DevStatus), s));
    // r = b, s = ||b||
    CK(launch_residual(ctx->L, A64, ctx->diag64, ctx->b0, ctx->xacc, ctx->rbuf, &ctx->dstat[1], s));
    double bn = 0.0;
    CKS(read_status(ctx, 1, nullptr, &bn, nullptr));
    int total = 0;
    double rr = bn == 0.0 ? 0.0 : 1.0;
    gabp_status st = GABP_E_NOT_CONVERGED;
    CKS(zero_messages(ctx, true, true));
    const int every = std::max(1, ctx->opt.check_every);
    // float sweeps per refinement step: a restarted solve re-uses GaBP's fast initial
    // phase, which is shorter for line and coloured GaBP (measured on the 2048^2
    // workload: 400 sweeps per step for the flood schedule, 150 for lines and red-black)
    const int inner_max = ctx->opt.ir_inner_max > 0 ? ctx->opt.ir_inner_max
                                                    : (ctx->lines_m > 0 || ctx->ncolors > 0 ? 150 : 400);
    const double inner_tol = ctx->opt.ir_inner_tol > 0 ? ctx->opt.ir_inner_tol : 1e-3;
    if (bn == 0.0) st = GABP_OK;
    for (int outer = 0; st == GABP_E_NOT_CONVERGED && outer < 200 && total < max_iter; ++outer) {
        // inner problem A e = r / ||r||: double copy for the checks, float copy for the sweeps
        CK(launch_scale_rhs(ctx->rbuf, &ctx->dstat[1], ctx->bres, ctx->bT, ctx->prec, n, s));
        if (ctx->lines_m > 0) CK(launch_transpose(ctx->prec, ctx->lines_m, ctx->bT, ctx->lbT, s));
        CKS(zero_messages(ctx, false, true));  // tilde-Lambda kept warm
        CKS(aggregate(ctx));
        int inner = 0;
        while (inner < inner_max && total < max_iter) {
            const int k = std::min(std::min(chunk_before_freeze(ctx, every), inner_max - inner), max_iter - total);
            CKS(run_chunk(ctx, k, transposed));
            inner += k;
            total += k;
            const DevStatus h = ctx->hstat[0];
            if (h.flags & FLAG_INDEX) { st = index_error(h.flags); break; }
            if (freeze_enabled(ctx) && !(h.flags & FLAG_BREAKDOWN)) CKS(maybe_freeze(ctx, transposed));
            if (h.flags & FLAG_BREAKDOWN) { st = fail(GABP_E_BREAKDOWN, "zero or non-finite message denominator"); break; }
            const double rin = bits_to_double(h.rmax);  // ||r/s||_inf == 1
            if ((h.flags & FLAG_NAN) || !std::isfinite(rin)) { st = fail(GABP_E_DIVERGED, "inner residual not finite"); break; }
            if (rin <= inner_tol) break;
        }
        if (st != GABP_E_NOT_CONVERGED) break;
        // x += s e;  r = b - A x;  s = ||r||
        CK(launch_axpy_status(ctx->xacc, ctx->xbuf, &ctx->dstat[1], n, s));
        CK(cudaMemsetAsync(&ctx->dstat[1], 0, 2 * sizeof(unsigned long long), s));
        CK(launch_residual(ctx->L, A64, ctx->diag64, ctx->b0, ctx->xacc, ctx->rbuf, &ctx->dstat[1], s));
        double rinf = 0.0;
        unsigned fl = 0;
        CKS(read_status(ctx, 1, &rinf, nullptr, &fl));
        if (fl & FLAG_INDEX) { st = index_error(fl); break; }
        rr = rinf / bn;
        if ((fl & FLAG_NAN) || !std::isfinite(rr) || rr > kDivergence) { st = fail(GABP_E_DIVERGED, "residual diverged"); break; }
        if (rr <= tol) st = GABP_OK;
    }
    if (st == GABP_E_NOT_CONVERGED) fail(st, "iteration cap reached");
    CKS(store_vector(ctx, ctx->xacc, x, s));
    CK(cudaStreamSynchronize(s));
    if (iters) *iters = total;
    if (relres) *relres = rr;
    return st;
}

}  // namespace gabp
