// The batched persistent solver's front end: batch set-up, the autotuner,
// the captured launch and the per-system results.
#include "host.h"

#define GABP_BATCH_RES_ITERS(h, i) (((int *)((char *)(h) + (i) * batch_result_bytes()))[0])
#define GABP_BATCH_RES_STATUS(h, i) (((int *)((char *)(h) + (i) * batch_result_bytes()))[1])
#define GABP_BATCH_RES_RR(h, i) (*(double *)((char *)(h) + (i) * batch_result_bytes() + 8))

// ---------------------------------------------------------------------------
// Batched persistent solver
// ---------------------------------------------------------------------------
void gabp_batch_destroy(gabp_batch *bt)
{
    if (!bt) return;
    cudaSetDevice(bt->dev);
    if (bt->stream) cudaStreamSynchronize(bt->stream);
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    free_all(bt->allocs);
    if (bt->h_b) cudaFreeHost((void *)bt->h_b);
    if (bt->h_x) cudaFreeHost(bt->h_x);
    if (bt->h_res) cudaFreeHost(bt->h_res);
    if (bt->cap_stream) cudaStreamDestroy(bt->cap_stream);
    if (bt->ev0) cudaEventDestroy(bt->ev0);
    if (bt->ev1) cudaEventDestroy(bt->ev1);
    delete bt;
}

gabp_status gabp_batch_setup(int nsys, gabp_ctx *const *systems, int check_every, void *stream,
                             gabp_batch **out)
{
    if (!out) return fail(GABP_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nsys < 1 || !systems || check_every < 0) return fail(GABP_E_INVALID_ARG, "bad argument");
    for (int i = 0; i < nsys; ++i) {
        const gabp_ctx *c = systems[i];
        if (!c) return fail(GABP_E_INVALID_ARG, "null system context");
        if (c->L.kind != GABP_LAYOUT_STENCIL) return fail(GABP_E_INVALID_ARG, "batched systems need the stencil layout");
        if (c->opt.precision != systems[0]->opt.precision || c->L.sp.K != systems[0]->L.sp.K ||
            c->dev != systems[0]->dev)
            return fail(GABP_E_INVALID_ARG, "batched systems need one precision, one diagonal count, one device");
        if (c->L.sp.K > 8) return fail(GABP_E_INVALID_ARG, "batched systems need at most 8 off-diagonal diagonals");
    }
    gabp_batch *bt = new (std::nothrow) gabp_batch;
    if (!bt) return fail(GABP_E_OOM, "host allocation");
    auto bail = [&](gabp_status st) {
        gabp_batch_destroy(bt);
        return st;
    };
    bt->dev = systems[0]->dev;
    gabp_status st;
    if ((st = set_dev(bt->dev)) != GABP_OK) return bail(st);
    bt->stream = (cudaStream_t)stream;
    bt->nsys = nsys;
    bt->prec = systems[0]->prec;
    bt->K = systems[0]->L.sp.K;
    bt->check_auto = check_every == 0;
    bt->check_every = check_every > 0 ? check_every : 10;
    bt->check_every0 = bt->check_every;
    bt->refine = systems[0]->opt.precision == GABP_FP32_IR ? 1 : 0;
    bt->inner_max = systems[0]->opt.ir_inner_max > 0 ? systems[0]->opt.ir_inner_max : 400;
    bt->inner_tol = systems[0]->opt.ir_inner_tol > 0 ? systems[0]->opt.ir_inner_tol : 1e-3;
    bt->freeze = freeze_enabled(systems[0]) ? 1 : 0;
    bt->sys.assign(systems, systems + nsys);
    cudaError_t e;
    if ((e = cudaDeviceGetAttribute(&bt->sms, cudaDevAttrMultiProcessorCount, bt->dev)) != cudaSuccess)
        return bail(fail_cuda(e, "cudaDeviceGetAttribute"));
    if ((e = cudaStreamCreateWithFlags(&bt->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(fail_cuda(e, "cudaStreamCreate"));
    if ((e = cudaEventCreate(&bt->ev0)) != cudaSuccess || (e = cudaEventCreate(&bt->ev1)) != cudaSuccess)
        return bail(fail_cuda(e, "cudaEventCreate"));
    const size_t dsz = batch_sys_bytes(bt->prec);
    std::vector<unsigned char> desc(dsz * nsys);
    for (int i = 0; i < nsys; ++i) {
        gabp_ctx *c = systems[i];
        if (!c->g) {
            if ((st = dalloc(c, &c->g, (size_t)c->L.slots * esz(c->prec))) != GABP_OK) return bail(st);
        }
        fill_batch_sys(bt->prec, desc.data() + i * dsz, c->n, c->L.sp, c->a, c->c, c->diagT, c->a64,
                       c->diag64, c->Lm, c->Mm, c->P, c->B, c->bT, c->xbuf, c->bres, c->g);
        c->frozen = false;  // the batch owns these buffers while it runs
    }
    std::vector<int> order(nsys);
    for (int i = 0; i < nsys; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return systems[x]->n > systems[y]->n; });
    if ((st = upload(bt, &bt->d_sys, desc.data(), desc.size())) != GABP_OK) return bail(st);
    if ((st = upload(bt, (void **)&bt->d_order, order.data(), order.size() * sizeof(int))) != GABP_OK) return bail(st);
    if ((st = dalloc(bt, (void **)&bt->d_queue, 2 * sizeof(int))) != GABP_OK) return bail(st);
    if ((st = dalloc(bt, (void **)&bt->d_b, nsys * sizeof(void *))) != GABP_OK) return bail(st);
    if ((st = dalloc(bt, (void **)&bt->d_x, nsys * sizeof(void *))) != GABP_OK) return bail(st);
    if ((st = dalloc(bt, &bt->d_res, nsys * batch_result_bytes())) != GABP_OK) return bail(st);
    if ((e = cudaMallocHost((void **)&bt->h_b, nsys * sizeof(void *))) != cudaSuccess ||
        (e = cudaMallocHost((void **)&bt->h_x, nsys * sizeof(void *))) != cudaSuccess ||
        (e = cudaMallocHost(&bt->h_res, nsys * batch_result_bytes())) != cudaSuccess)
        return bail(fail_cuda(e, "cudaMallocHost"));
    *out = bt;
    return GABP_OK;
}

namespace {

// Systems solved by whole clusters: those with at least min_rows rows per cluster thread.
int batch_nbig(const gabp_batch *bt, int block, int cs)
{
    const int64_t thr = (int64_t)bt->min_rows * block * cs;
    int nb = 0;
    for (auto *c : bt->sys)
        if (c->n >= thr) ++nb;
    return nb;  // systems are queued largest first
}

cudaError_t batch_enqueue(gabp_batch *bt, int block, int cs, int grid, double tol, int max_iter,
                          cudaStream_t s)
{
    const int nbig = batch_nbig(bt, block, cs);
    cudaError_t e;
    const size_t pb = (size_t)bt->nsys * sizeof(void *);
    if ((e = cudaMemcpyAsync((void *)bt->d_b, (const void *)bt->h_b, pb, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(bt->d_x, bt->h_x, pb, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bt->d_queue, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
    e = bt->prec == 0
            ? launch_batch<double>(bt->K, bt->rows, cs, grid, block, bt->d_sys, bt->d_order, bt->nsys, nbig,
                                   bt->d_b, bt->d_x, bt->d_queue, tol, max_iter, bt->check_every, bt->refine,
                                   bt->inner_tol, bt->inner_max, bt->freeze, bt->d_res, s)
            : launch_batch<float>(bt->K, bt->rows, cs, grid, block, bt->d_sys, bt->d_order, bt->nsys, nbig,
                                  bt->d_b, bt->d_x, bt->d_queue, tol, max_iter, bt->check_every, bt->refine,
                                  bt->inner_tol, bt->inner_max, bt->freeze, bt->d_res, s);
    if (e != cudaSuccess) return e;
    count_launches(s, 1);
    return cudaMemcpyAsync(bt->h_res, bt->d_res, (size_t)bt->nsys * batch_result_bytes(),
                           cudaMemcpyDeviceToHost, s);
}

gabp_status batch_stage(gabp_batch *bt, const double *const *b, double *const *x)
{
    if (!b || !x) return fail(GABP_E_INVALID_ARG, "null pointer table");
    for (int i = 0; i < bt->nsys; ++i) {
        if ((!b[i] || !x[i]) && bt->sys[i]->n > 0) return fail(GABP_E_INVALID_ARG, "null system vector");
        bt->h_b[i] = b[i];
        bt->h_x[i] = x[i];
    }
    return GABP_OK;
}

}  // namespace

static int batch_clusters(const gabp_batch *bt, int cs, int blk)
{
    return bt->prec == 0 ? batch_max_clusters<double>(bt->K, bt->rows, cs, blk)
                         : batch_max_clusters<float>(bt->K, bt->rows, cs, blk);
}

static gabp_status batch_set_shape(gabp_batch *bt, int blk, int cs)
{
    const int nc = batch_clusters(bt, cs, blk);
    if (nc < 1) return fail(GABP_E_INVALID_ARG, "launch shape does not fit the batched kernel");
    const int grid = nc * cs;  // every cluster resident: a persistent launch
    if (bt->exec && (bt->block != blk || bt->cs != cs || bt->grid != grid)) {
        cudaGraphExecDestroy(bt->exec);
        bt->exec = nullptr;
    }
    bt->block = blk;
    bt->cs = cs;
    bt->grid = grid;
    bt->nbig = batch_nbig(bt, blk, cs);
    return GABP_OK;
}

gabp_status gabp_batch_set_shape(gabp_batch *bt, int block, int cluster)
{
    if (!bt || (block != 256 && block != 512) ||
        !(cluster == 1 || cluster == 2 || cluster == 4 || cluster == 8 || cluster == 16))
        return fail(GABP_E_INVALID_ARG, "block must be 256 or 512, cluster 1, 2, 4, 8 or 16");
    CKS(set_dev(bt->dev));
    return batch_set_shape(bt, block, cluster);
}

gabp_status gabp_batch_set_params(gabp_batch *bt, int rows, int min_rows, int check_every)
{
    if (!bt || rows < 0 || min_rows < 0 || check_every < 0) return fail(GABP_E_INVALID_ARG, "bad argument");
    if (rows > 0 && !batch_rows_supported(bt->K, rows))
        return fail(GABP_E_INVALID_ARG, "rows in flight: 1, or 2 for 5- and 9-point systems");
    CKS(set_dev(bt->dev));
    if (bt->exec) {
        cudaGraphExecDestroy(bt->exec);
        bt->exec = nullptr;
    }
    if (rows > 0) bt->rows = rows;
    if (min_rows > 0) bt->min_rows = min_rows;
    if (check_every > 0) bt->check_every = check_every;
    if (bt->block > 0) return batch_set_shape(bt, bt->block, bt->cs);  // resident clusters may change
    return GABP_OK;
}

gabp_status gabp_batch_params(gabp_batch *bt, int *rows, int *min_rows, int *check_every)
{
    if (!bt) return fail(GABP_E_INVALID_ARG, "null batch");
    if (rows) *rows = bt->rows;
    if (min_rows) *min_rows = bt->min_rows;
    if (check_every) *check_every = bt->check_every;
    return GABP_OK;
}

// One timed solve of the staged batch with the current parameters and shape
// (blk, cs); a negative time when the shape does not fit.
static gabp_status batch_trial(gabp_batch *bt, int blk, int cs, double tol, int max_iter, float *ms)
{
    *ms = -1.0f;
    const int nc = batch_clusters(bt, cs, blk);
    if (nc < 1) return GABP_OK;
    const int save_block = bt->block, save_cs = bt->cs;
    bt->block = blk;  // batch_nbig reads the parameters of the shape being tried
    bt->cs = cs;
    CK(cudaEventRecord(bt->ev0, bt->stream));
    cudaError_t e = batch_enqueue(bt, blk, cs, nc * cs, tol, max_iter, bt->stream);
    bt->block = save_block;
    bt->cs = save_cs;
    if (e != cudaSuccess) return fail_cuda(e, "batch trial");
    CK(cudaEventRecord(bt->ev1, bt->stream));
    CK(cudaEventSynchronize(bt->ev1));
    CK(cudaEventElapsedTime(ms, bt->ev0, bt->ev1));
    return GABP_OK;
}

gabp_status gabp_batch_tune(gabp_batch *bt, const double *const *b, double *const *x, double tol,
                            int max_iter, int *block, int *cluster)
{
    if (!bt || max_iter < 1 || !(tol >= 0.0)) return fail(GABP_E_INVALID_ARG, "bad argument");
    CKS(set_dev(bt->dev));
    CKS(batch_stage(bt, b, x));
    if (bt->exec) {
        cudaGraphExecDestroy(bt->exec);
        bt->exec = nullptr;
    }
    // stage 1: block size x cluster size, one row in flight, the setup's check interval
    bt->rows = 1;
    bt->min_rows = 4;
    bt->check_every = bt->check_every0;
    const int blocks[] = {256, 512};
    const int clusters[] = {1, 2, 4, 8, 16};  // 16: non-portable cluster size, where it fits
    // the two fastest shapes go on to stage 2: its parameters can reorder them
    float best = -1.0f, second = -1.0f, ms = 0.0f;
    int bb = 0, bc = 0, sb = 0, sc = 0;
    for (int blk : blocks)
        for (int cs : clusters) {
            CKS(batch_trial(bt, blk, cs, tol, max_iter, &ms));
            if (ms < 0.0f) continue;
            if (best < 0.0f || ms < best) {
                second = best;
                sb = bb;
                sc = bc;
                best = ms;
                bb = blk;
                bc = cs;
            } else if (second < 0.0f || ms < second) {
                second = ms;
                sb = blk;
                sc = cs;
            }
        }
    if (best < 0.0f) return fail(GABP_E_CUDA, "no launch shape fits the batched kernel");
    // stage 2: rows in flight per thread (the edges per thread of a mean sweep are
    // rows x diagonals) and, with clusters, the rows per cluster thread from which a
    // system takes a whole cluster, on each of the two shapes
    int br = 1, bm = 4;
    const int rows_try[] = {1, 2}, minr_try[] = {2, 4, 8};
    const int shapes[2][2] = {{bb, bc}, {sb, sc}};
    const int nshapes = second < 0.0f ? 1 : 2;
    int fb = bb, fc = bc;
    for (int k = 0; k < nshapes; ++k) {
        const int blk = shapes[k][0], cs = shapes[k][1];
        for (int r : rows_try) {
            if (!batch_rows_supported(bt->K, r)) continue;
            for (int mr : minr_try) {
                if (cs == 1 && mr != 4) continue;     // no cluster teams: the threshold does not matter
                if (k == 0 && r == 1 && mr == 4) continue;  // stage 1's setting of the best shape
                bt->rows = r;
                bt->min_rows = mr;
                CKS(batch_trial(bt, blk, cs, tol, max_iter, &ms));
                if (ms >= 0.0f && ms < best) {
                    best = ms;
                    br = r;
                    bm = mr;
                    fb = blk;
                    fc = cs;
                }
            }
        }
    }
    bb = fb;
    bc = fc;
    bt->rows = br;
    bt->min_rows = bm;
    // stage 3 (only for a batch set up with a tuned check interval): residual checks
    // half as often (each check is a residual pass and team reductions; a system may
    // then run up to that many sweeps past its tolerance)
    int bce = bt->check_every0;
    if (bt->check_auto) {
        bt->check_every = 2 * bt->check_every0;
        CKS(batch_trial(bt, bb, bc, tol, max_iter, &ms));
        if (ms >= 0.0f && ms < best) {
            best = ms;
            bce = bt->check_every;
        }
    }
    bt->check_every = bce;
    CKS(batch_set_shape(bt, bb, bc));
    if (block) *block = bb;
    if (cluster) *cluster = bc;
    return GABP_OK;
}

gabp_status gabp_batch_solve(gabp_batch *bt, const double *const *b, double *const *x, double tol,
                             int max_iter, int *iters, double *relres, int *status)
{
    if (!bt || max_iter < 0 || !(tol >= 0.0)) return fail(GABP_E_INVALID_ARG, "bad argument");
    CKS(set_dev(bt->dev));
    CKS(batch_stage(bt, b, x));
    if (bt->block == 0) CKS(gabp_batch_tune(bt, b, x, tol, max_iter, nullptr, nullptr));
    if (!bt->exec || bt->g_tol != tol || bt->g_max_iter != max_iter) {
        if (bt->exec) {
            cudaGraphExecDestroy(bt->exec);
            bt->exec = nullptr;
        }
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(bt->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = batch_enqueue(bt, bt->block, bt->cs, bt->grid, tol, max_iter, bt->cap_stream);
        cudaError_t e2 = cudaStreamEndCapture(bt->cap_stream, &graph);
        if (e != cudaSuccess) return fail_cuda(e, "batch capture");
        if (e2 != cudaSuccess) return fail_cuda(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&bt->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail_cuda(e, "cudaGraphInstantiate");
        bt->g_tol = tol;
        bt->g_max_iter = max_iter;
    }
    CK(cudaGraphLaunch(bt->exec, bt->stream));
    count_launches(bt->stream, 1);
    CK(cudaStreamSynchronize(bt->stream));
    gabp_status worst = GABP_OK;
    for (int i = 0; i < bt->nsys; ++i) {
        const int st = GABP_BATCH_RES_STATUS(bt->h_res, i);
        if (iters) iters[i] = GABP_BATCH_RES_ITERS(bt->h_res, i);
        if (relres) relres[i] = GABP_BATCH_RES_RR(bt->h_res, i);
        if (status) status[i] = st;
        if (st != GABP_OK && (worst == GABP_OK || st == GABP_E_BREAKDOWN || st == GABP_E_DIVERGED))
            worst = (gabp_status)st;
    }
    if (worst != GABP_OK) fail(worst, "some batched systems did not converge (see status[])");
    return worst;
}

gabp_status gabp_batch_info(gabp_batch *bt, int *block, int *cluster, int *grid)
{
    if (!bt) return fail(GABP_E_INVALID_ARG, "null batch");
    if (block) *block = bt->block;
    if (cluster) *cluster = bt->cs;
    if (grid) *grid = bt->grid;
    return GABP_OK;
}
