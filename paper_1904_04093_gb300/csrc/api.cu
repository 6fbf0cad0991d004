// C ABI of the GaBP library: context set-up, solve drivers, multigrid.
// The declarations and their contracts are in include/gabp.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gabp_internal.h"

using namespace gabp;

namespace {

thread_local std::string g_last_error;

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

#define CK(call)                                            \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return fail_cuda(e_, #call); \
    } while (0)

#define CKS(expr)                            \
    do {                                     \
        gabp_status s_ = (expr);             \
        if (s_ != GABP_OK) return s_;        \
    } while (0)

constexpr double kDivergence = 1e8;  // relative residual that counts as divergence

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

struct GraphEntry {
    int k, parity, transposed, frozen;
    cudaGraphExec_t exec;
};

}  // namespace

namespace gabp {
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace gabp

struct gabp_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    gabp_options opt{};
    int prec = 0;  // message precision: 0 double, 1 float
    int n = 0;
    int64_t nnz = 0, edges = 0;
    DevLayout L{};
    // host copy of the caller's matrix
    std::vector<int64_t> h_indptr;
    std::vector<int32_t> h_indices;
    std::vector<double> h_data;
    // device allocations (tracked for cleanup)
    std::vector<void *> allocs;
    size_t dev_bytes = 0;
    // coefficients
    void *a = nullptr, *c = nullptr, *diagT = nullptr;  // message precision
    double *a64 = nullptr, *diag64 = nullptr;           // double (residual)
    void *aT = nullptr;                                 // transposed mean coefficients
    double *aT64 = nullptr;
    int64_t *slotmap = nullptr;                         // caller slot -> layout slot (-1: none)
    int64_t *diagpos = nullptr;                         // entry index of each row's diagonal (lazy)
    // internal renumbering (reverse Cuthill-McKee, CSR layout): internal node i
    // is the caller's node perm[i]; the CSR in internal order and, for every
    // caller entry, its position there
    bool reordered = false;
    int *d_perm = nullptr;
    std::vector<int32_t> h_perm;
    std::vector<int64_t> h_pindptr, h_pmap;
    std::vector<int32_t> h_pindices;
    int64_t *d_indptr = nullptr;                        // caller CSR on device (edge gradient)
    int *d_indices = nullptr;
    // state
    void *Lm[2] = {nullptr, nullptr}, *Mm[2] = {nullptr, nullptr};
    void *P[2] = {nullptr, nullptr}, *B[2] = {nullptr, nullptr};
    int cur = 0;
    void *bT = nullptr;       // rhs of the sweeps, message precision
    double *bres = nullptr;   // rhs of the residual checks (double)
    double *xbuf = nullptr;   // beliefs of the last sweep of a chunk
    double *b0 = nullptr, *xacc = nullptr, *rbuf = nullptr;  // refinement (lazy)
    double *sq_part = nullptr, *h_sq_part = nullptr;         // 2-norm partial sums (lazy)
    void *g = nullptr;           // frozen mean-message gains a_e / d_e (lazy)
    unsigned char *color = nullptr;  // coloured schedule (lazy); ncolors == 0: flood
    int ncolors = 0;
    bool has_masks = false;          // stencil layout: per-colour slot masks valid
    ColorMasks masks{};
    // coloured schedule on the parity-class layout (grids whose colours are
    // unions of parity classes): messages Lm/Mm held by sender, class by class
    bool parity = false;
    ParityGrid pg{};
    std::vector<PhaseClasses> phases;
    void *pa = nullptr, *pc = nullptr, *paT = nullptr;  // a, c, a^T in class layout
    // line schedule (lazy): grid side; couplings along rows (natural order, a
    // row line contiguous) and along columns (transposed order, a column line
    // contiguous) with the diagonal and b transposed; node messages of both
    // families in natural order, plus the transposed copies the column phase
    // reads (LHt, MHt) and writes (LVt, MVt); scratch for very long lines
    int lines_m = 0;
    void *lsubH = nullptr, *lsupH = nullptr, *lsubV = nullptr, *lsupV = nullptr;
    void *lsubHT = nullptr, *lsupHT = nullptr, *lsubVT = nullptr, *lsupVT = nullptr;  // of A^T (lazy)
    void *ldiagT = nullptr, *lbT = nullptr;
    void *LH = nullptr, *MH = nullptr, *LV = nullptr, *MV = nullptr;
    void *LHt = nullptr, *MHt = nullptr, *LVt = nullptr, *MVt = nullptr;
    void *lf = nullptr, *ly = nullptr;
    // frozen line coefficients (lazy): aF, aB, 1 / S per family, and the
    // precision messages of the last check (convergence test)
    void *laFH = nullptr, *laBH = nullptr, *lSH = nullptr;
    void *laFV = nullptr, *laBV = nullptr, *lSV = nullptr;
    void *laFVn = nullptr, *laBVn = nullptr, *lSVn = nullptr;  // the same in natural order
    void *lprevH = nullptr, *lprevV = nullptr;
    bool lprev_valid = false;
    // parity-class layout: messages reset lazily (bit 0 precision, bit 1 mean); the
    // next sweep reads every class that has not sent in it yet as zero
    unsigned zero_pending = 0;
    bool frozen = false;         // precision messages frozen (both L and P buffers equal)
    bool frozen_transposed = false;
    DevStatus *dstat = nullptr;  // [0] chunk checks, [1] refinement / misc, [2] Lambda change
    DevStatus *hstat = nullptr;  // pinned host mirror
    std::vector<GraphEntry> graphs;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

struct gabp_batch {
    int dev = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int nsys = 0, prec = 0, K = 0, check_every = 10;
    int refine = 0, inner_max = 2000;  // refinement (contexts created with GABP_FP32_IR)
    int freeze = 0;                    // freeze precision messages per system once converged
    double inner_tol = 1e-3;
    int block = 0, cs = 0, grid = 0, nbig = 0, sms = 0;  // launch shape (0 = not tuned)
    int rows = 1;       // rows in flight per thread in the mean-message sweeps
    int min_rows = 4;   // a system takes a whole cluster from this many rows per cluster thread
    int check_every0 = 10;  // the check interval given at setup
    bool check_auto = false;  // setup asked for a tuned check interval (check_every 0)
    std::vector<gabp_ctx *> sys;
    void *d_sys = nullptr;            // descriptors
    int *d_order = nullptr;           // largest first
    int *d_queue = nullptr;
    const double **d_b = nullptr;     // per-system rhs / output pointers
    double **d_x = nullptr;
    const double **h_b = nullptr;     // pinned staging of the pointer tables
    double **h_x = nullptr;
    void *d_res = nullptr, *h_res = nullptr;
    double g_tol = -1.0;              // parameters baked into the captured graph
    int g_max_iter = -1;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<void *> allocs;
    size_t dev_bytes = 0;
};

struct mg_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    int levels = 0;
    std::vector<gabp_ctx *> lv;
    std::vector<int> side;
    double scale = 4.0;
    int mode = MG_SMOOTH_COLD;
    std::vector<double *> b, x;  // per level >= 1
    double *coarse_inv = nullptr;
    int nc = 0;
    DevStatus *dstat = nullptr, *hstat = nullptr;
    std::vector<void *> allocs;
    size_t dev_bytes = 0;
    // mg_solve replays its cycles (V-cycle, convergence residual, status and
    // flag copies) as CUDA graphs captured on cap_stream, one per (b, x, nu)
    struct CycleGraph {
        const double *b;
        double *x;
        int nu_pre, nu_post;
        cudaGraphExec_t exec;
        unsigned long long kernels;
    };
    cudaStream_t cap_stream = nullptr;
    std::vector<CycleGraph> graphs;
    unsigned *hflags = nullptr;  // pinned: each level's breakdown flags after a replay
    // fused transfers (mg.cu): every level a grid stencil inside the 3 x 3
    // neighbourhood; tbuf holds the finest level's x + e between restriction and
    // prolongation
    bool fusable = false, fused = false;
    double *tbuf = nullptr;
};

namespace {

template <typename Ctx>
gabp_status dalloc(Ctx *ctx, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return fail_cuda(e, "cudaMalloc");
    ctx->allocs.push_back(*p);
    ctx->dev_bytes += bytes;
    return GABP_OK;
}

size_t esz(int prec) { return prec == 0 ? sizeof(double) : sizeof(float); }

gabp_status set_dev(int dev)
{
    CK(cudaSetDevice(dev));
    return GABP_OK;
}

// ---------------------------------------------------------------------------
// CSR validation and layout construction (host)
// ---------------------------------------------------------------------------
gabp_status validate_csr(int32_t n, int64_t nnz, const int64_t *indptr, const int32_t *indices,
                         const double *data)
{
    if (n < 0 || nnz < 0) return fail(GABP_E_INVALID_ARG, "negative size");
    if (n > 0 && (!indptr || (nnz > 0 && (!indices || !data))))
        return fail(GABP_E_INVALID_ARG, "null matrix array");
    if (n == 0) return GABP_OK;
    if (indptr[0] != 0 || indptr[n] != nnz) return fail(GABP_E_BAD_CSR, "indptr[0] != 0 or indptr[n] != nnz");
    for (int32_t r = 0; r < n; ++r) {
        if (indptr[r + 1] < indptr[r]) return fail(GABP_E_BAD_CSR, "indptr not monotone");
        bool diag = false;
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p) {
            const int32_t c = indices[p];
            if (c < 0 || c >= n) return fail(GABP_E_BAD_CSR, "column index out of range");
            if (p > indptr[r] && indices[p - 1] >= c)
                return fail(GABP_E_BAD_CSR, "columns not strictly ascending (unsorted or duplicate)");
            if (!std::isfinite(data[p])) return fail(GABP_E_BAD_CSR, "non-finite matrix value");
            if (c == r) {
                if (data[p] == 0.0) return fail(GABP_E_ZERO_DIAG, "zero diagonal entry in row " + std::to_string(r));
                diag = true;
            }
        }
        if (!diag) return fail(GABP_E_ZERO_DIAG, "missing diagonal entry in row " + std::to_string(r));
    }
    return GABP_OK;
}

// Host-side coefficient arrays of a layout (double), before upload.
struct HostLayout {
    int kind = GABP_LAYOUT_CSR;
    StencilParams sp{};
    int64_t slots = 0;
    std::vector<int> rowptr, col, rev;
    std::vector<double> a, c, diag;
    std::vector<int64_t> slotmap;
};

// Distinct off-diagonal offsets closed under negation; false if more than KMAX.
bool stencil_offsets(int32_t n, const int64_t *indptr, const int32_t *indices, StencilParams &sp)
{
    std::vector<int> absoff;
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p) {
            const int o = indices[p] - r;
            if (o == 0) continue;
            const int ao = o < 0 ? -o : o;
            if (std::find(absoff.begin(), absoff.end(), ao) == absoff.end()) {
                absoff.push_back(ao);
                if ((int)absoff.size() * 2 > KMAX) return false;
            }
        }
    std::sort(absoff.begin(), absoff.end());
    const int h = (int)absoff.size();
    sp.K = 2 * h;
    for (int i = 0; i < h; ++i) {
        sp.off[i] = -absoff[h - 1 - i];
        sp.off[h + i] = absoff[i];
    }
    for (int k = 0; k < sp.K; ++k) sp.krev[k] = sp.K - 1 - k;  // off sorted symmetric
    for (int k = sp.K; k < KMAX; ++k) sp.off[k] = sp.krev[k] = 0;
    return true;
}

void build_stencil(int32_t n, const int64_t *indptr, const int32_t *indices, const double *data,
                   const StencilParams &sp, HostLayout &H)
{
    H.kind = GABP_LAYOUT_STENCIL;
    H.sp = sp;
    const int K = sp.K;
    H.slots = (int64_t)K * n;
    H.a.assign((size_t)H.slots, 0.0);
    H.c.assign((size_t)H.slots, 0.0);
    H.diag.assign((size_t)n, 0.0);
    H.slotmap.assign((size_t)indptr[n], -1);
    for (int32_t r = 0; r < n; ++r) {
        int k = 0;
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p) {
            const int o = indices[p] - r;
            if (o == 0) {
                H.diag[r] = data[p];
                continue;
            }
            while (sp.off[k] != o) ++k;  // columns ascend, offsets ascend
            const int64_t e = (int64_t)k * n + r;
            H.a[e] = -data[p];
            H.slotmap[p] = e;
        }
    }
    for (int k = 0; k < K; ++k) {
        const int o = sp.off[k];
        const int64_t kr = sp.krev[k];
        for (int32_t r = 0; r < n; ++r) {
            const int64_t e = (int64_t)k * n + r;
            const int64_t s = (int64_t)r + o;
            if (H.a[e] != 0.0 && s >= 0 && s < n) H.c[e] = -H.a[e] * H.a[kr * n + s];
        }
    }
}

void build_csr(int32_t n, const int64_t *indptr, const int32_t *indices, const double *data,
               HostLayout &H)
{
    H.kind = GABP_LAYOUT_CSR;
    // symmetrised off-diagonal pattern
    std::vector<int64_t> cnt((size_t)n + 1, 0);
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p)
            if (indices[p] != r) {
                cnt[r + 1]++;
                cnt[indices[p] + 1]++;
            }
    for (int32_t r = 0; r < n; ++r) cnt[r + 1] += cnt[r];
    std::vector<int> tmp((size_t)cnt[n]);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p)
            if (indices[p] != r) {
                tmp[fill[r]++] = indices[p];
                tmp[fill[indices[p]]++] = r;
            }
    H.rowptr.assign((size_t)n + 1, 0);
    H.col.clear();
    H.col.reserve(tmp.size());
    for (int32_t r = 0; r < n; ++r) {
        auto b0 = tmp.begin() + cnt[r], b1 = tmp.begin() + cnt[r + 1];
        std::sort(b0, b1);
        auto e = std::unique(b0, b1);
        for (auto it = b0; it != e; ++it) H.col.push_back(*it);
        H.rowptr[r + 1] = (int)H.col.size();
    }
    H.slots = (int64_t)H.col.size();
    auto find = [&](int r, int s) -> int64_t {
        auto b0 = H.col.begin() + H.rowptr[r], b1 = H.col.begin() + H.rowptr[r + 1];
        auto it = std::lower_bound(b0, b1, s);
        return (it != b1 && *it == s) ? (int64_t)(it - H.col.begin()) : -1;
    };
    H.a.assign((size_t)H.slots, 0.0);
    H.c.assign((size_t)H.slots, 0.0);
    H.rev.assign((size_t)H.slots, 0);
    H.diag.assign((size_t)n, 0.0);
    H.slotmap.assign((size_t)indptr[n], -1);
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p) {
            if (indices[p] == r) {
                H.diag[r] = data[p];
                continue;
            }
            const int64_t e = find(r, indices[p]);
            H.a[e] = -data[p];
            H.slotmap[p] = e;
        }
    for (int32_t r = 0; r < n; ++r)
        for (int e = H.rowptr[r]; e < H.rowptr[r + 1]; ++e) {
            const int64_t q = find(H.col[e], r);
            H.rev[e] = (int)q;
            H.c[e] = -H.a[e] * H.a[q];
        }
}

template <typename T>
std::vector<T> cast_vec(const std::vector<double> &v)
{
    std::vector<T> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (T)v[i];
    return o;
}

template <typename Ctx>
gabp_status upload(Ctx *ctx, void **dst, const void *src, size_t bytes)
{
    CKS(dalloc(ctx, dst, bytes));
    if (bytes) CK(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return GABP_OK;
}

// Uploads the coefficient arrays (a, c, diag in both precisions) of H.
gabp_status upload_coeffs(gabp_ctx *ctx, const HostLayout &H, bool realloc)
{
    const size_t S = (size_t)H.slots, n = (size_t)ctx->n;
    auto put = [&](void **dst, const void *src, size_t bytes) -> gabp_status {
        if (realloc) return upload(ctx, dst, src, bytes);
        if (bytes) CK(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
        return GABP_OK;
    };
    CKS(put((void **)&ctx->a64, H.a.data(), S * sizeof(double)));
    CKS(put((void **)&ctx->diag64, H.diag.data(), n * sizeof(double)));
    if (ctx->prec == 0) {
        ctx->a = ctx->a64;
        ctx->diagT = ctx->diag64;
        CKS(put(&ctx->c, H.c.data(), S * sizeof(double)));
    } else {
        auto af = cast_vec<float>(H.a), cf = cast_vec<float>(H.c), df = cast_vec<float>(H.diag);
        CKS(put(&ctx->a, af.data(), S * sizeof(float)));
        CKS(put(&ctx->c, cf.data(), S * sizeof(float)));
        CKS(put(&ctx->diagT, df.data(), n * sizeof(float)));
    }
    return GABP_OK;
}

void free_all(std::vector<void *> &allocs)
{
    for (void *p : allocs) cudaFree(p);
    allocs.clear();
}

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

int block_of(const gabp_ctx *ctx) { return ctx->opt.block_size > 0 ? ctx->opt.block_size : 256; }

// One sweep from state cur into 1 - cur (mean messages only while frozen);
// with a coloured schedule, one in-place phase per colour class.
cudaError_t sweep_once(gabp_ctx *ctx, bool transposed, double *x, cudaStream_t s)
{
    const int c0 = ctx->cur, c1 = c0 ^ 1;
    // line couplings of A, or of A^T for the transposed solve
    void *lsH = transposed ? ctx->lsubHT : ctx->lsubH, *luH = transposed ? ctx->lsupHT : ctx->lsupH;
    void *lsV = transposed ? ctx->lsubVT : ctx->lsubV, *luV = transposed ? ctx->lsupVT : ctx->lsupV;
    if (ctx->lines_m > 0 && ctx->frozen && line_cols_natural(ctx->prec, ctx->lines_m)) {
        // frozen precision messages, both families in the natural order: no transposes
        const int m = ctx->lines_m, pr = ctx->prec;
        cudaError_t e;
        if ((e = launch_line_mean(pr, m, ctx->laFH, ctx->laBH, ctx->lSH, ctx->bT, ctx->MV, ctx->MH,
                                  ctx->ly, nullptr, 0, s)) != cudaSuccess)
            return e;
        return launch_line_mean_cols(pr, m, ctx->laFVn, ctx->laBVn, ctx->lSVn, ctx->bT, ctx->MH,
                                     ctx->MV, x, s);
    }
    if (ctx->lines_m > 0 && ctx->frozen) {
        // frozen precision messages: the mean messages move, rows then columns
        const int m = ctx->lines_m, pr = ctx->prec;
        cudaError_t e;
        if ((e = launch_line_mean(pr, m, ctx->laFH, ctx->laBH, ctx->lSH, ctx->bT, ctx->MV, ctx->MH,
                                  ctx->ly, nullptr, 0, s)) != cudaSuccess)
            return e;
        if ((e = launch_transpose(pr, m, ctx->MH, ctx->MHt, s)) != cudaSuccess) return e;
        if ((e = launch_line_mean(pr, m, ctx->laFV, ctx->laBV, ctx->lSV, ctx->lbT, ctx->MHt,
                                  ctx->MVt, ctx->ly, x, 1, s)) != cudaSuccess)
            return e;
        return launch_transpose(pr, m, ctx->MVt, ctx->MV, s);
    }
    if (ctx->lines_m > 0) {
        // Algorithm 2 over the rows (natural order), then the columns (transposed order)
        const int m = ctx->lines_m, pr = ctx->prec;
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
            cudaError_t e = launch_sweep_parity(ctx->pg, ph, ctx->prec, transposed ? ctx->paT : ctx->pa,
                                                ctx->pc, ctx->diagT, ctx->bT, ctx->Lm[c0],
                                                ctx->Mm[c0], x, &ctx->dstat[0].flags,
                                                (zp & 1u) ? later : 0u, (zp & 2u) ? later : 0u, s);
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

// Freezes once the last sweep changed no precision message by more than
// `rel` times the largest one (rounding level).
gabp_status maybe_freeze(gabp_ctx *ctx, bool transposed)
{
    if (ctx->frozen) return GABP_OK;
    if (ctx->lines_m > 0) return maybe_freeze_lines(ctx, ctx->prec == 0 ? 1e-14 : 1e-6, transposed);
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

bool freeze_enabled(const gabp_ctx *ctx)
{
    if (ctx->ncolors > 0) return false;  // frozen sweeps: flood and line schedules
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
            const int k = std::min(every, max_iter - it);
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
                     int *iters, double *relres, bool transposed = false)
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
    // phase, which is shorter for line GaBP (measured on the 2048^2 workload: 400 sweeps
    // per step for the flood schedule, 150 for lines)
    const int inner_max = ctx->opt.ir_inner_max > 0 ? ctx->opt.ir_inner_max : (ctx->lines_m > 0 ? 150 : 400);
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
            const int k = std::min(std::min(every, inner_max - inner), max_iter - total);
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

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

namespace {

// Symmetrised adjacency of A without the diagonal, rows sorted, no duplicates.
void sym_adjacency(int32_t n, const int64_t *indptr, const int32_t *indices,
                   std::vector<int64_t> &ap, std::vector<int32_t> &aj)
{
    std::vector<int64_t> cnt((size_t)n + 1, 0);
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p)
            if (indices[p] != r) {
                cnt[r + 1]++;
                cnt[indices[p] + 1]++;
            }
    for (int32_t r = 0; r < n; ++r) cnt[r + 1] += cnt[r];
    std::vector<int32_t> tmp((size_t)cnt[n]);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p)
            if (indices[p] != r) {
                tmp[fill[r]++] = indices[p];
                tmp[fill[indices[p]]++] = r;
            }
    ap.assign((size_t)n + 1, 0);
    aj.clear();
    aj.reserve(tmp.size());
    for (int32_t r = 0; r < n; ++r) {
        auto b0 = tmp.begin() + cnt[r], b1 = tmp.begin() + cnt[r + 1];
        std::sort(b0, b1);
        auto e = std::unique(b0, b1);
        aj.insert(aj.end(), b0, e);
        ap[r + 1] = (int64_t)aj.size();
    }
}

// Reverse Cuthill-McKee order of the symmetrised graph: for each connected
// component a breadth-first search from a pseudo-peripheral node (the last
// node a search from a minimum-degree node reaches), each node's unvisited
// neighbours taken by ascending degree; the whole order reversed.  perm[i] is
// the node placed at position i.  Returns whether the renumbering is worth it
// (`force`, or it at least halves the mean |i - j| over the coupled pairs).
bool rcm_order(int32_t n, const int64_t *indptr, const int32_t *indices, bool force,
               std::vector<int32_t> &perm)
{
    std::vector<int64_t> ap;
    std::vector<int32_t> aj;
    sym_adjacency(n, indptr, indices, ap, aj);
    auto deg = [&](int32_t v) { return ap[v + 1] - ap[v]; };
    std::vector<int32_t> byDeg((size_t)n);
    for (int32_t i = 0; i < n; ++i) byDeg[i] = i;
    std::stable_sort(byDeg.begin(), byDeg.end(), [&](int32_t a, int32_t b) { return deg(a) < deg(b); });
    std::vector<int32_t> stamp((size_t)n, -1);
    std::vector<char> placed((size_t)n, 0);
    std::vector<int32_t> order, queue, nb;
    order.reserve(n);
    queue.reserve(n);
    int32_t comp = 0;
    for (int32_t v0 : byDeg) {
        if (placed[v0]) continue;
        // pseudo-peripheral start: the last node reached from v0
        queue.clear();
        queue.push_back(v0);
        stamp[v0] = comp;
        for (size_t h = 0; h < queue.size(); ++h)
            for (int64_t p = ap[queue[h]]; p < ap[queue[h] + 1]; ++p)
                if (stamp[aj[p]] != comp) {
                    stamp[aj[p]] = comp;
                    queue.push_back(aj[p]);
                }
        const int32_t u = queue.back();
        // Cuthill-McKee from u
        const size_t first = order.size();
        order.push_back(u);
        placed[u] = 1;
        for (size_t h = first; h < order.size(); ++h) {
            const int32_t w = order[h];
            nb.clear();
            for (int64_t p = ap[w]; p < ap[w + 1]; ++p)
                if (!placed[aj[p]]) {
                    placed[aj[p]] = 1;
                    nb.push_back(aj[p]);
                }
            std::stable_sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) { return deg(a) < deg(b); });
            order.insert(order.end(), nb.begin(), nb.end());
        }
        ++comp;
    }
    std::reverse(order.begin(), order.end());
    perm.swap(order);
    if (force) return true;
    std::vector<int32_t> iperm((size_t)n);
    for (int32_t i = 0; i < n; ++i) iperm[perm[i]] = i;
    double before = 0.0, after = 0.0;
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = ap[r]; p < ap[r + 1]; ++p) {
            before += std::abs((double)aj[p] - r);
            after += std::abs((double)iperm[aj[p]] - iperm[r]);
        }
    return after * 2.0 <= before;
}

// The CSR of P A P^T for the order perm (internal row i = caller row perm[i]),
// rows sorted, and pmap[p] = position of the caller's entry p in it.
void permute_csr(int32_t n, const int64_t *indptr, const int32_t *indices,
                 const std::vector<int32_t> &perm, std::vector<int64_t> &pindptr,
                 std::vector<int32_t> &pindices, std::vector<int64_t> &pmap)
{
    std::vector<int32_t> iperm((size_t)n);
    for (int32_t i = 0; i < n; ++i) iperm[perm[i]] = i;
    pindptr.assign((size_t)n + 1, 0);
    for (int32_t i = 0; i < n; ++i) pindptr[i + 1] = pindptr[i] + (indptr[perm[i] + 1] - indptr[perm[i]]);
    pindices.assign((size_t)indptr[n], 0);
    pmap.assign((size_t)indptr[n], 0);
    std::vector<std::pair<int32_t, int64_t>> row;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t r = perm[i];
        row.clear();
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p) row.emplace_back(iperm[indices[p]], p);
        std::sort(row.begin(), row.end());
        int64_t q = pindptr[i];
        for (auto &cp : row) {
            pindices[q] = cp.first;
            pmap[cp.second] = q;
            ++q;
        }
    }
}

std::vector<double> permute_values(const std::vector<int64_t> &pmap, const double *data)
{
    std::vector<double> v(pmap.size());
    for (size_t p = 0; p < pmap.size(); ++p) v[pmap[p]] = data[p];
    return v;
}

}  // namespace

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

#define GABP_BATCH_RES_ITERS(h, i) (((int *)((char *)(h) + (i) * batch_result_bytes()))[0])
#define GABP_BATCH_RES_STATUS(h, i) (((int *)((char *)(h) + (i) * batch_result_bytes()))[1])
#define GABP_BATCH_RES_RR(h, i) (*(double *)((char *)(h) + (i) * batch_result_bytes() + 8))

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

static gabp_status setup_lines(gabp_ctx *ctx);

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

static gabp_status setup_lines(gabp_ctx *ctx)
{
    if (ctx->reordered)
        return fail(GABP_E_INVALID_ARG, "the line schedule needs the caller's grid numbering (reorder = 0)");
    const int n = ctx->n;
    int m = 0;
    while ((int64_t)m * m < n) ++m;
    if ((int64_t)m * m != n || n == 0) return fail(GABP_E_INVALID_ARG, "line schedule needs an m x m grid");
    const int64_t *ip = ctx->h_indptr.data();
    const int32_t *ix = ctx->h_indices.data();
    const double *dv = ctx->h_data.data();
    std::vector<double> subH(n, 0.0), supH(n, 0.0), subV(n, 0.0), supV(n, 0.0), dT(n, 0.0);
    std::vector<double> dg(n, 0.0);
    for (int r = 0; r < n; ++r) {
        const int rx = r % m, ry = r / m;
        for (int64_t p = ip[r]; p < ip[r + 1]; ++p) {
            const int j = ix[p];
            const int jx = j % m, jy = j / m;
            if (j == r) dg[r] = dv[p];
            else if (jy == ry && jx == rx - 1) subH[r] = dv[p];                      // west, along the row
            else if (jy == ry && jx == rx + 1) supH[r] = dv[p];                      // east
            else if (jx == rx && jy == ry - 1) subV[(size_t)rx * m + ry] = dv[p];   // south, along the column
            else if (jx == rx && jy == ry + 1) supV[(size_t)rx * m + ry] = dv[p];   // north
            else return fail(GABP_E_INVALID_ARG, "line schedule needs a 5-point grid matrix (every edge inside a row or a column)");
        }
    }
    for (int r = 0; r < n; ++r) dT[(size_t)(r % m) * m + r / m] = dg[r];
    const size_t nb = (size_t)n * esz(ctx->prec);
    auto put = [&](void **dst, const std::vector<double> &v) -> gabp_status {
        if (!*dst) CKS(dalloc(ctx, dst, nb));
        if (ctx->prec == 0) {
            CK(cudaMemcpy(*dst, v.data(), nb, cudaMemcpyHostToDevice));
        } else {
            auto f = cast_vec<float>(v);
            CK(cudaMemcpy(*dst, f.data(), nb, cudaMemcpyHostToDevice));
        }
        return GABP_OK;
    };
    CKS(put(&ctx->lsubH, subH));
    CKS(put(&ctx->lsupH, supH));
    CKS(put(&ctx->lsubV, subV));
    CKS(put(&ctx->lsupV, supV));
    CKS(put(&ctx->ldiagT, dT));
    void **bufs[] = {&ctx->lbT, &ctx->LH, &ctx->MH, &ctx->LV, &ctx->MV, &ctx->LHt, &ctx->MHt,
                     &ctx->LVt, &ctx->MVt};
    for (void **bp : bufs) {
        if (!*bp) CKS(dalloc(ctx, bp, nb));
        CK(cudaMemset(*bp, 0, nb));
    }
    if (line_needs_scratch(ctx->prec, m)) {
        if (!ctx->lf) CKS(dalloc(ctx, &ctx->lf, nb));
        if (!ctx->ly) CKS(dalloc(ctx, &ctx->ly, nb));
    }
    CK(prepare_line_kernels(ctx->prec, m));
    ctx->lines_m = m;
    return GABP_OK;
}

// Coloured schedule on the parity-class layout when A is an m x m grid
// stencil (m >= 3, every coupling inside the 3 x 3 neighbourhood, none
// wrapping around a grid row) and every colour is a union of parity classes.
// Leaves ctx->parity false when A or the colouring does not fit.
static gabp_status setup_parity(gabp_ctx *ctx, const std::vector<int> &col, int nc)
{
    ctx->parity = false;
    const int n = ctx->n;
    const StencilParams &sp = ctx->L.sp;
    if (ctx->L.kind != GABP_LAYOUT_STENCIL || sp.K == 0 || sp.K > KMAXPG) return GABP_OK;
    int m = 0;
    while ((int64_t)m * m < n) ++m;
    if ((int64_t)m * m != n || m < 3) return GABP_OK;
    ParityGrid g{};
    g.m = m;
    g.K = sp.K;
    for (int k = 0; k < sp.K; ++k) {
        bool found = false;
        for (int dy = -1; dy <= 1 && !found; ++dy)
            for (int dx = -1; dx <= 1 && !found; ++dx)
                if ((dx || dy) && dy * m + dx == sp.off[k]) {
                    g.dx[k] = dx;
                    g.dy[k] = dy;
                    found = true;
                }
        if (!found) return GABP_OK;
        g.krev[k] = sp.krev[k];
    }
    const int64_t *ip = ctx->h_indptr.data();
    const int32_t *ix = ctx->h_indices.data();
    for (int r = 0; r < n; ++r)
        for (int64_t p = ip[r]; p < ip[r + 1]; ++p) {
            const int j = ix[p];
            if (j == r) continue;
            const int ddx = j % m - r % m, ddy = j / m - r / m;
            if (ddx < -1 || ddx > 1 || ddy < -1 || ddy > 1) return GABP_OK;
        }
    int qc[4] = {-1, -1, -1, -1};
    for (int i = 0; i < n; ++i) {
        const int q = ((i % m) & 1) | (((i / m) & 1) << 1);
        if (qc[q] < 0) qc[q] = col[i];
        else if (qc[q] != col[i]) return GABP_OK;
    }
    long long size[4], acc = 0;
    for (int q = 0; q < 4; ++q) {
        g.w[q] = (m - (q & 1) + 1) / 2;
        g.h[q] = (m - (q >> 1) + 1) / 2;
        size[q] = (long long)g.w[q] * g.h[q];
        g.base[q] = acc;
        acc += size[q];
    }
    // the full 3 x 3 neighbourhood (or its 5-point part) in ascending order
    static const int dx4[4] = {0, -1, 1, 0}, dy4[4] = {-1, 0, 0, 1};
    static const int dx8[8] = {-1, 0, 1, -1, 1, -1, 0, 1}, dy8[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
    g.std_order = (g.K == 4 || g.K == 8) && (long long)g.K * n < (1LL << 31);
    for (int k = 0; k < g.K && g.std_order; ++k) {
        const int ex = g.K == 4 ? dx4[k] : dx8[k], ey = g.K == 4 ? dy4[k] : dy8[k];
        if (g.dx[k] != ex || g.dy[k] != ey || g.krev[k] != g.K - 1 - k) g.std_order = 0;
    }
    std::vector<PhaseClasses> phases((size_t)nc);
    for (int c = 0; c < nc; ++c) {
        PhaseClasses &ph = phases[(size_t)c];
        ph = PhaseClasses{};
        for (int q = 0; q < 4; ++q)
            if (qc[q] == c) {
                ph.q[ph.nq] = q;
                ph.start[ph.nq + 1] = ph.start[ph.nq] + size[q];
                ++ph.nq;
            }
    }
    const size_t S = (size_t)ctx->L.slots * esz(ctx->prec);
    if (!ctx->pa) CKS(dalloc(ctx, &ctx->pa, S));
    if (!ctx->pc) CKS(dalloc(ctx, &ctx->pc, S));
    CK(launch_parity_convert(g, ctx->prec, 1, ctx->a, ctx->pa, ctx->stream));
    CK(launch_parity_convert(g, ctx->prec, 1, ctx->c, ctx->pc, ctx->stream));
    ctx->pg = g;
    ctx->phases.swap(phases);
    ctx->parity = true;
    if (ctx->aT) CKS(ensure_parity_transpose(ctx));
    return GABP_OK;
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
    if (MH) CK(launch_to_double(ctx->prec, ctx->MH, MH, n, ctx->stream));
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
    return GABP_OK;
}

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

gabp_status mg_cycle_fused(mg_ctx *mg, int l, int last, int nu_pre, int nu_post, const double *b,
                           double *x, MgRes top)
{
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
    CKS(mg_cycle_fused(mg, l + 1, last, nu_pre, nu_post, mg->b[l + 1], mg->x[l + 1], MG_RES_BT));
    // x2 = x1 + P e_c into x, and the post-smoothing right-hand side b - A x2
    const double *Xin = X ? mg->tbuf : nullptr;
    const double *Ein = X ? nullptr : E;
    CK(launch_mg_prolong_residual(c->L.sp, mg->side[l], c->a64, c->diag64, b, Xin, Ein,
                                  mg->x[l + 1], x, c->prec == 0 ? c->bres : nullptr,
                                  c->prec == 1 ? (float *)c->bT : nullptr, &c->dstat[0].flags, s));
    if (nu_post > 0) {
        CKS(mg_fused_sweeps(mg, l, nu_post));
        CK(launch_axpy(x, c->xbuf, 1.0, c->n, s));
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
    float best = -1.0f, ms = 0.0f;
    int bb = 0, bc = 0;
    for (int blk : blocks)
        for (int cs : clusters) {
            CKS(batch_trial(bt, blk, cs, tol, max_iter, &ms));
            if (ms >= 0.0f && (best < 0.0f || ms < best)) {
                best = ms;
                bb = blk;
                bc = cs;
            }
        }
    if (best < 0.0f) return fail(GABP_E_CUDA, "no launch shape fits the batched kernel");
    // stage 2: rows in flight per thread (the edges per thread of a mean sweep are
    // rows x diagonals) and, with clusters, the rows per cluster thread from which a
    // system takes a whole cluster
    int br = 1, bm = 4;
    const int rows_try[] = {1, 2}, minr_try[] = {2, 4, 8};
    for (int r : rows_try) {
        if (!batch_rows_supported(bt->K, r)) continue;
        for (int mr : minr_try) {
            if (bc == 1 && mr != 4) continue;  // no cluster teams: the threshold does not matter
            if (r == 1 && mr == 4) continue;   // stage 1's setting
            bt->rows = r;
            bt->min_rows = mr;
            CKS(batch_trial(bt, bb, bc, tol, max_iter, &ms));
            if (ms >= 0.0f && ms < best) {
                best = ms;
                br = r;
                bm = mr;
            }
        }
    }
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

}  // extern "C"
