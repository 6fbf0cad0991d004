// Host-side definitions shared by the library's C ABI files (not part of the
// C ABI): the context, batch and multigrid structs, error and allocation
// helpers, and the layout and solver-driver functions that api.cu,
// layout.cu, solve.cu, mg_driver.cu and batch_driver.cu share.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gabp_internal.h"

namespace gabp {

// Sets the calling thread's last-error message and returns s (api.cu).
gabp_status fail(gabp_status s, const std::string &msg);
// The message of a failed CUDA call; clears a non-sticky error (api.cu).
gabp_status fail_cuda(cudaError_t e, const char *what);

}  // namespace gabp

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

namespace gabp {

constexpr double kDivergence = 1e8;  // relative residual that counts as divergence

double bits_to_double(unsigned long long u);
gabp_status index_error(unsigned fl);

struct GraphEntry {
    int k, parity, transposed, frozen;
    cudaGraphExec_t exec;
};

}  // namespace gabp

using namespace gabp;

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
    void *pprevL = nullptr;  // parity-class layout: the precision messages at the previous check
    bool lprev_valid = false;
    // parity-class layout: messages reset lazily (bit 0 precision, bit 1 mean); the
    // next sweep reads every class that has not sent in it yet as zero
    unsigned zero_pending = 0;
    bool frozen = false;         // precision messages frozen (both L and P buffers equal)
    bool frozen_transposed = false;
    // the row mean messages MH hold b + m' (the last sweep was a frozen
    // natural-order float sweep that wrote no beliefs)
    bool mh_sum = false;
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

namespace gabp {

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

inline size_t esz(int prec) { return prec == 0 ? sizeof(double) : sizeof(float); }

inline gabp_status set_dev(int dev)
{
    CK(cudaSetDevice(dev));
    return GABP_OK;
}

template <typename Ctx>
gabp_status upload(Ctx *ctx, void **dst, const void *src, size_t bytes)
{
    CKS(dalloc(ctx, dst, bytes));
    if (bytes) CK(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return GABP_OK;
}

inline void free_all(std::vector<void *> &allocs)
{
    for (void *p : allocs) cudaFree(p);
    allocs.clear();
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

// ---- layout.cu: validation, layouts, renumbering, line and parity-class set-up ----
gabp_status validate_csr(int32_t n, int64_t nnz, const int64_t *indptr, const int32_t *indices,
                         const double *data);
bool stencil_offsets(int32_t n, const int64_t *indptr, const int32_t *indices, StencilParams &sp);
void build_stencil(int32_t n, const int64_t *indptr, const int32_t *indices, const double *data,
                   const StencilParams &sp, HostLayout &H);
void build_csr(int32_t n, const int64_t *indptr, const int32_t *indices, const double *data,
               HostLayout &H);
gabp_status upload_coeffs(gabp_ctx *ctx, const HostLayout &H, bool realloc);
void sym_adjacency(int32_t n, const int64_t *indptr, const int32_t *indices,
                   std::vector<int64_t> &ap, std::vector<int32_t> &aj);
bool rcm_order(int32_t n, const int64_t *indptr, const int32_t *indices, bool force,
               std::vector<int32_t> &perm);
void permute_csr(int32_t n, const int64_t *indptr, const int32_t *indices,
                 const std::vector<int32_t> &perm, std::vector<int64_t> &pindptr,
                 std::vector<int32_t> &pindices, std::vector<int64_t> &pmap);
std::vector<double> permute_values(const std::vector<int64_t> &pmap, const double *data);
gabp_status setup_lines(gabp_ctx *ctx);
gabp_status setup_parity(gabp_ctx *ctx, const std::vector<int> &col, int nc);

// ---- solve.cu: sweeps, chunks, freezing, the plain and refinement solve drivers ----
gabp_status zero_messages(gabp_ctx *ctx, bool lam, bool mean);
gabp_status load_rhs(gabp_ctx *ctx, const double *b);
gabp_status store_vector(gabp_ctx *ctx, const double *in, double *out, cudaStream_t s);
gabp_status aggregate(gabp_ctx *ctx);
cudaError_t sweep_once(gabp_ctx *ctx, bool transposed, double *x, cudaStream_t s);
cudaError_t enqueue_chunk(gabp_ctx *ctx, int k, bool transposed, cudaStream_t s);
gabp_status run_chunk(gabp_ctx *ctx, int k, bool transposed);
gabp_status read_status(gabp_ctx *ctx, int which, double *rinf, double *binf, unsigned *flags);
gabp_status ensure_parity_transpose(gabp_ctx *ctx);
gabp_status ensure_transpose(gabp_ctx *ctx);
gabp_status ensure_ir(gabp_ctx *ctx);
gabp_status freeze(gabp_ctx *ctx, bool transposed);
gabp_status freeze_lines(gabp_ctx *ctx, bool transposed);
gabp_status maybe_freeze_lines(gabp_ctx *ctx, double rel, bool transposed);
gabp_status maybe_freeze(gabp_ctx *ctx, bool transposed);
bool freeze_enabled(const gabp_ctx *ctx);
gabp_status solve_plain(gabp_ctx *ctx, const double *b, double *x, double tol, int max_iter,
                        int *iters, double *relres, bool transposed);
gabp_status solve_ir(gabp_ctx *ctx, const double *b, double *x, double tol, int max_iter,
                     int *iters, double *relres, bool transposed = false);
int block_of(const gabp_ctx *ctx);

}  // namespace gabp
