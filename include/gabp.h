/*
 * gabp.h -- C ABI of the GB300 Gaussian belief propagation (GaBP) library for
 * sparse nonsymmetric systems A x = b.
 *
 * The method: each directed edge j -> i of the graph of A (the edge exists iff
 * A_ij != 0, Sec. 2.3) carries a precision message tilde-Lambda_ji and a mean
 * message m_ji (eq. nonsymmetric_GaBP_messages).  One flood sweep (Sec. 2.2)
 * first forms the beliefs
 *     x_i = (b_i + sum_j m_ji) / (A_ii + sum_j tilde-Lambda_ji A_ji)
 * from the current messages and then replaces every message at once by
 *     tilde-Lambda_ji = -A_ij / (A_jj + sum_{k in N(j)\i} tilde-Lambda_kj A_kj)
 *     m_ji            =  tilde-Lambda_ji (b_j + sum_{k in N(j)\i} m_kj)
 * (eq. nonsymmetric_GaBP_rules; the belief-before-update order of
 * Algorithm 1).  Solves stop on ||b - A x||_inf / ||b||_inf (Algorithm 1).
 *
 * Conventions shared by every entry point:
 *  - Matrices are square CSR: int64 row pointers (n+1), int32 column indices
 *    sorted strictly ascending in each row, double values, the diagonal
 *    stored and non-zero.  Matrix arrays passed to a setup call are HOST
 *    arrays; the library copies them and the caller keeps ownership.
 *  - Vectors (b, x, g, r, ...) are DEVICE pointers to double unless stated,
 *    on the device that was current at setup, owned by the caller.  Work is
 *    enqueued on the context's CUDA stream (the `stream` given at setup, NULL
 *    = legacy default stream); calls that return a result on the host
 *    synchronise that stream.
 *  - Every call returns a gabp_status; nothing aborts.  gabp_last_error()
 *    returns a message for the last non-OK status of the calling thread.
 *  - A context is not thread-safe: one host thread at a time per context.
 *  - Per-slot arrays (messages, gradients) follow the caller's CSR slot order
 *    (length nnz); slots on the diagonal or holding an explicit zero carry
 *    no message and read as 0.
 */
#ifndef GABP_H
#define GABP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gabp_ctx gabp_ctx;
typedef struct mg_ctx mg_ctx;
typedef struct gabp_batch gabp_batch;

typedef enum {
    GABP_OK = 0,
    GABP_E_INVALID_ARG = 1,   /* null pointer, negative size, bad option */
    GABP_E_BAD_CSR = 2,       /* unsorted / duplicate / out-of-range index, non-finite value */
    GABP_E_ZERO_DIAG = 3,     /* a diagonal entry missing or zero */
    GABP_E_BREAKDOWN = 4,     /* a message denominator was zero or not finite */
    GABP_E_DIVERGED = 5,      /* relative residual not finite or above 1e8 */
    GABP_E_NOT_CONVERGED = 6, /* iteration cap reached; the outputs hold the last iterate */
    GABP_E_CUDA = 7,          /* a CUDA runtime call failed (message in gabp_last_error) */
    GABP_E_OOM = 8            /* device or host allocation failed */
} gabp_status;

typedef enum {
    GABP_FP64 = 0,    /* messages, beliefs and residual in double */
    GABP_FP32 = 1,    /* messages and beliefs in float, residual check in double */
    GABP_FP32_IR = 2  /* float GaBP inside double iterative refinement (solve only) */
} gabp_precision;

typedef enum {
    GABP_LAYOUT_AUTO = 0,    /* stencil layout when the matrix has few distinct diagonals */
    GABP_LAYOUT_CSR = 1,     /* general layout: symmetrised CSR with a reverse-edge index */
    GABP_LAYOUT_STENCIL = 2  /* per-diagonal (DIA) layout; GABP_E_INVALID_ARG if > 16 diagonals */
} gabp_layout;

typedef struct {
    int precision;       /* gabp_precision */
    int layout;          /* gabp_layout */
    int check_every;     /* sweeps between residual checks in gabp_solve (>= 1) */
    int use_graphs;      /* 1: replay each chunk of sweeps as a captured CUDA graph */
    int ir_inner_max;    /* GABP_FP32_IR: float sweeps per refinement step, at most
                            (0: 150 under the line and coloured schedules, 400 otherwise) */
    double ir_inner_tol; /* GABP_FP32_IR: inner relative residual that ends a refinement step */
    int block_size;      /* threads per block of the sweep kernel (0 = tuned default) */
    int freeze_lambda;   /* precomputed precision messages (Sec. 4.2): 1 on, 0 off,
                            -1 default (on for GABP_FP32_IR, off otherwise); see gabp_solve */
    int reorder;         /* CSR layout only: renumber the unknowns internally by reverse
                            Cuthill-McKee (1), keep the caller's numbering (0), or -1 (default)
                            renumber when that at least halves the mean index distance |i - j|
                            of the coupled unknowns.  Invisible at the interface: vectors,
                            per-slot arrays and colours stay in the caller's order. */
} gabp_options;

/* Fills `opt` with the defaults: FP64, auto layout, check_every 10, graphs on,
 * ir_inner_max 0 (400, or 150 under the line and coloured schedules),
 * ir_inner_tol 1e-3, block_size 0, freeze_lambda -1, reorder -1.  (Short
 * refinement steps win: restarting the float solve on a fresh double residual
 * every few hundred sweeps -- fewer for line and coloured GaBP, whose fast
 * initial phase is shorter -- reaches 1e-10 in fewer total sweeps than long
 * inner solves.) */
void gabp_default_options(gabp_options *opt);

/* Text for a status code (static storage). */
const char *gabp_status_str(gabp_status s);

/* Message of the last non-OK status returned on the calling thread ("" if none). */
const char *gabp_last_error(void);

/* Number of CUDA kernel launches this library has enqueued in the process so
 * far (a replayed graph counts each kernel it contains). */
unsigned long long gabp_launch_count(void);

/* 1 for the bounds-checked build of the library (compiled with GABP_DEBUG:
 * kernels test the indices they compute or read -- CSR row pointers, columns
 * and reverse edges, parity-class positions, multigrid tile indices, and that
 * a stored non-zero coefficient has its neighbour inside the grid -- skip an
 * access that fails and report it as GABP_E_CUDA "a device index check
 * failed"), 0 for the release build.  No counterpart in the paper. */
int gabp_debug_build(void);

/*
 * Builds a context for the n x n CSR matrix A (host arrays, copied; Sec. 2.3:
 * the graph of A).  Validates the matrix, symmetrises its pattern with
 * explicit zeros (a message over an edge whose matrix entry is zero is zero,
 * Sec. 2.3), builds the reverse-edge index, the per-edge coefficients and the
 * device layout, allocates the double-buffered message state on the current
 * device and zeroes it.  `opt` may be NULL (defaults).  `stream` is a
 * cudaStream_t (NULL = default stream).  On success *out owns device memory
 * until gabp_destroy.
 * Errors: GABP_E_INVALID_ARG, GABP_E_BAD_CSR, GABP_E_ZERO_DIAG, GABP_E_OOM, GABP_E_CUDA.
 */
gabp_status gabp_setup(int32_t n, int64_t nnz, const int64_t *indptr, const int32_t *indices,
                       const double *data, const gabp_options *opt, void *stream,
                       gabp_ctx **out);

/* Replaces the matrix values on the same pattern (host array `data`, nnz
 * doubles in the setup slot order) and zeroes the messages.  Used when A
 * depends on parameters (the differentiable solve). */
gabp_status gabp_set_values(gabp_ctx *ctx, const double *data);

/* gabp_set_values with the values in DEVICE memory (nnz doubles on the
 * context's device, setup slot order, owned by the caller): the coefficient
 * arrays are rebuilt by kernels from the values where they lie, so a caller
 * that assembles A on the GPU (the differentiable solve) has no host round
 * trip for them.  The library still copies the values to the host once per
 * call to validate them (same checks and errors as gabp_set_values) and to
 * keep its host-side consumers (line couplings, the multigrid coarse solve)
 * in step.  Zeroes the messages. */
gabp_status gabp_set_values_device(gabp_ctx *ctx, const double *data);

/* Releases the context and its device memory (NULL is ignored). */
void gabp_destroy(gabp_ctx *ctx);

/*
 * Selects the message schedule of every later sweep (gabp_sweep, gabp_solve,
 * the multigrid smoother); the messages restart from zero.
 *  schedule = 0: the flood schedule (Sec. 2.2, the default).
 *  schedule = 1: a coloured schedule (red-black / 4-colour GaBP, Sec. 5.1): a
 *    sweep visits the colour classes in order and, for every node of the
 *    current class, forms its belief and replaces the messages it sends from
 *    the current messages (Algorithm 1 with the nodes of one class processed
 *    together).  `color` (host, n ints, nullable) gives each node's class in
 *    [0, 254]; adjacent nodes must differ (GABP_E_INVALID_ARG otherwise).
 *    NULL colours the graph greedily in natural order, which gives red-black
 *    for 5-point and 4 colours for 9-point grids.  *ncolors (nullable)
 *    receives the number of classes.
 *  schedule = 2: line GaBP -- Algorithm 2 (Sec. 3) with the rows and columns
 *    of an m x m grid (node i = ix + m iy) as large regions and single nodes
 *    as small regions: a sweep updates every row region, then every column
 *    region (regions of one family share no node), each by an exact
 *    tridiagonal solve; the beliefs are the column regions' solutions.
 *    Needs n = m^2 and every edge inside a row or a column (5-point grids),
 *    GABP_E_INVALID_ARG otherwise.  The transposed solve runs the same
 *    schedule on A^T (line couplings sub_i, sup_i become sup_{i-1},
 *    sub_{i+1}); gabp_get_line_state reads the messages.
 *    On an m x m grid stencil (m >= 3, couplings inside the 3 x 3
 *    neighbourhood) whose colours are unions of the parity classes
 *    (x mod 2, y mod 2) -- red-black and the 4-colour grid colouring -- the
 *    messages are kept by sender, class by class, so a sweep streams every
 *    message once; gabp_info.parity_layout reports it.  Other colourings run
 *    on the slot layout.
 * Under schedule 2 the precision messages freeze as under the flood schedule
 * (freeze_lambda): once both families' messages stop changing, the lines'
 * elimination multipliers are stored and later sweeps move only the mean
 * messages.  Under schedule 1 they freeze likewise on the parity-class layout
 * (once they moved by less than rounding between two checks, the gains
 * a_e / d_e of every slot and the aggregates P are stored and a phase moves
 * only the mean messages: gabp_info.colored_mean_sweep_bytes); other
 * colourings are not frozen.  The batched solver always floods.
 */
gabp_status gabp_set_schedule(gabp_ctx *ctx, int schedule, const int32_t *color, int *ncolors);

/*
 * Line schedule: copies the node messages out (device arrays of n doubles,
 * natural node order): LH/MH = (Lambda, m) from each node's row region,
 * LV/MV from its column region.  Any pointer may be NULL.  Float lines of at
 * most 2048 nodes with frozen precision messages hand the row messages to the
 * column phase as b + m; a sweep that writes beliefs (every solve chunk,
 * gabp_sweep, a multigrid smoother) stores m again.  After sweeps that wrote
 * none (gabp_time_sweeps), MH is (b + m) - b with the context's current
 * right-hand side, so read it before loading another one.
 */
gabp_status gabp_get_line_state(gabp_ctx *ctx, double *LH, double *MH, double *LV, double *MV);

/* Sets every message to zero (the initial state of Algorithm 1). */
gabp_status gabp_reset(gabp_ctx *ctx);

/*
 * Runs `nsweeps` >= 0 flood sweeps (Sec. 2.2, eq. nonsymmetric_GaBP_rules)
 * from the current messages with right-hand side b (device, n doubles).  If
 * x is not NULL it receives the beliefs formed in the last sweep (Algorithm
 * 1 forms x_j before updating j's messages), so after one sweep from zero
 * messages x = b / diag(A).  The messages stay in the context for the next
 * call.  Asynchronous except for the status read at the end (one 16-byte
 * device-to-host copy); GABP_E_BREAKDOWN if a denominator was zero or not finite.
 */
gabp_status gabp_sweep(gabp_ctx *ctx, const double *b, int nsweeps, double *x);

/*
 * Solves A x = b with GaBP from zero messages (Algorithm 1, flood schedule):
 * sweeps in chunks of opt.check_every, after each chunk the relative residual
 * rr = ||b - A x||_inf / ||b||_inf of the last beliefs in double; stops at
 * rr <= tol (GABP_OK), at `max_iter` sweeps (GABP_E_NOT_CONVERGED), on
 * GABP_E_BREAKDOWN or GABP_E_DIVERGED.  With GABP_FP32_IR the float solver
 * runs inside double iterative refinement (x += s e, e from float GaBP on
 * A e = r / s, s = ||r||_inf; tilde-Lambda messages are reused across
 * refinement steps since they do not depend on the right-hand side, Sec.
 * 2.3) and `max_iter` caps the total float sweeps.  With freeze_lambda the
 * precision messages are frozen once a sweep changes none of them by more
 * than rounding (1e-14 relative in double, 1e-6 in float; until then a solve
 * checks every min(check_every, 5) sweeps): they do not depend
 * on b (Sec. 2.3) and the paper precomputes them (Sec. 4.2); from then on a
 * sweep moves only the mean messages with the fixed gains a_e / d_e, which is
 * the same update up to rounding.  x (device, n doubles)
 * receives the last iterate in every case; iters / relres (host, nullable)
 * receive the sweeps done and the final rr.  b == 0 gives x = 0, rr = 0.
 */
gabp_status gabp_solve(gabp_ctx *ctx, const double *b, double *x, double tol, int max_iter,
                       int *iters, double *relres);

/*
 * Solves A^T lam = g the same way (the adjoint solve).  The transpose has the
 * pattern of A after symmetrisation and the same precision messages (the
 * diagonal corrections tilde-Lambda_ji A_ji are symmetric in the pair), so
 * only the mean-message coefficients change.  Arguments as gabp_solve.
 */
gabp_status gabp_solve_transpose(gabp_ctx *ctx, const double *g, double *lam, double tol,
                                  int max_iter, int *iters, double *relres);

/*
 * Gradient of a loss with respect to the stored entries of A at x = A^{-1} b,
 * given lam = A^{-T} dL/dx: dA[p] = -lam_i x_j for the slot p of entry (i, j)
 * (implicit differentiation; no counterpart in the paper).  lam, x: device,
 * n doubles; dA: device, nnz doubles in setup slot order.
 */
gabp_status gabp_edge_grad(gabp_ctx *ctx, const double *lam, const double *x, double *dA);

/*
 * r = b - A x in double (device vectors; r may be NULL) and, on the host,
 * rinf = ||r||_inf and binf = ||b||_inf (either may be NULL).  The stopping
 * quantity of Algorithm 1.
 */
gabp_status gabp_residual(gabp_ctx *ctx, const double *b, const double *x, double *r,
                          double *rinf, double *binf);

/*
 * 2-norms of the residual and of the right-hand side: *r2 = ||b - A x||_2,
 * *b2 = ||b||_2 (host doubles), logged beside the infinity norm that
 * Algorithm 1 stops on.  The residual is formed in double as in
 * gabp_residual; the sums of squares run over a fixed partition of the
 * unknowns in a fixed order, so repeated calls give identical results.
 * Synchronises the context's stream.  Errors: GABP_E_INVALID_ARG, GABP_E_OOM,
 * GABP_E_CUDA.
 */
gabp_status gabp_residual_2norm(gabp_ctx *ctx, const double *b, const double *x, double *r2,
                                double *b2);

/*
 * Copies the message state out (device arrays in setup slot order, as
 * double): lam[p] = tilde-Lambda_ji A_ji (the message's correction to the
 * diagonal of row i) and m[p] = m_ji for the slot p of entry (i, j).  Either
 * pointer may be NULL.
 */
gabp_status gabp_get_state(gabp_ctx *ctx, double *lam, double *m);

/* Loads a message state in the format of gabp_get_state (device arrays). */
gabp_status gabp_set_state(gabp_ctx *ctx, const double *lam, const double *m);

/* Description of a context (host struct). */
typedef struct {
    int32_t n;              /* unknowns */
    int64_t nnz;            /* stored entries of the setup matrix */
    int64_t edges;          /* directed edges: off-diagonal entries with A_ij != 0 */
    int layout;             /* gabp_layout actually used (STENCIL or CSR) */
    int ndiag;              /* stencil layout: number of off-diagonal diagonals */
    int precision;          /* gabp_precision */
    int64_t slots;          /* message slots per buffer (padded edges) */
    double sweep_bytes;     /* compulsory DRAM bytes of one sweep kernel launch */
    double mean_sweep_bytes; /* the same for a sweep with frozen precision messages */
    double residual_bytes;  /* compulsory DRAM bytes of one residual kernel launch */
    size_t device_bytes;    /* device memory held by the context */
    int parity_layout;      /* 1: the coloured schedule runs on the parity-class layout */
    double colored_sweep_bytes; /* compulsory DRAM bytes of one sweep on that layout */
    int reordered;          /* 1: the unknowns are renumbered internally (gabp_options.reorder) */
    double colored_mean_sweep_bytes; /* the same with frozen precision messages */
} gabp_info;

gabp_status gabp_get_info(gabp_ctx *ctx, gabp_info *info);

/*
 * Times the sweep kernel alone: runs `nsweeps` sweeps like gabp_sweep, with
 * CUDA events recorded on the context's stream around the sweep launches
 * only; *ms receives their total device time.  frozen = 1 times the
 * mean-message sweep of a context whose precision messages a solve has
 * frozen (GABP_E_INVALID_ARG otherwise).  For the bench's roofline figure.
 */
gabp_status gabp_time_sweeps(gabp_ctx *ctx, const double *b, int nsweeps, int frozen, float *ms);

/*
 * Measured FP64 instruction throughput of the current device, the ceiling of
 * the double message sweep (which is bound by the FP64 pipe, not by HBM).  No
 * counterpart in the paper, whose cost model counts serial FLOPs only
 * (Sec. 4.2).  One resident wave of blocks, each thread running eight
 * independent chains of `iters` x 16 instructions of one kind: op 0 = fma,
 * 1 = add, 2 = mul, 3 = rcp.approx.ftz.f64.  Every block records its SM and
 * the SM cycle counter, so per_cycle_per_sm does not depend on the clock;
 * per_second comes from CUDA events around the launch and clock_mhz =
 * per_second / (per_cycle_per_sm x sms).  Allocates and frees small scratch
 * buffers and its own stream, synchronises the device's work on that stream.
 * Errors: GABP_E_INVALID_ARG (op outside 0..3, iters < 1, out NULL),
 * GABP_E_CUDA.
 */
typedef struct {
    int sms;                     /* SMs of the device */
    int sms_seen;                /* SMs that ran a block of the wave */
    int blocks;                  /* blocks launched (one wave) */
    float ms;                    /* device time of the timed launch */
    double instructions;         /* instructions of the kind retired in the timed launch */
    double per_cycle_per_sm;     /* mean over SMs of instructions per SM cycle */
    double per_cycle_per_sm_min; /* slowest SM */
    double per_cycle_per_sm_max; /* fastest SM */
    double per_second;           /* instructions per second of the whole device */
    double clock_mhz;            /* SM clock implied by the two rates */
} gabp_peak_result;

gabp_status gabp_fp64_peak(int op, int iters, gabp_peak_result *out);

/*
 * The paper has no counterpart to this entry point: it serves callers that
 * cannot allocate device memory (code that runs while another component owns
 * every allocation, such as a framework's memory arena or a loop that forbids
 * allocation after start-up, and callers handed only device pointers).
 * Runs `nsweeps` >= 1 flood sweeps from zero messages, exactly like
 * gabp_reset + gabp_sweep, on a CSR matrix the caller already holds on the
 * device (indptr: n+1 int64, indices: nnz int32 sorted per row, data: nnz
 * double, non-zero diagonal), right-hand side b (n doubles) and output x (n
 * doubles, the beliefs of the last sweep).  It allocates nothing: all working
 * state lives in one fixed __device__ array of 10 MiB that every device
 * loading the library holds until the process exits, so n <= 65536 and
 * nnz <= 262144; larger sizes return GABP_E_INVALID_ARG without launching.
 * The first call on a device looks up that array's address
 * (cudaGetSymbolAddress).  Every call shares the one array and leaves its
 * last contents there (each call starts from zero messages and clears the
 * error word itself), so calls whose work overlaps on the GPU (other streams,
 * other host threads) race and give undefined results.  Each call is
 * synchronous: it enqueues its sweeps on `stream` (a cudaStream_t, NULL =
 * default), copies the error word to host memory and synchronises `stream`
 * before it returns the status:
 * GABP_E_BAD_CSR for a row pointer or column index out of range or columns
 * not strictly ascending in a row, GABP_E_ZERO_DIAG for a missing or zero
 * diagonal, both found on the device, and GABP_E_BREAKDOWN as in gabp_sweep.
 */
gabp_status gabp_sweep_noalloc(int32_t n, int64_t nnz, const int64_t *indptr,
                               const int32_t *indices, const double *data, const double *b,
                               int nsweeps, double *x, void *stream);

/* ---------------------------------------------------------------------------
 * Batched solver: many independent systems in one persistent launch.  The
 * paper solves one system at a time; this is the same Algorithm 1 per
 * system (flood sweeps, residual check every check_every sweeps, the same
 * per-row arithmetic as gabp_solve, so a batched system follows gabp_solve's
 * iterates), scheduled so that one kernel launch, replayed as a CUDA graph,
 * serves the whole batch.
 * ------------------------------------------------------------------------- */

/*
 * Groups `nsys` >= 1 contexts (created by gabp_setup, all in the stencil
 * layout with at most 8 off-diagonal diagonals, one message precision, one
 * device) into a batch.  The batch uses the contexts' coefficient and message
 * buffers (their message state is overwritten by batch solves); the contexts
 * stay owned by the caller and must outlive the batch.  Systems are queued
 * largest first.  check_every: sweeps between residual checks, or 0 to let
 * gabp_batch_tune choose it (starting from 10).
 */
gabp_status gabp_batch_setup(int nsys, gabp_ctx *const *systems, int check_every, void *stream,
                             gabp_batch **out);

/*
 * Autotuner: times whole batched solves (tolerance `tol`, sweep cap
 * `max_iter`, as gabp_batch_solve) and keeps the fastest setting, in three
 * stages.  (1) The launch shape: 256 or 512 threads per CTA x 1, 2, 4, 8 or
 * 16 CTAs per thread-block cluster (16 where the non-portable cluster size
 * fits), as many clusters as can be resident.  (2) At the two fastest
 * shapes (its settings can reorder them), the rows each thread keeps in
 * flight in the sweeps with frozen precision messages
 * (1, or 2 for 5- and 9-point systems: the edges per thread of one step are
 * rows x diagonals) and, with clusters, the rows per cluster thread from
 * which a system is solved by a whole cluster instead of one CTA (2, 4 or 8).
 * (3) Only for a batch set up with check_every 0: the residual check
 * interval, 10 or 20 (a system may then sweep up to that many times past its
 * tolerance); otherwise the setup's interval is kept.  b, x: host arrays of
 * nsys device pointers (n_i doubles each); x receives scratch values.  The
 * first gabp_batch_solve tunes itself (with its own tol and max_iter) unless
 * a shape was set.  block / cluster (nullable) receive the shape;
 * gabp_batch_params the rest.
 */
gabp_status gabp_batch_tune(gabp_batch *batch, const double *const *b, double *const *x, double tol,
                            int max_iter, int *block, int *cluster);

/* Sets the launch shape without tuning: block 256 or 512, cluster 1, 2, 4, 8 or 16
 * (GABP_E_INVALID_ARG when the shape cannot be resident). */
gabp_status gabp_batch_set_shape(gabp_batch *batch, int block, int cluster);

/*
 * Sets the other tuned parameters (0 keeps one): rows in flight per thread
 * (1, or 2 for 5- and 9-point systems), rows per cluster thread from which a
 * system takes a whole cluster (default 4), residual check interval (default:
 * the setup's).  Any setting gives each system the iterates of gabp_solve with
 * that check interval.  Errors: GABP_E_INVALID_ARG.
 */
gabp_status gabp_batch_set_params(gabp_batch *batch, int rows, int min_rows, int check_every);

/* The parameters in use (each pointer nullable). */
gabp_status gabp_batch_params(gabp_batch *batch, int *rows, int *min_rows, int *check_every);

/*
 * Solves every system A_i x_i = b_i from zero messages in one persistent
 * launch: each thread-block cluster takes the next system from a queue
 * (largest first), sweeps it with all its threads until
 * ||b_i - A_i x_i||_inf / ||b_i||_inf <= tol (checked in double every
 * check_every sweeps), breakdown, divergence or max_iter sweeps, then takes
 * the next.  Contexts created with GABP_FP32_IR run float GaBP inside double
 * iterative refinement per system (as gabp_solve does; max_iter caps the
 * float sweeps).  b, x: host arrays of nsys device pointers.  iters / relres /
 * status (host arrays of nsys, nullable) receive each system's sweeps, final
 * relative residual and gabp_status.  Returns GABP_OK if every system
 * converged, else the most severe per-system status.  Synchronises the
 * stream.
 */
gabp_status gabp_batch_solve(gabp_batch *batch, const double *const *b, double *const *x, double tol,
                             int max_iter, int *iters, double *relres, int *status);

/* Launch shape in use: threads per CTA, CTAs per cluster, CTAs (0 before tuning). */
gabp_status gabp_batch_info(gabp_batch *batch, int *block, int *cluster, int *grid);

void gabp_batch_destroy(gabp_batch *batch);

/* ---------------------------------------------------------------------------
 * Geometric multigrid with GaBP as the smoother (Sec. 4).
 * ------------------------------------------------------------------------- */

typedef enum {
    MG_SMOOTH_COLD = 0,    /* each smoother call: nu sweeps of Algorithm 1 from zero messages */
    MG_SMOOTH_WARM = 1,    /* tilde-Lambda persists per level across calls, means restart at 0 */
    MG_SMOOTH_PERSIST = 2  /* both kinds of messages persist across calls */
} mg_smooth_mode;

/*
 * Builds a V-cycle over `levels` >= 1 contexts, finest first, on square grids
 * of side grid_side[l] = 2^J_l - 1 with lexicographic numbering i = ix + m*iy
 * (Sec. 4: grids with 2^J + 1 points including the boundary; the coarse point
 * (I, J) is the fine point (2I+1, 2J+1), 0-based).  Consecutive sides must
 * satisfy m_fine = 2 m_coarse + 1.  `transfer_scale` multiplies every
 * restricted residual (4 when the rows of every level are scaled by h^2).
 * The level contexts stay owned by the caller and must outlive the mg
 * context; their messages are used as the smoother state.  The coarsest
 * level is solved directly (its inverse is formed once here by LU with
 * partial pivoting, the paper's coarse solver); it must have at most 4096
 * unknowns.  `mode` is an mg_smooth_mode.
 */
gabp_status mg_setup(int levels, gabp_ctx *const *level_ctx, const int32_t *grid_side,
                     double transfer_scale, int mode, void *stream, mg_ctx **out);

/*
 * One V-cycle in place on x (device, fine-level doubles) for right-hand side
 * b: on each level nu_pre smoothing sweeps as Algorithm 3 (r = b - A x,
 * nu sweeps of GaBP on A e = r, x += e), residual, full-weighting
 * restriction (Trottenberg eq. 2.3.3), recursion, bilinear prolongation
 * (eq. 2.3.7) and correction, nu_post smoothing sweeps; direct solve on the
 * coarsest level.  `levels` = number of levels to use (0 = all).  Smoothing
 * runs in the precision of each level context; residuals and transfers in
 * double.
 */
gabp_status mg_vcycle(mg_ctx *mg, int levels, int nu_pre, int nu_post, const double *b,
                      double *x);

/* V-cycles from x = 0 until ||b - A x||_inf / ||b||_inf <= tol or max_cycles. */
gabp_status mg_solve(mg_ctx *mg, const double *b, double *x, double tol, int max_cycles,
                     int nu_pre, int nu_post, int *cycles, double *relres);

/*
 * Chooses how a cycle moves between levels.  fused = 1 (the default whenever
 * every level is a grid stencil inside the 3 x 3 neighbourhood): the
 * residual, the full-weighting restriction and the pre-smoothing correction
 * in one kernel, the bilinear prolongation, the coarse-grid correction and the
 * post-smoothing residual in another, each writing the next smoother's
 * right-hand side in its precision.  fused = 0: one kernel per step
 * (residual, restriction, prolongation, correction, conversion).  Both
 * compute the same operations in the same order.  The transfers are the
 * V-cycle of Sec. 4 with Algorithm 3 as the smoother either way.
 * Errors: GABP_E_INVALID_ARG (null context, or fused = 1 on levels that do not
 * allow it), GABP_E_CUDA.
 */
gabp_status mg_set_fused(mg_ctx *mg, int fused);

void mg_destroy(mg_ctx *mg);

#ifdef __cplusplus
}
#endif

#endif /* GABP_H */
