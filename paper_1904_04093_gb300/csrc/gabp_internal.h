// Internal declarations of the GaBP library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/gabp.h"

// Programmatic dependent launch (sm_90 and later): a kernel launched through
// launch_pdl may be placed on the SMs while the kernel before it in the
// stream is still finishing; it waits in pdl_wait() until that kernel has
// completed and its writes are visible, so every such kernel calls pdl_wait()
// before its first access to global memory.  What overlaps is the launch and
// the placement of CTAs on the SMs the previous kernel has left, never a
// memory access, so the results are those of plain stream order.
// pdl_trigger() lets the next kernel be launched once every CTA of this one
// has passed it.  Building with -DGABP_PDL=0 gives plain launches.
#ifndef GABP_PDL
#define GABP_PDL 1
#endif

namespace gabp {

__device__ __forceinline__ void pdl_wait()
{
#if GABP_PDL
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

__device__ __forceinline__ void pdl_trigger()
{
#if GABP_PDL
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// Launches kernel k (whose body starts with pdl_wait) with programmatic
// stream serialisation; the arguments are converted to k's parameter types.
// Errors are returned and also left for cudaGetLastError.  Inside a stream
// capture the launch is a plain one: a graph replay already starts each
// kernel as soon as its predecessor ends, and programmatic edges in the
// captured graphs made the multigrid and frozen line solves about 2 % slower.
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A &&...args)
{
#if GABP_PDL
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        k<<<grid, block, smem, s>>>(std::forward<A>(args)...);
        return cudaGetLastError();
    }
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
#else
    k<<<grid, block, smem, s>>>(std::forward<A>(args)...);
    return cudaGetLastError();
#endif
}

constexpr int KMAX = 16;  // most off-diagonal diagonals the stencil layout takes

// Offsets of the stored diagonals (column - row), ascending, and for each the
// index of the diagonal holding the reverse edges (offset -off[k]).
struct StencilParams {
    int K;
    int off[KMAX];
    int krev[KMAX];
};

// Coloured schedule on a stencil layout: m[cr][c] has bit k set when slot k of
// a row of colour cr carries a message sent by colour c.
constexpr int KMAXCOLOR = 8;
struct ColorMasks {
    unsigned short m[KMAXCOLOR][KMAXCOLOR];
};

// Coloured schedule on an m x m grid (node i = x + m y) whose colours are
// constant on the four parity classes q = (x mod 2) + 2 (y mod 2).  Messages
// are stored by their sender: slot k * n + pos(s) holds the message s -> s +
// off[k] (as its effect on the recipient, like the slot layout), where pos(s)
// = base[q] + (y / 2) w[q] + x / 2 numbers the class of s row by row.  One
// phase reads only other classes' slots and writes only its own, contiguously.
constexpr int KMAXPG = 8;
// std_order = 1: the diagonals are the full 5-point (K = 4) or 9-point (K = 8)
// neighbourhood in ascending offset order and K n < 2^31, which the sweep
// specialises at compile time.
struct ParityGrid {
    int m, K;
    int dx[KMAXPG], dy[KMAXPG], krev[KMAXPG];
    int w[4], h[4];
    long long base[4];
    int std_order;
};
// The parity classes one colour covers: q[j] for j < nq, its threads
// start[j] <= t < start[j + 1].
struct PhaseClasses {
    int nq;
    int q[4];
    long long start[5];
};

// Device status word: residual and rhs maxima (bit patterns of non-negative
// doubles, ordered like unsigned integers) and error flags.
struct DevStatus {
    unsigned long long rmax;
    unsigned long long bmax;
    unsigned int flags;
    unsigned int pad;
};
enum : unsigned { FLAG_BREAKDOWN = 1u, FLAG_NAN = 2u, FLAG_INDEX = 4u };

// The bounds-checked build (compiled with -DGABP_DEBUG, gabp_debug_build()
// returns 1): kernels test the indices they compute or read (CSR columns,
// reverse edges and row pointers, parity-class positions, multigrid tile
// indices, and that a stored non-zero coefficient has its neighbour inside the
// grid), skip an access that fails and set FLAG_INDEX in their status word;
// the host turns the flag into GABP_E_CUDA.  Release builds compile the tests
// out (kIndexChecks false).
#ifdef GABP_DEBUG
constexpr bool kIndexChecks = true;
#else
constexpr bool kIndexChecks = false;
#endif

// Pointers one sweep kernel launch needs (T = float or double, erased).
struct SweepArgs {
    int n;
    const void *a, *c, *diag, *b;
    const void *Lin, *Min, *Pin, *Bin;
    void *Lout, *Mout, *Pout, *Bout;
    double *x;  // beliefs of this sweep (nullable)
    unsigned *flags;
};

// Matrix description on the device in one layout.
struct DevLayout {
    int kind;  // GABP_LAYOUT_STENCIL or GABP_LAYOUT_CSR
    int n;
    int64_t slots;       // K*n (stencil) or symmetrised off-diagonal count (CSR)
    StencilParams sp;    // stencil
    const int *rowptr;   // CSR (int32, n+1)
    const int *col;      // CSR
    const int *rev;      // CSR reverse-edge index
};

// Sets the message gabp_last_error() returns on the calling thread (api.cu).
void set_last_error(const std::string &msg);

// ---- launch accounting (kernels.cu) ----
void count_launches(cudaStream_t s, unsigned long long k);
unsigned long long launch_count();

// ---- launchers (kernels.cu) ----
// prec: 0 = double, 1 = float (message precision)
cudaError_t launch_sweep(const DevLayout &L, int prec, const SweepArgs &a, int block, cudaStream_t s);
// CSR layout, edge-parallel (csr.cu): the full sweep and the mean-only sweep with gains g
cudaError_t launch_sweep_csr_edge(const DevLayout &L, int prec, const SweepArgs &a, cudaStream_t s);
cudaError_t launch_sweep_mean_csr_edge(const DevLayout &L, int prec, const void *g, const void *b,
                                       const void *P, const void *Min, const void *Bin, void *Mout,
                                       void *Bout, double *x, unsigned *flags, cudaStream_t s);
cudaError_t launch_aggregate(const DevLayout &L, int prec, const void *diag, const void *b,
                             const void *Lm, const void *Mm, void *P, void *B, cudaStream_t s);
// r = b - A x in double with off-diagonal coefficients a64 = -A (layout slots), max |r|, |b| into st
cudaError_t launch_residual(const DevLayout &L, const double *a64, const double *diag64,
                            const double *b, const double *x, double *r, DevStatus *st,
                            cudaStream_t s);
// the same, the residual also written in float into rf (nullable; stencil layout only)
cudaError_t launch_residual2(const DevLayout &L, const double *a64, const double *diag64,
                             const double *b, const double *x, double *r, float *rf,
                             DevStatus *st, cudaStream_t s);
cudaError_t launch_convert_d2f(const double *in, float *out, int64_t n, cudaStream_t s);
// per-block partial sums of u^2 and v^2 (part: 2 * nblocks doubles), a fixed order on every call
constexpr int kSumsqBlocks = 1024;
cudaError_t launch_sumsq2(const double *u, const double *v, int64_t n, double *part, int nblocks,
                          cudaStream_t s);
cudaError_t launch_copy_vec(const double *in, double *out, int64_t n, cudaStream_t s);
// out = in / ||in||_inf (scale read from st->rmax) in double, and as precision prec into outT
cudaError_t launch_scale_rhs(const double *in, const DevStatus *st, double *out, void *outT,
                             int prec, int64_t n, cudaStream_t s);
// x += scale * e, scale = ||r||_inf read from st->rmax
cudaError_t launch_axpy_status(double *x, const double *e, const DevStatus *st, int64_t n,
                               cudaStream_t s);
cudaError_t launch_axpy(double *x, const double *e, double alpha, int64_t n, cudaStream_t s);
// state export / import through the caller's slot map (-1 = no message)
// Parity-class layout (parity.cu).  to_class = 1: dst (class layout) from src
// (slot layout); 0: the reverse.  Both K * n elements of message precision.
cudaError_t launch_parity_convert(const ParityGrid &g, int prec, int to_class, const void *src,
                                  void *dst, cudaStream_t s);
// One in-place phase of the coloured schedule over the classes of ph:
// a, c in class layout; diag, b in natural order; Lo, Mo the class-layout state.
// zl, zm: parity classes whose precision / mean messages read as zero (the
// first sweep after a reset of the messages, instead of clearing the arrays).
// mean = 1 (frozen precision messages): a = the gains, diag = the frozen
// aggregates P (natural order), only Mo moves; c, Lo, zl unused.
cudaError_t launch_sweep_parity(const ParityGrid &g, const PhaseClasses &ph, int prec,
                                const void *a, const void *c, const void *diag, const void *b,
                                void *Lo, void *Mo, double *x, unsigned *flags, unsigned zl,
                                unsigned zm, int mean, cudaStream_t s);
// Frozen precision messages on the class layout: gains g = a / (P_s - L[rev])
// (class layout) and the aggregates P (natural order) from the current Lo.
cudaError_t launch_freeze_parity(const ParityGrid &g, int prec, const void *a, const void *diag,
                                 const void *Lo, void *gains, void *Pf, unsigned *flags, cudaStream_t s);
cudaError_t launch_get_state(const int64_t *slotmap, int64_t nnz, int prec, const void *Lm,
                             const void *Mm, double *lam, double *m, cudaStream_t s);
cudaError_t launch_set_state(const int64_t *slotmap, int64_t nnz, int prec, const double *lam,
                             const double *m, void *Lm, void *Mm, cudaStream_t s);
cudaError_t launch_edge_grad(int n, const int64_t *indptr, const int *indices, const double *lam,
                             const double *x, double *dA, cudaStream_t s);
// frozen precision messages: g = a / (P_s - L[rev]); mean-only sweep; convergence of L
cudaError_t launch_freeze(const DevLayout &L, int prec, const void *a, const void *P, const void *Lm,
                          void *g, unsigned *flags, cudaStream_t s);
cudaError_t launch_sweep_mean(const DevLayout &L, int prec, const void *g, const void *b,
                              const void *P, const void *Min, const void *Bin, void *Mout,
                              void *Bout, double *x, int block, unsigned *flags, cudaStream_t s);
cudaError_t launch_lambda_change(int64_t slots, int prec, const void *L0, const void *L1,
                                 DevStatus *st, cudaStream_t s);
// one colour phase of the coloured schedule (in place on L, M, P, B)
// (cm = nullptr: read each sender's colour instead of the table)
cudaError_t launch_sweep_color(const DevLayout &L, int prec, const unsigned char *color, int cphase,
                               const ColorMasks *cm, const void *a, const void *c, void *Lm,
                               void *Mm, void *P, void *B, double *x, unsigned *flags,
                               cudaStream_t s);
// line GaBP (lines.cu): one phase over the m lines of a layout in which line c
// is contiguous (element i at c * m + i); x (nullable) receives the lines'
// solutions at c * m + i, or at i * m + c when x_transposed; f, y: scratch of
// m * m elements, needed only when line_needs_scratch(prec, m)
cudaError_t launch_line_phase(int prec, int m, const void *sub, const void *sup, const void *diag,
                              const void *b, const void *Loth, const void *Moth, void *Lown,
                              void *Mown, void *f, void *y, double *x, int x_transposed,
                              unsigned *flags, cudaStream_t s);
bool line_needs_scratch(int prec, int m);
// line couplings (rows natural, columns transposed) and the transposed
// diagonal from the stencil layout of a 5-point m x m grid
cudaError_t launch_line_couplings_from_stencil(int prec, int m, const StencilParams &sp,
                                               const double *a64, const double *diag64,
                                               void *subH, void *supH, void *subV, void *supV,
                                               void *diagV, cudaStream_t s);
// couplings of A^T along the same contiguous lines: subT_i = sup_{i-1}, supT_i = sub_{i+1}
cudaError_t launch_line_couplings_transpose(int prec, int m, const void *sub, const void *sup,
                                            void *subT, void *supT, cudaStream_t s);
// frozen precision messages: the line's multipliers aF_i = -sub_i / f_{i-1},
// aB_i = -sup_i / g_{i+1} and 1 / S_i from the current other-family Loth;
// then phases that move the mean messages only
cudaError_t launch_line_freeze(int prec, int m, const void *sub, const void *sup,
                               const void *diag, const void *Loth, void *f, void *y, void *aF,
                               void *aB, void *sinv, unsigned *flags, cudaStream_t s);
// the frozen column phase on the natural node order (no transposes): float
// messages and m <= 2048 only (line_cols_natural); aF, aB, sinv, b, S, Mown
// and x in natural order; S = b + m'_row as the row phase left it (sum_out),
// replaced by the row messages S - b when x is written
bool line_cols_natural(int prec, int m);
cudaError_t launch_line_mean_cols(int prec, int m, const void *aF, const void *aB,
                                  const void *sinv, const void *b, void *S, void *Mown,
                                  double *x, unsigned *flags, cudaStream_t s);
// sum_out (float, lines of at most 4096): Mown = b + m' for the natural-order column phase
cudaError_t launch_line_mean(int prec, int m, const void *aF, const void *aB, const void *sinv,
                             const void *b, const void *Moth, void *Mown, void *y, double *x,
                             int x_transposed, int sum_out, unsigned *flags, cudaStream_t s);
// out = S - b in double: the row messages back from their folded form
cudaError_t launch_line_unfold(int64_t n, const void *S, const void *b, double *out, cudaStream_t s);
// raises the kernel's dynamic shared-memory limit for lines of length m (once, at setup)
cudaError_t prepare_line_kernels(int prec, int m);
cudaError_t launch_transpose(int prec, int m, const void *in, void *out, cudaStream_t s);
cudaError_t launch_to_double(int prec, const void *in, double *out, int64_t n, cudaStream_t s);
// internal renumbering: out[i] = in[idx[i]] (scatter = 0) or out[idx[i]] = in[i]
cudaError_t launch_permute(int n, const int *idx, const double *in, double *out, int scatter,
                           cudaStream_t s);
// a64, diag64 (and a, c, diagT in the message precision) from CSR values on
// the device: slotmap[p] = layout slot of entry p (-1 on the diagonal),
// diagpos[r] = entry index of the diagonal of row r
cudaError_t launch_coeffs_from_values(const DevLayout &L, int prec, int64_t nnz,
                                      const int64_t *slotmap, const int64_t *diagpos,
                                      const double *data, double *a64, double *diag64, void *a,
                                      void *c, void *diagT, cudaStream_t s);
// a^T[e] = a[rev(e)] (mean-message coefficients of the transposed system)
cudaError_t launch_transpose_coeffs(const DevLayout &L, int prec, const void *a, void *aT,
                                    cudaStream_t s);
// multigrid transfers on square grids (lexicographic, m_f = 2 m_c + 1)
cudaError_t launch_restrict_fw(const double *rf, int mf, double scale, double *rc, cudaStream_t s);
cudaError_t launch_prolong_add(const double *ec, int mc, double *xf, cudaStream_t s);
// fused transfers (mg.cu) on an m x m grid level whose stencil lies in the 3 x 3
// neighbourhood (mg_fusable): x1 = X + E (nullable terms) and, optionally, x1 into
// T for the tile's own points; r = b - A x1 restricted by full weighting, times
// scale, into rc (double) and optionally rcf (float) / rcd (a second double copy);
// flags: the status word of the bounds-checked build
bool mg_fusable(const StencilParams &sp, int m);
cudaError_t launch_mg_restrict_residual(const StencilParams &sp, int mf, const double *a64,
                                        const double *diag64, const double *b, const double *X,
                                        const double *E, double *T, double scale, double *rc,
                                        float *rcf, double *rcd, unsigned *flags, cudaStream_t s);
// x2 = Xin + Ein + P (ec + ec2) (nullable Xin, Ein, ec2; the coarse sum is formed
// before the interpolation) into Xout (Xout may not alias Xin or Ein);
// r = b - A x2 into r (double) and / or rf (float)
cudaError_t launch_mg_prolong_residual(const StencilParams &sp, int mf, const double *a64,
                                       const double *diag64, const double *b, const double *Xin,
                                       const double *Ein, const double *ec, const double *ec2,
                                       double *Xout, double *r, float *rf, unsigned *flags,
                                       cudaStream_t s);
// y = M x for a dense row-major n x n matrix (coarse-grid solve)
cudaError_t launch_dense_gemv(const double *M, const double *x, double *y, int n, cudaStream_t s);

// ---- batched persistent solver (batch.cu) ----
// cs = CTAs per thread-block cluster (1..16), grid a multiple of cs; the first
// nbig systems of `order` are solved by whole clusters, the rest by single CTAs;
// rows = rows in flight per thread (batch_rows_supported)
bool batch_rows_supported(int K, int rows);
template <typename T>
cudaError_t launch_batch(int K, int rows, int cs, int grid, int block, const void *sys, const int *order,
                         int nsys, int nbig, const double *const *bptr, double *const *xptr, int *queue,
                         double tol, int max_iter, int check_every, int refine, double inner_tol,
                         int inner_max, int freeze, void *res, cudaStream_t s);
template <typename T>
int batch_max_clusters(int K, int rows, int cs, int block);
void fill_batch_sys(int prec, void *dst, int n, const StencilParams &sp, const void *a, const void *c,
                    const void *diag, const double *a64, const double *diag64, void *const L[2],
                    void *const M[2], void *const P[2], void *const B[2], void *bT, double *e,
                    double *r, void *g);
size_t batch_sys_bytes(int prec);
size_t batch_result_bytes();  // {int iters; int status; double rr;}

}  // namespace gabp
