// Flood sweeps for callers that cannot allocate device memory.
//
// gabp_sweep_noalloc runs the same message sweep as gabp_sweep, but on a CSR
// matrix the caller already holds on the device, with all of its working
// state (double-buffered messages, node aggregates, an error word) in one
// file-scope __device__ array instead of memory from cudaMalloc.  It is meant
// for code that must not allocate: work recorded while another component owns
// every allocation (a host framework's arena, a real-time loop that forbids
// allocation after start-up), or callers that are only handed device pointers.
//
// Every device that loads this library holds the array until the process
// exits: kNoallocMaxEntries * 32 + kNoallocMaxRows * 32 bytes (10 MiB).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gabp_internal.h"

namespace {

constexpr int64_t kNoallocMaxEntries = int64_t(1) << 18;  // stored CSR entries (nnz)
constexpr int64_t kNoallocMaxRows = int64_t(1) << 16;     // unknowns (n)
constexpr int kMaxDevices = 64;

// [L0 | M0 | L1 | M1] per stored entry, [P0 | B0 | P1 | B1] per row, then the error word.
constexpr int64_t kMsgOff = 0;
constexpr int64_t kAggOff = 4 * kNoallocMaxEntries;
constexpr int64_t kFlagOff = kAggOff + 4 * kNoallocMaxRows;
constexpr int64_t kScratchDoubles = kFlagOff + 32;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

enum : unsigned { NA_BREAKDOWN = 1u, NA_BAD_INDEX = 2u, NA_ZERO_DIAG = 4u };

// Position of entry (row, col) in the caller's CSR, -1 if it is not stored.
__device__ __forceinline__ int64_t find_entry(const int64_t *__restrict__ indptr,
                                              const int *__restrict__ indices, int64_t nnz,
                                              int row, int col, unsigned &bad)
{
    int64_t lo = indptr[row], hi = indptr[row + 1] - 1;
    if (lo < 0 || hi >= nnz || lo > hi + 1) {
        bad |= NA_BAD_INDEX;
        return -1;
    }
    while (lo <= hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        const int c = indices[mid];
        if (c == col) return mid;
        if (c < col) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// One flood sweep over the caller's CSR (messages per stored slot; the slot
// of entry (r, s) carries the message s -> r as L = tilde-Lambda_sr A_sr and
// M = m_sr).  `first` = the sweep starts from zero messages, so the sender
// aggregates are P_s = A_ss, B_s = b_s and nothing is read from the scratch.
__global__ void __launch_bounds__(256) k_sweep_noalloc(
    int n, int64_t nnz, const int64_t *__restrict__ indptr, const int *__restrict__ indices,
    const double *__restrict__ data, const double *__restrict__ b, double *__restrict__ scratch,
    int cur, int first, double *__restrict__ x)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int nxt = cur ^ 1;
    const double *Lin = scratch + kMsgOff + (2 * cur) * kNoallocMaxEntries;
    const double *Min = Lin + kNoallocMaxEntries;
    double *Lout = scratch + kMsgOff + (2 * nxt) * kNoallocMaxEntries;
    double *Mout = Lout + kNoallocMaxEntries;
    const double *Pin = scratch + kAggOff + (2 * cur) * kNoallocMaxRows;
    const double *Bin = Pin + kNoallocMaxRows;
    double *Pout = scratch + kAggOff + (2 * nxt) * kNoallocMaxRows;
    double *Bout = Pout + kNoallocMaxRows;
    unsigned bad = 0;

    const int64_t pd = find_entry(indptr, indices, nnz, r, r, bad);
    const double arr = pd >= 0 ? data[pd] : 0.0;
    if (arr == 0.0) bad |= NA_ZERO_DIAG;
    const double Pr = first ? arr : Pin[r];
    const double Br = first ? b[r] : Bin[r];
    if (x) x[r] = Br / Pr;
    double pn = arr, bn = b[r];
    const int64_t lo = indptr[r], hi = indptr[r + 1];
    if (lo < 0 || hi > nnz || lo > hi) bad |= NA_BAD_INDEX;
    for (int64_t p = (bad ? hi : lo); p < hi; ++p) {
        const int s = indices[p];
        double lam = 0.0, mu = 0.0;
        // columns must ascend strictly within the row, or the searches above
        // and below would miss entries (a duplicate or unsorted row)
        if (p > lo && s <= indices[p - 1]) bad |= NA_BAD_INDEX;
        if (s < 0 || s >= n) {
            bad |= NA_BAD_INDEX;
        } else if (s != r && data[p] != 0.0) {
            const double a_e = -data[p];  // -A_rs
            double Ps, Bs, Lrev = 0.0, Mrev = 0.0, Asr = 0.0;
            const int64_t q = find_entry(indptr, indices, nnz, s, r, bad);
            if (q >= 0) Asr = data[q];
            if (first) {
                const int64_t ps = find_entry(indptr, indices, nnz, s, s, bad);
                Ps = ps >= 0 ? data[ps] : 0.0;
                if (Ps == 0.0) bad |= NA_ZERO_DIAG;
                Bs = b[s];
            } else {
                Ps = Pin[s];
                Bs = Bin[s];
                if (q >= 0) {
                    Lrev = Lin[q];
                    Mrev = Min[q];
                }
            }
            const double d = Ps - Lrev;
            if (d == 0.0 || !isfinite(d)) bad |= NA_BREAKDOWN;
            const double qd = 1.0 / d;
            lam = a_e * Asr * qd;  // c_e / d_e with c_e = -A_rs A_sr
            mu = a_e * (Bs - Mrev) * qd;
        }
        Lout[p] = lam;
        Mout[p] = mu;
        pn += lam;
        bn += mu;
    }
    Pout[r] = pn;
    Bout[r] = bn;
    if (bad) atomicOr(reinterpret_cast<unsigned *>(scratch + kFlagOff), bad);
}

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" gabp_status gabp_sweep_noalloc(int32_t n, int64_t nnz, const int64_t *indptr,
                                          const int32_t *indices, const double *data,
                                          const double *b, int nsweeps, double *x, void *stream)
{
    auto fail = [&](gabp_status s, const std::string &m) {
        gabp::set_last_error(m);
        return s;
    };
    if (n < 0 || nnz < 0 || nsweeps < 1) return fail(GABP_E_INVALID_ARG, "need n >= 0, nnz >= 0, nsweeps >= 1");
    if ((int64_t)n > kNoallocMaxRows || nnz > kNoallocMaxEntries)
        return fail(GABP_E_INVALID_ARG,
                    "matrix too large for the fixed scratch: at most 65536 rows and 262144 stored entries");
    if (n == 0) return GABP_OK;
    if (!indptr || !indices || !data || !b || !x) return fail(GABP_E_INVALID_ARG, "null device pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(GABP_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(GABP_E_INVALID_ARG, "device ordinal above 63");
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            // first call on this device: resolve the array's device address
            e = cudaGetSymbolAddress((void **)&g_scratch_ptr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_scratch_ptr[dev] = nullptr;
                return fail(GABP_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *flags = reinterpret_cast<unsigned *>(scratch + kFlagOff);
    if ((e = cudaMemsetAsync(flags, 0, sizeof(unsigned), s)) != cudaSuccess)
        return fail(GABP_E_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int block = 256, grid = (n + block - 1) / block;
    int cur = 0;
    for (int i = 0; i < nsweeps; ++i) {
        k_sweep_noalloc<<<grid, block, 0, s>>>(n, nnz, indptr, indices, data, b, scratch, cur,
                                                i == 0, i == nsweeps - 1 ? x : nullptr);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return fail(GABP_E_CUDA, std::string("sweep launch: ") + cudaGetErrorString(e));
        gabp::count_launches(s, 1);
        cur ^= 1;
    }
    unsigned hflags = 0;
    if ((e = cudaMemcpyAsync(&hflags, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(GABP_E_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    if (hflags & NA_BAD_INDEX)
        return fail(GABP_E_BAD_CSR, "row pointer or column index out of range, or columns not ascending");
    if (hflags & NA_ZERO_DIAG) return fail(GABP_E_ZERO_DIAG, "missing or zero diagonal entry");
    if (hflags & NA_BREAKDOWN) return fail(GABP_E_BREAKDOWN, "zero or non-finite message denominator");
    return GABP_OK;
}
