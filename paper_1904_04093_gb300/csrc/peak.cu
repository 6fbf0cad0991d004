// FP64 instruction throughput of this GPU, measured (gabp_fp64_peak).
//
// The double message sweep is bound by the FP64 pipe, not by HBM, so its
// roofline needs the rate at which an SM retires FP64 instructions.  Each
// thread runs eight independent dependency chains of one instruction kind
// (so the pipe, not the chain latency, limits the rate), every block of a
// single resident wave records its SM and the SM cycle counter at start and
// end, and the host divides the instructions retired on each SM by the
// cycles that SM spent.  The result is per cycle, independent of the clock;
// the wall-clock rate over CUDA events gives the clock it ran at.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "gabp_internal.h"

namespace gabp {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kBlock = 256;

__device__ __forceinline__ unsigned smid()
{
    unsigned s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

template <int OP>
__device__ __forceinline__ double step(double x, double a, double b)
{
    if (OP == 0) return fma(x, a, b);
    if (OP == 1) return x + b;
    if (OP == 2) return x * a;
    double y;
    asm volatile("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

// clk[3 * block] = {SM id, start cycle, end cycle}
template <int OP>
__global__ void __launch_bounds__(kBlock) k_fp64_peak(int iters, double a, double b, double *sink,
                                                      long long *clk)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.5 + 1e-7 * (threadIdx.x + c);
    __syncthreads();
    long long t0 = 0;
    if (threadIdx.x == 0) t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = step<OP>(x[c], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long t1 = clock64();
        clk[3 * blockIdx.x] = smid();
        clk[3 * blockIdx.x + 1] = t0;
        clk[3 * blockIdx.x + 2] = t1;
    }
    if (s == -1.0) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

template <int OP>
cudaError_t launch_peak(int grid, int iters, double *sink, long long *clk, cudaStream_t s)
{
    // a = 1 - 2^-30 and b = 2^-30 keep every chain near 1.5 for any iters
    k_fp64_peak<OP><<<grid, kBlock, 0, s>>>(iters, 1.0 - 0x1p-30, 0x1p-30, sink, clk);
    return cudaGetLastError();
}

template <int OP>
int blocks_per_sm()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fp64_peak<OP>, kBlock, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

}  // namespace
}  // namespace gabp

using namespace gabp;

extern "C" gabp_status gabp_fp64_peak(int op, int iters, gabp_peak_result *out)
{
    if (!out || op < 0 || op > 3 || iters < 1) {
        set_last_error("gabp_fp64_peak: op in 0..3, iters >= 1, out not null");
        return GABP_E_INVALID_ARG;
    }
    std::memset(out, 0, sizeof(*out));
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_last_error("gabp_fp64_peak: no CUDA device");
        cudaGetLastError();
        return GABP_E_CUDA;
    }
    const int per_sm = op == 0 ? blocks_per_sm<0>() : op == 1 ? blocks_per_sm<1>()
                     : op == 2 ? blocks_per_sm<2>() : blocks_per_sm<3>();
    if (per_sm < 1) {
        set_last_error("gabp_fp64_peak: kernel does not fit on an SM");
        return GABP_E_CUDA;
    }
    const int grid = per_sm * sms;  // one wave: every block resident at once
    double *sink = nullptr;
    long long *clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    gabp_status st = GABP_OK;
    std::vector<long long> h((size_t)3 * grid);
    auto run = [&](int it) {
        switch (op) {
            case 0: return launch_peak<0>(grid, it, sink, clk, s);
            case 1: return launch_peak<1>(grid, it, sink, clk, s);
            case 2: return launch_peak<2>(grid, it, sink, clk, s);
            default: return launch_peak<3>(grid, it, sink, clk, s);
        }
    };
    float ms = 0.0f;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&sink, (size_t)grid * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&clk, h.size() * sizeof(long long));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = run(std::max(1, iters / 8));  // warm-up: clocks up, code loaded
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = run(iters);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess)
        e = cudaMemcpy(h.data(), clk, h.size() * sizeof(long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_last_error(std::string("gabp_fp64_peak: ") + cudaGetErrorString(e));
        cudaGetLastError();
        st = GABP_E_CUDA;
    } else {
        // per SM: instructions of its blocks over the cycles from its first start to its last end
        const double per_block = (double)kBlock * kChains * kUnroll * (double)iters;
        std::vector<long long> lo(sms, 0), hi(sms, 0);
        std::vector<int> cnt(sms, 0);
        for (int i = 0; i < grid; ++i) {
            const long long id = h[3 * i], t0 = h[3 * i + 1], t1 = h[3 * i + 2];
            if (id < 0 || id >= sms) continue;
            if (cnt[id] == 0 || t0 < lo[id]) lo[id] = t0;
            if (cnt[id] == 0 || t1 > hi[id]) hi[id] = t1;
            ++cnt[id];
        }
        std::vector<double> rate;
        for (int i = 0; i < sms; ++i)
            if (cnt[i] > 0 && hi[i] > lo[i]) rate.push_back(per_block * cnt[i] / (double)(hi[i] - lo[i]));
        std::sort(rate.begin(), rate.end());
        double mean = 0.0;
        for (double r : rate) mean += r;
        out->sms = sms;
        out->sms_seen = (int)rate.size();
        out->blocks = grid;
        out->ms = ms;
        out->instructions = per_block * grid;
        out->per_cycle_per_sm = rate.empty() ? 0.0 : mean / rate.size();
        out->per_cycle_per_sm_min = rate.empty() ? 0.0 : rate.front();
        out->per_cycle_per_sm_max = rate.empty() ? 0.0 : rate.back();
        out->per_second = ms > 0.0f ? out->instructions / (ms * 1e-3) : 0.0;
        out->clock_mhz = out->per_cycle_per_sm > 0.0
                             ? out->per_second / (out->per_cycle_per_sm * sms) / 1e6 : 0.0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (clk) cudaFree(clk);
    if (s) cudaStreamDestroy(s);
    return st;
}
