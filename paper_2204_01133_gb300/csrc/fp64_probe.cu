// fp64_probe.cu -- FP64 pipe throughput probe (libat_probe.so).
//
// The stage kernels are bound by FP64 arithmetic, not by HBM.  This probe
// measures the FP64 FMA rate the GPU sustains: every thread runs 8
// independent fma chains, so the pipe, not latency, limits the rate.  Used
// by the benchmark to put the roofline denominator next to the nominal one.
// It also exports the stage kernels' exponential and reciprocal for testing.
#include <cuda_runtime.h>

#include <cstdint>

#include "at_device.cuh"

namespace {

__global__ void __launch_bounds__(256) dfma_chains(double* out, int iters, double a, double b, int active_lanes)
{
    if ((int)(threadIdx.x & 31) >= active_lanes) return;
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 0.1, x2 = x0 + 0.2, x3 = x0 + 0.3;
    double x4 = x0 + 0.4, x5 = x0 + 0.5, x6 = x0 + 0.6, x7 = x0 + 0.7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b);
        x1 = fma(x1, a, b);
        x2 = fma(x2, a, b);
        x3 = fma(x3, a, b);
        x4 = fma(x4, a, b);
        x5 = fma(x5, a, b);
        x6 = fma(x6, a, b);
        x7 = fma(x7, a, b);
    }
    const double s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == 12345.678) out[blockIdx.x] = s;  // keeps the chains alive, never true
}

// one dependent chain per thread: the time per fma is the FP64 latency seen
// by a warp that has nothing else to issue
__global__ void dfma_chain1(double* out, int iters, double a, double b)
{
    double x = threadIdx.x * 1e-3;
    for (int i = 0; i < iters; ++i) x = fma(x, a, b);
    if (x == 12345.678) out[blockIdx.x] = x;
}

} // namespace

// latency probe: `warps` warps per SM, each one dependent fma chain;
// returns the average SM cycles between two dependent fmas of one warp
extern "C" int at_probe_fp64_latency(int device, int warps_per_sm, int iters, double* cycles_per_fma)
{
    if (cudaSetDevice(device) != cudaSuccess) return -3;
    int sms = 0, clk_khz = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, device);
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * sms) != cudaSuccess) return -2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    dfma_chain1<<<sms, 32 * warps_per_sm>>>(out, iters / 10 + 1, 0.999999, 1e-7);
    cudaEventRecord(e0);
    dfma_chain1<<<sms, 32 * warps_per_sm>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *cycles_per_fma = (double)ms * 1e-3 * clk_khz * 1e3 / iters;
    return cudaGetLastError() != cudaSuccess ? -3 : 0;
}

// lanes: active lanes per warp (1..32); the rate counts active lanes only
extern "C" int at_probe_fp64_fma_lanes(int device, void* stream, int iters, int reps, int lanes, double* tflops,
                                       double* ms_best)
{
    if (cudaSetDevice(device) != cudaSuccess) return -3;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * 8, threads = 256;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks) != cudaSuccess) return -2;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    dfma_chains<<<blocks, threads, 0, st>>>(out, iters / 10 + 1, 0.999999, 1e-7, 32);  // warm-up
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, st);
        dfma_chains<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7, lanes);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (t < best) best = t;
    }
    const int err = cudaGetLastError() != cudaSuccess ? -3 : 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    const double flops = 2.0 * 8.0 * (double)iters * blocks * (threads / 32) * lanes;
    *ms_best = best;
    *tflops = flops / (best * 1e-3) / 1e12;
    return err;
}

extern "C" int at_probe_fp64_fma(int device, void* stream, int iters, int reps, double* tflops, double* ms_best)
{
    return at_probe_fp64_fma_lanes(device, stream, iters, reps, 32, tflops, ms_best);
}

namespace {
__global__ void fn_eval(const double* __restrict__ x, double* __restrict__ y, int64_t n, int which)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        y[i] = which == 0 ? atk::at_exp(v) : which == 1 ? exp(v) : which == 2 ? atk::at_rcp(v) : 1.0 / v;
    }
}
} // namespace

// y[i] = f(x[i]) for device arrays of n doubles, on the default stream,
// synchronous: which = 0 the kernels' table-driven exponential at_exp,
// 1 CUDA's exp, 2 the kernels' Newton reciprocal at_rcp, 3 IEEE 1/x.
extern "C" int at_probe_fn(const double* x, double* y, int64_t n, int which)
{
    if (n <= 0) return 0;
    if (which < 0 || which > 3) return -1;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    fn_eval<<<blocks, 256>>>(x, y, n, which);
    if (cudaGetLastError() != cudaSuccess) return -3;
    return cudaDeviceSynchronize() != cudaSuccess ? -3 : 0;
}
