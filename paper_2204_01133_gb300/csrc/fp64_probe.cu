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

// pipe-sharing probe: every thread runs 8 independent chains of `kind`
// (0: FP64 fma; 1: 64-bit integer multiply-add; 2: 64-bit integer add;
// 3: 32-bit integer multiply-add) and, when with_fp64, also the 8 FP64 fma
// chains of kind 0.  If a kind shares the FP64 pipe, running it beside the
// fma chains costs about the sum of the two times, otherwise about the max.
__global__ void __launch_bounds__(256) mixed_chains(double* out, uint64_t* iout, int iters, double a, double b,
                                                    uint64_t m, uint64_t c, int kind, int with_fp64)
{
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 0.1, x2 = x0 + 0.2, x3 = x0 + 0.3;
    double x4 = x0 + 0.4, x5 = x0 + 0.5, x6 = x0 + 0.6, x7 = x0 + 0.7;
    uint64_t i0 = threadIdx.x + 1, i1 = i0 + 3, i2 = i0 + 5, i3 = i0 + 7, i4 = i0 + 11, i5 = i0 + 13, i6 = i0 + 17,
             i7 = i0 + 19;
    uint32_t j0 = (uint32_t)i0, j1 = j0 + 3, j2 = j0 + 5, j3 = j0 + 7, j4 = j0 + 11, j5 = j0 + 13, j6 = j0 + 17,
             j7 = j0 + 19;
    const bool f = with_fp64 || kind == 0;
    for (int it = 0; it < iters; ++it) {
        if (f) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
        if (kind == 1) {
            i0 = i0 * m + c; i1 = i1 * m + c; i2 = i2 * m + c; i3 = i3 * m + c;
            i4 = i4 * m + c; i5 = i5 * m + c; i6 = i6 * m + c; i7 = i7 * m + c;
        } else if (kind == 2) {
            i0 += c ^ i7; i1 += c ^ i0; i2 += c ^ i1; i3 += c ^ i2;
            i4 += c ^ i3; i5 += c ^ i4; i6 += c ^ i5; i7 += c ^ i6;
        } else if (kind == 3) {
            const uint32_t mm = (uint32_t)m, cc = (uint32_t)c;
            j0 = j0 * mm + cc; j1 = j1 * mm + cc; j2 = j2 * mm + cc; j3 = j3 * mm + cc;
            j4 = j4 * mm + cc; j5 = j5 * mm + cc; j6 = j6 * mm + cc; j7 = j7 * mm + cc;
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    iout[blockIdx.x * blockDim.x + threadIdx.x] = (i0 ^ i1 ^ i2 ^ i3 ^ i4 ^ i5 ^ i6 ^ i7) + (j0 ^ j1 ^ j2 ^ j3 ^ j4 ^ j5 ^ j6 ^ j7);
}

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
        y[i] = which == 0 ? atk::at_exp(v) : which == 1 ? exp(v) : which == 2 ? atk::at_rcp(v)
             : which == 4 ? atk::at_rcp3(v) : 1.0 / v;
    }
}
} // namespace

// y[i] = f(x[i]) for device arrays of n doubles, on the default stream,
// synchronous: which = 0 the kernels' table-driven exponential at_exp,
// 1 CUDA's exp, 2 the kernels' Newton reciprocal at_rcp, 3 IEEE 1/x, 4 the
// kernels' cubic-step reciprocal at_rcp3.
extern "C" int at_probe_fn(const double* x, double* y, int64_t n, int which)
{
    if (n <= 0) return 0;
    if (which < 0 || which > 4) return -1;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    fn_eval<<<blocks, 256>>>(x, y, n, which);
    if (cudaGetLastError() != cudaSuccess) return -3;
    return cudaDeviceSynchronize() != cudaSuccess ? -3 : 0;
}

// Best-of-`reps` time (ms) of mixed_chains(kind, with_fp64) on a grid of
// 4 CTAs of 256 threads per SM; see mixed_chains for what the times show.
extern "C" int at_probe_pipe_mix(int device, int kind, int with_fp64, int iters, int reps, double* ms_best)
{
    if (kind < 0 || kind > 3 || iters < 1 || reps < 1) return -1;
    if (cudaSetDevice(device) != cudaSuccess) return -3;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * 4, threads = 256;
    double* out = nullptr;
    uint64_t* iout = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return -2;
    if (cudaMalloc(&iout, sizeof(uint64_t) * blocks * threads) != cudaSuccess) {
        cudaFree(out);
        return -2;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    mixed_chains<<<blocks, threads>>>(out, iout, iters / 10 + 1, 0.999999, 1e-7, 0x9E3779B97F4A7C15ull, 12345, kind,
                                      with_fp64);
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        mixed_chains<<<blocks, threads>>>(out, iout, iters, 0.999999, 1e-7, 0x9E3779B97F4A7C15ull, 12345, kind,
                                          with_fp64);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (t < best) best = t;
    }
    const int err = cudaGetLastError() != cudaSuccess ? -3 : 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(iout);
    *ms_best = best;
    return err;
}
