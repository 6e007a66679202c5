// at_cluster.cu -- advection-diffusion on a few PEs: the whole domain in one
// thread-block cluster, all steps of an at_step call in one launch.
//
// For small problems (config 0: 32 PEs of 64 points) the cost of a step is
// the hand-off between neighbouring PEs, not arithmetic.  Here every CTA of
// one cluster (up to 16, one per SM) holds m consecutive PEs: their state,
// stage argument, RK accumulator and their edge windows of the history ring
// stay in shared memory, a PE reads its neighbour's ring through distributed
// shared memory, and one cluster barrier per stage orders the ring writes of
// a stage before the reads of the next (split into arrive after the update
// and wait before the neighbour reads, with the stage's local work between).  One warp per PE, point j of the PE
// on lane j % 32.  The delays, the AT extrapolation, the stencil and the RK
// update are those of the per-stage kernels, with the same arithmetic in the
// same order, so results are bitwise equal to them.  The global history ring
// is read at the start of a launch and written back at its end, so runs can
// switch between paths between at_step calls.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "at_device.cuh"

namespace cg = cooperative_groups;

namespace atk {

template <int H, int PPL>
__global__ void __launch_bounds__(128) cluster_advdiff(const StageArgs a, int64_t level0, int64_t nsteps)
{
    constexpr int B = 32 * PPL;
    cg::cluster_group cl = cg::this_cluster();
    const int m = (int)(blockDim.x >> 5);  // PEs of this CTA
    const int lane = threadIdx.x & 31;
    const int lp = threadIdx.x >> 5;       // local PE of this warp
    const int64_t pe = (int64_t)blockIdx.x * m + lp;
    const int S = a.S, R = a.R;
    extern __shared__ double sm[];
    double* U = sm;                                 // u^n                [m][B]
    double* X = U + m * B;                          // stage argument     [m][B]
    double* ACC = X + m * B;                        // RK accumulator     [m][B]
    double* W = ACC + m * B;                        // stencil rows       [m][B + 2H]
    double* RING = W + m * (B + 2 * H);             // edge windows       [R][S][m][2][H]
    auto ridx = [&](int64_t level, int stage, int l, int side, int h) {
        const int r = (int)((uint32_t)level % (uint32_t)R);
        return (((r * S + stage) * m + l) * 2 + side) * H + h;
    };
    for (int i = threadIdx.x; i < m * B; i += blockDim.x) {
        const int l = i / B, j = i - l * B;
        const double x = a.u[(int64_t)blockIdx.x * m * B + (int64_t)l * B + j];
        U[i] = x;
        X[i] = x;
    }
    for (int i = threadIdx.x; i < R * S * m * 2 * H; i += blockDim.x) {
        const int h = i % H, side = (i / H) % 2, l = (i / (2 * H)) % m, st = (i / (2 * H * m)) % S;
        const int r = i / (2 * H * m * S);
        RING[i] = a.ring[ring_index(a, r, st, (int64_t)blockIdx.x * m + l, side, h, 0)];
    }
    cl.sync();

    const int nw = (a.mode == AT) ? a.q + 1 : 1;
    double* Wl = W + lp * (B + 2 * H);
    bool bad = false;
    for (int64_t n = level0; n < level0 + nsteps; ++n) {
        for (int s = 0; s < S; ++s) {
            const bool last = (s == S - 1);
            const int64_t Ln = last ? n + 1 : n;
            const int sn = last ? 0 : s + 1;
            // local work first, while the previous stage's cluster barrier completes:
            // the delays of this stage and the own points of the stencil row
            int k = 0;
            const int side = lane < H ? 0 : 1;
            const int h = lane - side * H;
            if (lane < 2 * H) {
                k = keff_at(a, n, s, pe, side);
                if (h == 0) log_delay(a, n, s, pe, side, k);
            }
#pragma unroll
            for (int i = 0; i < PPL; ++i) Wl[H + lane + 32 * i] = X[lp * B + lane + 32 * i];
            if (n > level0 || s > 0) cl.barrier_wait();  // every CTA's ring writes of the previous stage
            if (lane < 2 * H) {  // one buffer point: delayed levels of the neighbour's ring, extrapolation
                const int64_t nbr = side == 0 ? (pe == 0 ? a.P - 1 : pe - 1) : (pe == a.P - 1 ? 0 : pe + 1);
                const int rank = (int)(nbr / m), nl = (int)(nbr - (int64_t)rank * m);
                const double* src = rank == (int)blockIdx.x ? RING : cl.map_shared_rank(RING, rank);
                double v[AT_QMAX + 1];
#pragma unroll
                for (int l = 0; l <= AT_QMAX; ++l) {
                    v[l] = 0.0;  // a level with weight 0 is not part of the scheme (and may not exist yet)
                    if (l < nw && ((a.wnz[k] >> l) & 1)) v[l] = src[ridx(n - k - l, s, nl, 1 - side, h)];
                }
                double acc = ((a.mode == AT) ? a.w[k][0] : 1.0) * v[0];
#pragma unroll
                for (int l = 1; l <= AT_QMAX; ++l)
                    if (l < nw) acc = fma(a.w[k][l], v[l], acc);
                Wl[side == 0 ? h : H + B + h] = acc;
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < PPL; ++i) {
                const int j = lane + 32 * i;
                const int it = lp * B + j;
                double K = 0.0;
#pragma unroll
                for (int o = -H; o <= H; ++o) K = fma(a.cm[o + H], Wl[H + j + o], K);
                // the update of the per-stage kernels (rk_update), into shared memory
                const double dt = a.dt, un = U[it], x = Wl[H + j];
                double y;
                if (a.rk == RK4) {
                    if (s == 0) {
                        ACC[it] = K;
                        y = fma(a.hdt, K, un);
                    } else if (s < 3) {
                        ACC[it] = fma(2.0, K, ACC[it]);
                        y = fma(s == 1 ? a.hdt : dt, K, un);
                    } else {
                        y = fma(a.dt6, ACC[it] + K, un);
                    }
                } else if (a.rk == RK3TVD) {
                    if (s == 0) y = fma(dt, K, x);
                    else if (s == 1) y = fma(0.75, un, 0.25 * fma(dt, K, x));
                    else y = fma(1.0 / 3.0, un, (2.0 / 3.0) * fma(dt, K, x));
                } else {
                    if (s == 0) {
                        ACC[it] = K;
                        y = fma(dt, K, un);
                    } else {
                        y = fma(a.hdt, ACC[it] + K, un);
                    }
                }
                X[it] = y;
                if (last) U[it] = y;
                if (nonfinite(y)) bad = true;
                if (j < H) RING[ridx(Ln, sn, lp, 0, j)] = y;
                else if (j >= B - H) RING[ridx(Ln, sn, lp, 1, j - (B - H))] = y;
            }
            cl.barrier_arrive();  // this stage's ring writes (and reads) done: release to the cluster
        }
    }
    if (nsteps > 0) cl.barrier_wait();  // no CTA leaves while another may still read its ring
    for (int i = threadIdx.x; i < m * B; i += blockDim.x) {
        const int l = i / B, j = i - l * B;
        a.Y[(int64_t)blockIdx.x * m * B + (int64_t)l * B + j] = U[i];
    }
    for (int i = threadIdx.x; i < R * S * m * 2 * H; i += blockDim.x) {
        const int h = i % H, side = (i / H) % 2, l = (i / (2 * H)) % m, st = (i / (2 * H * m)) % S;
        const int r = i / (2 * H * m * S);
        a.ring[ring_index(a, r, st, (int64_t)blockIdx.x * m + l, side, h, 0)] = RING[i];
    }
    if (bad) atomicOr(a.status, 1);
}

} // namespace atk

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

void* cluster_fn(int H, int ppl)
{
#define AT_CL(HH)                                                        \
    switch (ppl) {                                                       \
    case 1: return (void*)atk::cluster_advdiff<HH, 1>;                   \
    case 2: return (void*)atk::cluster_advdiff<HH, 2>;                   \
    case 4: return (void*)atk::cluster_advdiff<HH, 4>;                   \
    default: return (void*)atk::cluster_advdiff<HH, 8>;                  \
    }
    if (H == 1) { AT_CL(1) }
    if (H == 2) { AT_CL(2) }
    AT_CL(3)
#undef AT_CL
}

size_t cluster_smem(int B, int H, int m, int R, int S)
{
    return sizeof(double) * ((size_t)3 * m * B + (size_t)m * (B + 2 * H) + (size_t)R * S * m * 2 * H);
}

} // namespace

// CTAs of the cluster (one per SM) for P PEs of B points of advection-
// diffusion, or 0 when the cluster path does not apply: B of 32..256 points
// (a multiple of 32), at most 4 PEs per CTA, at most 16 CTAs (sizes above 8
// are non-portable; every size is checked with the occupancy query).
int atk_cluster_size(int pde, int order, int B, int64_t P, int R, int S, int device)
{
    if (pde != atk::ADVDIFF || !(B == 32 || B == 64 || B == 128 || B == 256)) return 0;
    const int H = order / 2;
    int C = 0;
    // the smallest cluster with at most 4 PEs per CTA: more warps per CTA hide
    // more latency and fewer CTAs meet at the barrier (measured on GB300 for
    // 32 PEs of 64 points: 8 CTAs 8.3, 16 CTAs 8.9, 4 CTAs 10.2 us per step)
    for (int c = 1; c <= (int)(P < 16 ? P : 16); ++c)
        if (P % c == 0 && P / c <= 4) {
            C = c;
            break;
        }
    if (C == 0) return 0;
    const int m = (int)(P / C);
    void* fn = cluster_fn(H, B / 32);
    const size_t smem = cluster_smem(B, H, m, R, S);
    if (cudaSetDevice(device) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(32 * m);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return 0;
    }
    return C;
}

cudaError_t atk_launch_cluster(const atk::StageArgs& a, int order, int csize, int64_t level0, int64_t nsteps,
                               cudaStream_t st)
{
    const int H = order / 2, m = (int)(a.P / csize);
    void* fn = cluster_fn(H, a.B / 32);
    const size_t smem = cluster_smem(a.B, H, m, a.R, a.S);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(32 * m);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    atk::StageArgs args = a;
    void* params[] = {(void*)&args, (void*)&level0, (void*)&nsteps};
    return cudaLaunchKernelExC(&cfg, fn, params);
}
