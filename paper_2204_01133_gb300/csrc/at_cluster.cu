// at_cluster.cu -- advection-diffusion on a few PEs: the whole domain in one
// thread-block cluster, all steps of an at_step call in one launch.
//
// For small problems (2,048 points in 32 PEs of 64 points) the cost of a
// step is the hand-off between neighbouring PEs, not arithmetic.  Here every
// CTA of one cluster (up to 16, one per SM) holds m consecutive PEs: their
// state, stage argument, RK accumulator and their edge windows of the history
// ring stay in shared memory, a PE reads its neighbour's ring through
// distributed shared memory, and one cluster barrier per stage orders the ring
// writes of a stage before the reads of the next.  The barrier is split into
// an arrive after the update and a wait before the one read that needs it (the
// neighbour's level of this step, delay 0); the delays, the neighbour's older
// levels and the copy of the own points into the stencil row go between the
// two.  A PE takes 1, 2, 4 or 8 warps (as many as bring the CTA to 8 warps,
// at most one per 32 points); each warp has its share of the points, point j
// of the share on lane j % 32, and its own stencil row, the first and last
// warp of a PE also its left and right buffer points.  The stage argument is
// double-buffered, so the warps of a PE meet only at the cluster barrier.  The
// delays, the AT extrapolation, the stencil and the RK update are those of
// the per-stage kernels, with the same arithmetic in the same order (a delay-0
// buffer value is the neighbour's value itself: its weights are the exact
// ratios (1, +-0, ...), which change at most the sign of a zero, and no
// stencil sum sees that), so results are bitwise equal to them.  The global
// history ring is read at the start of a launch and written back at its end,
// so runs can switch between paths between at_step calls.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "at_device.cuh"

namespace cg = cooperative_groups;

namespace atk {

template <int H, int PPL, int WPP>
__global__ void __launch_bounds__(256) cluster_advdiff(const StageArgs a, int64_t level0, int64_t nsteps)
{
    constexpr int B = 32 * PPL;       // PE size
    constexpr int PPW = PPL / WPP;    // points per lane of each of the PE's WPP warps
    constexpr int SW = 32 * PPW;      // points of a warp's share of its PE
    cg::cluster_group cl = cg::this_cluster();
    const int m = (int)(blockDim.x >> 5) / WPP;  // PEs of this CTA
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int lp = wib / WPP;                      // local PE of this warp
    const int hw = wib - lp * WPP;                 // which share of the PE's points
    const int j0 = hw * SW;                        // first point of the share
    const int64_t pe = (int64_t)blockIdx.x * m + lp;
    const int S = a.S, R = a.R;
    extern __shared__ double sm[];
    double* U = sm;                                 // u^n                          [m][B]
    double* X = U + m * B;                          // stage argument, two parities [2][m][B]
    double* ACC = X + 2 * m * B;                    // RK accumulator               [m][B]
    double* W = ACC + m * B;                        // stencil row of each warp     [m * WPP][SW + 2H]
    double* RING = W + m * WPP * (SW + 2 * H);      // edge windows                 [R][S][m][2][H]
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
    double* Wr = W + wib * (SW + 2 * H);
    // Buffer points: both sides on the warp of a one-warp PE, else the left
    // side on the PE's first warp and the right side on its last.  Between
    // the warps of a PE the stencil reads H points of the neighbouring share.
    const bool buf = WPP == 1 ? lane < 2 * H : (lane < H && (hw == 0 || hw == WPP - 1));
    const int side = WPP == 1 ? (lane < H ? 0 : 1) : (hw == 0 ? 0 : 1);
    const int h = WPP == 1 ? lane - side * H : lane;
    const bool halo_l = WPP > 1 && hw > 0 && lane < H;          // left H points from the previous share
    const bool halo_r = WPP > 1 && hw < WPP - 1 && lane < H;    // right H points from the next share
    const int64_t nbr = side == 0 ? (pe == 0 ? a.P - 1 : pe - 1) : (pe == a.P - 1 ? 0 : pe + 1);
    const int rank = (int)(nbr / m), nl = (int)(nbr - (int64_t)rank * m);
    const double* src = rank == (int)blockIdx.x ? RING : cl.map_shared_rank(RING, rank);
    bool bad = false;
    int par = 0;  // parity of the stage argument this stage reads
    for (int64_t n = level0; n < level0 + nsteps; ++n) {
        for (int s = 0; s < S; ++s) {
            const bool last = (s == S - 1);
            const int64_t Ln = last ? n + 1 : n;
            const int sn = last ? 0 : s + 1;
            const double* Xc = X + par * m * B + lp * B;      // this stage's argument of the PE
            double* Xn = X + (1 - par) * m * B + lp * B;      // the next one
            // Before the previous stage's cluster barrier completes: the delays,
            // the neighbour's levels for delays k >= 1 (written at least a step
            // ago, and their slots are not written in the stage in flight) and
            // the warp's own points of the stencil row (written by the same
            // lanes in the previous stage).
            int k = 0;
            double bv = 0.0;
            double v[AT_QMAX + 1];
            if (buf) {
                k = keff_at(a, n, s, pe, side);
                if (h == 0) log_delay(a, n, s, pe, side, k);
#pragma unroll
                for (int l = 0; l <= AT_QMAX; ++l) {
                    v[l] = 0.0;  // a level with weight 0 is not part of the scheme (and may not exist yet)
                    if (k >= 1 && l < nw && ((a.wnz[k] >> l) & 1)) v[l] = src[ridx(n - k - l, s, nl, 1 - side, h)];
                }
            }
#pragma unroll
            for (int i = 0; i < PPW; ++i) Wr[H + lane + 32 * i] = Xc[j0 + lane + 32 * i];
            // every CTA's ring writes and the other warps' stage arguments of the
            // previous stage
            if (n > level0 || s > 0) cl.barrier_wait();
            if (buf) {
                // delay 0: the weights are exact integer ratios (1, +-0, ..., +-0),
                // so the extrapolation is this level's value, just written, up to
                // the sign of a zero; the stencil sum starts from +0, where a zero
                // adds nothing whatever its sign (bitwise the per-stage results)
                if (k == 0) bv = src[ridx(n, s, nl, 1 - side, h)];
                else {
                    bv = ((a.mode == AT) ? a.w[k][0] : 1.0) * v[0];
#pragma unroll
                    for (int l = 1; l <= AT_QMAX; ++l)
                        if (l < nw) bv = fma(a.w[k][l], v[l], bv);
                }
                Wr[side == 0 ? h : H + SW + h] = bv;
            }
            if (halo_l) Wr[lane] = Xc[j0 - H + lane];
            if (halo_r) Wr[H + SW + lane] = Xc[j0 + SW + lane];
            __syncwarp();
#pragma unroll
            for (int i = 0; i < PPW; ++i) {
                const int jw = lane + 32 * i;  // point of the share
                const int j = j0 + jw;         // point of the PE
                const int it = lp * B + j;
                double K = 0.0;
#pragma unroll
                for (int o = -H; o <= H; ++o) K = fma(a.cm[o + H], Wr[H + jw + o], K);
                // the update of the per-stage kernels (rk_update), into shared memory
                const double dt = a.dt, un = U[it], x = Wr[H + jw];
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
                Xn[j] = y;
                if (last) U[it] = y;
                if (nonfinite(y)) bad = true;
                if (j < H) RING[ridx(Ln, sn, lp, 0, j)] = y;
                else if (j >= B - H) RING[ridx(Ln, sn, lp, 1, j - (B - H))] = y;
            }
            __syncwarp();  // the row is read by all lanes before the next stage rewrites it
            cl.barrier_arrive();  // this stage's ring and stage-argument writes done: release to the cluster
            par = 1 - par;
        }
    }
    if (nsteps > 0) cl.barrier_wait();  // no CTA leaves while another may still read its ring
    for (int i = threadIdx.x; i < m * B; i += blockDim.x) {
        const int l = i / B, j = i - l * B;
        a.Y[(int64_t)blockIdx.x * m * B + (int64_t)l * B + j] = U[i];
    }
    for (int i = threadIdx.x; i < R * S * m * 2 * H; i += blockDim.x) {
        const int h2 = i % H, sd = (i / H) % 2, l = (i / (2 * H)) % m, st = (i / (2 * H * m)) % S;
        const int r = i / (2 * H * m * S);
        a.ring[ring_index(a, r, st, (int64_t)blockIdx.x * m + l, sd, h2, 0)] = RING[i];
    }
    if (bad) atomicOr(a.status, 1);
}

} // namespace atk

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

// warps per PE: as many as bring a CTA of m PEs to kClusterWarps warps (at
// most one per 32 points), so the FP64 work of a PE is issued from several SM
// sub-partitions
constexpr int kClusterMaxPePerCta = 4;
constexpr int kClusterWarps = 8;
int cluster_wpp(int B, int m)
{
    int w = kClusterWarps / m;
    if (w > B / 32) w = B / 32;
    return w >= 8 ? 8 : w >= 4 ? 4 : w >= 2 ? 2 : 1;
}

void* cluster_fn(int H, int ppl, int wpp)
{
#define AT_CL(HH)                                                                  \
    if (wpp == 1) {                                                                \
        switch (ppl) {                                                             \
        case 1: return (void*)atk::cluster_advdiff<HH, 1, 1>;                      \
        case 2: return (void*)atk::cluster_advdiff<HH, 2, 1>;                      \
        case 4: return (void*)atk::cluster_advdiff<HH, 4, 1>;                      \
        default: return (void*)atk::cluster_advdiff<HH, 8, 1>;                     \
        }                                                                          \
    }                                                                              \
    if (wpp == 2) {                                                                \
        switch (ppl) {                                                             \
        case 2: return (void*)atk::cluster_advdiff<HH, 2, 2>;                      \
        case 4: return (void*)atk::cluster_advdiff<HH, 4, 2>;                      \
        default: return (void*)atk::cluster_advdiff<HH, 8, 2>;                     \
        }                                                                          \
    }                                                                              \
    if (wpp == 4) {                                                                \
        if (ppl == 4) return (void*)atk::cluster_advdiff<HH, 4, 4>;                \
        return (void*)atk::cluster_advdiff<HH, 8, 4>;                              \
    }                                                                              \
    return (void*)atk::cluster_advdiff<HH, 8, 8>;
    if (H == 1) { AT_CL(1) }
    if (H == 2) { AT_CL(2) }
    AT_CL(3)
#undef AT_CL
}

size_t cluster_smem(int B, int H, int m, int R, int S)
{
    const int w = cluster_wpp(B, m);
    return sizeof(double) *
           ((size_t)4 * m * B + (size_t)m * w * (B / w + 2 * H) + (size_t)R * S * m * 2 * H);
}

cudaLaunchConfig_t cluster_config(int B, int csize, int m, size_t smem, cudaStream_t st, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(32 * m * cluster_wpp(B, m));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
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
    // the largest cluster (the work of a stage spread over the most SMs) with
    // at most 4 PEs per CTA
    for (int c = (int)(P < 16 ? P : 16); c >= 1; --c)
        if (P % c == 0) {
            C = c;
            break;
        }
    if (C == 0 || P / C > kClusterMaxPePerCta) return 0;
    const int m = (int)(P / C);
    void* fn = cluster_fn(H, B / 32, cluster_wpp(B, m));
    const size_t smem = cluster_smem(B, H, m, R, S);
    if (cudaSetDevice(device) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(B, C, m, smem, 0, attr);
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
    void* fn = cluster_fn(H, a.B / 32, cluster_wpp(a.B, m));
    const size_t smem = cluster_smem(a.B, H, m, a.R, a.S);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(a.B, csize, m, smem, st, attr);
    atk::StageArgs args = a;
    void* params[] = {(void*)&args, (void*)&level0, (void*)&nsteps};
    return cudaLaunchKernelExC(&cfg, fn, params);
}
