// at_persist.cu -- persistent, neighbour-synchronised AT kernel (central PDEs).
//
// One CTA owns one virtual PE for a whole run of steps.  The PE's u^n, RK
// accumulator and stage argument live in shared memory between stages and
// steps; only the edge windows go through the history ring in global memory
// (L2), exactly as in the per-stage path, so the arithmetic and its order are
// identical and the results agree bit for bit.
//
// The CTAs synchronise only pairwise, through per-PE progress counters
// done[p] = n*S + s + 1 after stage s of step n.  Before stage s of step n,
// PE p needs its neighbour's stage-s argument at level n-k: it waits for
// done[nbr] >= (n-k)*S + s.  With a drawn delay k >= 1 that is usually
// already true, so the asynchrony the AT scheme tolerates (Sec. 2.1-2.3)
// becomes slack in the GPU's own synchronisation: no grid barrier, no launch
// per stage.  Before overwriting a ring slot a PE waits until both
// neighbours are past every stage that can still read the slot's old level
// (the ring keeps `slack` spare levels, so this rarely binds).  Results do
// not depend on timing: what is read is fixed by the Philox draws.
//
// Every wait is bounded (wait_limit polls with a short sleep).  A wait that
// runs out sets status bit 1 and a global abort flag; every other wait sees
// the flag and returns, and the kernel ends: the host reports AT_ETIMEOUT.
// The launch is cooperative, so all CTAs are resident at once.
#include <cuda/atomic>
#include <cuda_runtime.h>

#include "at_device.cuh"

namespace atk {

__device__ __forceinline__ int64_t load_acquire(int64_t* p)
{
    cuda::atomic_ref<int64_t, cuda::thread_scope_device> r(*p);
    return r.load(cuda::memory_order_acquire);
}

__device__ __forceinline__ void store_release(int64_t* p, int64_t v)
{
    cuda::atomic_ref<int64_t, cuda::thread_scope_device> r(*p);
    r.store(v, cuda::memory_order_release);
}

// bounded wait for *ctr >= target; false if it ran out or another wait did
__device__ bool wait_ge(const StageArgs& a, int64_t* ctr, int64_t target)
{
    if (load_acquire(ctr) >= target) return true;
    for (int64_t it = 0; it < a.wait_limit; ++it) {
        __nanosleep(128);
        if (load_acquire(ctr) >= target) return true;
        if ((it & 63) == 0 && *(volatile int*)a.abort_flag) return false;
    }
    atomicOr(a.status, 2);
    atomicExch(a.abort_flag, 1);
    return false;
}

// stencil, source and RK update of own point (v, jl) for stage s, in shared
// memory: the same arithmetic, in the same order, as the per-stage kernels
// (the Arrhenius factor exp(-Ea/T) arrives precomputed in E)
template <int PDE, int H>
__device__ __forceinline__ double point_update(const StageArgs& a, int s, int v, int jl, const double* G,
                                               const double* E, double* X, double* U, double* ACC, int W2, int B,
                                               bool last)
{
    const int it = v * B + jl;
    const int c = jl + H;
    double K = 0.0;
    const double x = X[it];
    if constexpr (PDE == ADVDIFF) {
#pragma unroll
        for (int o = -H; o <= H; ++o) K = fma(a.cm[o + H], G[c + o], K);
    } else {
        const double* F = G + v * W2;
#pragma unroll
        for (int o = -H; o <= H; ++o)
            if (o != 0) K = fma(a.c1[o + H], F[c + o], K);
        if (v > 0) {
            const double* D = G + (3 + v) * W2;
#pragma unroll
            for (int o = -H; o <= H; ++o) K = fma(a.c2v[v - 1][o + H], D[c + o], K);
        }
        if (v == 3) K = fma(-a.prm[4] * x, E[jl], K);
    }
    const double dt = a.dt;
    const double un = U[it];
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
        const double xs = fma(dt, K, x);
        if (s == 0) y = xs;
        else if (s == 1) y = fma(0.75, un, 0.25 * xs);
        else y = fma(1.0 / 3.0, un, (2.0 / 3.0) * xs);
    } else {
        if (s == 0) {
            ACC[it] = K;
            y = fma(dt, K, un);
        } else {
            y = fma(a.hdt, ACC[it] + K, un);
        }
    }
    X[it] = y;  // next stage argument (u^{n+1} after the last stage)
    if (last) U[it] = y;
    return y;
}

// named barriers (ids 1..5; 0 is __syncthreads): bar.sync waits until
// `count` threads have arrived, bar.arrive counts this warp without waiting
template <int ID>
__device__ __forceinline__ void bar_sync(int count)
{
    asm volatile("bar.sync %0, %1;" ::"n"(ID), "r"(count) : "memory");
}
template <int ID>
__device__ __forceinline__ void bar_arrive(int count)
{
    asm volatile("bar.arrive %0, %1;" ::"n"(ID), "r"(count) : "memory");
}
// the barrier of parity p among a pair (ids B0, B0 + 1), with immediate ids
template <int B0>
__device__ __forceinline__ void bar_sync_p(int p, int count)
{
    if (p) bar_sync<B0 + 1>(count);
    else bar_sync<B0>(count);
}
template <int B0>
__device__ __forceinline__ void bar_arrive_p(int p, int count)
{
    if (p) bar_arrive<B0 + 1>(count);
    else bar_arrive<B0>(count);
}

// GB300's FP64 unit spends the same time on a warp instruction whatever the
// number of active lanes, so the work is laid out in whole, uniform warps
// with fixed roles.  Stage t (= step n, stage s) of a PE:
//   (A) derive warps: own-point derived quantities into G[t % 2] and the
//       Arrhenius factor exp(-Ea/T) from the temperature among them;
//   (C) all worker warps: stencil, source and RK update of every (point,
//       variable), one variable per warp, the edge points straight into the
//       ring; then the progress counter is published.
// After a stage, warp 0 derives the new stage argument at the PE's 2H edge
// points into a ring of derived quantities and publishes the stage.  The
// halo warp runs one stage ahead of the workers: while they do stage t it
// takes the delays of stage t + 1, waits (boundedly) for the neighbours'
// data, reads their derived quantities of the delayed levels and writes the
// weighted buffer values into the halo columns of G[(t + 1) % 2], so that
// its latency hides behind the workers' arithmetic (a drawn delay of 0
// then costs the neighbour's edge derivation, not a derivation under the
// contention of the receiving SM).  Named barriers, by
// the parity p of the stage:
//   1 + p  halo of stage t ready      (halo warp arrives, workers sync)
//   3 + p  G[p] no longer read        (workers arrive after stage t, the
//                                      halo warp syncs before filling G[p]
//                                      for stage t + 2)
//   5      workers' phase C done      (workers only, before publishing)
// A failed wait records the stage in s_abort_at before the halo warp
// arrives; the workers stop at that stage and the halo warp matches the one
// arrival it would otherwise have consumed, so every barrier completes.
template <int PDE, int H>
__global__ void __launch_bounds__(288, 2) persist_central(const StageArgs a, int64_t level0, int64_t nsteps)
{
    using P = Phys<PDE>;
    constexpr int NV = P::NV, ND = P::ND;
    const int B = a.B, W2 = B + 2 * H, S = a.S;
    const int64_t pe = place_rank(a);
    const int64_t nbr[2] = {pe == 0 ? a.P - 1 : pe - 1, pe == a.P - 1 ? 0 : pe + 1};
    extern __shared__ double sm[];
    double* U = sm;                // u^n                 [NV][B]
    double* ACC = U + NV * B;      // RK accumulator      [NV][B]
    double* X = ACC + NV * B;      // stage argument      [NV][B]
    double* G2 = X + NV * B;       // derived, by stage parity [2][ND][W2]
    double* HS = G2 + 2 * ND * W2; // halo levels         [2H(q+1)][ND]
    double* E = HS + 2 * H * (AT_QMAX + 1) * ND;  // exp(-Ea/T) of own points [B]
    __shared__ long long s_abort_at;  // first stage whose halo could not be formed
    __shared__ int s_k[2];
    __shared__ int s_fail;
    const int nw = (a.mode == AT) ? a.q + 1 : 1;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int hwarp = (int)(blockDim.x >> 5) - 1;  // the halo warp
    const int nwork = hwarp * 32;                    // threads of the worker warps
    const int nall = nwork + 32;
    // warps per role in phase A: enough for one point per lane
    int bw = (B + 31) / 32;
    if (bw > hwarp) bw = hwarp;
    if (bw < 1) bw = 1;
    // Roles of the worker warps in phase A.  Warp w runs on SM sub-partition
    // w % 4 and the halo warp on hwarp % 4 (sub-partition 0 with 8 workers).
    // The derive warps start at warp 1, so that two of them (a 64-point PE)
    // take sub-partitions 1 and 2, away from the halo warp.
    int derive_rank = -1;
    if (warp < hwarp) {
        const int r = (warp + hwarp - 1) % hwarp;  // warp 1 -> rank 0, warp 2 -> rank 1, ...
        if (r < bw) derive_rank = r;
    }

    for (int i = threadIdx.x; i < NV * B; i += blockDim.x) {
        const int v = i / B, j = i - v * B;
        const double x = a.u[v * a.N + pe * B + j];
        U[i] = x;
        X[i] = x;
    }
    if (threadIdx.x == 0) s_abort_at = 0x7fffffffffffffffLL;
    int bad = 0;
    // this PE's ring of derived quantities of its edge windows, from its ring
    // of stage arguments (steps before this launch may have run elsewhere);
    // the neighbours read it only after the release below
    for (int i = threadIdx.x; i < a.R * S * 2 * H; i += blockDim.x) {
        const int h = i % H, side = (i / H) % 2, st = (i / (2 * H)) % S, r = i / (2 * H * S);
        double Q[NV], g[ND];
#pragma unroll
        for (int v = 0; v < NV; ++v) Q[v] = a.ring[ring_index(a, r, st, pe, side, h, v)];
        P::derive(a, Q, g);
        const int64_t gi = gring_index(a, r, st, pe, side, h, ND);
#pragma unroll
        for (int d = 0; d < ND; ++d) a.gring[gi + d] = g[d];
    }
    __syncthreads();
    if (threadIdx.x == 0 && pe != a.withhold_pe) store_release(a.done + pe, level0 * S);
    const int64_t T = nsteps * S;

    if (warp == hwarp) {
        // ---- the halo warp: stage t's buffer values, one stage ahead ----
        int64_t n = level0;
        int s = 0;
        for (int64_t t = 0; t < T; ++t) {
            const int p = (int)(t & 1);
            double* G = G2 + p * ND * W2;
            const bool last = (s == S - 1);
            const int64_t Ln = last ? n + 1 : n;  // the stage argument stage t produces: (Ln, sn)
            const int sn = last ? 0 : s + 1;
            if (t >= 2) bar_sync_p<3>(p, nall);  // the workers are done with G[p] (stage t - 2)
            if (lane == 0) s_fail = 0;
            __syncwarp();
            if (lane < 2) {
                const int side = lane;
                int k;
                bool ok;
                // one bounded wait for both conditions on the neighbour's
                // progress: the stage-s argument this stage reads has been
                // published, and the ring slot of (Ln, sn) this stage writes is
                // no longer read by it
                const int64_t free_at = (Ln - a.slack - 1) * S + sn + 1;
                if (a.arrival) {
                    // the freshest stage-s argument of the neighbour that has
                    // arrived, once one recent enough for the clamp is there
                    const int kc = kcap_at(a, n);
                    const int64_t need = (n - kc) * S + s;
                    ok = wait_ge(a, a.done + nbr[side], need > free_at ? need : free_at);
                    const int64_t m = (load_acquire(a.done + nbr[side]) - s) / S;
                    k = m >= n ? 0 : (int)(n - m);
                    if (k > kc) k = kc;  // only if the wait gave up
                } else {
                    // the neighbour's stage-s argument at the drawn level n-k
                    k = keff_at(a, n, s, pe, side);
                    const int64_t need = (n - k) * S + s;
                    ok = wait_ge(a, a.done + nbr[side], need > free_at ? need : free_at);
                }
                s_k[side] = k;
                log_delay(a, n, s, pe, side, k);
                if (!ok) s_fail = 1;
            }
            __syncwarp();
            const bool failed = *(volatile int*)&s_fail != 0;
            if (!failed) {
                // A side with delay 0 has weights (1, +-0, ...), exact integer
                // ratios: its buffer values are the neighbour's level-n quantities
                // themselves, up to the sign of a zero, which no stencil sum sees
                // (they start from +0 and take the buffer columns as factors), so
                // they are copied without FP64 work.  Their loads go first, so
                // that they are in flight with those of the other side.  (With
                // one derived quantity the weighted sum is a few instructions on
                // 2H lanes and the staging of the general case measured faster:
                // there every side takes it.)
                constexpr bool copy0 = ND > 1;
                constexpr int NI = 2 * H * ND, NP = (NI + 31) / 32;
                double cur[NP];
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    const int c = lane + 32 * i;
                    cur[i] = 0.0;
                    if (c < NI) {
                        const int hp = c / ND, d = c - hp * ND;
                        const int side = hp < H ? 0 : 1;
                        if (copy0 && s_k[side] == 0)
                            cur[i] = __ldcg(a.gring + gring_index(a, n, s, nbr[side], 1 - side,
                                                                 side == 0 ? hp : hp - H, ND) + d);
                    }
                }
                // the other sides: their levels n-k-l into HS
                const int tt = lane;
                if (tt < 2 * H * nw) {
                    const int hp = tt / nw, l = tt - hp * nw;
                    const int side = hp < H ? 0 : 1;
                    const int h = side == 0 ? hp : hp - H;
                    const int k = s_k[side];
                    const bool staged = !copy0 || k >= 1;
                    if (staged && ((a.wnz[k] >> l) & 1)) {
                        // the neighbour's own derived quantities of that level
                        const int64_t gi = gring_index(a, n - k - l, s, nbr[side], 1 - side, h, ND);
#pragma unroll
                        for (int d = 0; d < ND; ++d) HS[tt * ND + d] = __ldcg(a.gring + gi + d);
                    } else if (staged) {
#pragma unroll
                        for (int d = 0; d < ND; ++d) HS[tt * ND + d] = 0.0;
                    }
                }
                __syncwarp();
                // weighted sum over levels, in level order: lanes (buffer point, quantity)
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    const int c = lane + 32 * i;
                    if (c < NI) {
                        const int hp = c / ND, d = c - hp * ND;
                        const int k = s_k[hp < H ? 0 : 1];
                        double acc = cur[i];
                        if (!copy0 || k >= 1) {
                            acc = ((a.mode == AT) ? a.w[k][0] : 1.0) * HS[(hp * nw) * ND + d];
                            for (int l = 1; l < nw; ++l) acc = fma(a.w[k][l], HS[(hp * nw + l) * ND + d], acc);
                        }
                        G[d * W2 + (hp < H ? hp : B + hp)] = acc;
                    }
                }
            } else if (lane == 0) {
                s_abort_at = t;
            }
            __syncwarp();
            bar_arrive_p<1>(p, nall);  // stage t's halo is ready (or the run stops at t)
            if (failed) {
                // the workers arrive on 3 + parity after stage t - 1 and stop at t:
                // consume that arrival so the barrier completes
                if (t >= 1 && t + 1 < T) bar_sync_p<3>((int)((t - 1) & 1), nall);
                break;
            }
            if (++s == S) {
                s = 0;
                ++n;
            }
        }
    } else {
        // ---- the worker warps ----
        int64_t n = level0;
        int s = 0;
        for (int64_t t = 0; t < T; ++t) {
            const int p = (int)(t & 1);
            double* G = G2 + p * ND * W2;
            const bool last = (s == S - 1);
            const int64_t Ln = last ? n + 1 : n;
            const int sn = last ? 0 : s + 1;
            // (A)
            if (derive_rank >= 0) {
                for (int it = derive_rank * 32 + lane; it < B; it += bw * 32) {
                    double g[ND];
                    double Q[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) Q[v] = X[v * B + it];
                    P::derive(a, Q, g);
#pragma unroll
                    for (int d = 0; d < ND; ++d) G[d * W2 + H + it] = g[d];
                    if constexpr (PDE == RNS) E[it] = at_exp(-a.prm[5] * at_rcp3(g[7]));  // g[7] = T
                }
            }
            bar_sync_p<1>(p, nall);  // own derived quantities and stage t's halo in G[p]
            if (t >= *(volatile long long*)&s_abort_at) break;
            // (C) item (v, jl).  With one warp per 32 points of a variable, warp w
            // takes variable w % NV: the two warps of the density equation (first
            // derivatives only, the lightest) then share sub-partition 0 with the
            // halo warp, which is on the critical path when a drawn delay is 0.
            const bool by_warp = (nwork == NV * B) && (B % 32 == 0);
            for (int it = threadIdx.x; it < NV * B; it += nwork) {
                const int v = by_warp ? warp % NV : it / B;
                const int jl = by_warp ? (warp / NV) * 32 + lane : it - v * B;
                const double y = point_update<PDE, H>(a, s, v, jl, G, E, X, U, ACC, W2, B, last);
                if (nonfinite(y)) bad = 1;
                int side = -1, h = 0;
                if (jl < H) {
                    side = 0;
                    h = jl;
                } else if (jl >= B - H) {
                    side = 1;
                    h = jl - (B - H);
                }
                if (side >= 0) __stcg(a.ring + ring_index(a, Ln, sn, pe, side, h, v), y);
            }
            bar_sync<5>(nwork);
            // the derived quantities of the new stage argument at the edge
            // points, for the neighbours' halos; then publish: the barriers
            // order every worker's ring writes before lane 0's device-scope
            // release store, which is cumulative
            if (warp == 0) {
                if (lane < 2 * H) {
                    const int side = lane < H ? 0 : 1;
                    const int h = lane - side * H;
                    const int jl = side == 0 ? h : B - H + h;
                    double Q[NV], g[ND];
#pragma unroll
                    for (int v = 0; v < NV; ++v) Q[v] = X[v * B + jl];
                    P::derive(a, Q, g);
                    const int64_t gi = gring_index(a, Ln, sn, pe, side, h, ND);
#pragma unroll
                    for (int d = 0; d < ND; ++d) __stcg(a.gring + gi + d, g[d]);
                }
                __syncwarp();
                if (lane == 0 && pe != a.withhold_pe) store_release(a.done + pe, n * S + s + 1);
            }
            if (t + 2 < T) bar_arrive_p<3>(p, nall);  // G[p] may be refilled for stage t + 2
            if (++s == S) {
                s = 0;
                ++n;
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NV * B; i += blockDim.x) {
        const int v = i / B, j = i - v * B;
        a.Y[v * a.N + pe * B + j] = U[i];
    }
    if (bad) atomicOr(a.status, 1);
}

__global__ void counters_set(int64_t* done, int64_t P, int64_t value, int* abort_flag, int* place_count)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
        done[i] = value;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *abort_flag = 0;
        *place_count = 0;
    }
}

template <int PDE, int H>
void* persist_fn()
{
    return (void*)persist_central<PDE, H>;
}

} // namespace atk

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {
void* persist_kernel(int pde, int order)
{
    if (pde == atk::ADVDIFF) {
        if (order == 2) return atk::persist_fn<atk::ADVDIFF, 1>();
        if (order == 4) return atk::persist_fn<atk::ADVDIFF, 2>();
        return atk::persist_fn<atk::ADVDIFF, 3>();
    }
    if (pde == atk::RNS) {
        if (order == 2) return atk::persist_fn<atk::RNS, 1>();
        if (order == 4) return atk::persist_fn<atk::RNS, 2>();
        return atk::persist_fn<atk::RNS, 3>();
    }
    return nullptr;
}
} // namespace

size_t atk_persist_smem_bytes(int pde, int B, int H)
{
    const int nv = pde == atk::RNS ? 4 : 1, nd = pde == atk::RNS ? 8 : 1;
    return sizeof(double) *
           ((size_t)3 * nv * B + (size_t)2 * nd * (B + 2 * H) + (size_t)2 * H * (AT_QMAX + 1) * nd + (size_t)B);
}

// worker warps for the PE's points (at least two roles' worth for phase A)
// plus one halo warp
int atk_persist_block(int pde, int B)
{
    const int nv = pde == atk::RNS ? 4 : 1;
    const int bw = (B + 31) / 32;
    int want = ((nv * B + 31) / 32) * 32;
    if (want > 256) want = 256;
    if (want < 64 * bw) want = 64 * bw;
    if (want > 256) want = 256;
    return want + 32;
}

// how many PEs one cooperative launch can hold (0: not available)
int64_t atk_persist_capacity(int pde, int order, int B, int device)
{
    void* fn = persist_kernel(pde, order);
    if (!fn) return 0;
    const int H = order / 2;
    const size_t smem = atk_persist_smem_bytes(pde, B, H);
    if (smem > 200 * 1024) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int per_sm = 0, sms = 0, coop = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, atk_persist_block(pde, B), smem) != cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop) return 0;
    return (int64_t)per_sm * sms;
}

cudaError_t atk_launch_persist(const atk::StageArgs& a, int pde, int order, int64_t level0, int64_t nsteps,
                               cudaStream_t st)
{
    void* fn = persist_kernel(pde, order);
    if (!fn) return cudaErrorInvalidValue;
    atk::counters_set<<<(unsigned)((a.P + 255) / 256 < 1024 ? (a.P + 255) / 256 : 1024), 256, 0, st>>>(
        a.done, a.P, (level0 - a.R) * a.S, a.abort_flag, a.place_count);  // raised to level0 S by each PE's prologue
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = atk_persist_smem_bytes(pde, a.B, order / 2);
    // the attribute is per kernel, not per context: set it for this launch
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    atk::StageArgs args = a;
    void* params[] = {(void*)&args, (void*)&level0, (void*)&nsteps};
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)a.P), dim3(atk_persist_block(pde, a.B)), params, smem, st);
}
