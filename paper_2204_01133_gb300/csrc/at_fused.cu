// at_fused.cu -- advection-diffusion, one launch per RK step: all S stages
// of a step in one pass over the state (the step-fused kernel).
//
// The per-stage path reads and writes the stage argument, u^n and the RK
// accumulator once per stage (17 arrays of the field per RK4 step).  Here a
// CTA holds W consecutive PEs, one warp each, and keeps their stage
// arguments in shared memory and u^n and the accumulator in registers for
// the whole step: the field is read once (u^n) and written once (u^{n+1}).
//
// What a PE needs from outside its own points at stage s is its buffer
// values: the extrapolation (Eq. 7 / Appendix A) of the neighbour's edge
// window at the delayed levels n-k-l (Sec. 2.3: the stage-level history).
// Levels older than n come from the global history ring, written by earlier
// steps.  Level n itself (k = 0) is the neighbour's stage argument of this
// very step: inside the CTA it is in shared memory; for the two PEs beyond
// the CTA's ends (the outer neighbours) it is recomputed here, by a strip
// warp, from u^n over the S H points of the neighbour nearest the CTA
// (the overlapped halo of a step-fused scheme: stage s needs the
// neighbour's stage-(s-1) values H points deeper, so the strip shrinks by H
// per stage).  The recomputation uses the outer neighbour's own delay draws
// and the same arithmetic in the same order as the neighbour's owner, so the
// values are bitwise those the owner computes, and the whole path is bitwise
// equal to the per-stage kernels.
//
// The step reads u^n from one buffer and writes u^{n+1} to another (a
// neighbouring CTA may still read the edge points of u^n); the host
// alternates the two.
#include <cuda/atomic>
#include <cuda_runtime.h>

#include "at_device.cuh"

namespace atk {

// The buffer value of one edge point (the extrapolation of Eq. 7 with the
// weights of delay k, in the order of the per-stage kernels), split by
// where the levels come from.  k >= 1: every level is older than n and in
// the global ring, so the value is known at the start of the step.
__device__ __forceinline__ double fused_extrap_old(const StageArgs& a, int k, const double* v)
{
    const int nw = (a.mode == AT) ? a.q + 1 : 1;
    double acc = ((a.mode == AT) ? a.w[k][0] : 1.0) * v[0];
#pragma unroll
    for (int l = 1; l <= AT_QMAX; ++l)
        if (l < nw) acc = fma(a.w[k][l], v[l], acc);
    return acc;
}

// k = 0: the weights are exact integer ratios, (1, +-0, ..., +-0), and the
// neighbour's level-n value cur comes out unchanged, up to the sign of a zero
// (1 x cur plus the +-0 terms).  The stencil sum starts from +0, so a zero
// buffer value adds nothing whatever its sign: taking cur itself gives the
// per-stage path's results bit for bit, with no FP64 instruction.
__device__ __forceinline__ double fused_extrap_cur(double cur) { return cur; }

// the buffer value of one edge point of PE nbr's window for a delay k >= 1,
// from the ring levels n-k-l
__device__ __forceinline__ double fused_buffer_old(const StageArgs& a, int64_t n, int s, int k, int64_t nbr, int side,
                                                   int h)
{
    const int nw = (a.mode == AT) ? a.q + 1 : 1;
    double v[AT_QMAX + 1];
#pragma unroll
    for (int l = 0; l <= AT_QMAX; ++l) {
        v[l] = 0.0;  // a level with weight 0 is not part of the scheme (and may not exist yet)
        if (l < nw && ((a.wnz[k] >> l) & 1)) v[l] = __ldcg(a.ring + ring_index(a, n - k - l, s, nbr, side, h, 0));
    }
    return fused_extrap_old(a, k, v);
}

// One CTA: W PE warps and one strip warp (warp W).  Shared memory:
//   ROW  [2][W][B + 2H]        stage arguments of the PEs with their buffer
//                              values, by stage parity
//   SROW [2][2][D + 2H]        the strips of the left and right outer
//                              neighbours (D = S H points nearest the CTA), by
//                              stage parity
//   SUN  [2][D]                u^n on the strips
//   BV   [W][S][2][H]          buffer values of the PEs with delays k >= 1,
//                              all stages
//   SBV  [2][S-1][H]           the same for the strips' buffer points
//   KS   [W][S][2], SKS [2][S-1]  the delays
// The delays of all S stages are drawn at the start of the step and the
// buffer values with k >= 1 formed from the ring then (with u^n in flight),
// one warp instruction for all stages and both sides of a PE; a stage only
// reads shared memory, and fills a k = 0 buffer point with the neighbour's
// stage argument itself (no FP64 instruction).
template <int H, int PPL, int RK, int W>
__device__ __forceinline__ void fused_step(const StageArgs& a, const double* __restrict__ uin,
                                           double* __restrict__ uout, int64_t n, double* sm, int64_t cta)
{
    constexpr int B = 32 * PPL;
    constexpr int S = RkS<RK>::S;
    constexpr int D = S * H;
    constexpr int RW = B + 2 * H, SW = D + 2 * H;
    double* ROW = sm;
    double* SROW = ROW + 2 * W * RW;
    double* SUN = SROW + 2 * 2 * SW;
    double* BV = SUN + 2 * D;
    double* SBV = BV + W * S * 2 * H;
    int* KS = (int*)(SBV + 2 * (S - 1) * H);
    int* SKS = KS + W * S * 2;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t P = a.P;
    const int64_t p0 = cta * W;  // the CTA's first PE
    const int nW = (int)(P - p0 < W ? P - p0 : W);  // PEs of this CTA
    const int64_t pl = p0 == 0 ? P - 1 : p0 - 1;     // outer neighbours
    const int64_t pr = p0 + nW == P ? 0 : p0 + nW;
    const int64_t plast = p0 + nW - 1;

    if (wid < W) {
        // ---------------- PE warps ----------------
        const bool active = wid < nW;
        const int64_t pe = p0 + wid;
        double x[PPL], un[PPL], ac[PPL];
        if (active) {
#pragma unroll
            for (int i = 0; i < PPL; ++i) {
                const double v = uin[pe * B + lane + 32 * i];
                x[i] = v;
                un[i] = v;
                ac[i] = 0.0;
                ROW[wid * RW + H + lane + 32 * i] = v;
            }
        }
        // the delays of every stage and the buffer values of delays >= 1: lane
        // e < 2 S H takes stage e / 2H, side (e / H) % 2, point e % H of the
        // edge window
        if (active && lane < 2 * S * H) {
            const int s = lane / (2 * H), side = (lane / H) & 1, h = lane % H;
            const int64_t nb = side == 0 ? (pe == 0 ? P - 1 : pe - 1) : (pe == P - 1 ? 0 : pe + 1);
            const int k = keff_at(a, n, s, pe, side);
            if (h == 0) {
                log_delay(a, n, s, pe, side, k);
                KS[(wid * S + s) * 2 + side] = k;
            }
            if (k >= 1) BV[((wid * S + s) * 2 + side) * H + h] = fused_buffer_old(a, n, s, k, nb, 1 - side, h);
        }
        // buffer lanes of the stages: left side on lanes 0..H-1, right side on H..2H-1
        const bool buf = active && lane < 2 * H;
        const int side = lane < H ? 0 : 1;
        const int h = lane - side * H;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int par = s & 1;
            double* R0 = ROW + par * W * RW;
            double* R1 = ROW + (par ^ 1) * W * RW;
            double* Rw = R0 + wid * RW;
            __syncthreads();  // the stage arguments of stage s, of every warp and strip
            if (buf) {
                const int k = KS[(wid * S + s) * 2 + side];
                // k = 0: the neighbour's stage argument at the point facing this
                // PE (its point B-H+h on the left, h on the right)
                double b;
                if (k == 0) {
                    double cur;
                    if (side == 0)
                        cur = wid > 0 ? R0[(wid - 1) * RW + H + B - H + h]
                                      : SROW[(par * 2 + 0) * SW + H + D - H + h];
                    else
                        cur = wid < nW - 1 ? R0[(wid + 1) * RW + H + h] : SROW[(par * 2 + 1) * SW + H + h];
                    b = fused_extrap_cur(cur);
                } else {
                    b = BV[((wid * S + s) * 2 + side) * H + h];
                }
                Rw[side == 0 ? h : H + B + h] = b;
            }
            __syncwarp();
            if (active) {
                const bool last = s == S - 1;
#pragma unroll
                for (int i = 0; i < PPL; ++i) {
                    const int j = lane + 32 * i;
                    double K = 0.0;
#pragma unroll
                    for (int o = -H; o <= H; ++o) K = fma(a.cm[o + H], Rw[H + j + o], K);
                    const double y = fused_update<RK>(a, s, K, x[i], un[i], ac[i]);
                    if (nonfinite(y)) atomicOr(a.status, 1);
                    if (j < H)
                        a.ring[ring_index(a, last ? n + 1 : n, last ? 0 : s + 1, pe, 0, j, 0)] = y;
                    else if (j >= B - H)
                        a.ring[ring_index(a, last ? n + 1 : n, last ? 0 : s + 1, pe, 1, j - (B - H), 0)] = y;
                    if (last)
                        uout[pe * B + j] = y;
                    else
                        R1[wid * RW + H + j] = y;
                    x[i] = y;
                }
            }
        }
    } else {
        // ---------------- strip warp ----------------
        // lanes 0..15: the left outer neighbour pl, its points B-D..B-1 at strip
        // index 0..D-1 (its right buffer after them); lanes 16..31: the right
        // outer neighbour pr, its points 0..D-1 (its left buffer before them)
        const int st = lane >> 4;          // 0: left strip, 1: right strip
        const int sl = lane & 15;          // lane within the strip
        const int64_t spe = st == 0 ? pl : pr;
        const int64_t soff = st == 0 ? (int64_t)(B - D) : 0;  // first strip point within spe
        if (sl < D) {
            const double v = __ldcg(uin + spe * B + soff + sl);  // written by another CTA
            SUN[st * D + sl] = v;
            SROW[(0 * 2 + st) * SW + H + sl] = v;
        }
        // the strips' buffers, on the side facing the CTA: pl's right side
        // (from p0's left window), pr's left side (from plast's right window);
        // the delays of every stage and the buffer values of delays >= 1, lane
        // e < 2 (S-1) H taking strip e / ((S-1) H), stage (e / H) % (S-1),
        // point e % H
        if (lane < 2 * (S - 1) * H) {
            const int t = lane / ((S - 1) * H), s = (lane / H) % (S - 1), hh = lane % H;
            const int64_t tpe = t == 0 ? pl : pr;
            const int tside = t == 0 ? 1 : 0;
            const int k = keff_at(a, n, s, tpe, tside);
            if (hh == 0) SKS[t * (S - 1) + s] = k;
            if (k >= 1) SBV[(t * (S - 1) + s) * H + hh] = fused_buffer_old(a, n, s, k, t == 0 ? p0 : plast, 1 - tside, hh);
        }
        const bool buf = sl < H;
#pragma unroll
        for (int s = 0; s < S - 1; ++s) {
            const int par = s & 1;
            double* Rs = SROW + (par * 2 + st) * SW;
            double* Rn = SROW + ((par ^ 1) * 2 + st) * SW;
            __syncthreads();
            if (buf) {
                const int k = SKS[st * (S - 1) + s];
                double b;
                if (k == 0) {
                    const double* R0 = ROW + par * W * RW;
                    b = fused_extrap_cur(st == 0 ? R0[0 * RW + H + sl] : R0[(nW - 1) * RW + H + B - H + sl]);
                } else {
                    b = SBV[(st * (S - 1) + s) * H + sl];
                }
                Rs[st == 0 ? H + D + sl : sl] = b;
            }
            __syncwarp();
            // K at the d = (S-1-s) H strip points nearest the CTA: stage s+1
            // needs them there
            const int d = (S - 1 - s) * H;
            if (sl < d) {
                const int idx = st == 0 ? D - d + sl : sl;  // strip index
                double K = 0.0;
#pragma unroll
                for (int o = -H; o <= H; ++o) K = fma(a.cm[o + H], Rs[H + idx + o], K);
                double acc_unused = 0.0;
                Rn[H + idx] = fused_update<RK>(a, s, K, Rs[H + idx], SUN[st * D + idx], acc_unused);
            }
        }
        // the PE warps' last stage has one more barrier
        __syncthreads();
    }
}

// one step n: u^n from uin, u^{n+1} to uout
template <int H, int PPL, int RK, int W>
__global__ void __launch_bounds__(32 * (W + 1)) step_fused_advdiff(const StageArgs a, const double* __restrict__ uin,
                                                                   double* __restrict__ uout, int64_t n)
{
    extern __shared__ double sm[];
    fused_step<H, PPL, RK, W>(a, uin, uout, n, sm, blockIdx.x);
}

__device__ __forceinline__ int64_t fused_load_acquire(int64_t* p)
{
    cuda::atomic_ref<int64_t, cuda::thread_scope_device> r(*p);
    return r.load(cuda::memory_order_acquire);
}

__device__ __forceinline__ void fused_store_release(int64_t* p, int64_t v)
{
    cuda::atomic_ref<int64_t, cuda::thread_scope_device> r(*p);
    r.store(v, cuda::memory_order_release);
}

// bounded wait for *ctr >= target; false if it ran out (status bit 2, abort
// flag raised) or another CTA's wait did
__device__ bool fused_wait_ge(const StageArgs& a, int64_t* ctr, int64_t target)
{
    if (fused_load_acquire(ctr) >= target) return true;
    for (int64_t it = 0; it < a.wait_limit; ++it) {
        __nanosleep(128);
        if (fused_load_acquire(ctr) >= target) return true;
        if ((it & 63) == 0 && *(volatile int*)a.abort_flag) return false;
    }
    atomicOr(a.status, 2);
    atomicExch(a.abort_flag, 1);
    return false;
}

// All steps of an at_step call in one cooperative launch (every CTA
// resident).  The CTA at position c (its rank by SM, place_rank: neighbouring
// positions on neighbouring SMs) takes PEs c W .. c W + W - 1 and publishes
// in done[c] the level it has reached; before
// step n it waits for its two neighbour CTAs to have finished step n-1.  That
// one wait covers everything a step reads from outside the CTA: the
// neighbours' u^n on the strips (written at their step n-1), and ring levels
// older than n.  It also protects what the step writes: u^{n+1} goes to the
// buffer that held u^{n-1}, which the neighbours read during their step n-1,
// and the ring slots of levels n and n+1, which no CTA at step n or n+1 reads
// (the CTAs are at most one step apart, the ring keeps k_max + q + 3 levels).
template <int H, int PPL, int RK, int W>
__global__ void __launch_bounds__(32 * (W + 1)) steps_fused_advdiff(const StageArgs a, double* __restrict__ b0,
                                                                    double* __restrict__ b1, int64_t level0,
                                                                    int64_t nsteps)
{
    extern __shared__ double sm[];
    __shared__ int s_fail;
    const int64_t C = gridDim.x, c = place_rank(a);  // CTA c takes PEs c W .. c W + W - 1
    const int64_t cl = c == 0 ? C - 1 : c - 1, cr = c == C - 1 ? 0 : c + 1;
    const bool withheld = a.withhold_pe >= 0 && a.withhold_pe / W == c;  // fault injection: never publishes
    for (int64_t i = 0; i < nsteps; ++i) {
        const int64_t n = level0 + i;
        if (i > 0) {
            if (threadIdx.x == 0) s_fail = (fused_wait_ge(a, a.done + cl, n) && fused_wait_ge(a, a.done + cr, n)) ? 0 : 1;
            __syncthreads();
            if (s_fail) break;
        }
        fused_step<H, PPL, RK, W>(a, (i & 1) ? b1 : b0, (i & 1) ? b0 : b1, n, sm, c);
        __syncthreads();  // every thread's writes of step n
        if (threadIdx.x == 0 && !withheld) {
            __threadfence();
            fused_store_release(a.done + c, n + 1);
        }
    }
}

// done[c] = level0 for the CTAs of a launch, the abort flag and the placement count cleared
__global__ void fused_counters_set(int64_t* done, int64_t C, int64_t level0, int* abort_flag, int* place_count)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C; i += (int64_t)gridDim.x * blockDim.x)
        done[i] = level0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *abort_flag = 0;
        *place_count = 0;
    }
}

} // namespace atk

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

constexpr int kFusedW = 8;  // PEs per CTA (measured on GB300: 8 ahead of 4 and 16)

template <int H, int RK>
void* fused_fn_ppl(int ppl)
{
    switch (ppl) {
    case 1: return (void*)atk::step_fused_advdiff<H, 1, RK, kFusedW>;
    case 2: return (void*)atk::step_fused_advdiff<H, 2, RK, kFusedW>;
    case 4: return (void*)atk::step_fused_advdiff<H, 4, RK, kFusedW>;
    default: return (void*)atk::step_fused_advdiff<H, 8, RK, kFusedW>;
    }
}

template <int H>
void* fused_fn_rk(int rk, int ppl)
{
    if (rk == atk::RK4) return fused_fn_ppl<H, atk::RK4>(ppl);
    if (rk == atk::RK3TVD) return fused_fn_ppl<H, atk::RK3TVD>(ppl);
    return fused_fn_ppl<H, atk::RK2>(ppl);
}

void* fused_fn(int H, int rk, int ppl)
{
    if (H == 1) return fused_fn_rk<1>(rk, ppl);
    if (H == 2) return fused_fn_rk<2>(rk, ppl);
    return fused_fn_rk<3>(rk, ppl);
}

// the multi-step kernel with W = 4 or 8 PEs per CTA
template <int H, int RK, int W>
void* fused_steps_fn_ppl(int ppl)
{
    switch (ppl) {
    case 1: return (void*)atk::steps_fused_advdiff<H, 1, RK, W>;
    case 2: return (void*)atk::steps_fused_advdiff<H, 2, RK, W>;
    case 4: return (void*)atk::steps_fused_advdiff<H, 4, RK, W>;
    default: return (void*)atk::steps_fused_advdiff<H, 8, RK, W>;
    }
}

template <int H, int W>
void* fused_steps_fn_rk(int rk, int ppl)
{
    if (rk == atk::RK4) return fused_steps_fn_ppl<H, atk::RK4, W>(ppl);
    if (rk == atk::RK3TVD) return fused_steps_fn_ppl<H, atk::RK3TVD, W>(ppl);
    return fused_steps_fn_ppl<H, atk::RK2, W>(ppl);
}

template <int W>
void* fused_steps_fn_h(int H, int rk, int ppl)
{
    if (H == 1) return fused_steps_fn_rk<1, W>(rk, ppl);
    if (H == 2) return fused_steps_fn_rk<2, W>(rk, ppl);
    return fused_steps_fn_rk<3, W>(rk, ppl);
}

void* fused_steps_fn(int H, int rk, int ppl, int W)
{
    return W == 4 ? fused_steps_fn_h<4>(H, rk, ppl) : fused_steps_fn_h<8>(H, rk, ppl);
}

size_t fused_smem(int B, int H, int S, int W = kFusedW)
{
    const int D = S * H;
    return sizeof(double) * ((size_t)2 * W * (B + 2 * H) + (size_t)4 * (D + 2 * H) + (size_t)2 * D +
                             (size_t)W * S * 2 * H + (size_t)2 * (S - 1) * H) +
           sizeof(int) * ((size_t)W * S * 2 + (size_t)2 * (S - 1));
}

} // namespace

// whether the fused path takes this problem: advection-diffusion with
// central stencils, PEs of 32, 64, 128 or 256 points, at least S H points
bool atk_fused_supported(int pde, int order, int B, int S)
{
    return pde == atk::ADVDIFF && (B == 32 || B == 64 || B == 128 || B == 256) && B >= S * (order / 2);
}

// CTAs (of W = 4 or 8 PEs) that one cooperative launch of the multi-step
// kernel holds at once (0: not available)
int64_t atk_fused_capacity(int order, int rk, int B, int S, int W, int device)
{
    const int H = order / 2;
    void* fn = fused_steps_fn(H, rk, B / 32, W);
    const size_t smem = fused_smem(B, H, S, W);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0, sms = 0, coop = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * (W + 1), smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop) {
        cudaGetLastError();
        return 0;
    }
    return (int64_t)per_sm * sms;
}

int64_t atk_fused_ctas(int64_t P, int W) { return (P + W - 1) / W; }

// PEs per CTA of the multi-step kernel for P PEs, or 0 when its CTAs do not
// fit one cooperative launch: 4 where they fit (more SMs share the stages of
// a small problem), else 8 (measured on GB300, PEs of 64 points, us per
// step: 2^14 points 7.3 with 4 against 8.9 with 8; 2^18 points 20.6 with 8,
// where 4 no longer fits and takes one launch per step: 22.5)
int atk_fused_multi_w(int order, int rk, int B, int S, int64_t P, int device)
{
    for (int W = 4; W <= 8; W += 4)
        if (atk_fused_ctas(P, W) <= atk_fused_capacity(order, rk, B, S, W, device)) return W;
    return 0;
}

// steps level0 .. level0 + nsteps - 1 in one cooperative launch of CTAs of W
// PEs: u^{level0} in b0, the result in b0 (even nsteps) or b1 (odd)
cudaError_t atk_launch_fused_steps(const atk::StageArgs& a, int order, int W, int64_t level0, int64_t nsteps,
                                   double* b0, double* b1, cudaStream_t st)
{
    const int H = order / 2;
    const int64_t C = atk_fused_ctas(a.P, W);
    void* fn = fused_steps_fn(H, a.rk, a.B / 32, W);
    const size_t smem = fused_smem(a.B, H, a.S, W);
    atk::fused_counters_set<<<(unsigned)((C + 255) / 256 < 1024 ? (C + 255) / 256 : 1024), 256, 0, st>>>(
        a.done, C, level0, a.abort_flag, a.place_count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    atk::StageArgs args = a;
    void* params[] = {(void*)&args, (void*)&b0, (void*)&b1, (void*)&level0, (void*)&nsteps};
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)C), dim3(32 * (W + 1)), params, smem, st);
}

// one step n: u^n from uin, u^{n+1} to uout (distinct buffers)
cudaError_t atk_launch_fused(const atk::StageArgs& a, int order, int64_t n, const double* uin, double* uout,
                             cudaStream_t st)
{
    const int H = order / 2;
    void* fn = fused_fn(H, a.rk, a.B / 32);
    const size_t smem = fused_smem(a.B, H, a.S);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (a.P + kFusedW - 1) / kFusedW;
    atk::StageArgs args = a;
    void* params[] = {(void*)&args, (void*)&uin, (void*)&uout, (void*)&n};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(32 * (kFusedW + 1)), params, smem, st);
}
