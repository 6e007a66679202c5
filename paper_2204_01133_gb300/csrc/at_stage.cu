// at_stage.cu -- the RK-stage kernels of the asynchrony-tolerant solver.
//
// One launch evaluates one Runge-Kutta stage over the whole domain.  A CTA
// owns a window of Tw consecutive points of one virtual PE (Tw divides the PE
// size, so a window never straddles a PE edge).  Per CTA:
//
//  1. fill: the derived quantities (fluxes, velocity, temperature, ...) of
//     the Tw + 2H points the window's stencils touch are staged in shared
//     memory.  Points inside the PE are read from the stage-argument field.
//     Points beyond the PE edge are buffer points (Sec. 2.1, Fig. 1): the
//     thread draws the delay k of that PE boundary from Philox, reads the
//     neighbour's edge window at levels n-k-l from the history ring and
//     combines the derived quantities with the temporal extrapolation weights
//     (AT: Eq. at1 / Appendix A / Eq. atRecon; AS: the plain delayed value).
//  2. compute: central stencils (Sec. 2.2; the AT scheme is the standard one
//     on the extrapolated halo) or WENO5 / AT-WENO5 reconstructions with
//     local Lax-Friedrichs splitting (Sec. 3, Eqs. Csplit, wender, omg,
//     betaS), the Arrhenius source fused in.
//  3. update: the RK update of this stage (Sec. 2.3), the edge points of the
//     new stage argument pushed into the history ring (the per-step message
//     of S stages x stencil of Sec. 2.3), a non-finite check.
//
// All arithmetic is FP64.  Stencil and RK coefficients arrive pre-scaled in
// the argument block.
#include <cuda_runtime.h>

#include "at_device.cuh"

namespace atk {

// What changes from one stage evaluation to the next: the level, the stage,
// the stage argument read by the stencils (X), the output (Y) and u^n.
struct Cx {
    int64_t level;
    int stage;
    const double* X;
    double* Y;
    const double* u;
};

__device__ __forceinline__ Cx launch_cx(const StageArgs& a) { return Cx{a.level, a.stage, a.X, a.Y, a.u}; }

// ---------------------------------------------------------------------------
// 1. fill the window
//
// Work items: one per point of the window inside the PE (read the field,
// derive), plus one per (buffer point, time level) pair of the window's PE
// boundaries (read the ring at level n-k-l, derive).  All items run
// concurrently, one per thread of the window's thread group (lt of gs); the
// level contributions are then combined per buffer point with the
// extrapolation weights.  HS stages the level contributions: [2 H (q+1)][ND].
// ---------------------------------------------------------------------------
template <int PDE, bool WENO>
__device__ __forceinline__ void fill_window(const StageArgs& a, const Cx& cx, double* __restrict__ G,
                                            double* __restrict__ SP, double* __restrict__ HS, int64_t pe, int chunk,
                                            int64_t t0, int W2, int lt, int gs, double* __restrict__ ARR = nullptr)
{
    using P = Phys<PDE>;
    constexpr int NV = P::NV, ND = P::ND;
    const int H = a.H;
    const int L0 = (chunk == 0) ? H : 0;             // ring-halo points on the left
    const int R0 = (chunk == a.wpp - 1) ? H : 0;     // and on the right
    const int nw = (a.mode == AT) ? a.q + 1 : 1;     // time levels per ring-halo point
    const int own = W2 - L0 - R0;
    const int items = own + (L0 + R0) * nw;
    for (int it = lt; it < items; it += gs) {
        double g[ND];
        double Q[NV];
        if (it < own) {
            const int i = L0 + it;
            const int64_t m = t0 - H + i;
#pragma unroll
            for (int v = 0; v < NV; ++v) Q[v] = cx.X[v * a.N + m];
            if constexpr (WENO) {
                double sp, arr;
                P::template derive_weno<PDE == EULER>(a, Q, g, sp, arr);
                SP[i] = sp;
                if constexpr (PDE == EULER) ARR[i] = arr;  // the reaction source's exp(-Ea rho / p)
            } else {
                P::derive(a, Q, g);
            }
#pragma unroll
            for (int d = 0; d < ND; ++d) G[d * W2 + i] = g[d];
        } else {
            const int t = it - own;
            const int hp = t / nw, l = t - hp * nw;         // buffer point, level
            const int side = hp < L0 ? 0 : 1;
            const int h = side == 0 ? hp : hp - L0;         // position in the neighbour's edge window
            const int k = keff_at(a, cx.level, cx.stage, pe, side);
            if (h == 0 && l == 0) log_delay(a, cx.level, cx.stage, pe, side, k);
            if ((a.wnz[k] >> l) & 1) {  // a level with weight 0 is not part of the scheme (and may not exist yet)
                const double* src = halo_window(a, cx.level - k - l, cx.stage, pe, side, h);
#pragma unroll
                for (int v = 0; v < NV; ++v) Q[v] = src[v];
                if constexpr (WENO) {
                    if (l == 0) {  // the (half) wave speed at level n-k, not extrapolated
                        double sp, unused;
                        P::template derive_weno<false>(a, Q, g, sp, unused);
                        SP[side == 0 ? h : W2 - R0 + h] = sp;
                    } else {
                        P::derive(a, Q, g);
                    }
                } else {
                    P::derive(a, Q, g);
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) HS[t * ND + d] = g[d];
            } else {
#pragma unroll
                for (int d = 0; d < ND; ++d) HS[t * ND + d] = 0.0;
            }
        }
    }
    __syncthreads();  // unconditional: every thread group of the CTA passes the same barriers
    // weighted sum of the level contributions of every buffer point, in level order
    for (int c = lt; c < (L0 + R0) * ND; c += gs) {
        const int hp = c / ND, d = c - hp * ND;
        const int side = hp < L0 ? 0 : 1;
        const int k = keff_at(a, cx.level, cx.stage, pe, side);
        double acc = ((a.mode == AT) ? a.w[k][0] : 1.0) * HS[(hp * nw) * ND + d];
        for (int l = 1; l < nw; ++l) acc = fma(a.w[k][l], HS[(hp * nw + l) * ND + d], acc);
        const int i = hp < L0 ? hp : W2 - R0 + (hp - L0);
        G[d * W2 + i] = acc;
    }
}

// ---------------------------------------------------------------------------
// 3. RK update of this stage, ring push, non-finite check
// ---------------------------------------------------------------------------
// The RK scheme and stage of a launch as one kind.  Kernels that take it as
// a template argument get straight-line update code; with RKS_ANY it is read
// at run time (the compiler may then predicate the alternatives, and
// predicated-off FP64 instructions still take FP64 issue slots).
enum { RKS_ANY = -1, RKS_RK4_0, RKS_RK4_MID, RKS_RK4_LAST, RKS_RK3_0, RKS_RK3_1, RKS_RK3_2, RKS_RK2_0, RKS_RK2_1 };

__host__ __device__ __forceinline__ int rk_stage_kind(int rk, int stage)
{
    if (rk == RK4) return stage == 0 ? RKS_RK4_0 : (stage < 3 ? RKS_RK4_MID : RKS_RK4_LAST);
    if (rk == RK3TVD) return RKS_RK3_0 + stage;
    return stage == 0 ? RKS_RK2_0 : RKS_RK2_1;
}

// pointwise operands of one update besides K and the stage argument: u^n and
// the accumulator, loaded only where the scheme reads them
struct RkIn {
    double un, ac;
};

template <int RKS = RKS_ANY>
__device__ __forceinline__ RkIn rk_load(const StageArgs& a, const Cx& cx, int64_t idx)
{
    const int k = RKS >= 0 ? RKS : rk_stage_kind(a.rk, cx.stage);
    RkIn r{0.0, 0.0};
    if (k != RKS_RK3_0) r.un = cx.u[idx];
    if (k == RKS_RK4_MID || k == RKS_RK4_LAST || k == RKS_RK2_1) r.ac = a.acc[idx];
    return r;
}

template <int RKS = RKS_ANY>
__device__ __forceinline__ void rk_update(const StageArgs& a, const Cx& cx, int v, int64_t j, int jpe, int64_t pe,
                                          double K, double x, RkIn in)
{
    const int k = RKS >= 0 ? RKS : rk_stage_kind(a.rk, cx.stage);
    const int64_t idx = v * a.N + j;
    const double dt = a.dt;
    const double un = in.un;
    double y;
    if (k == RKS_RK4_0) {
        a.acc[idx] = K;
        y = fma(a.hdt, K, un);
    } else if (k == RKS_RK4_MID) {
        a.acc[idx] = fma(2.0, K, in.ac);
        y = fma(cx.stage == 1 ? a.hdt : dt, K, un);
    } else if (k == RKS_RK4_LAST) {
        y = fma(a.dt6, in.ac + K, un);
    } else if (k == RKS_RK3_0) {
        y = fma(dt, K, x);
    } else if (k == RKS_RK3_1) {
        y = fma(0.75, un, 0.25 * fma(dt, K, x));
    } else if (k == RKS_RK3_2) {
        y = fma(1.0 / 3.0, un, (2.0 / 3.0) * fma(dt, K, x));
    } else if (k == RKS_RK2_0) {
        a.acc[idx] = K;
        y = fma(dt, K, un);
    } else {  // RK2 (Heun), second stage
        y = fma(a.hdt, in.ac + K, un);
    }
    cx.Y[idx] = y;
    if (nonfinite(y)) atomicOr(a.status, 1);
    int side = -1, h = 0;
    if (jpe < a.H) {
        side = 0;
        h = jpe;
    } else if (jpe >= a.B - a.H) {
        side = 1;
        h = jpe - (a.B - a.H);
    }
    if (side >= 0 && !a.hist_recompute) {
        const bool last = (cx.stage == a.S - 1);
        a.ring[ring_index(a, last ? cx.level + 1 : cx.level, last ? 0 : cx.stage + 1, pe, side, h, v)] = y;
    }
}

// ---------------------------------------------------------------------------
// central stencils: advection-diffusion and reacting Navier-Stokes
// ---------------------------------------------------------------------------
// Reacting N-S in chain-rule form (Sec. 4) at own point j (window column c):
// with m_f = sum_o c1_o f_{j+o} = -f_x and f_xx from the c2 taps,
//   K_rho  = -(rho_x u + rho u_x)
//   K_rhou = -(rho_x u^2 + 2 rho u u_x) - p_x + 4/3 mu u_xx
//   K_rhoE = -(u_x (rho E + p) + u ((rho E)_x + p_x)) + 4/3 mu (u_x^2 + u u_xx)
//            + lam T_xx + q_c rhoD Y_xx
//   K_rhoY = -(rho_x u Y + rho u_x Y + rho u Y_x) + rhoD Y_xx - A rho Y exp(-Ea/T)
// (tau = 4/3 mu u_x, q = -lam T_x + q_c J_F, J_F = -rhoD Y_x), the factors
// being the point's own current values; then the four RK updates.
template <int H, int RKS>
__device__ __forceinline__ void chain_point(const StageArgs& a, const Cx& cx, const double* G, int W2, int64_t pe,
                                            int jpe, int64_t j, int c)
{
    double m[5];  // -d/dx of rho, u, p, rho E, Y
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double t = 0.0;
#pragma unroll
        for (int o = -H; o <= H; ++o)
            if (o != 0) t = fma(a.c1[o + H], G[q * W2 + c + o], t);
        m[q] = t;
    }
    double uxx = 0.0, Yxx = 0.0, Txx = 0.0;
#pragma unroll
    for (int o = -H; o <= H; ++o) {
        uxx = fma(a.c2[o + H], G[1 * W2 + c + o], uxx);
        Yxx = fma(a.c2[o + H], G[4 * W2 + c + o], Yxx);
        Txx = fma(a.c2[o + H], G[5 * W2 + c + o], Txx);
    }
    const double rho = G[c], u = G[W2 + c], p = G[2 * W2 + c], rE = G[3 * W2 + c], Y = G[4 * W2 + c];
    const double T = G[5 * W2 + c];
    const double ru = rho * u;
    double K[4];
    K[0] = fma(m[0], u, rho * m[1]);
    K[1] = fma(m[0] * u, u, fma(2.0 * ru, m[1], fma(a.k0, uxx, m[2])));
    K[2] = fma(m[1], rE + p, fma(u, m[3] + m[2], fma(a.k0, fma(m[1], m[1], u * uxx), fma(a.k2, Txx, a.prm[6] * a.k3 * Yxx))));
    const double x3 = cx.X[3 * a.N + j];
    K[3] = fma(m[0] * u, Y, fma(rho * m[1], Y, fma(ru, m[4], fma(a.k3, Yxx, -a.prm[4] * x3 * at_exp(-a.prm[5] * at_rcp3(T))))));
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const double x = v == 3 ? x3 : cx.X[v * a.N + j];
        rk_update<RKS>(a, cx, v, j, jpe, pe, K[v], x, rk_load<RKS>(a, cx, v * a.N + j));
    }
}

template <int PDE, int H, int RKS = RKS_ANY>
__device__ __forceinline__ void central_window(const StageArgs& a, const Cx& cx, int64_t win, double* sm, int lt,
                                               int gs)
{
    using P = Phys<PDE>;
    constexpr int NV = P::NV;
    const int W2 = a.Tw + 2 * H;
    double* G = sm;
    double* HS = G + P::ND * W2;
    const int64_t pe = a.wpp == 1 ? win : win / a.wpp;  // a 64-bit division only where PEs hold several windows
    const int chunk = (int)(win - pe * a.wpp);
    const int64_t t0 = pe * a.B + (int64_t)chunk * a.Tw;
    if constexpr (PDE == RNS_CHAIN) {  // one item per point: its derivatives feed all four equations
        fill_window<PDE, false>(a, cx, G, nullptr, HS, pe, chunk, t0, W2, lt, gs);
        __syncthreads();
        for (int jl = lt; jl < a.Tw; jl += gs)
            chain_point<H, RKS>(a, cx, G, W2, pe, chunk * a.Tw + jl, t0 + jl, jl + H);
        return;
    }
    const int items = NV * a.Tw;
    // advection-diffusion (few FP64 operations per byte): the pointwise
    // operands of the thread's first update item are loaded before the fill,
    // so that their latency overlaps it
    constexpr bool kPrefetch = (PDE == ADVDIFF);
    double x0 = 0.0;
    RkIn in0{0.0, 0.0};
    if (kPrefetch && lt < items) {
        const int v = lt / a.Tw;
        const int64_t idx = v * a.N + t0 + (lt - v * a.Tw);
        if constexpr (PDE != ADVDIFF) x0 = cx.X[idx];
        in0 = rk_load<RKS>(a, cx, idx);
    }
    fill_window<PDE, false>(a, cx, G, nullptr, HS, pe, chunk, t0, W2, lt, gs);
    __syncthreads();
    for (int it = lt; it < items; it += gs) {
        const int v = it / a.Tw;
        const int jl = it - v * a.Tw;
        const int64_t j = t0 + jl;
        const int c = jl + H;
        double x = x0;
        RkIn in = in0;
        if (!kPrefetch || it != lt) {
            if constexpr (PDE != ADVDIFF) x = cx.X[v * a.N + j];
            in = rk_load<RKS>(a, cx, v * a.N + j);
        }
        double K = 0.0;
        if constexpr (PDE == ADVDIFF) {
#pragma unroll
            for (int o = -H; o <= H; ++o) K = fma(a.cm[o + H], G[c + o], K);
            x = G[c];
        } else {
            const double* F = G + v * W2;
#pragma unroll
            for (int o = -H; o <= H; ++o)
                if (o != 0) K = fma(a.c1[o + H], F[c + o], K);
            if (v > 0) {
                const double* D = G + (3 + v) * W2;  // u | energy diffusion / lambda | Y (constants in the taps)
#pragma unroll
                for (int o = -H; o <= H; ++o) K = fma(a.c2v[v - 1][o + H], D[c + o], K);
            }
            if (v == 3) K = fma(-a.prm[4] * x, at_exp(-a.prm[5] * at_rcp3(G[7 * W2 + c])), K);
        }
        rk_update<RKS>(a, cx, v, j, chunk * a.Tw + jl, pe, K, x, in);
    }
}

// One CTA evaluates a.wpc consecutive windows, one thread group each (a.wpc
// > 1 only when every window spans a whole PE, so all groups pass the same
// barriers, and a.wpc divides the window count).
template <int PDE, int H, int RKS>
__global__ void __launch_bounds__(256, PDE == ADVDIFF ? 6 : 5) stage_central(const StageArgs a)
{
    extern __shared__ double sm[];
    const int gs = blockDim.x / a.wpc;
    const int g = threadIdx.x / gs;
    central_window<PDE, H, RKS>(a, launch_cx(a), (int64_t)blockIdx.x * a.wpc + g, sm + (size_t)g * a.win_smem,
                                threadIdx.x - g * gs, gs);
}

// ---------------------------------------------------------------------------
// advection-diffusion on PEs of 32 PPL points: one warp per PE
//
// With one variable and a 3-, 5- or 7-point stencil a point carries too
// little work for a CTA-wide fill and barriers to pay for.  A warp owns one
// PE; point j of the PE belongs to lane j % 32 (coalesced loads and stores);
// lanes 0..H-1 synthesise the left buffer points and lanes H..2H-1 the right
// ones from the ring; the PE's row with its two halos is staged in the
// warp's slice of shared memory, and the warp synchronises with __syncwarp
// only.  The arithmetic, and its order, is that of central_window<ADVDIFF, H>.
// ---------------------------------------------------------------------------
template <int H, int PPL, int RKS>
__global__ void __launch_bounds__(256, PPL <= 2 ? 6 : (PPL == 4 ? 4 : 3)) stage_advdiff_warp(const StageArgs a)
{
    extern __shared__ double sm[];
    constexpr int B = 32 * PPL;  // the PE size
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t pe = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    if (pe >= a.P) return;  // whole warps only
    double* W = sm + wid * (B + 2 * H);  // [H left halo | B own points | H right halo]
    const Cx cx = launch_cx(a);
    const int64_t base = pe * B;
    double x[PPL];
    RkIn in[PPL];
#pragma unroll
    for (int i = 0; i < PPL; ++i) {
        x[i] = cx.X[base + lane + 32 * i];
        in[i] = rk_load<RKS>(a, cx, base + lane + 32 * i);
    }
    if (lane < 2 * H) {  // one buffer point: delay draw, delayed ring levels, extrapolation
        const int side = lane < H ? 0 : 1;
        const int h = lane - side * H;  // position in the neighbour's edge window
        const int k = keff_at(a, cx.level, cx.stage, pe, side);
        if (h == 0) log_delay(a, cx.level, cx.stage, pe, side, k);
        const int nw = (a.mode == AT) ? a.q + 1 : 1;
        double v[AT_QMAX + 1];
#pragma unroll
        for (int l = 0; l <= AT_QMAX; ++l) {
            v[l] = 0.0;  // a level with weight 0 is not part of the scheme (and may not exist yet)
            if (l < nw && ((a.wnz[k] >> l) & 1)) v[l] = *halo_window(a, cx.level - k - l, cx.stage, pe, side, h);
        }
        double acc = ((a.mode == AT) ? a.w[k][0] : 1.0) * v[0];
#pragma unroll
        for (int l = 1; l <= AT_QMAX; ++l)
            if (l < nw) acc = fma(a.w[k][l], v[l], acc);
        W[side == 0 ? h : H + B + h] = acc;
    }
#pragma unroll
    for (int i = 0; i < PPL; ++i) W[H + lane + 32 * i] = x[i];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < PPL; ++i) {
        const int j = lane + 32 * i;
        double K = 0.0;
#pragma unroll
        for (int o = -H; o <= H; ++o) K = fma(a.cm[o + H], W[H + j + o], K);
        rk_update<RKS>(a, cx, 0, base + j, j, pe, K, x[i], in[i]);
    }
}

// ---------------------------------------------------------------------------
// WENO5 / AT-WENO5 fluxes: reactive Euler and scalar advection
// ---------------------------------------------------------------------------
template <int PDE, int RKS = RKS_ANY>
__device__ __forceinline__ void weno_window(const StageArgs& a, const Cx& cx, int64_t win, double* sm)
{
    using P = Phys<PDE>;
    constexpr int NV = P::NV, ND = P::ND;
    static_assert(ND == 2 * NV, "the WENO PDEs derive C/2 and Q for each variable");
    constexpr int H = 3;
    const int Tw = a.Tw;
    const int W2 = Tw + 2 * H;
    const int E = Tw + 1;  // edges of the window: edge e sits between points e-1 and e
    double* G = sm;
    double* DG = G + ND * W2;  // first differences along the window: DG[d W2 + j] = G[d W2 + j] - G[d W2 + j - 1]
    double* SP = DG + ND * W2;
    double* ARR = SP + W2;
    double* LAM = ARR + W2;
    double* FL = LAM + E;      // the flux at every edge, [NV][E]
    double* HS = FL + NV * E;
    const int64_t pe = a.wpp == 1 ? win : win / a.wpp;  // a 64-bit division only where PEs hold several windows
    const int chunk = (int)(win - pe * a.wpp);
    const int64_t t0 = pe * a.B + (int64_t)chunk * Tw;
    fill_window<PDE, true>(a, cx, G, SP, HS, pe, chunk, t0, W2, threadIdx.x, blockDim.x, ARR);
    __syncthreads();
    for (int e = threadIdx.x; e < E; e += blockDim.x)
        LAM[e] = fmax(SP[e - 1 + H], SP[e + H]);  // half the edge's local wave speed (SP: half speeds)
    for (int it = threadIdx.x; it < ND * (W2 - 1); it += blockDim.x) {
        const int d = it / (W2 - 1);
        const int j = 1 + it - d * (W2 - 1);
        DG[d * W2 + j] = G[d * W2 + j] - G[d * W2 + j - 1];
    }
    __syncthreads();
    const double eps = (PDE == EULER) ? a.prm[4] : a.prm[1];
    for (int it = threadIdx.x; it < NV * E; it += blockDim.x) {
        const int v = it / E;
        const int e = it - v * E;
        const double* dC = DG + v * W2;
        const double* dQ = DG + (NV + v) * W2;
        FL[it] = weno_flux(G + v * W2, [&](int j) { return dC[j]; },
                           [&](int j) { return dQ[j]; }, e + H, LAM[e], eps);
    }
    __syncthreads();
    const double rdx = a.k0;  // 1 / dx
    for (int it = threadIdx.x; it < NV * Tw; it += blockDim.x) {
        const int v = it / Tw;
        const int jl = it - v * Tw;
        const int64_t j = t0 + jl;
        const int c = jl + H;
        double K = (FL[v * E + jl] - FL[v * E + jl + 1]) * rdx;
        const double x = G[(NV + v) * W2 + c];
        if constexpr (PDE == EULER) {
            if (v == 3) K = fma(-a.prm[1] * x, ARR[c], K);  // x = rho Y; ARR from the fill
        }
        rk_update<RKS>(a, cx, v, j, chunk * Tw + jl, pe, K, x, rk_load<RKS>(a, cx, v * a.N + j));
    }
}

template <int PDE, int RKS>
__global__ void __launch_bounds__(256, 4) stage_weno(const StageArgs a)
{
    extern __shared__ double sm[];
    weno_window<PDE, RKS>(a, launch_cx(a), blockIdx.x, sm);
}

// ---------------------------------------------------------------------------
// The interpolation form (Sec. 3, Eqs. interpS, fullSten, omg): the value at
// the right edge of f[2] from f[0..4] by the third-order interpolants
// u0 = 3/8 f0 - 5/4 f1 + 15/8 f2, u1 = -1/8 f1 + 3/4 f2 + 3/8 f3,
// u2 = 3/8 f2 + 3/4 f3 - 1/8 f4, ideal weights {1/16, 5/8, 5/16}, the
// indicators of Eq. betaS and the weights of Eq. omg, arranged as weno5d():
// u0 - u1 = 3/8 (s_0 - s_1), u2 - u1 = 1/8 (s_1 - s_2), and with the common
// factor E_0 E_1 E_2 and a scaling by 128,
//   num = E_1 (3 E_2 (s_0 - s_1) + 5 E_0 (s_1 - s_2)),
//   den = E_1 (8 E_2 + 40 E_0) + 80 E_0 E_2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double weno5_interp(double f0, double f1, double f2, double f3, double f4, double eps4)
{
    const double s0 = fma(-2.0, f1, f0) + f2;
    const double s1 = fma(-2.0, f2, f1) + f3;
    const double s2 = fma(-2.0, f3, f2) + f4;
    const double r0 = fma(2.0, f2 - f1, s0);
    const double r1 = f1 - f3;
    const double r2 = fma(2.0, f2 - f3, s2);
    const double d0 = fma((13.0 / 3.0) * s0, s0, fma(r0, r0, eps4));
    const double d1 = fma((13.0 / 3.0) * s1, s1, fma(r1, r1, eps4));
    const double d2 = fma((13.0 / 3.0) * s2, s2, fma(r2, r2, eps4));
    const double e0 = d0 * d0, e1 = d1 * d1, e2 = d2 * d2;
    const double num = e1 * fma(3.0 * e2, s0 - s1, (5.0 * e0) * (s1 - s2));
    const double den = fma(e1, fma(8.0, e2, 40.0 * e0), 80.0 * (e0 * e2));
    const double u1 = fma(-0.125, f1, fma(0.75, f2, 0.375 * f3));
    return fma(num, at_rcp3(den), u1);
}

// A window of Tw points with a halo of H = 4: the edge values F of the
// Tw + 3 edges between points p and p+1, p = -2 .. Tw (window coordinates),
// then at each point the fourth-order staggered difference
//   -dC/dx = (9/8 (F_{j-1/2} - F_{j+1/2}) + 1/24 (F_{j+3/2} - F_{j-3/2})) / dx.
// Shared memory: G [ND][W2], SP [W2], ARR [W2], LAM [E], REC [NV][2][E], HS.
template <int PDE, int RKS = RKS_ANY>
__device__ __forceinline__ void weno_interp_window(const StageArgs& a, const Cx& cx, int64_t win, double* sm)
{
    using P = Phys<PDE>;
    constexpr int NV = P::NV, ND = P::ND;
    constexpr int H = 4;
    const int Tw = a.Tw;
    const int W2 = Tw + 2 * H;
    const int E = Tw + 3;  // edge t sits between points t-2 and t-1 of the window (shared index t+2, t+3)
    double* G = sm;
    double* SP = G + ND * W2;
    double* ARR = SP + W2;
    double* LAM = ARR + W2;
    double* REC = LAM + E;
    double* HS = REC + NV * 2 * E;
    const int64_t pe = a.wpp == 1 ? win : win / a.wpp;
    const int chunk = (int)(win - pe * a.wpp);
    const int64_t t0 = pe * a.B + (int64_t)chunk * Tw;
    fill_window<PDE, true>(a, cx, G, SP, HS, pe, chunk, t0, W2, threadIdx.x, blockDim.x, ARR);
    __syncthreads();
    for (int t = threadIdx.x; t < E; t += blockDim.x)
        LAM[t] = fmax(SP[t + 2], SP[t + 3]);  // SP holds half speeds
    __syncthreads();
    const double eps4 = 4.0 * ((PDE == EULER) ? a.prm[4] : a.prm[1]);
    const int items = NV * 2 * E;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int r = it / E;
        const int t = it - r * E;
        const int v = r >> 1;
        const double hl = LAM[t];
        const double* C = G + v * W2;
        const double* Qv = G + (NV + v) * W2;
        double rec;
        if ((r & 1) == 0) {  // f+ on points t-4 .. t, shared index t .. t+4
            rec = weno5_interp(fma(hl, Qv[t], C[t]), fma(hl, Qv[t + 1], C[t + 1]), fma(hl, Qv[t + 2], C[t + 2]),
                               fma(hl, Qv[t + 3], C[t + 3]), fma(hl, Qv[t + 4], C[t + 4]), eps4);
        } else {  // f- on points t+1 .. t-3 (mirrored), shared index t+5 .. t+1
            rec = weno5_interp(fma(-hl, Qv[t + 5], C[t + 5]), fma(-hl, Qv[t + 4], C[t + 4]),
                               fma(-hl, Qv[t + 3], C[t + 3]), fma(-hl, Qv[t + 2], C[t + 2]),
                               fma(-hl, Qv[t + 1], C[t + 1]), eps4);
        }
        REC[r * E + t] = rec;
    }
    __syncthreads();
    const double rdx = a.k0;
    for (int it = threadIdx.x; it < NV * Tw; it += blockDim.x) {
        const int v = it / Tw;
        const int jl = it - v * Tw;
        const int64_t j = t0 + jl;
        const int c = jl + H;
        const double* Rp = REC + (2 * v) * E;
        const double* Rm = REC + (2 * v + 1) * E;
        // edges of point jl: j-3/2 -> t = jl, j-1/2 -> jl+1, j+1/2 -> jl+2, j+3/2 -> jl+3
        const double Fl2 = Rp[jl] + Rm[jl], Fl = Rp[jl + 1] + Rm[jl + 1];
        const double Fr = Rp[jl + 2] + Rm[jl + 2], Fr2 = Rp[jl + 3] + Rm[jl + 3];
        double K = fma(9.0 / 8.0, Fl - Fr, (1.0 / 24.0) * (Fr2 - Fl2)) * rdx;
        const double x = G[(NV + v) * W2 + c];
        if constexpr (PDE == EULER) {
            if (v == 3) K = fma(-a.prm[1] * x, ARR[c], K);
        }
        rk_update<RKS>(a, cx, v, j, chunk * Tw + jl, pe, K, x, rk_load<RKS>(a, cx, v * a.N + j));
    }
}

template <int PDE, int RKS>
__global__ void __launch_bounds__(256, 4) stage_weno_interp(const StageArgs a)
{
    extern __shared__ double sm[];
    weno_interp_window<PDE, RKS>(a, launch_cx(a), blockIdx.x, sm);
}

// ---------------------------------------------------------------------------
// batched solves: a persistent grid pulls whole instances (largest first) from
// a queue; one CTA runs every stage and step of its instance, so all of an
// instance's PE-to-PE dependencies stay inside the CTA (a barrier between
// stages, none between CTAs).  Per-slot level and remaining steps live on
// the device, so a launch is the same from one chunk of steps to the next.
// ---------------------------------------------------------------------------
template <int PDE, int H, bool WENO>
__global__ void __launch_bounds__(256) batch_run(const StageArgs* __restrict__ tab, int64_t* lvl, int64_t* left,
                                                 const int* __restrict__ order, int n_order, int* queue,
                                                 int64_t chunk)
{
    extern __shared__ double sm[];
    __shared__ int s_q;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_q = atomicAdd(queue, 1);
        __syncthreads();
        const int q = s_q;
        if (q >= n_order) return;
        const int slot = order[q];
        const StageArgs& a = tab[slot];
        const int64_t L0 = lvl[slot];
        const int64_t rem = left[slot];
        const int64_t nst = rem < chunk ? rem : chunk;
        const int64_t nwin = a.P * a.wpp;
        for (int64_t n = L0; n < L0 + nst; ++n) {
            for (int s = 0; s < a.S; ++s) {
                // same buffers, stage by stage, as the per-stage launch sequence
                const double* X = (s == 0) ? a.state : ((s & 1) ? a.bufA : a.bufB);
                double* Y = (s == a.S - 1) ? a.state : ((s & 1) ? a.bufB : a.bufA);
                const Cx cx{n, s, X, Y, a.state};
                for (int64_t w = 0; w < nwin; ++w) {
                    if constexpr (WENO)
                        weno_window<PDE>(a, cx, w, sm);
                    else
                        central_window<PDE, H>(a, cx, w, sm, threadIdx.x, blockDim.x);
                    __syncthreads();
                }
            }
        }
        if (threadIdx.x == 0) {
            lvl[slot] = L0 + nst;
            left[slot] = rem - nst;
        }
    }
}

// Flat mode: one launch per stage over the windows of every bound instance
// of a kernel variant, so large instances spread over all SMs; an instance
// with no steps left, or whose RK scheme has fewer stages, skips the launch.
// CTA c takes window win_idx[c] & AT_BATCH_WIN_MASK of slot win_slot[c] and,
// when bit 30 of win_idx[c] is set (central PDEs), the next window of the
// same slot too, one half of the threads each with win_smem doubles of
// shared memory apiece: two windows' fill items then share the barrier phases
// of one CTA, as on the per-stage path.
constexpr int AT_BATCH_WIN_MASK = 0x3fffffff;
template <int PDE, int H, bool WENO>
__global__ void __launch_bounds__(256, 4) batch_stage(const StageArgs* __restrict__ tab, const int64_t* __restrict__ lvl,
                                                   const int64_t* __restrict__ left, const int* __restrict__ win_slot,
                                                   const int* __restrict__ win_idx, int stage, int win_smem)
{
    extern __shared__ double sm[];
    const int slot = win_slot[blockIdx.x];
    if (left[slot] <= 0) return;  // the whole CTA: both windows belong to the slot
    const StageArgs& a = tab[slot];
    if (stage >= a.S) return;
    const double* X = (stage == 0) ? a.state : ((stage & 1) ? a.bufA : a.bufB);
    double* Y = (stage == a.S - 1) ? a.state : ((stage & 1) ? a.bufB : a.bufA);
    const Cx cx{lvl[slot], stage, X, Y, a.state};
    const int e = win_idx[blockIdx.x];
    const int w0 = e & AT_BATCH_WIN_MASK;
    if constexpr (WENO) {
        weno_window<PDE>(a, cx, w0, sm);
    } else {
        if (e >> 30) {
            const int half = blockDim.x >> 1;
            const int g = threadIdx.x >= half ? 1 : 0;
            central_window<PDE, H>(a, cx, w0 + g, sm + (size_t)g * win_smem, threadIdx.x - g * half, half);
        } else {
            central_window<PDE, H>(a, cx, w0, sm, threadIdx.x, blockDim.x);
        }
    }
}

// after every stage of a step: advance the level of each slot with steps left
__global__ void batch_advance(int64_t* lvl, int64_t* left, const int* __restrict__ slots, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = slots[i];
        if (left[s] > 0) {
            lvl[s] += 1;
            left[s] -= 1;
        }
    }
}

// copy every slot's status word into one array (one read for the host)
__global__ void batch_status(const StageArgs* __restrict__ tab, const int* __restrict__ slots, int n, int* out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = *tab[slots[i]].status;
}

// seed the ring with the edge windows of the state at level 0, stage 0
__global__ void ring_seed(const StageArgs a)
{
    const int64_t total = a.P * 2 * a.H * a.nvar;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(t % a.nvar);
        const int h = (int)((t / a.nvar) % a.H);
        const int side = (int)((t / ((int64_t)a.nvar * a.H)) % 2);
        const int64_t pe = t / ((int64_t)a.nvar * a.H * 2);
        const int64_t j = pe * a.B + (side == 0 ? h : a.B - a.H + h);
        a.ring[ring_index(a, 0, 0, pe, side, h, v)] = a.u[v * a.N + j];
    }
}

// ---------------------------------------------------------------------------
// Reading A of the stage history (Sec. 2.3: the stage values a PE's buffer
// points need are formed from the neighbour's u^m rather than received): for
// every PE boundary, the stage arguments U^{m,(s)} of the two edge windows
// next to it, recomputed as a synchronous RK step from u^m would form them,
// written into the ring at level m for every stage s.  Stage s at the
// window needs K_{s-1} there, which needs U^{(s-1)} H points further out, so
// the strip is 2 S H points centred on the boundary (S H on each side) and
// the points where U^{(r)} is known shrink by H per stage.  One warp per
// boundary, lane i = strip point i (2 S H <= 32).  The right-hand side and
// the update are those of the per-stage kernels, operation for operation
// (the derived quantities, the central taps in the same order, the Arrhenius
// source, rk_update's formulas), so with no delays the recomputed values are
// bit for bit the ones the PEs compute themselves.
// ---------------------------------------------------------------------------
template <int PDE, int H, int RK>
__global__ void __launch_bounds__(128) ring_recompute(const StageArgs a, const double* __restrict__ um, int64_t m)
{
    using P = Phys<PDE>;
    constexpr int NV = P::NV, ND = P::ND;
    constexpr int S = RK == RK4 ? 4 : (RK == RK3TVD ? 3 : 2);
    constexpr int SH = S * H, W = 2 * SH;
    __shared__ double sG[4][ND][W];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * 4 + wid;  // boundary between PE b-1 and PE b
    if (b >= a.P) return;                              // whole warps only
    double* G = &sG[wid][0][0];
    const bool in = lane < W;
    int64_t j = (b * a.B - SH + lane) % a.N;  // the lane's point (periodic; the strip may wrap)
    if (j < 0) j += a.N;
    double un[NV], x[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) un[v] = x[v] = in ? um[v * a.N + j] : 0.0;
    // the window: points SH-H .. SH+H-1 of the strip; left of the boundary the
    // right edge window of PE b-1, right of it the left edge window of PE b
    const bool win = lane >= SH - H && lane < SH + H;
    const int64_t pe = lane < SH ? (b == 0 ? a.P - 1 : b - 1) : b;
    const int side = lane < SH ? 1 : 0;
    const int h = lane < SH ? lane - (SH - H) : lane - SH;
    const int r0 = (int)((uint32_t)m % (uint32_t)a.R);
    auto put = [&](int s) {
        if (win) {
            const int64_t base = (((((int64_t)r0 * a.S + s) * a.P + pe) * 2 + side) * a.H + h) * a.nvar;
#pragma unroll
            for (int v = 0; v < NV; ++v) a.ring[base + v] = x[v];
        }
    };
    put(0);
#pragma unroll 1
    for (int r = 0; r < S - 1; ++r) {
        // U^{(r)} is known on [r H, W - r H): its derived quantities
        if (lane >= r * H && lane < W - r * H) {
            double g[ND];
            P::derive(a, x, g);
#pragma unroll
            for (int d = 0; d < ND; ++d) G[d * W + lane] = g[d];
        }
        __syncwarp();
        double y[NV];
        const bool upd = lane >= (r + 1) * H && lane < W - (r + 1) * H;
        if (upd) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                double K = 0.0;
                if constexpr (PDE == ADVDIFF) {
#pragma unroll
                    for (int o = -H; o <= H; ++o) K = fma(a.cm[o + H], G[lane + o], K);
                } else {
                    const double* F = G + v * W;
#pragma unroll
                    for (int o = -H; o <= H; ++o)
                        if (o != 0) K = fma(a.c1[o + H], F[lane + o], K);
                    if (v > 0) {
                        const double* D = G + (3 + v) * W;
#pragma unroll
                        for (int o = -H; o <= H; ++o) K = fma(a.c2v[v - 1][o + H], D[lane + o], K);
                    }
                    if (v == 3) K = fma(-a.prm[4] * x[v], at_exp(-a.prm[5] * at_rcp3(G[7 * W + lane])), K);
                }
                // the stage-(r+1) argument as rk_update forms it
                if (RK == RK4) y[v] = fma(r == 2 ? a.dt : a.hdt, K, un[v]);
                else if (RK == RK3TVD) y[v] = r == 0 ? fma(a.dt, K, x[v]) : fma(0.75, un[v], 0.25 * fma(a.dt, K, x[v]));
                else y[v] = fma(a.dt, K, un[v]);
            }
        }
        __syncwarp();
        if (upd) {
#pragma unroll
            for (int v = 0; v < NV; ++v) x[v] = y[v];
        }
        put(r + 1);
    }
}

} // namespace atk

// ---------------------------------------------------------------------------
// host-side launchers (C++ linkage, used by at_abi.cu)
// ---------------------------------------------------------------------------
// reading A: the recomputed stage arguments of every PE boundary at level m
// into the ring (advection-diffusion and the reacting flow in flux form)
cudaError_t atk_launch_ring_recompute(const atk::StageArgs& a, int pde, int order, int rk, const double* um,
                                      int64_t m, cudaStream_t st)
{
    const dim3 grid((unsigned)((a.P + 3) / 4)), block(128);
#define AT_RR(PDE, HH)                                                                                   \
    do {                                                                                                 \
        if (rk == atk::RK4) atk::ring_recompute<PDE, HH, atk::RK4><<<grid, block, 0, st>>>(a, um, m);      \
        else if (rk == atk::RK3TVD) atk::ring_recompute<PDE, HH, atk::RK3TVD><<<grid, block, 0, st>>>(a, um, m); \
        else atk::ring_recompute<PDE, HH, atk::RK2><<<grid, block, 0, st>>>(a, um, m);                   \
    } while (0)
    if (pde == atk::ADVDIFF) {
        if (order == 2) AT_RR(atk::ADVDIFF, 1);
        else if (order == 4) AT_RR(atk::ADVDIFF, 2);
        else AT_RR(atk::ADVDIFF, 3);
    } else if (pde == atk::RNS) {
        if (order == 2) AT_RR(atk::RNS, 1);
        else if (order == 4) AT_RR(atk::RNS, 2);
        else AT_RR(atk::RNS, 3);
    } else {
        return cudaErrorInvalidValue;
    }
#undef AT_RR
    return cudaGetLastError();
}

size_t atk_stage_smem_bytes(int pde, int Tw, int H)
{
    const size_t W2 = Tw + 2 * H, E = Tw + 1;
    const size_t hs = (size_t)2 * H * (AT_QMAX + 1);  // ring-halo (point, level) items
    switch (pde) {
    case atk::ADVDIFF: return sizeof(double) * (W2 + hs * 1);
    case atk::RNS: return sizeof(double) * (8 * W2 + hs * 8);
    case atk::RNS_CHAIN: return sizeof(double) * (6 * W2 + hs * 6);
    // WENO: G and its first differences (2 ND W2), SP, ARR (2 W2), LAM (E),
    // the edge fluxes (NV E), HS
    case atk::EULER: return sizeof(double) * (18 * W2 + E + 4 * E + hs * 8);
    default: return sizeof(double) * (6 * W2 + E + E + hs * 2);
    }
}

int atk_stage_block(int pde, int Tw)
{
    int nv = (pde == atk::RNS || pde == atk::EULER) ? 4 : 1;
    int want = (pde == atk::EULER || pde == atk::ADV_WENO || pde == atk::BURGERS) ? 256 : nv * Tw;
    // reacting N-S: half a thread per (point, variable) item, so that a CTA of
    // 256 threads takes two whole-PE windows (below).  A window's fill has
    // fewer items than its update (own points plus ring levels, against 4 per
    // point), and two windows' fills keep more of the CTA busy before the
    // barrier (measured on GB300 at N = 2^24, PEs of 64: 15.1 ms per step with
    // one window per CTA, 13.7 with two or four)
    if (pde == atk::RNS) want = nv * Tw / 2;
    if (want > 256) want = 256;
    want = ((want + 31) / 32) * 32;
    return want < 32 ? 32 : want;
}

cudaError_t atk_launch_stage(const atk::StageArgs& a, int pde, int order, cudaStream_t st)
{
    const int64_t windows = a.P * a.wpp;
    const int b1 = atk_stage_block(pde, a.Tw);
    size_t smem1 = atk_stage_smem_bytes(pde, a.Tw, a.H);
    if (a.weno_interp) {  // G [ND][W2], SP, ARR [W2], LAM [E], REC [NV][2][E], HS with W2 = Tw + 8, E = Tw + 3
        const size_t nd = pde == atk::EULER ? 8 : 2, nv = nd / 2, W2 = a.Tw + 2 * a.H, E = a.Tw + 3;
        smem1 = sizeof(double) * (nd * W2 + 2 * W2 + E + 2 * nv * E + (size_t)2 * a.H * (AT_QMAX + 1) * nd);
    }
    // central stencils on small windows: several windows per CTA (whole PEs
    // only, dividing the window count), so a CTA carries up to 256 threads
    int m = 1;
    if ((pde == atk::ADVDIFF || pde == atk::RNS || pde == atk::RNS_CHAIN) && a.wpp == 1) {
        for (int c = 4; c >= 2; c /= 2)
            if (c * b1 <= 256 && windows % c == 0) {
                m = c;
                break;
            }
    }
    atk::StageArgs b = a;
    b.wpc = m;
    b.win_smem = (int)(smem1 / sizeof(double));
    const dim3 grid((unsigned)(windows / m)), block(b1 * m);
    const size_t smem = smem1 * m;
    // advection-diffusion on whole PEs of 32, 64, 128 or 256 points: one warp per PE
    if (pde == atk::ADVDIFF && a.wpp == 1 && (a.B == 32 || a.B == 64 || a.B == 128 || a.B == 256)) {
        const unsigned g8 = (unsigned)((a.P + 7) / 8);
        const size_t sw = sizeof(double) * 8 * (size_t)(a.B + 2 * a.H);
        const int ppl = a.B / 32;
        // classic RK4 (the advection-diffusion configuration) gets one kernel per stage kind
        const int kind = atk::rk_stage_kind(a.rk, a.stage);
#define AT_WARP_LAUNCH(HH, PP)                                                                          \
    do {                                                                                                \
        if (kind == atk::RKS_RK4_0) atk::stage_advdiff_warp<HH, PP, atk::RKS_RK4_0><<<g8, 256, sw, st>>>(b);       \
        else if (kind == atk::RKS_RK4_MID) atk::stage_advdiff_warp<HH, PP, atk::RKS_RK4_MID><<<g8, 256, sw, st>>>(b); \
        else if (kind == atk::RKS_RK4_LAST) atk::stage_advdiff_warp<HH, PP, atk::RKS_RK4_LAST><<<g8, 256, sw, st>>>(b); \
        else atk::stage_advdiff_warp<HH, PP, atk::RKS_ANY><<<g8, 256, sw, st>>>(b);                   \
    } while (0)
#define AT_WARP_PPL(HH)                                                                                 \
    do {                                                                                                \
        if (ppl == 1) AT_WARP_LAUNCH(HH, 1);                                                            \
        else if (ppl == 2) AT_WARP_LAUNCH(HH, 2);                                                       \
        else if (ppl == 4) AT_WARP_LAUNCH(HH, 4);                                                       \
        else AT_WARP_LAUNCH(HH, 8);                                                                     \
    } while (0)
        if (order == 2) AT_WARP_PPL(1);
        else if (order == 4) AT_WARP_PPL(2);
        else AT_WARP_PPL(3);
#undef AT_WARP_PPL
#undef AT_WARP_LAUNCH
        return cudaGetLastError();
    }
    // the benchmarked combinations (6th-order reacting N-S with RK4, reactive
    // Euler with RK3-TVD) get one kernel per RK stage kind
    const int kind = atk::rk_stage_kind(a.rk, a.stage);
    constexpr int ANY = atk::RKS_ANY;
    switch (pde) {
    case atk::ADVDIFF:
        if (order == 2) atk::stage_central<atk::ADVDIFF, 1, ANY><<<grid, block, smem, st>>>(b);
        else if (order == 4) atk::stage_central<atk::ADVDIFF, 2, ANY><<<grid, block, smem, st>>>(b);
        else atk::stage_central<atk::ADVDIFF, 3, ANY><<<grid, block, smem, st>>>(b);
        break;
    case atk::RNS:
        if (order == 2) atk::stage_central<atk::RNS, 1, ANY><<<grid, block, smem, st>>>(b);
        else if (order == 4) atk::stage_central<atk::RNS, 2, ANY><<<grid, block, smem, st>>>(b);
        else if (kind == atk::RKS_RK4_0) atk::stage_central<atk::RNS, 3, atk::RKS_RK4_0><<<grid, block, smem, st>>>(b);
        else if (kind == atk::RKS_RK4_MID) atk::stage_central<atk::RNS, 3, atk::RKS_RK4_MID><<<grid, block, smem, st>>>(b);
        else if (kind == atk::RKS_RK4_LAST) atk::stage_central<atk::RNS, 3, atk::RKS_RK4_LAST><<<grid, block, smem, st>>>(b);
        else atk::stage_central<atk::RNS, 3, ANY><<<grid, block, smem, st>>>(b);
        break;
    case atk::RNS_CHAIN:
        if (order == 2) atk::stage_central<atk::RNS_CHAIN, 1, ANY><<<grid, block, smem, st>>>(b);
        else if (order == 4) atk::stage_central<atk::RNS_CHAIN, 2, ANY><<<grid, block, smem, st>>>(b);
        else atk::stage_central<atk::RNS_CHAIN, 3, ANY><<<grid, block, smem, st>>>(b);
        break;
    case atk::EULER:
        if (a.weno_interp) atk::stage_weno_interp<atk::EULER, ANY><<<grid, block, smem, st>>>(b);
        else if (kind == atk::RKS_RK3_0) atk::stage_weno<atk::EULER, atk::RKS_RK3_0><<<grid, block, smem, st>>>(b);
        else if (kind == atk::RKS_RK3_1) atk::stage_weno<atk::EULER, atk::RKS_RK3_1><<<grid, block, smem, st>>>(b);
        else if (kind == atk::RKS_RK3_2) atk::stage_weno<atk::EULER, atk::RKS_RK3_2><<<grid, block, smem, st>>>(b);
        else atk::stage_weno<atk::EULER, ANY><<<grid, block, smem, st>>>(b);
        break;
    case atk::BURGERS:
        if (a.weno_interp) atk::stage_weno_interp<atk::BURGERS, ANY><<<grid, block, smem, st>>>(b);
        else atk::stage_weno<atk::BURGERS, ANY><<<grid, block, smem, st>>>(b);
        break;
    default:
        if (a.weno_interp) atk::stage_weno_interp<atk::ADV_WENO, ANY><<<grid, block, smem, st>>>(b);
        else atk::stage_weno<atk::ADV_WENO, ANY><<<grid, block, smem, st>>>(b);
        break;
    }
    return cudaGetLastError();
}

cudaError_t atk_launch_ring_seed(const atk::StageArgs& a, cudaStream_t st)
{
    const int64_t total = a.P * 2 * a.H * a.nvar;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    atk::ring_seed<<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t atk_set_smem_limits()
{
    constexpr int ANY = atk::RKS_ANY;
    const int big = 200 * 1024;
    const void* fns[] = {
        (const void*)atk::stage_weno<atk::EULER, ANY>, (const void*)atk::stage_weno<atk::EULER, atk::RKS_RK3_0>,
        (const void*)atk::stage_weno<atk::EULER, atk::RKS_RK3_1>, (const void*)atk::stage_weno<atk::EULER, atk::RKS_RK3_2>,
        (const void*)atk::stage_weno<atk::ADV_WENO, ANY>, (const void*)atk::stage_weno<atk::BURGERS, ANY>,
        (const void*)atk::stage_weno_interp<atk::EULER, ANY>, (const void*)atk::stage_weno_interp<atk::ADV_WENO, ANY>,
        (const void*)atk::stage_weno_interp<atk::BURGERS, ANY>,
        (const void*)atk::stage_central<atk::RNS, 3, ANY>, (const void*)atk::stage_central<atk::RNS, 3, atk::RKS_RK4_0>,
        (const void*)atk::stage_central<atk::RNS, 3, atk::RKS_RK4_MID>,
        (const void*)atk::stage_central<atk::RNS, 3, atk::RKS_RK4_LAST>, (const void*)atk::stage_central<atk::RNS, 2, ANY>,
        (const void*)atk::stage_central<atk::RNS, 1, ANY>, (const void*)atk::stage_central<atk::RNS_CHAIN, 1, ANY>,
        (const void*)atk::stage_central<atk::RNS_CHAIN, 2, ANY>, (const void*)atk::stage_central<atk::RNS_CHAIN, 3, ANY>,
        (const void*)atk::stage_central<atk::ADVDIFF, 1, ANY>, (const void*)atk::stage_central<atk::ADVDIFF, 2, ANY>,
        (const void*)atk::stage_central<atk::ADVDIFF, 3, ANY>};
    for (const void* f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// batched path launchers.  Kernel variants: 0..2 advection-diffusion with
// H = 1..3, 3..5 reacting N-S with H = 1..3, 6 reactive Euler, 7 scalar WENO
// advection, 8 Burgers.
// ---------------------------------------------------------------------------
int atk_batch_variant(int pde, int order)
{
    if (pde == atk::ADVDIFF) return order / 2 - 1;
    if (pde == atk::RNS) return 3 + order / 2 - 1;
    if (pde == atk::BURGERS) return 8;
    if (pde == atk::RNS_CHAIN) return 9 + order / 2 - 1;
    return pde == atk::EULER ? 6 : 7;
}

static void* batch_fn(int variant)
{
    switch (variant) {
    case 0: return (void*)atk::batch_run<atk::ADVDIFF, 1, false>;
    case 1: return (void*)atk::batch_run<atk::ADVDIFF, 2, false>;
    case 2: return (void*)atk::batch_run<atk::ADVDIFF, 3, false>;
    case 3: return (void*)atk::batch_run<atk::RNS, 1, false>;
    case 4: return (void*)atk::batch_run<atk::RNS, 2, false>;
    case 5: return (void*)atk::batch_run<atk::RNS, 3, false>;
    case 6: return (void*)atk::batch_run<atk::EULER, 3, true>;
    case 8: return (void*)atk::batch_run<atk::BURGERS, 3, true>;
    case 9: return (void*)atk::batch_run<atk::RNS_CHAIN, 1, false>;
    case 10: return (void*)atk::batch_run<atk::RNS_CHAIN, 2, false>;
    case 11: return (void*)atk::batch_run<atk::RNS_CHAIN, 3, false>;
    default: return (void*)atk::batch_run<atk::ADV_WENO, 3, true>;
    }
}

cudaError_t atk_launch_batch(int variant, const atk::StageArgs* tab, int64_t* lvl, int64_t* left, const int* order,
                             int n_order, int* queue, int64_t chunk, int grid, int block, size_t smem, cudaStream_t st)
{
    void* fn = batch_fn(variant);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* params[] = {(void*)&tab, (void*)&lvl, (void*)&left, (void*)&order, (void*)&n_order, (void*)&queue,
                      (void*)&chunk};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), params, smem, st);
}

static void* batch_stage_fn(int variant)
{
    switch (variant) {
    case 0: return (void*)atk::batch_stage<atk::ADVDIFF, 1, false>;
    case 1: return (void*)atk::batch_stage<atk::ADVDIFF, 2, false>;
    case 2: return (void*)atk::batch_stage<atk::ADVDIFF, 3, false>;
    case 3: return (void*)atk::batch_stage<atk::RNS, 1, false>;
    case 4: return (void*)atk::batch_stage<atk::RNS, 2, false>;
    case 5: return (void*)atk::batch_stage<atk::RNS, 3, false>;
    case 6: return (void*)atk::batch_stage<atk::EULER, 3, true>;
    case 8: return (void*)atk::batch_stage<atk::BURGERS, 3, true>;
    case 9: return (void*)atk::batch_stage<atk::RNS_CHAIN, 1, false>;
    case 10: return (void*)atk::batch_stage<atk::RNS_CHAIN, 2, false>;
    case 11: return (void*)atk::batch_stage<atk::RNS_CHAIN, 3, false>;
    default: return (void*)atk::batch_stage<atk::ADV_WENO, 3, true>;
    }
}

cudaError_t atk_launch_batch_stage(int variant, const atk::StageArgs* tab, const int64_t* lvl, const int64_t* left,
                                   const int* win_slot, const int* win_idx, int nwin, int stage, int block,
                                   size_t smem, int win_smem, cudaStream_t st)
{
    void* fn = batch_stage_fn(variant);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* params[] = {(void*)&tab, (void*)&lvl, (void*)&left, (void*)&win_slot, (void*)&win_idx, (void*)&stage,
                      (void*)&win_smem};
    return cudaLaunchKernel(fn, dim3(nwin), dim3(block), params, smem, st);
}

cudaError_t atk_launch_batch_advance(int64_t* lvl, int64_t* left, const int* slots, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    atk::batch_advance<<<(n + 255) / 256, 256, 0, st>>>(lvl, left, slots, n);
    return cudaGetLastError();
}

int atk_batch_max_ctas_per_sm(int variant, int block, size_t smem)
{
    int n = 0;
    if (cudaFuncSetAttribute(batch_fn(variant), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_fn(variant), block, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t atk_launch_batch_status(const atk::StageArgs* tab, const int* slots, int n, int* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    atk::batch_status<<<(n + 255) / 256, 256, 0, st>>>(tab, slots, n, out);
    return cudaGetLastError();
}
