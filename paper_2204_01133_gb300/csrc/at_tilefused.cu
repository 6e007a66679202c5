// at_tilefused.cu -- the step-fused path for the reacting flow: all S stages
// of an RK step in one launch.
//
// A CTA holds a tile of W consecutive PEs and, on each side, a strip of the
// D = S H points of the neighbouring PE nearest the tile.  Stage s of the
// tile's PEs needs the neighbours' stage-s arguments at their edge points
// (delay 0), and stage s at a point needs stage s-1 at the points H around
// it; so the strips are recomputed here from u^n, stage by stage, on the
// points where they are known, which shrink by H per stage (the paper's
// remark that stage values at buffer points can be computed locally, Sec.
// 2.3).  Levels older than n come from the history ring, written by earlier
// steps.  Everything a step needs stays in shared memory: u^n is read once
// and u^{n+1} written once (to the other of two buffers: the neighbouring
// CTAs read the strips' u^n during the same step).
//
// The arithmetic, and its order, is that of the per-stage kernels: the
// derived quantities, the extrapolation of buffer values with the weights of
// the drawn delay (Eq. at1, Appendix A; a delay-0 buffer value goes through
// the same weighted sum, with the level-n value taken from the tile instead
// of the ring), the central taps, the Arrhenius source and the RK update.
// So the results are bit for bit those of the per-stage path.
#include <cuda_runtime.h>

#include "at_device.cuh"

namespace atk {

// Shared memory (doubles), E = W B + 2 D extended points (extended index i
// <-> global point p0 B - D + i):
//   UN  [NV][E]             u^n
//   XS  [2][NV][E]          stage arguments by stage parity
//   AC  [NV][E]             RK accumulator (RK2, RK4)
//   G   [W+2][ND][B + 2H]   derived quantities by PE row: row 0 the left
//                           strip's PE, rows 1..W the tile, row W+1 the
//                           right strip's PE; own point j at column H + j,
//                           buffer values at 0..H-1 and H+B..H+B+H-1
//   HS  [W+1][2][H][q+1][ND] buffer (point, level) derivations
template <int PDE, int H, int RK>
__global__ void __launch_bounds__(256) tile_fused(const StageArgs a, const double* __restrict__ uin,
                                                   double* __restrict__ uout, int64_t n, int W)
{
    using P = Phys<PDE>;
    constexpr int NV = P::NV, ND = P::ND;
    constexpr int S = RkS<RK>::S;
    constexpr int D = S * H;
    const int B = a.B;
    const int T = W * B, E = T + 2 * D, RW = B + 2 * H;
    const int64_t PP = a.P;
    const int64_t p0 = (int64_t)blockIdx.x * W;
    const int nW = (int)(PP - p0 < W ? PP - p0 : W);  // PEs of this tile (the last tile may hold fewer)
    const int Tn = nW * B, En = Tn + 2 * D;            // this tile's points, extended
    const int nw = (a.mode == AT) ? a.q + 1 : 1;
    extern __shared__ double sm[];
    double* UN = sm;
    double* XS = UN + NV * E;
    double* AC = XS + 2 * NV * E;
    double* G = AC + NV * E;
    double* HS = G + (W + 2) * ND * RW;
    __shared__ int s_k[2 * 9];  // delays of the buffer sides, [boundary][side] (W + 1 <= 9)

    // the PE of row r (0: left strip, 1..nW: tile, nW + 1: right strip)
    auto pe_of = [&](int r) -> int64_t {
        int64_t pe = p0 - 1 + r;
        if (pe < 0) pe += PP;
        if (pe >= PP) pe -= PP;
        return pe;
    };
    // extended index of point j of row r
    auto ext_of = [&](int r, int j) -> int { return r == 0 ? j - (B - D) : D + (r - 1) * B + j; };

    // u^n on the tile and the strips
    for (int it = threadIdx.x; it < NV * En; it += blockDim.x) {
        const int v = it / En, i = it - v * En;
        int64_t g = p0 * B - D + i;
        if (g < 0) g += a.N;
        if (g >= a.N) g -= a.N;
        const double x = __ldcg(uin + v * a.N + g);  // the strips are other CTAs' points
        UN[v * E + i] = x;
        XS[v * E + i] = x;
        AC[v * E + i] = 0.0;
    }
    __syncthreads();

    for (int s = 0; s < S; ++s) {
        const double* X = XS + (s & 1) * NV * E;
        double* Xn = XS + ((s + 1) & 1) * NV * E;
        const int lo = s * H, hi = En - s * H;  // where X is known
        // delays of the buffer sides: boundary b lies between rows b and b+1;
        // side 0 is row b's right buffer (PE pe_of(b), side 1), side 1 is row
        // b+1's left buffer (PE pe_of(b + 1), side 0)
        if (threadIdx.x < 2 * (nW + 1)) {
            const int b = threadIdx.x >> 1, w = threadIdx.x & 1;
            const int64_t pe = pe_of(w == 0 ? b : b + 1);
            const int side = w == 0 ? 1 : 0;
            const int k = keff_at(a, n, s, pe, side);
            s_k[threadIdx.x] = k;
            const bool tile_pe = w == 0 ? (b >= 1) : (b + 1 <= nW);
            if (tile_pe) log_delay(a, n, s, pe, side, k);  // the owner logs its own delays
        }
        // own points: derived quantities where X is known
        for (int it = threadIdx.x; it < En; it += blockDim.x) {
            if (it < lo || it >= hi) continue;
            int r, j;
            if (it < D) {
                r = 0;
                j = B - D + it;
            } else if (it < D + Tn) {
                r = 1 + (it - D) / B;
                j = (it - D) - (r - 1) * B;
            } else {
                r = nW + 1;
                j = it - D - Tn;
            }
            double Q[NV], g[ND];
#pragma unroll
            for (int v = 0; v < NV; ++v) Q[v] = X[v * E + it];
            P::derive(a, Q, g);
            double* Gr = G + r * ND * RW;
#pragma unroll
            for (int d = 0; d < ND; ++d) Gr[d * RW + H + j] = g[d];
        }
        __syncthreads();
        // buffer (point, level) items: the level n-k-l value of the neighbour's
        // edge point, derived (level n: the neighbour's stage argument here;
        // older levels: the ring)
        const int nitems = (nW + 1) * 2 * H * nw;
        for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
            const int l = it % nw, h = (it / nw) % H, w = (it / (nw * H)) & 1, b = it / (nw * H * 2);
            const int k = s_k[b * 2 + w];
            double g[ND];
            if ((a.wnz[k] >> l) & 1) {  // a level with weight 0 is not part of the scheme
                double Q[NV];
                // row b's right buffer reads row b+1's point h; row b+1's left
                // buffer reads row b's point B-H+h
                const int rn = w == 0 ? b + 1 : b;
                const int jn = w == 0 ? h : B - H + h;
                if (k + l == 0) {
                    const int i = ext_of(rn, jn);
#pragma unroll
                    for (int v = 0; v < NV; ++v) Q[v] = X[v * E + i];
                } else {
                    const int64_t base = ring_index(a, n - k - l, s, pe_of(rn), w == 0 ? 0 : 1, h, 0);
#pragma unroll
                    for (int v = 0; v < NV; ++v) Q[v] = __ldcg(a.ring + base + v);
                }
                P::derive(a, Q, g);
            } else {
#pragma unroll
                for (int d = 0; d < ND; ++d) g[d] = 0.0;
            }
#pragma unroll
            for (int d = 0; d < ND; ++d) HS[it * ND + d] = g[d];
        }
        __syncthreads();
        // weighted sums into the buffer columns, in level order
        for (int it = threadIdx.x; it < (nW + 1) * 2 * H * ND; it += blockDim.x) {
            const int d = it % ND, h = (it / ND) % H, w = (it / (ND * H)) & 1, b = it / (ND * H * 2);
            const int k = s_k[b * 2 + w];
            const int base = ((b * 2 + w) * H + h) * nw;
            double acc = ((a.mode == AT) ? a.w[k][0] : 1.0) * HS[base * ND + d];
            for (int l = 1; l < nw; ++l) acc = fma(a.w[k][l], HS[(base + l) * ND + d], acc);
            const int r = w == 0 ? b : b + 1;
            G[r * ND * RW + d * RW + (w == 0 ? H + B + h : h)] = acc;
        }
        __syncthreads();
        // stencil, source and update where stage s+1 is needed: the tile, and
        // for s < S-1 the strip points where X_{s+1} will be known
        const bool last = s == S - 1;
        const int klo = last ? D : (s + 1) * H, khi = last ? D + Tn : En - (s + 1) * H;
        const int nk = khi - klo;
        for (int it = threadIdx.x; it < NV * nk; it += blockDim.x) {
            const int v = it / nk, i = klo + (it - v * nk);
            int r, j;
            if (i < D) {
                r = 0;
                j = B - D + i;
            } else if (i < D + Tn) {
                r = 1 + (i - D) / B;
                j = (i - D) - (r - 1) * B;
            } else {
                r = nW + 1;
                j = i - D - Tn;
            }
            const double* Gr = G + r * ND * RW;
            const int c = j + H;
            const double x = X[v * E + i];
            double K = 0.0;
            if constexpr (PDE == ADVDIFF) {
#pragma unroll
                for (int o = -H; o <= H; ++o) K = fma(a.cm[o + H], Gr[c + o], K);
            } else {
                const double* F = Gr + v * RW;
#pragma unroll
                for (int o = -H; o <= H; ++o)
                    if (o != 0) K = fma(a.c1[o + H], F[c + o], K);
                if (v > 0) {
                    const double* Dq = Gr + (3 + v) * RW;
#pragma unroll
                    for (int o = -H; o <= H; ++o) K = fma(a.c2[o + H], Dq[c + o], K);
                }
                if (v == 3) K = fma(-a.prm[4] * x, at_exp(-a.prm[5] * at_rcp(Gr[7 * RW + c])), K);
            }
            double acc = AC[v * E + i];
            const double y = fused_update<RK>(a, s, K, x, UN[v * E + i], acc);
            AC[v * E + i] = acc;
            if (r >= 1 && r <= nW) {
                const int64_t pe = p0 + (r - 1);
                if (nonfinite(y)) atomicOr(a.status, 1);
                if (j < H || j >= B - H) {
                    const int side = j < H ? 0 : 1;
                    const int h = j < H ? j : j - (B - H);
                    a.ring[ring_index(a, last ? n + 1 : n, last ? 0 : s + 1, pe, side, h, v)] = y;
                }
                if (last) uout[v * a.N + pe * B + j] = y;
            }
            if (!last) Xn[v * E + i] = y;
        }
        __syncthreads();
    }
}

} // namespace atk

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {
// PEs per tile: tiles of 256 points (one PE when larger), at most 8 PEs
int tile_pes(int B) { return B >= 256 ? 1 : (256 / B > 8 ? 8 : 256 / B); }

int tile_stages(int rk) { return rk == atk::RK4 ? 4 : (rk == atk::RK3TVD ? 3 : 2); }

size_t tile_smem(int pde, int B, int H, int rk, int q)
{
    const int NV = pde == atk::RNS ? 4 : 1, ND = pde == atk::RNS ? 8 : 1;
    const int W = tile_pes(B), S = tile_stages(rk), D = S * H;
    const size_t E = (size_t)W * B + 2 * D, RW = B + 2 * H;
    return sizeof(double) * (4 * NV * E + (W + 2) * ND * RW + (size_t)(W + 1) * 2 * H * (q + 1) * ND);
}

template <int PDE, int H>
const void* tile_fn_rk(int rk)
{
    if (rk == atk::RK4) return (const void*)atk::tile_fused<PDE, H, atk::RK4>;
    if (rk == atk::RK3TVD) return (const void*)atk::tile_fused<PDE, H, atk::RK3TVD>;
    return (const void*)atk::tile_fused<PDE, H, atk::RK2>;
}

const void* tile_fn(int pde, int H, int rk)
{
    if (pde == atk::RNS) return H == 1 ? tile_fn_rk<atk::RNS, 1>(rk) : H == 2 ? tile_fn_rk<atk::RNS, 2>(rk)
                                                                             : tile_fn_rk<atk::RNS, 3>(rk);
    return H == 1 ? tile_fn_rk<atk::ADVDIFF, 1>(rk) : H == 2 ? tile_fn_rk<atk::ADVDIFF, 2>(rk)
                                                             : tile_fn_rk<atk::ADVDIFF, 3>(rk);
}
} // namespace

// the tile-fused kernel takes the reacting flow in flux form with PEs of at
// least S H points and tiles that fit shared memory
bool atk_tile_fused_supported(int pde, int order, int B, int rk, int q)
{
    if (pde != atk::RNS) return false;
    const int H = order / 2, S = tile_stages(rk);
    if (B < S * H || B > 1024) return false;
    return tile_smem(pde, B, H, rk, q) <= 200 * 1024;
}

cudaError_t atk_launch_tile_fused(const atk::StageArgs& a, int pde, int order, int64_t n, const double* uin,
                                  double* uout, cudaStream_t st)
{
    const int H = order / 2;
    const void* fn = tile_fn(pde, H, a.rk);
    const size_t smem = tile_smem(pde, a.B, H, a.rk, a.q);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int W = tile_pes(a.B);
    const int64_t grid = (a.P + W - 1) / W;
    atk::StageArgs args = a;
    void* params[] = {(void*)&args, (void*)&uin, (void*)&uout, (void*)&n, (void*)&W};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(256), params, smem, st);
}
