// at_tilefused.cu -- the step-fused path for the reacting flow and the WENO
// PDEs (the detonation): all S stages of an RK step in one launch.
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
                    for (int o = -H; o <= H; ++o) K = fma(a.c2v[v - 1][o + H], Dq[c + o], K);
                }
                if (v == 3) K = fma(-a.prm[4] * x, at_exp(-a.prm[5] * at_rcp3(Gr[7 * RW + c])), K);
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

// ---------------------------------------------------------------------------
// The WENO PDEs (the detonation): a tile is one window of Tw points of a PE
// (the per-stage kernels' windows), plus strips of D = S H points on each
// side, which belong to the same PE (the neighbouring window) or, for the
// first and last window of a PE, to the neighbouring PE.  Points are grouped
// in rows by PE: row 1 the window's PE over its points in the region, rows 0
// and 2 the neighbouring PEs' strips when the window touches a PE edge.  A
// row sees its own points and, beyond a PE edge inside the region, H buffer
// columns formed with its own delay for that side.  Stage s: the fluxes of
// the edges around every point where stage s+1 is needed, as the row that
// owns the point sees them (the two PEs at a PE edge each form their own
// flux there, as in the per-stage kernels), then the update.
//
// Shared memory (doubles), E = Tw + 2 D; row 1 has RC = E + 2 H columns,
// rows 0 and 2 (strips) RS = D + 2 H; a quantity of row r sits at the row's
// base with the row's stride:
//   G [ND] per row, SP, ARR, LAM one per row   derived, half wave speed,
//                                             Arrhenius factor, edge speed;
//                                             the derived quantities NV..2NV-1
//                                             are the state itself, so the
//                                             own columns of G hold the stage
//                                             argument, updated in place
//   REC [NV] per row                          fluxes at the edges
//   HS [2][2][H][2][ND]                       buffer (point, level) items
//   AC [NV][E]                                accumulator (RK2, RK4 only)
// u^n is read from global memory where the update needs it (L2 holds the
// tile's part, read at the start of the step).
// ---------------------------------------------------------------------------
template <int PDE, int RK>
__global__ void __launch_bounds__(256) tile_fused_weno(const StageArgs a, const double* __restrict__ uin,
                                                        double* __restrict__ uout, int64_t n)
{
    using P = Phys<PDE>;
    constexpr int NV = P::NV, ND = P::ND;
    constexpr int H = 3;
    constexpr int S = RkS<RK>::S;
    constexpr int D = S * H;
    const int B = a.B, Tw = a.Tw;
    const int E = Tw + 2 * D, RC = E + 2 * H, RS = D + 2 * H, RT = RC + 2 * RS;
    constexpr bool has_acc = RK != RK3TVD;
    const int64_t PP = a.P;
    const int64_t win = blockIdx.x;
    const int64_t pe = a.wpp == 1 ? win : win / a.wpp;
    const int chunk = (int)(win - pe * a.wpp);
    const int64_t t0 = pe * B + (int64_t)chunk * Tw;       // first point of the window
    const bool left_edge = chunk == 0, right_edge = chunk == a.wpp - 1;
    const int64_t pl = pe == 0 ? PP - 1 : pe - 1, pr = pe == PP - 1 ? 0 : pe + 1;
    const int nw = (a.mode == AT) ? a.q + 1 : 1;
    // rows: own extended range [lo_r, hi_r) and PE
    const int lo1 = left_edge ? D : 0, hi1 = right_edge ? D + Tw : E;
    extern __shared__ double sm[];
    double* G = sm;
    double* SP = G + ND * RT;
    double* ARR = SP + RT;
    double* LAM = ARR + RT;
    double* REC = LAM + RT;
    double* HS = REC + NV * RT;
    double* AC = HS + 2 * 2 * H * 2 * ND;  // (not there for RK3)
    __shared__ int s_k[4];  // [boundary 0 (left), 1 (right)][0: outer row's side, 1: the window's side]
    auto row_of = [&](int i) -> int { return i < lo1 ? 0 : (i < hi1 ? 1 : 2); };
    auto row_lo = [&](int r) -> int { return r == 0 ? 0 : (r == 1 ? lo1 : hi1); };
    // column of extended point i in its row
    auto col_of = [&](int i) -> int { return H + i - row_lo(row_of(i)); };
    // a row's stride and the offset of its first column in a one-per-row array
    auto rstride = [&](int r) -> int { return r == 1 ? RC : RS; };
    auto roff = [&](int r) -> int { return r == 0 ? 0 : (r == 1 ? RS : RS + RC); };
    // a per-row array of m quantities: row r's quantity d at column c is
    // base[m * roff(r) + d * rstride(r) + c]
    // variable v of the stage argument at extended point i (row r, column c)
    auto xq = [&](int r, int c, int v) -> double& { return G[ND * roff(r) + (NV + v) * rstride(r) + c]; };
    // its global point
    auto glob = [&](int i) -> int64_t {
        int64_t g = t0 - D + i;
        if (g < 0) g += a.N;
        if (g >= a.N) g -= a.N;
        return g;
    };

    for (int it = threadIdx.x; it < NV * E; it += blockDim.x) {
        const int v = it / E, i = it - v * E;
        xq(row_of(i), col_of(i), v) = __ldcg(uin + v * a.N + glob(i));
        if (has_acc) AC[v * E + i] = 0.0;
    }
    __syncthreads();

    for (int s = 0; s < S; ++s) {
        const int lo = s * H, hi = E - s * H;
        // the delays at the PE edges inside the region: at the left edge the
        // left PE's right side and the window PE's left side, at the right
        // edge the window PE's right side and the right PE's left side
        if (threadIdx.x < 4) {
            const int b = threadIdx.x >> 1, w = threadIdx.x & 1;
            if (b == 0 ? left_edge : right_edge) {
                const int64_t q = w == 1 ? pe : (b == 0 ? pl : pr);
                const int side = b == 0 ? (w == 1 ? 0 : 1) : (w == 1 ? 1 : 0);
                const int k = keff_at(a, n, s, q, side);
                s_k[threadIdx.x] = k;
                if (w == 1) log_delay(a, n, s, pe, side, k);
            }
        }
        // own points where X is known: derived quantities, half wave speed, Arrhenius factor
        for (int i = threadIdx.x + lo; i < hi; i += blockDim.x) {
            const int r = row_of(i), c = col_of(i);
            double Q[NV], g[ND], sp, arr;
#pragma unroll
            for (int v = 0; v < NV; ++v) Q[v] = xq(r, c, v);
            P::template derive_weno<PDE == EULER>(a, Q, g, sp, arr);
            double* Gr = G + ND * roff(r);
#pragma unroll
            for (int d = 0; d < ND; ++d) Gr[d * rstride(r) + c] = g[d];
            SP[roff(r) + c] = sp;
            if constexpr (PDE == EULER) ARR[roff(r) + c] = arr;
        }
        __syncthreads();
        // buffer (point, level) items at the PE edges of the region
        const int nitems = 2 * 2 * H * nw;
        for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
            const int l = it % nw, h = (it / nw) % H, w = (it / (nw * H)) & 1, b = it / (nw * H * 2);
            if (!(b == 0 ? left_edge : right_edge)) continue;
            const int k = s_k[b * 2 + w];
            // the row whose buffer this is, its side, and the facing row's PE
            // and edge point: at the left edge the left row's right buffer
            // (w = 0) faces the window's first points, the window's left
            // buffer (w = 1) faces the left PE's last points; mirrored at the right edge
            const int64_t nb = b == 0 ? (w == 0 ? pe : pl) : (w == 0 ? pe : pr);
            const int nside = b == 0 ? (w == 0 ? 0 : 1) : (w == 0 ? 1 : 0);  // the facing window's side
            // extended index of the facing point (level n), in increasing x
            const int fi = b == 0 ? (w == 0 ? D + h : D - H + h) : (w == 0 ? D + Tw - H + h : D + Tw + h);
            double g[ND];
            double sp = 0.0, unused;
            if ((a.wnz[k] >> l) & 1) {
                double Q[NV];
                if (k + l == 0) {
                    const int fr = row_of(fi), fc = col_of(fi);
#pragma unroll
                    for (int v = 0; v < NV; ++v) Q[v] = xq(fr, fc, v);
                } else {
                    const int64_t base = ring_index(a, n - k - l, s, nb, nside, h, 0);
#pragma unroll
                    for (int v = 0; v < NV; ++v) Q[v] = __ldcg(a.ring + base + v);
                }
                if (l == 0) {
                    P::template derive_weno<false>(a, Q, g, sp, unused);  // the speed at level n-k
                } else {
                    P::derive(a, Q, g);
                }
            } else {
#pragma unroll
                for (int d = 0; d < ND; ++d) g[d] = 0.0;
            }
#pragma unroll
            for (int d = 0; d < ND; ++d) HS[it * ND + d] = g[d];
            if (l == 0) {
                // the buffer column: the row on the other side of the PE edge from the facing point
                const int r = b == 0 ? (w == 0 ? 0 : 1) : (w == 0 ? 2 : 1);
                const int rlen = (r == 0 ? lo1 : (r == 1 ? hi1 - lo1 : E - hi1));
                const int c = (b == 0 ? (w == 0 ? H + rlen + h : h) : (w == 0 ? h : H + rlen + h));
                if ((a.wnz[k] & 1)) SP[roff(r) + c] = sp;
            }
        }
        __syncthreads();
        for (int it = threadIdx.x; it < 2 * 2 * H * ND; it += blockDim.x) {
            const int d = it % ND, h = (it / ND) % H, w = (it / (ND * H)) & 1, b = it / (ND * H * 2);
            if (!(b == 0 ? left_edge : right_edge)) continue;
            const int k = s_k[b * 2 + w];
            const int base = ((b * 2 + w) * H + h) * nw;
            double acc = ((a.mode == AT) ? a.w[k][0] : 1.0) * HS[base * ND + d];
            for (int l = 1; l < nw; ++l) acc = fma(a.w[k][l], HS[(base + l) * ND + d], acc);
            const int r = b == 0 ? (w == 0 ? 0 : 1) : (w == 0 ? 2 : 1);
            const int rlen = (r == 0 ? lo1 : (r == 1 ? hi1 - lo1 : E - hi1));
            const int c = (b == 0 ? (w == 0 ? H + rlen + h : h) : (w == 0 ? h : H + rlen + h));
            G[ND * roff(r) + d * rstride(r) + c] = acc;
        }
        __syncthreads();
        // edges: for each row, the edges around its points in the update range
        const bool last = s == S - 1;
        const int klo = last ? D : (s + 1) * H, khi = last ? D + Tw : E - (s + 1) * H;
        int ka[3], kb[3], ne[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int rlo = row_lo(r), rhi = r == 0 ? lo1 : (r == 1 ? hi1 : E);
            ka[r] = rlo > klo ? rlo : klo;
            kb[r] = rhi < khi ? rhi : khi;
            ne[r] = kb[r] > ka[r] ? kb[r] - ka[r] + 1 : 0;  // edge t sits left of point ka + t
        }
        for (int t = threadIdx.x; t < ne[0] + ne[1] + ne[2]; t += blockDim.x) {
            const int r = t < ne[0] ? 0 : (t < ne[0] + ne[1] ? 1 : 2);
            const int e = t - (r == 0 ? 0 : (r == 1 ? ne[0] : ne[0] + ne[1]));
            const int c = H + ka[r] + e - row_lo(r);  // column of the point right of the edge
            LAM[roff(r) + c] = fmax(SP[roff(r) + c - 1], SP[roff(r) + c]);  // SP holds half speeds
        }
        __syncthreads();
        const double eps = (PDE == EULER) ? a.prm[4] : a.prm[1];
        const int nrec = NV * (ne[0] + ne[1] + ne[2]);
        for (int it = threadIdx.x; it < nrec; it += blockDim.x) {
            const int t = it % (ne[0] + ne[1] + ne[2]);
            const int v = it / (ne[0] + ne[1] + ne[2]);
            const int r = t < ne[0] ? 0 : (t < ne[0] + ne[1] ? 1 : 2);
            const int e = t - (r == 0 ? 0 : (r == 1 ? ne[0] : ne[0] + ne[1]));
            const int c = H + ka[r] + e - row_lo(r);
            const double* Cr = G + ND * roff(r) + v * rstride(r);
            const double* Qr = G + ND * roff(r) + (NV + v) * rstride(r);
            // the rows' first differences formed where they are used: the same
            // operations, so the same values, as the per-stage kernels' stored ones
            REC[NV * roff(r) + v * rstride(r) + c] =
                weno_flux(Cr, [&](int j) { return Cr[j] - Cr[j - 1]; }, [&](int j) { return Qr[j] - Qr[j - 1]; }, c,
                          LAM[roff(r) + c], eps);
        }
        __syncthreads();
        const double rdx = a.k0;
        const int nk = khi - klo;
        for (int it = threadIdx.x; it < NV * nk; it += blockDim.x) {
            const int v = it / nk, i = klo + (it - v * nk);
            const int r = row_of(i), c = col_of(i);
            const double* F = REC + NV * roff(r) + v * rstride(r);
            double K = (F[c] - F[c + 1]) * rdx;
            const double x = xq(r, c, v);
            if constexpr (PDE == EULER) {
                if (v == 3) K = fma(-a.prm[1] * x, ARR[roff(r) + c], K);
            }
            double acc = has_acc ? AC[v * E + i] : 0.0;
            // u^n where the update reads it (RK3-TVD's first stage does not)
            const double un = (RK == RK3TVD && s == 0) ? 0.0 : __ldcg(uin + v * a.N + glob(i));
            const double y = fused_update<RK>(a, s, K, x, un, acc);
            if (has_acc) AC[v * E + i] = acc;
            if (i >= D && i < D + Tw) {  // the window: this CTA's points
                const int jpe = chunk * Tw + (i - D);
                if (nonfinite(y)) atomicOr(a.status, 1);
                if (jpe < H || jpe >= B - H) {
                    const int side = jpe < H ? 0 : 1;
                    const int h = jpe < H ? jpe : jpe - (B - H);
                    a.ring[ring_index(a, last ? n + 1 : n, last ? 0 : s + 1, pe, side, h, v)] = y;
                }
                if (last) uout[v * a.N + t0 + (i - D)] = y;
            }
            if (!last) xq(r, c, v) = y;  // in place: nothing else reads it in this phase
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

size_t tile_weno_smem(int pde, int Tw, int rk)
{
    const int NV = pde == atk::EULER ? 4 : 1, ND = pde == atk::EULER ? 8 : 2, H = 3;
    const size_t D = (size_t)tile_stages(rk) * H, E = (size_t)Tw + 2 * D;
    const size_t RT = (E + 2 * H) + 2 * (D + 2 * H);  // the three rows' columns
    const size_t acc = rk == atk::RK3TVD ? 0 : NV * E;  // the accumulator
    return sizeof(double) * (ND * RT + 3 * RT + NV * RT + 2 * 2 * H * 2 * ND + acc);
}

// the tile-fused kernels take the reacting flow in flux form (tiles of whole
// PEs of at least S H points) and the WENO PDEs in the reconstruction form
// (tiles of one window, PEs of at least S H points)
bool atk_tile_fused_supported(int pde, int order, int B, int rk, int q)
{
    const int S = tile_stages(rk);
    if (pde == atk::EULER || pde == atk::ADV_WENO || pde == atk::BURGERS) return B >= S * 3;
    if (pde != atk::RNS) return false;
    const int H = order / 2;
    if (B < S * H || B > 1024) return false;
    return tile_smem(pde, B, H, rk, q) <= 200 * 1024;
}

template <int PDE>
const void* tile_weno_fn(int rk)
{
    if (rk == atk::RK4) return (const void*)atk::tile_fused_weno<PDE, atk::RK4>;
    if (rk == atk::RK3TVD) return (const void*)atk::tile_fused_weno<PDE, atk::RK3TVD>;
    return (const void*)atk::tile_fused_weno<PDE, atk::RK2>;
}

cudaError_t atk_launch_tile_fused(const atk::StageArgs& a, int pde, int order, int64_t n, const double* uin,
                                  double* uout, cudaStream_t st)
{
    if (pde == atk::EULER || pde == atk::ADV_WENO || pde == atk::BURGERS) {
        const void* fn = pde == atk::EULER ? tile_weno_fn<atk::EULER>(a.rk)
                         : pde == atk::BURGERS ? tile_weno_fn<atk::BURGERS>(a.rk) : tile_weno_fn<atk::ADV_WENO>(a.rk);
        const size_t smem = tile_weno_smem(pde, a.Tw, a.rk);
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        atk::StageArgs args = a;
        void* params[] = {(void*)&args, (void*)&uin, (void*)&uout, (void*)&n};
        return cudaLaunchKernel(fn, dim3((unsigned)(a.P * a.wpp)), dim3(256), params, smem, st);
    }
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
