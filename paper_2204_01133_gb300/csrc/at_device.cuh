// at_device.cuh -- device-side pieces of the AT stage kernels (sm_103a, FP64).
//
// Everything a stage kernel needs that is not the kernel itself: the launch
// argument block, the Philox4x32-10 delay draw, the temporal extrapolation of
// halo values from the history ring, and the per-PDE derived quantities.
#pragma once
#include <cuda/atomic>

#include <cstdint>

#include "exp_table.h"

#define AT_KMAX_LIMIT 15
#define AT_QMAX 3
#define AT_HMAX 3
#define AT_NDER 8

namespace atk {

enum { ADVDIFF = 0, RNS = 1, EULER = 2, ADV_WENO = 3, BURGERS = 4, RNS_CHAIN = 5 };
enum { RK2 = 0, RK3TVD = 1, RK4 = 2 };
enum { SYNC = 0, AS = 1, AT = 2 };

// Everything one stage launch needs, passed by value (well under the
// kernel-parameter limit).
struct StageArgs {
    const double* X;   // stencil source: the stage argument U^{n,(s)}   [nvar][N]
    const double* u;   // u^n (read pointwise)                            [nvar][N]
    double* acc;       // RK accumulator (RK2, RK4)                       [nvar][N]
    double* Y;         // output: next stage argument, or u^{n+1} in place [nvar][N]
    double* ring;      // edge windows of stage arguments [R][S][P][2][H][nvar]
    uint8_t* dlog;     // delays of this step [S][P][2]
    int* status;       // bit 0: a non-finite value was written
    int64_t N, P;
    int64_t level;     // n: the step being computed
    int B, Tw, wpp;    // PE size, window length, windows per PE
    int wpc, win_smem; // per-stage central kernels: windows per CTA, shared doubles per window
    int stage, S, R, H, q, nvar;
    int mode, kmax, per_stage, rk;
    uint32_t instance, key0, key1;
    double dt, hdt, dt6;                      // dt, dt/2, dt/6 (formed once on the host)
    uint64_t thr[AT_KMAX_LIMIT];              // Philox word-0 thresholds
    double w[AT_KMAX_LIMIT + 1][AT_QMAX + 1]; // extrapolation weights by delay
    uint8_t wnz[AT_KMAX_LIMIT + 1];           // bit l: level l enters at delay k (weight != 0)
    double c1[2 * AT_HMAX + 1];               // -d1_m / dx  (central)
    double c2[2 * AT_HMAX + 1];               //  d2_m / dx^2 (central)
    double cm[2 * AT_HMAX + 1];               // merged advection-diffusion taps
    double prm[16];                           // physics constants (see at.h)
    double k0, k1, k2, k3;                    // derived physics constants
    // reacting flow: the diffusion rows are u, the energy term over lambda and
    // Y, with the constants in the taps: c2v[v-1][m] = c2[m] times (4/3) mu,
    // lambda, lambda / (cp Le) for v = 1, 2, 3; kd1 = k1 / k2, kd3 = qc k3 / k2
    double c2v[3][2 * AT_HMAX + 1];
    double kd1, kd3;
    // persistent path only
    int64_t* done;       // per PE: stages completed, as the index n*S + s + 1 [P]
    double* gring;       // derived quantities of the edge windows [R][S][P][2][H][ND]
    int* abort_flag;     // set by the first wait that runs out
    int* place;          // per CTA: the SM it runs on, for the PE placement [P]
    int* place_count;    // CTAs that have written their SM
    int64_t wait_limit;  // polls before a wait gives up (bounded spin)
    int64_t withhold_pe; // fault injection: this PE never publishes (-1: none)
    int slack;           // ring levels beyond k_max + q + 1
    int arrival;         // 1: a delay is the age of the freshest neighbour data that has arrived
    int hist_recompute;  // 1: the ring holds stage values recomputed from u^m (reading A); the
                         //    stage kernels then push nothing into it
    int weno_interp;     // WENO PDEs: 1 the interpolation form (edge values, halo 4)
    // a PE range of a larger domain (split over ranks)
    int open_ends;       // 1: the range's outer buffer points read ext, not the ring
    double* ext;         // windows beyond the range's ends [R][S][2][H][nvar]
    int64_t pe_base, pe_total;  // global index of PE 0 and the domain's PE count (0: P)
    // delay trace (optional): the delay of every (step, stage, PE, side) of
    // levels trace_n0 .. trace_n0 + trace_steps - 1, [steps][S][P][2]
    uint8_t* trace;
    int64_t trace_n0, trace_steps;
    // batched path: the solve's own buffers (the stage kernels get X/Y/u per launch)
    double* bufA;
    double* bufB;
    double* state;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products
// with a Weyl key schedule; only output word 0 is used.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t philox_w0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c0;
}

// Delay seen by PE `pe` at its `side` (0 left, 1 right) at (level, stage),
// clamped so that no level below 0 is ever read.
__device__ __forceinline__ int keff_at(const StageArgs& a, int64_t level, int stage, int64_t pe, int side)
{
    if (a.mode == SYNC) return 0;
    const uint32_t sc = a.per_stage ? (uint32_t)stage : 0u;
    int64_t gpe = pe;  // the global PE index (a range of a larger domain draws the domain's delays)
    if (a.pe_total > 0) {
        gpe += a.pe_base;
        if (gpe >= a.pe_total) gpe -= a.pe_total;
    }
    const uint32_t x = philox_w0((uint32_t)level, (uint32_t)gpe, sc | ((uint32_t)side << 8), a.instance,
                                 a.key0, a.key1);
    int k = 0;
    for (int i = 0; i < a.kmax; ++i) k += ((uint64_t)x >= a.thr[i]) ? 1 : 0;
    const int qq = (a.mode == AT) ? a.q : 0;
    int64_t avail = level - qq;
    if (avail < 0) avail = 0;
    return (int64_t)k < avail ? k : (int)avail;
}

// largest delay the start-up clamp allows at `level` (no level below 0 is read)
__device__ __forceinline__ int kcap_at(const StageArgs& a, int64_t level)
{
    if (a.mode == SYNC) return 0;
    int64_t avail = level - ((a.mode == AT) ? a.q : 0);
    if (avail < 0) avail = 0;
    return avail < a.kmax ? (int)avail : a.kmax;
}

// record the delay used at (level, stage, PE, side): the per-step log and,
// when one is attached, the trace
__device__ __forceinline__ void log_delay(const StageArgs& a, int64_t level, int stage, int64_t pe, int side, int k)
{
    a.dlog[((int64_t)stage * a.P + pe) * 2 + side] = (uint8_t)k;
    if (a.trace) {
        const int64_t t = level - a.trace_n0;
        if (t >= 0 && t < a.trace_steps) a.trace[((t * a.S + stage) * a.P + pe) * 2 + side] = (uint8_t)k;
    }
}

__device__ __forceinline__ int keff(const StageArgs& a, int64_t pe, int side)
{
    return keff_at(a, a.level, a.stage, pe, side);
}

// exp(x) by Tang's table-driven method (P. T. P. Tang, ACM TOMS 15(2), 1989)
// with 256 table entries: x = (256 M + j) ln2/256 + r, |r| <= ln2/512, and
// exp(x) = 2^M 2^(j/256) (1 + expm1(r)), expm1(r) by its Taylor polynomial of
// degree 4 (the first omitted term, r^5/120, is below 4e-17).  The product
// with 2^M is an integer add to the exponent field, exact while the result is
// normal, which the fast path |x| < 512 guarantees (tested on the high word
// with integer instructions); every other x (and Inf, NaN) goes to exp().
// Nine FP64 instructions; within 2 ulp of the correctly rounded value.
__device__ __forceinline__ double at_exp(double x)
{
    static_assert(AT_EXP_N == 256, "the table has 256 entries");
    if ((__double2hiint(x) & 0x7fffffff) >= 0x40800000) return exp(x);
    const double shift = 0x1.8p52;                  // round to integer, result in the low word
    const double t = fma(x, AT_EXP_INV_L, shift);
    const int n = __double2loint(t);                // 256 M + j
    const double nf = t - shift;
    double r = fma(-nf, AT_EXP_L_HI, x);
    r = fma(-nf, AT_EXP_L_LO, r);
    double c = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    c = fma(c, r, 0.5);
    const double em1 = fma(c, r * r, r);            // expm1(r)
    const double tj = __ldg(&at_exp_tab[n & 255]);  // 2^(j/256)
    const double e = fma(tj, em1, tj);
    return __hiloint2double(__double2hiint(e) + ((n >> 8) << 20), __double2loint(e));
}

// 1/x by two Newton-Raphson steps r <- r + r (1 - x r) from the hardware's
// approximate reciprocal (rcp.approx.ftz.f64): each step squares the
// relative error, leaving the result within about an ulp of 1/x for the
// normal, finite, nonzero x the kernels divide by (densities, pressures,
// temperatures, WENO weight sums).  Zero, Inf or subnormal x give Inf or
// NaN, which the non-finite check reports.  Five FP64-pipe instructions, about
// half of an IEEE division.  The kernels use at_rcp3 below (one instruction
// fewer); this form is exported by the probe library beside it for the
// reciprocal tests.
__device__ __forceinline__ double at_rcp(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// 1/x by one cubic Newton step from the hardware's approximate reciprocal:
// with e = 1 - x r, 1/x = r (1 + e + e^2 + ...), so r + r (e + e^2) cubes the
// relative error of r (Householder's method of order 3, e.g. Householder,
// "The Numerical Treatment of a Single Nonlinear Equation", 1970), one FP64
// instruction fewer than at_rcp's two quadratic steps, within about an ulp
// of 1/x for normal, finite, nonzero x (both are tested against 1/x).  The
// kernels' reciprocals (densities, temperatures, pressures, WENO weight
// sums) all use this one.
__device__ __forceinline__ double at_rcp3(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// Inf or NaN: exponent field all ones, tested on the high word with integer
// instructions (the FP64 pipe is the scarce one on this chip)
__device__ __forceinline__ bool nonfinite(double v)
{
    return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000;
}

// Ring element of (level, stage, PE, side, point h of the edge window,
// variable v).  Levels read or written are never negative (start-up clamp)
// and stay below 2^31 (the library refuses longer runs), so the slot comes
// from a 32-bit remainder: a 64-bit one is a long software sequence that
// occupies the FP64 pipe.
__device__ __forceinline__ int64_t ring_index(const StageArgs& a, int64_t level, int stage, int64_t pe, int side,
                                              int h, int v)
{
    const int64_t r = (int64_t)((uint32_t)level % (uint32_t)a.R);
    return ((((r * a.S + stage) * a.P + pe) * 2 + side) * a.H + h) * a.nvar + v;
}

// The nvar values buffer point h beyond PE pe's `side` edge reads at level m,
// stage s: the neighbour's edge window in the ring (the neighbour's side
// 1 - side), or, at the outer edges of a range with open ends, the window
// supplied from outside the range.
__device__ __forceinline__ const double* halo_window(const StageArgs& a, int64_t m, int s, int64_t pe, int side, int h)
{
    if (a.open_ends && (side == 0 ? pe == 0 : pe == a.P - 1)) {
        const int64_t r = (int64_t)((uint32_t)m % (uint32_t)a.R);
        return a.ext + (((r * a.S + s) * 2 + side) * a.H + h) * a.nvar;
    }
    const int64_t nbr = side == 0 ? (pe == 0 ? a.P - 1 : pe - 1) : (pe == a.P - 1 ? 0 : pe + 1);
    return a.ring + ring_index(a, m, s, nbr, 1 - side, h, 0);
}

// the same slot in the ring of derived quantities (nd per point)
__device__ __forceinline__ int64_t gring_index(const StageArgs& a, int64_t level, int stage, int64_t pe, int side,
                                               int h, int nd)
{
    const int64_t r = (int64_t)((uint32_t)level % (uint32_t)a.R);
    return ((((r * a.S + stage) * a.P + pe) * 2 + side) * a.H + h) * nd;
}

// ---------------------------------------------------------------------------
// Physics: derived quantities of one state vector.  Coefficients that only
// scale a derived quantity are folded in here (they commute with the
// temporal extrapolation, which is linear).
// ---------------------------------------------------------------------------
template <int PDE>
struct Phys;

// u_t + c u_x = a u_xx: the only derived quantity is u itself.
template <>
struct Phys<ADVDIFF> {
    static constexpr int NV = 1, ND = 1;
    __device__ static void derive(const StageArgs&, const double* Q, double* g) { g[0] = Q[0]; }
};

// Reacting Navier-Stokes: g = [rho u, rho u^2 + p, u (rho E + p), rho u Y,
// u, ((2/3) mu u^2 + lam T + q_c rhoD Y) / lam, Y, T]; the diffusion rows
// 4..6 are differentiated with the taps c2v, which carry their constants
// (4/3) mu, lam and rhoD.  k0 = (4/3) mu, k1 = (2/3) mu, k2 = lam, k3 = rhoD.
template <>
struct Phys<RNS> {
    static constexpr int NV = 4, ND = 8;
    __device__ static void derive(const StageArgs& a, const double* Q, double* g)
    {
        const double gm1 = a.prm[0] - 1.0, qc = a.prm[6];
        const double rinv = at_rcp3(Q[0]);
        const double u = Q[1] * rinv;
        const double p = gm1 * (Q[2] - fma(0.5 * Q[1], u, qc * Q[3]));
        const double T = p * rinv;
        const double Y = Q[3] * rinv;
        g[0] = Q[1];
        g[1] = fma(Q[1], u, p);
        g[2] = u * (Q[2] + p);
        g[3] = Q[3] * u;
        g[4] = u;                                      // times (4/3) mu in the taps
        g[5] = fma(a.kd1 * u, u, fma(a.kd3, Y, T));    // (k1 u^2 + k2 T + qc k3 Y) / k2; times k2 in the taps
        g[6] = Y;                                      // times k3 in the taps
        g[7] = T;
    }
    // the temperature exactly as derive() forms it (same operations, same rounding)
    __device__ static double temperature(const StageArgs& a, const double* Q)
    {
        const double gm1 = a.prm[0] - 1.0, qc = a.prm[6];
        const double rinv = at_rcp3(Q[0]);
        const double u = Q[1] * rinv;
        const double p = gm1 * (Q[2] - fma(0.5 * Q[1], u, qc * Q[3]));
        return p * rinv;
    }
};

// Reacting Navier-Stokes in chain-rule form (Sec. 4): the product
// derivatives are expanded, so only the primitives g = [rho, u, p, rho E, Y,
// T] are differentiated (and extrapolated at buffer points).
template <>
struct Phys<RNS_CHAIN> {
    static constexpr int NV = 4, ND = 6;
    __device__ static void derive(const StageArgs& a, const double* Q, double* g)
    {
        const double gm1 = a.prm[0] - 1.0, qc = a.prm[6];
        const double rinv = at_rcp3(Q[0]);
        const double u = Q[1] * rinv;
        const double p = gm1 * (Q[2] - fma(0.5 * Q[1], u, qc * Q[3]));
        g[0] = Q[0];
        g[1] = u;
        g[2] = p;
        g[3] = Q[2];
        g[4] = Q[3] * rinv;
        g[5] = p * rinv;
    }
};

// Reactive Euler, WENO form: g = [C/2 (4), Q (4)], C = (rho u, rho u^2 + p,
// u (rho E + p), rho u Y); the split fluxes are C/2 +- (lam/2) Q.
template <>
struct Phys<EULER> {
    static constexpr int NV = 4, ND = 8;
    __device__ static double pressure(const StageArgs& a, const double* Q, double u)
    {
        return (a.prm[0] - 1.0) * (Q[2] - fma(0.5 * Q[1], u, a.prm[3] * Q[3]));
    }
    __device__ static void derive(const StageArgs& a, const double* Q, double* g)
    {
        const double u = Q[1] * at_rcp3(Q[0]);
        const double uh = 0.5 * u;
        const double p = pressure(a, Q, u);
        g[0] = 0.5 * Q[1];
        g[1] = 0.5 * fma(Q[1], u, p);
        g[2] = uh * (Q[2] + p);  // = (u (E + p)) / 2 exactly
        g[3] = Q[3] * uh;
        g[4] = Q[0];
        g[5] = Q[1];
        g[6] = Q[2];
        g[7] = Q[3];
    }
    // derive() and half the wave speed, (|u| + c) / 2, of one point at once
    // (1/rho, u and p formed once, by the same operations), and with ARR the
    // Arrhenius factor exp(-Ea rho / p) of the point's reaction source.
    // Halving is exact, so g[2] = (u/2)(E + p), g[3] = rho Y (u/2) and the half
    // speed |u/2| + sqrt(gamma p / (4 rho)) equal the halved products and the
    // halved speed bit for bit (sqrt is correctly rounded).
    template <bool ARR>
    __device__ static void derive_weno(const StageArgs& a, const double* Q, double* g, double& sph, double& arr)
    {
        const double rinv = at_rcp3(Q[0]);
        const double u = Q[1] * rinv;
        const double uh = 0.5 * u;
        const double p = pressure(a, Q, u);
        g[0] = 0.5 * Q[1];
        g[1] = 0.5 * fma(Q[1], u, p);
        g[2] = uh * (Q[2] + p);
        g[3] = Q[3] * uh;
        g[4] = Q[0];
        g[5] = Q[1];
        g[6] = Q[2];
        g[7] = Q[3];
        sph = fabs(uh) + sqrt((0.25 * a.prm[0]) * p * rinv);
        if constexpr (ARR) arr = at_exp(-a.prm[2] * Q[0] * at_rcp3(p));
    }
};

// Scalar linear advection, WENO form: g = [c u / 2, u].
template <>
struct Phys<ADV_WENO> {
    static constexpr int NV = 1, ND = 2;
    __device__ static void derive(const StageArgs& a, const double* Q, double* g)
    {
        g[0] = 0.5 * a.prm[0] * Q[0];
        g[1] = Q[0];
    }
    template <bool ARR>
    __device__ static void derive_weno(const StageArgs& a, const double* Q, double* g, double& sph, double&)
    {
        derive(a, Q, g);
        sph = 0.5 * fabs(a.prm[0]);  // half the wave speed
    }
};

// Inviscid Burgers, WENO form: g = [u^2 / 4, u] (C/2 with C = u^2/2); wave speed |u|.
template <>
struct Phys<BURGERS> {
    static constexpr int NV = 1, ND = 2;
    __device__ static void derive(const StageArgs&, const double* Q, double* g)
    {
        g[0] = 0.5 * (0.5 * Q[0] * Q[0]);
        g[1] = Q[0];
    }
    template <bool ARR>
    __device__ static void derive_weno(const StageArgs& a, const double* Q, double* g, double& sph, double&)
    {
        derive(a, Q, g);
        sph = 0.5 * fabs(Q[0]);  // half the wave speed |u|
    }
};

// the SM this thread runs on
__device__ __forceinline__ int sm_id()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return (int)r;
}

// The position of this CTA in a cooperative launch whose CTAs hand data to
// their neighbours (the persistent kernel: one PE per CTA; the multi-step
// fused kernel: a range of PEs per CTA).  A hand-off between SMs far apart
// (GB300's two dies) costs more than one between SMs that share a GPC, and
// the blocks of a launch are spread over the SMs in an order the program
// does not choose, so positions are dealt out by the SMs the CTAs landed on:
// every CTA records its SM, meets the others at a one-time bounded barrier
// (the launch is cooperative, so all CTAs are resident), and takes as its
// position its rank in (SM, block) order.  Consecutive positions then sit on
// the same or neighbouring SMs.  The arithmetic does not depend on where it
// runs, so results are the same bit for bit; a barrier that runs out keeps
// position = block (status bit 2 and the abort flag stop the run).  The
// caller resets *a.place_count before the launch.
__device__ __forceinline__ int64_t place_rank(const StageArgs& a)
{
    __shared__ int s_pe;
    if (threadIdx.x == 0) {
        int rank = (int)blockIdx.x;
        if (a.place && a.place_count) {
            const int me = sm_id();
            a.place[blockIdx.x] = me;
            cuda::atomic_ref<int, cuda::thread_scope_device> cnt(*a.place_count);
            cnt.fetch_add(1, cuda::memory_order_release);
            bool ok = cnt.load(cuda::memory_order_acquire) >= (int)gridDim.x;
            for (int64_t it = 0; !ok && it < a.wait_limit; ++it) {
                __nanosleep(128);
                ok = cnt.load(cuda::memory_order_acquire) >= (int)gridDim.x;
                if (!ok && (it & 63) == 0 && *(volatile int*)a.abort_flag) break;
            }
            if (ok) {
                rank = 0;
                for (int j = 0; j < (int)gridDim.x; ++j) {
                    const int sj = __ldcg(a.place + j);
                    rank += (sj < me) || (sj == me && j < (int)blockIdx.x);
                }
            } else {
                atomicOr(a.status, 2);
                atomicExch(a.abort_flag, 1);
            }
        }
        s_pe = rank;
    }
    __syncthreads();
    return s_pe;
}

// ---------------------------------------------------------------------------
// WENO5-JS reconstruction at the right edge of f[2] from f[0..4]
// (candidates of Eq. atRecon at k = 0, ideal weights {1/10, 3/5, 3/10},
// indicators of Eq. betaS, weights of Eq. omg with power 2), taken from the
// first differences a_k = f[k] - f[k-1] (k = 1..4), and arranged for few
// FP64 instructions without changing the mathematics:
//  * the second differences s_i (centred on f[i+1]) are s_0 = a_2 - a_1,
//    s_1 = a_3 - a_2, s_2 = a_4 - a_3, and the first-difference terms of the
//    indicators r_0 = f0 - 4 f1 + 3 f2 = s_0 + 2 a_2, r_1 = f1 - f3 =
//    -(a_2 + a_3) = -(s_1 + 2 a_2), r_2 = 3 f2 - 4 f3 + f4 = s_2 - 2 a_3;
//    then beta_i = (13 s_i^2 + 3 r_i^2) / 12, and with r_i expanded
//      D_0 = eps + beta_0 = s_0 ((4/3) s_0 + a_2) + a_2^2 + eps,
//      D_1 = eps + beta_1 = s_1 ((4/3) s_1 + a_2) + a_2^2 + eps,
//      D_2 = eps + beta_2 = s_2 ((4/3) s_2 - a_3) + a_3^2 + eps
//    (each a positive definite form in (s_i, a), so the sum does not
//    cancel), D_0 and D_1 sharing a_2^2 + eps;//  * the middle candidate p_1 = (-f1 + 5 f2 + 2 f3) / 6 = f2 + a_2/6 + a_3/3,
//    and the others differ from it by third differences,
//    p_0 - p_1 = (s_0 - s_1) / 3 and p_2 - p_1 = (s_1 - s_2) / 6, so
//    sum omega_i p_i = p_1 + omega_0 (p_0 - p_1) + omega_2 (p_2 - p_1);
//  * alpha_i ~ gamma_i / D_i^2 times the common factor D_0^2 D_1^2 D_2^2, and
//    numerator and denominator scaled by 10 (ideal weights 1 : 6 : 3); with
//    E_i = D_i^2, A = 3 E_0 and B = 2 E_2,
//      num = E_1 (B (s_0 - s_1) + A (s_1 - s_2))   (6 times the corrections'
//            numerator E_1 (E_2 (s_0 - s_1) / 3 + E_0 (s_1 - s_2) / 2)),
//      den = E_1 (A + E_2) + A B                   (= E_1 (3 E_0 + E_2) + 6 E_0 E_2),
//    so the reconstruction is p_1 + num / (6 den).
// Returned: num, den and s_1 (the caller forms p_1 of both signs at once and
// shares one reciprocal between the two reconstructions of an edge).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void weno5d(double a1, double a2, double a3, double a4, double eps, double& num,
                                       double& den, double& s1)
{
    const double s0 = a2 - a1;
    s1 = a3 - a2;
    const double s2 = a4 - a3;
    const double t2 = fma(a2, a2, eps);
    const double d0 = fma(s0, fma(4.0 / 3.0, s0, a2), t2);
    const double d1 = fma(s1, fma(4.0 / 3.0, s1, a2), t2);
    const double d2 = fma(s2, fma(4.0 / 3.0, s2, -a3), fma(a3, a3, eps));
    const double e0 = d0 * d0, e1 = d1 * d1, e2 = d2 * d2;
    const double A = 3.0 * e0, B = 2.0 * e2;
    num = e1 * fma(B, s0 - s1, A * (s1 - s2));
    den = fma(e1, A + e2, A * B);
}

// The LLF-split WENO5 flux at the edge left of column c of a row: the
// reconstruction of f+ = C + hl Q from columns c-3..c+1 plus that of
// f- = C - hl Q from columns c+2..c-2 (mirrored), hl half the edge's wave
// speed (Eq. Csplit).  The split fluxes' first differences are those of C
// and Q combined, P(j) = dC(j) + hl dQ(j) and M(j) = hl dQ(j) - dC(j) with
// dC(j) = C[j] - C[j-1], so they come from the rows' own first differences,
// formed once per column and shared by every edge and both signs; dC(j),
// dQ(j) are callables returning them.
// The two middle candidates add up to a centred value: p+ = f+(c-1) +
// P(c-1)/6 + P(c)/3 and p- = f-(c) + M(c+1)/6 + M(c)/3, and with
// f+(c-1) + f-(c) = C[c-1] + C[c] - hl dQ(c) and P(c) + M(c) = 2 hl dQ(c),
//   p+ + p- = C[c-1] + C[c] + (P(c-1) - P(c) + M(c+1) - M(c)) / 6
//           = C[c-1] + C[c] - (s1+ + s1-) / 6,
// s1+ = P(c) - P(c-1) and s1- = M(c) - M(c+1) being the two
// reconstructions' middle second differences.  The corrections
// num+ / (6 den+) + num- / (6 den-) share one reciprocal,
// (num+ den- + num- den+) / (6 den+ den-), and the 1/6 of both parts is
// applied once (den is at least 10 eps^4 ~ 1e-23 with eps = 1e-6 and grows
// with the fourth power of the differences, so the product stays far inside
// the double range for the states these PDEs carry).
template <class DC, class DQ>
__device__ __forceinline__ double weno_flux(const double* C, DC dC, DQ dQ, int c, double hl, double eps)
{
    double np, dp, s1p, nm, dm, s1m;
    weno5d(fma(hl, dQ(c - 2), dC(c - 2)), fma(hl, dQ(c - 1), dC(c - 1)), fma(hl, dQ(c), dC(c)),
           fma(hl, dQ(c + 1), dC(c + 1)), eps, np, dp, s1p);
    // mirrored: a_k of f- is M at columns c+2, c+1, c, c-1
    weno5d(fma(hl, dQ(c + 2), -dC(c + 2)), fma(hl, dQ(c + 1), -dC(c + 1)), fma(hl, dQ(c), -dC(c)),
           fma(hl, dQ(c - 1), -dC(c - 1)), eps, nm, dm, s1m);
    return fma(1.0 / 6.0, fma(fma(np, dm, nm * dp), at_rcp3(dp * dm), -(s1p + s1m)), C[c - 1] + C[c]);
}

// ---------------------------------------------------------------------------
// The RK update of the step-fused kernels, stage by stage: the next stage
// argument (u^{n+1} after the last stage) from K, the stage argument x and
// u^n, with the formulas and operation order of the per-stage kernels'
// update; the accumulator (RK2, RK4) is carried by the caller.
// ---------------------------------------------------------------------------
template <int RK>
struct RkS {
    static constexpr int S = RK == RK4 ? 4 : (RK == RK3TVD ? 3 : 2);
};

// the update of the per-stage kernels (rk_update), stage by stage: y from K,
// the stage argument x and u^n; the accumulator is carried by the caller
template <int RK>
__device__ __forceinline__ double fused_update(const StageArgs& a, int s, double K, double x, double un, double& acc)
{
    if (RK == RK4) {
        if (s == 0) {
            acc = K;
            return fma(a.hdt, K, un);
        }
        if (s < 3) {
            acc = fma(2.0, K, acc);
            return fma(s == 1 ? a.hdt : a.dt, K, un);
        }
        return fma(a.dt6, acc + K, un);
    }
    if (RK == RK3TVD) {
        if (s == 0) return fma(a.dt, K, x);
        if (s == 1) return fma(0.75, un, 0.25 * fma(a.dt, K, x));
        return fma(1.0 / 3.0, un, (2.0 / 3.0) * fma(a.dt, K, x));
    }
    if (s == 0) {
        acc = K;
        return fma(a.dt, K, un);
    }
    return fma(a.hdt, acc + K, un);
}

} // namespace atk
