/*
 * at_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * What it computes, following Kumari, Aditya & Donzis (arXiv 2204.01133):
 *
 *  - The domain is periodic and split into P processing elements (PEs) of B
 *    points (Sec. 2.1, Fig. 1).  Every stencil tap that leaves its PE is a
 *    "buffer point" whose value may be delayed.
 *  - A delay k in {0..k_max} is drawn for every PE boundary (Sec. 2.1, Sec. 5
 *    "delays are introduced using a random number generator at each
 *    processor boundary").  The generator is Philox4x32-10 (Salmon et al.,
 *    SC'11), used as a counter-based hash of (step, PE, stage|side<<8,
 *    instance) keyed by the seed; word 0 is compared with the cumulative
 *    probability thresholds floor(2^32 * CDF(i)).
 *  - AT schemes (Eq. geDer, Eq. at1, Appendix A): the spatial stencil is the
 *    standard central one; every buffer value u_m is replaced by the
 *    combination sum_l w_l(k) u_m^{n-k-l}, l = 0..q, where w_l are the
 *    Lagrange weights that extrapolate from the time levels n-k-l to n.
 *    q = 1 reproduces Eq. at1 (second order), q = 2 reproduces Appendix A
 *    (fourth order), q = 3 is the sixth-order member of the same family.
 *    AS schemes (Eq. async-fde) use the plain delayed value u_m^{n-k}.
 *  - AT-WENO5 (Sec. 3, Eqs. atRecon, idRec, beta2AT0-2; Appendix B): the
 *    WENO5-JS reconstruction (candidates of Eq. atRecon at k = 0, ideal
 *    weights {1/10, 3/5, 3/10}, smoothness indicators of Eq. betaS, weights of
 *    Eq. omg) applied to buffer values extrapolated linearly (q = 1).
 *  - Derived quantities (fluxes, velocity, temperature, ...) at buffer points
 *    are computed from the stored state at each delayed level and then
 *    combined across levels (the "on the fly" option of Sec. 6).
 *  - Runge-Kutta in Butcher form (Eq. rk1).  Each stage argument
 *    U^{n,(s)} = u^n + dt sum_{i<s} a_si K_i is kept for every level, and the
 *    buffer points of stage s read U^{n-k-l,(s)}: the message of Sec. 2.3
 *    carries all stages of a step, so stage s of an old level is available.
 *  - Inviscid Burgers u_t + (u^2/2)_x = 0 with WENO5 / AT-WENO5 (the
 *    nonlinear order test of Sec. 3).
 *  - Governing equations (Sec. 4, Eqs. ge, convEq) reduced to two species
 *    (fuel -> product, equal molecular weights and heat capacities) with
 *    constant transport and a one-step irreversible Arrhenius rate (Sec. 5.2
 *    uses one-step chemistry for this purpose).  Reactive Euler for the
 *    detonation (Sec. 5.6).
 *
 * Where the paper leaves a point open, the reading taken is stated at the
 * code that depends on it.
 */
#include "at_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXD 8 /* most derived quantities per point */

struct orc_ctx {
    orc_problem pb;
    int nvar, S, H, q, R, nder;
    int64_t N, P, B;
    double a[4][4], b[4];
    double* u;     /* u^n          [nvar][N]          */
    double* hist;  /* U^{m,(s)}    [R][S][nvar][N]    */
    double* K;     /* K_s          [S][nvar][N]       */
    uint64_t thr[16];
    int64_t level;
    int32_t* keff; /* delays in use  [S][P][2]        */
    uint8_t* dlog; /* last step's    [S][P][2]        */
    int32_t* kfix; /* forced raw delays [P][2], or NULL to draw them */
    uint8_t* trace;            /* delays of every (step, stage, PE, side) to replay, or NULL */
    int64_t trace_n0, trace_steps;
    double* ext;   /* open ends: edge windows beyond the window [R][S][2][H][nvar] */
    double* syncf; /* reading A: synchronous stage arguments [R][S][nvar][N] */
    struct orc_ctx* shadow; /* reading A: the same problem in SYNC mode    */
};

/* ------------------------------------------------------------------ */
/* Philox4x32-10, Salmon, Moraes, Dror & Shaw, SC'11, Sec. 3.2/4.2.    */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * x0;
        uint64_t p1 = (uint64_t)M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

/* Probabilities p_0..p_kmax (Sec. 2.1: sum p_k = 1) -> thresholds.
 * Table entries are normalised by their sum (a table that does not sum to 1,
 * like p = [0.3, 0.3, 0.3] of Table wenoLin, is read as proportional).
 * Geometric: p_k proportional to r (1-r)^k on {0..kmax}. */
void orc_thresholds(int k_max, int dist, const double* prob, uint64_t* thr)
{
    double w[16];
    for (int i = 0; i <= k_max; ++i) {
        if (dist == ORC_UNIFORM)
            w[i] = 1.0;
        else if (dist == ORC_TABLE)
            w[i] = prob[i];
        else {
            double r = prob[0], t = r;
            for (int j = 0; j < i; ++j) t *= (1.0 - r);
            w[i] = t;
        }
    }
    double total = 0.0;
    for (int i = 0; i <= k_max; ++i) total += w[i];
    double cum = 0.0;
    for (int i = 0; i < k_max; ++i) {
        cum += w[i];
        double cdf = cum / total;
        double t = floor(cdf * 4294967296.0);
        if (t < 0.0) t = 0.0;
        if (t > 4294967296.0) t = 4294967296.0;
        thr[i] = (uint64_t)t;
    }
}

int orc_draw(const orc_ctx* c, int64_t level, int stage, int64_t pe, int side)
{
    const orc_problem* pb = &c->pb;
    uint32_t s_ctr = pb->per_stage ? (uint32_t)stage : 0u;
    int64_t gpe = pe;
    if (pb->pe_total > 0) {
        gpe = (pb->pe_base + pe) % pb->pe_total;
        if (gpe < 0) gpe += pb->pe_total;
    }
    uint32_t ctr[4] = {(uint32_t)level, (uint32_t)gpe, s_ctr | ((uint32_t)side << 8), pb->instance};
    uint32_t key[2] = {(uint32_t)(pb->seed & 0xffffffffu), (uint32_t)(pb->seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    int k = 0;
    for (int i = 0; i < pb->k_max; ++i)
        if ((uint64_t)out[0] >= c->thr[i]) ++k;
    return k;
}

/* Start-up clamp (the paper is silent): never read a level below 0.  A delay
 * is never larger than k_max, the oldest level the history keeps. */
static int clamp_k(const orc_ctx* c, int64_t level, int k)
{
    if (c->pb.mode == ORC_SYNC) return 0;
    if (k > c->pb.k_max) k = c->pb.k_max;
    if (k < 0) k = 0;
    int qq = (c->pb.mode == ORC_AT) ? c->q : 0;
    int64_t avail = level - qq;
    if (avail < 0) avail = 0;
    return (k < avail) ? k : (int)avail;
}

/* Lagrange weights that extrapolate values at times -k, -k-1, ..., -k-q to
 * time 0:  w_l = prod_{m != l} (k+m) / (m-l).  Numerator and denominator are
 * formed as integers first, so the weights are exact. */
void orc_lagrange_weights(int q, int k, double* w)
{
    for (int l = 0; l <= q; ++l) {
        long long num = 1, den = 1;
        for (int m = 0; m <= q; ++m) {
            if (m == l) continue;
            num *= (long long)(k + m);
            den *= (long long)(m - l);
        }
        w[l] = (double)num / (double)den;
    }
}

/* ------------------------------------------------------------------ */
/* Central stencils (textbook), numerators over a common denominator. */
/* ------------------------------------------------------------------ */
static const double D1_2[3] = {-1, 0, 1}, D1_2den = 2;
static const double D2_2[3] = {1, -2, 1}, D2_2den = 1;
static const double D1_4[5] = {1, -8, 0, 8, -1}, D1_4den = 12;
static const double D2_4[5] = {-1, 16, -30, 16, -1}, D2_4den = 12;
static const double D1_6[7] = {-1, 9, -45, 0, 45, -9, 1}, D1_6den = 60;
static const double D2_6[7] = {2, -27, 270, -490, 270, -27, 2}, D2_6den = 180;

static void central_tables(int order, const double** d1, double* d1den, const double** d2, double* d2den)
{
    if (order == 2) {
        *d1 = D1_2; *d1den = D1_2den; *d2 = D2_2; *d2den = D2_2den;
    } else if (order == 4) {
        *d1 = D1_4; *d1den = D1_4den; *d2 = D2_4; *d2den = D2_4den;
    } else {
        *d1 = D1_6; *d1den = D1_6den; *d2 = D2_6; *d2den = D2_6den;
    }
}

/* ------------------------------------------------------------------ */
/* WENO5-JS reconstruction at x_{j+1/2} from v = f_{j-2..j+2}.         */
/* Candidates: Eq. atRecon at k = 0.  Ideal weights: Eq. idRec.        */
/* Smoothness indicators: Eq. betaS.  Nonlinear weights: Eq. omg.      */
/* ------------------------------------------------------------------ */
double orc_weno5_js(const double v[5], double eps)
{
    double p0 = v[0] / 3.0 - 7.0 * v[1] / 6.0 + 11.0 * v[2] / 6.0;
    double p1 = -v[1] / 6.0 + 5.0 * v[2] / 6.0 + v[3] / 3.0;
    double p2 = v[2] / 3.0 + 5.0 * v[3] / 6.0 - v[4] / 6.0;
    double b0 = (4.0 * v[0] * v[0] + (11.0 * v[2] - 19.0 * v[1]) * v[0] + 25.0 * v[1] * v[1]
                 + 10.0 * v[2] * v[2] - 31.0 * v[1] * v[2]) / 3.0;
    double b1 = (4.0 * v[1] * v[1] + (5.0 * v[3] - 13.0 * v[2]) * v[1] + 13.0 * v[2] * v[2]
                 + 4.0 * v[3] * v[3] - 13.0 * v[2] * v[3]) / 3.0;
    double b2 = (10.0 * v[2] * v[2] + (11.0 * v[4] - 31.0 * v[3]) * v[2] + 25.0 * v[3] * v[3]
                 + 4.0 * v[4] * v[4] - 19.0 * v[3] * v[4]) / 3.0;
    double a0 = 0.1 / ((eps + b0) * (eps + b0));
    double a1 = 0.6 / ((eps + b1) * (eps + b1));
    double a2 = 0.3 / ((eps + b2) * (eps + b2));
    double s = a0 + a1 + a2;
    return (a0 / s) * p0 + (a1 / s) * p1 + (a2 / s) * p2;
}

/* ------------------------------------------------------------------ */
/* WENO5 interpolation of the point value at x_{j+1/2} from            */
/* v = u_{j-2..j+2}: the third-order interpolants of Eq. interpS on    */
/* the three candidate stencils, combined by Eq. fullSten with the     */
/* weights of Eq. omg, ideal weights {1/16, 5/8, 5/16} (their          */
/* combination is the printed five-point fifth-order interpolant), and */
/* the smoothness indicators of Eq. betaS.                             */
/* ------------------------------------------------------------------ */
double orc_weno5_interp(const double v[5], double eps)
{
    double u0 = 3.0 / 8.0 * v[0] - 5.0 / 4.0 * v[1] + 15.0 / 8.0 * v[2];
    double u1 = -1.0 / 8.0 * v[1] + 3.0 / 4.0 * v[2] + 3.0 / 8.0 * v[3];
    double u2 = 3.0 / 8.0 * v[2] + 3.0 / 4.0 * v[3] - 1.0 / 8.0 * v[4];
    double b0 = (4.0 * v[0] * v[0] + (11.0 * v[2] - 19.0 * v[1]) * v[0] + 25.0 * v[1] * v[1]
                 + 10.0 * v[2] * v[2] - 31.0 * v[1] * v[2]) / 3.0;
    double b1 = (4.0 * v[1] * v[1] + (5.0 * v[3] - 13.0 * v[2]) * v[1] + 13.0 * v[2] * v[2]
                 + 4.0 * v[3] * v[3] - 13.0 * v[2] * v[3]) / 3.0;
    double b2 = (10.0 * v[2] * v[2] + (11.0 * v[4] - 31.0 * v[3]) * v[2] + 25.0 * v[3] * v[3]
                 + 4.0 * v[4] * v[4] - 19.0 * v[3] * v[4]) / 3.0;
    double a0 = (1.0 / 16.0) / ((eps + b0) * (eps + b0));
    double a1 = (5.0 / 8.0) / ((eps + b1) * (eps + b1));
    double a2 = (5.0 / 16.0) / ((eps + b2) * (eps + b2));
    double s = a0 + a1 + a2;
    return (a0 / s) * u0 + (a1 / s) * u1 + (a2 / s) * u2;
}

/* ------------------------------------------------------------------ */
/* Physics: derived quantities of one state vector                     */
/* ------------------------------------------------------------------ */
static int nvar_of(int pde) { return (pde == ORC_RNS || pde == ORC_EULER || pde == ORC_RNS_CHAIN) ? 4 : 1; }

static double* field(const orc_ctx* c, int64_t level, int s)
{
    int64_t r = level % c->R;
    if (r < 0) r += c->R;
    return c->hist + ((size_t)r * c->S + s) * (size_t)c->nvar * c->N;
}

static void state_at(const orc_ctx* c, const double* f, int64_t m, double* Q)
{
    for (int v = 0; v < c->nvar; ++v) Q[v] = f[(size_t)v * c->N + m];
}

/* ADVDIFF: [u].  ADV_WENO: [c u, u].  BURGERS: [u^2 / 2, u].
 * RNS (Eq. convEq with two species, R = 1, p = rho T):
 *   [rho u, rho u^2 + p, u (rho E + p), rho u Y, u, u^2, T, Y]
 * RNS_CHAIN (the primitive quantities whose derivatives the chain-rule
 * form of Sec. 4 takes): [rho, u, p, rho E, Y, T]
 * EULER: [rho u, rho u^2 + p, u (rho E + p), rho u Y, rho, rho u, rho E, rho Y] */
static void derive(const orc_ctx* c, const double* Q, double* g)
{
    const double* pr = c->pb.prm;
    switch (c->pb.pde) {
    case ORC_ADVDIFF:
        g[0] = Q[0];
        break;
    case ORC_ADV_WENO:
        g[0] = pr[0] * Q[0];
        g[1] = Q[0];
        break;
    case ORC_BURGERS:
        g[0] = 0.5 * Q[0] * Q[0];
        g[1] = Q[0];
        break;
    case ORC_RNS: {
        double gam = pr[0], qc = pr[6];
        double rho = Q[0], u = Q[1] / rho;
        double p = (gam - 1.0) * (Q[2] - 0.5 * Q[1] * u - qc * Q[3]);
        g[0] = Q[1];
        g[1] = Q[1] * u + p;
        g[2] = u * (Q[2] + p);
        g[3] = Q[3] * u;
        g[4] = u;
        g[5] = u * u;
        g[6] = p / rho;
        g[7] = Q[3] / rho;
        break;
    }
    case ORC_RNS_CHAIN: {
        double gam = pr[0], qc = pr[6];
        double rho = Q[0], u = Q[1] / rho;
        double p = (gam - 1.0) * (Q[2] - 0.5 * Q[1] * u - qc * Q[3]);
        g[0] = rho;
        g[1] = u;
        g[2] = p;
        g[3] = Q[2];
        g[4] = Q[3] / rho;
        g[5] = p / rho;
        break;
    }
    case ORC_EULER: {
        double gam = pr[0], qc = pr[3];
        double rho = Q[0], u = Q[1] / rho;
        double p = (gam - 1.0) * (Q[2] - 0.5 * Q[1] * u - qc * Q[3]);
        g[0] = Q[1];
        g[1] = Q[1] * u + p;
        g[2] = u * (Q[2] + p);
        g[3] = Q[3] * u;
        g[4] = Q[0];
        g[5] = Q[1];
        g[6] = Q[2];
        g[7] = Q[3];
        break;
    }
    }
}

/* largest characteristic speed |u| + c (local Lax-Friedrichs, Eq. Csplit) */
static double wave_speed(const orc_ctx* c, const double* Q)
{
    const double* pr = c->pb.prm;
    if (c->pb.pde == ORC_ADV_WENO) return fabs(pr[0]);
    if (c->pb.pde == ORC_BURGERS) return fabs(Q[0]);
    double gam = pr[0], qc = pr[3];
    double rho = Q[0], u = Q[1] / rho;
    double p = (gam - 1.0) * (Q[2] - 0.5 * Q[1] * u - qc * Q[3]);
    return fabs(u) + sqrt(gam * p / rho);
}

/* ------------------------------------------------------------------ */
/* Stencil taps as seen from PE p                                      */
/* ------------------------------------------------------------------ */
static int64_t wrap(const orc_ctx* c, int64_t m)
{
    m %= c->N;
    if (m < 0) m += c->N;
    return m;
}

/* the state at buffer position m (unwrapped) of U^{level,(s)}: the stored
 * field, or with open ends beyond the window the supplied edge window of the
 * PE there */
static void buffer_state(const orc_ctx* c, int64_t level, int s, int64_t m, double* Q)
{
    if (c->pb.history == 1) { /* reading A: the synchronous recomputation from u^level */
        int64_t r = level % c->R;
        if (r < 0) r += c->R;
        state_at(c, c->syncf + ((size_t)r * c->S + s) * (size_t)c->nvar * c->N, wrap(c, m), Q);
        return;
    }
    if (c->pb.open_ends && (m < 0 || m >= c->N)) {
        int side = (m < 0) ? 0 : 1;
        int64_t h = (m < 0) ? m + c->H : m - c->N;
        int64_t r = level % c->R;
        if (r < 0) r += c->R;
        const double* w = c->ext + ((((size_t)r * c->S + s) * 2 + side) * c->H + h) * c->nvar;
        for (int v = 0; v < c->nvar; ++v) Q[v] = w[v];
        return;
    }
    state_at(c, field(c, level, s), wrap(c, m), Q);
}

/* derived quantities at global position m (unwrapped), as PE p sees them at
 * stage s of level `level`: own points read U^{level,(s)}; buffer points
 * combine delayed levels with the AT (or AS) weights. */
static void tap(const orc_ctx* c, int64_t level, int s, int64_t p, int64_t m, double* g)
{
    int64_t lo = p * c->B, hi = lo + c->B;
    double Q[4];
    if (m >= lo && m < hi) {
        state_at(c, field(c, level, s), m, Q);
        derive(c, Q, g);
        return;
    }
    int side = (m < lo) ? 0 : 1;
    int k = c->keff[((size_t)s * c->P + p) * 2 + side];
    double w[8];
    int nw;
    if (c->pb.mode == ORC_AT) {
        orc_lagrange_weights(c->q, k, w);
        nw = c->q + 1;
    } else {
        w[0] = 1.0;
        nw = 1;
    }
    for (int d = 0; d < c->nder; ++d) g[d] = 0.0;
    for (int l = 0; l < nw; ++l) {
        double gl[MAXD];
        /* a level with weight 0 (l >= 1 at k = 0) is not part of the scheme;
         * it may not exist yet (start-up), so it is not evaluated at all */
        if (w[l] == 0.0) continue;
        buffer_state(c, level - k - l, s, m, Q);
        derive(c, Q, gl);
        for (int d = 0; d < c->nder; ++d) g[d] += w[l] * gl[d];
    }
}

/* wave speed at m as PE p sees it: own points at `level`, buffer points at
 * the most recent delayed level n-k (not extrapolated). */
static double tap_speed(const orc_ctx* c, int64_t level, int s, int64_t p, int64_t m)
{
    int64_t lo = p * c->B, hi = lo + c->B;
    double Q[4];
    if (m >= lo && m < hi) {
        state_at(c, field(c, level, s), m, Q);
    } else {
        int side = (m < lo) ? 0 : 1;
        int k = c->keff[((size_t)s * c->P + p) * 2 + side];
        buffer_state(c, level - k, s, m, Q);
    }
    return wave_speed(c, Q);
}

/* numerical flux at the edge between points i and i+1, as PE p sees it */
static void edge_flux(const orc_ctx* c, int64_t level, int s, int64_t p, int64_t i, double* F)
{
    int nv = c->nvar;
    double eps = (c->pb.pde == ORC_EULER) ? c->pb.prm[4] : c->pb.prm[1];
    double l0 = tap_speed(c, level, s, p, i), l1 = tap_speed(c, level, s, p, i + 1);
    double lam = (l0 > l1) ? l0 : l1;
    double G[6][MAXD];
    for (int o = -2; o <= 3; ++o) tap(c, level, s, p, i + o, G[o + 2]);
    for (int v = 0; v < nv; ++v) {
        double fp[6], fm[6];
        for (int o = 0; o < 6; ++o) {
            fp[o] = 0.5 * (G[o][v] + lam * G[o][nv + v]);
            fm[o] = 0.5 * (G[o][v] - lam * G[o][nv + v]);
        }
        double vp[5] = {fp[0], fp[1], fp[2], fp[3], fp[4]};
        double vm[5] = {fm[5], fm[4], fm[3], fm[2], fm[1]};
        if (c->pb.weno_interp)
            F[v] = orc_weno5_interp(vp, eps) + orc_weno5_interp(vm, eps);
        else
            F[v] = orc_weno5_js(vp, eps) + orc_weno5_js(vm, eps);
    }
}

static void rhs_point(const orc_ctx* c, int64_t level, int s, int64_t p, int64_t j, double* K)
{
    const double* pr = c->pb.prm;
    const double dx = c->pb.dx;
    int pde = c->pb.pde;
    if (pde == ORC_ADVDIFF || pde == ORC_RNS || pde == ORC_RNS_CHAIN) {
        const double *d1, *d2;
        double d1den, d2den;
        central_tables(c->pb.order, &d1, &d1den, &d2, &d2den);
        int H = c->H;
        double G[7][MAXD];
        for (int o = -H; o <= H; ++o) tap(c, level, s, p, j + o, G[o + H]);
        double D1[MAXD], D2[MAXD];
        for (int d = 0; d < c->nder; ++d) {
            double s1 = 0.0, s2 = 0.0;
            for (int o = 0; o <= 2 * H; ++o) {
                s1 += d1[o] * G[o][d];
                s2 += d2[o] * G[o][d];
            }
            D1[d] = s1 / (d1den * dx);
            D2[d] = s2 / (d2den * dx * dx);
        }
        if (pde == ORC_ADVDIFF) {
            K[0] = -pr[0] * D1[0] + pr[1] * D2[0];
        } else if (pde == ORC_RNS_CHAIN) {
            /* Eq. ge with every derivative of a product expanded by the chain
             * rule (Sec. 4), so that only the primitives rho, u, p, rho E, Y
             * and T are differentiated (and extrapolated at buffer points);
             * the factors multiplying the derivatives are the point's own
             * current values.  tau = 4/3 mu u_x, (tau u)_x = 4/3 mu (u_x^2 +
             * u u_xx), q = -lam T_x + q_c J_F, J_F = -rhoD Y_x. */
            double gam = pr[0], mu = pr[1], Pr = pr[2], Le = pr[3], A = pr[4], Ea = pr[5], qc = pr[6];
            double cp = gam / (gam - 1.0);
            double lam = mu * cp / Pr;
            double rhoD = lam / (cp * Le);
            double Q[4], g[MAXD];
            state_at(c, field(c, level, s), j, Q);
            derive(c, Q, g);
            double rho = g[0], u = g[1], p_ = g[2], rE = g[3], Y = g[4], T = g[5];
            double rho_x = D1[0], u_x = D1[1], p_x = D1[2], rE_x = D1[3], Y_x = D1[4];
            double u_xx = D2[1], Y_xx = D2[4], T_xx = D2[5];
            double wdot = A * Q[3] * exp(-Ea / T);
            K[0] = -(rho_x * u + rho * u_x);
            K[1] = -(rho_x * u * u + 2.0 * rho * u * u_x) - p_x + (4.0 / 3.0) * mu * u_xx;
            K[2] = -(u_x * (rE + p_) + u * (rE_x + p_x)) + (4.0 / 3.0) * mu * (u_x * u_x + u * u_xx)
                   + lam * T_xx + qc * rhoD * Y_xx;
            K[3] = -(rho_x * u * Y + rho * u_x * Y + rho * u * Y_x) + rhoD * Y_xx - wdot;
        } else {
            double gam = pr[0], mu = pr[1], Pr = pr[2], Le = pr[3], A = pr[4], Ea = pr[5], qc = pr[6];
            double cp = gam / (gam - 1.0);
            double lam = mu * cp / Pr;      /* thermal conductivity          */
            double rhoD = lam / (cp * Le);  /* rho * D, Fick diffusion        */
            double Q[4];
            state_at(c, field(c, level, s), j, Q);
            double g[MAXD];
            derive(c, Q, g);
            double T = g[6];
            double wdot = A * Q[3] * exp(-Ea / T);
            /* D1 of the convective fluxes; D2 of u, u^2, T, Y (Sec. 4 with
             * tau = 4/3 mu u_x, q = -lam T_x + q_c J_F, J_F = -rhoD Y_x). */
            K[0] = -D1[0];
            K[1] = -D1[1] + (4.0 / 3.0) * mu * D2[4];
            K[2] = -D1[2] + (2.0 / 3.0) * mu * D2[5] + lam * D2[6] + qc * rhoD * D2[7];
            K[3] = -D1[3] + rhoD * D2[7] - wdot;
        }
    } else {
        double Fr[4], Fl[4];
        edge_flux(c, level, s, p, j, Fr);
        edge_flux(c, level, s, p, j - 1, Fl);
        if (c->pb.weno_interp) {
            /* edge point values: the fourth-order staggered difference
             * f'_j = (9/8 (F_{j+1/2} - F_{j-1/2}) - 1/24 (F_{j+3/2} - F_{j-3/2})) / dx
             * (the paper gives no derivative formula for interpolated edge
             * values; this difference is conservative and keeps the fourth
             * order the paper states for the AT interpolant's full stencil) */
            double Fr2[4], Fl2[4];
            edge_flux(c, level, s, p, j + 1, Fr2);
            edge_flux(c, level, s, p, j - 2, Fl2);
            for (int v = 0; v < c->nvar; ++v)
                K[v] = -(9.0 / 8.0 * (Fr[v] - Fl[v]) - 1.0 / 24.0 * (Fr2[v] - Fl2[v])) / dx;
        } else {
            for (int v = 0; v < c->nvar; ++v) K[v] = -(Fr[v] - Fl[v]) / dx;
        }
        if (pde == ORC_EULER) {
            double A = pr[1], Ea = pr[2];
            double Q[4];
            state_at(c, field(c, level, s), j, Q);
            double g[MAXD];
            derive(c, Q, g);
            double rho = Q[0], u = Q[1] / rho;
            double p_ = (pr[0] - 1.0) * (Q[2] - 0.5 * Q[1] * u - pr[3] * Q[3]);
            double T = p_ / rho;
            K[3] -= A * Q[3] * exp(-Ea / T);
        }
    }
}

/* delays of stage s at `level`: a replayed trace (delays observed in a run
 * whose delays were not drawn, e.g. taken from arrival order), else forced
 * ones, else the Philox draw; always through the start-up clamp */
static void set_keff(orc_ctx* c, int64_t level, int s, const int32_t* kforce)
{
    const uint8_t* tr = NULL;
    if (c->trace && level >= c->trace_n0 && level < c->trace_n0 + c->trace_steps)
        tr = c->trace + ((size_t)(level - c->trace_n0) * c->S + s) * (size_t)c->P * 2;
    for (int64_t p = 0; p < c->P; ++p)
        for (int side = 0; side < 2; ++side) {
            int k = tr ? tr[p * 2 + side] : (kforce ? kforce[p * 2 + side] : orc_draw(c, level, s, p, side));
            c->keff[((size_t)s * c->P + p) * 2 + side] = clamp_k(c, level, k);
        }
}

/* The PEs are independent given the delays (each writes K at its own points
 * only and reads the stored stage arguments), so with OpenMP they are shared
 * among the host's threads; a point's arithmetic is the same either way. */
void orc_rhs(orc_ctx* c, int64_t level, int stage, const int32_t* kforce, double* K)
{
    set_keff(c, level, stage, kforce);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < c->P; ++p) {
        double Kp[4];
        for (int64_t jl = 0; jl < c->B; ++jl) {
            int64_t j = p * c->B + jl;
            rhs_point(c, level, stage, p, j, Kp);
            for (int v = 0; v < c->nvar; ++v) K[(size_t)v * c->N + j] = Kp[v];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Runge-Kutta in Butcher form (Eq. rk1)                               */
/* ------------------------------------------------------------------ */
static void tableau(orc_ctx* c)
{
    memset(c->a, 0, sizeof c->a);
    memset(c->b, 0, sizeof c->b);
    if (c->pb.rk == ORC_RK2) { /* Eq. rk2 */
        c->S = 2;
        c->a[1][0] = 1.0;
        c->b[0] = 0.5; c->b[1] = 0.5;
    } else if (c->pb.rk == ORC_RK3TVD) { /* Shu-Osher TVD RK3 in Butcher form */
        c->S = 3;
        c->a[1][0] = 1.0;
        c->a[2][0] = 0.25; c->a[2][1] = 0.25;
        c->b[0] = 1.0 / 6.0; c->b[1] = 1.0 / 6.0; c->b[2] = 2.0 / 3.0;
    } else { /* classic RK4 */
        c->S = 4;
        c->a[1][0] = 0.5;
        c->a[2][1] = 0.5;
        c->a[3][2] = 1.0;
        c->b[0] = 1.0 / 6.0; c->b[1] = 1.0 / 3.0; c->b[2] = 1.0 / 3.0; c->b[3] = 1.0 / 6.0;
    }
}

/* Reading A (Sec. 2.3, the receiver forms the stage values at old levels
 * itself): the stage arguments of level m as a synchronous RK step from the
 * actual u^m would form them, no delay anywhere (the shadow context runs the
 * same problem in SYNC mode), kept for every level a buffer point can read. */
static void sync_stages(orc_ctx* c)
{
    orc_ctx* sh = c->shadow;
    size_t nf = (size_t)c->nvar * c->N;
    memcpy(sh->u, c->u, nf * sizeof(double));
    sh->level = c->level;
    int64_t r = c->level % c->R;
    for (int s = 0; s < c->S; ++s) {
        orc_stage_begin(sh, s);
        memcpy(c->syncf + ((size_t)r * c->S + s) * nf, field(sh, sh->level, s), nf * sizeof(double));
        if (s < c->S - 1) orc_stage_rhs(sh, s);
    }
}

void orc_stage_begin(orc_ctx* c, int s)
{
    int64_t n = c->level;
    if (s == 0 && c->pb.history == 1) sync_stages(c);
    size_t nf = (size_t)c->nvar * c->N;
    double* U = field(c, n, s);
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < nf; ++i) {
        double acc = 0.0;
        for (int r = 0; r < s; ++r) acc += c->a[s][r] * c->K[(size_t)r * nf + i];
        U[i] = c->u[i] + c->pb.dt * acc;
    }
}

void orc_stage_rhs(orc_ctx* c, int s)
{
    size_t nf = (size_t)c->nvar * c->N;
    orc_rhs(c, c->level, s, c->kfix, c->K + (size_t)s * nf);
}

int orc_step_end(orc_ctx* c)
{
    size_t nf = (size_t)c->nvar * c->N;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (size_t i = 0; i < nf; ++i) {
        double acc = 0.0;
        for (int s = 0; s < c->S; ++s) acc += c->b[s] * c->K[(size_t)s * nf + i];
        c->u[i] = c->u[i] + c->pb.dt * acc;
        if (!isfinite(c->u[i])) bad = 1;
    }
    for (size_t i = 0; i < (size_t)c->S * c->P * 2; ++i) c->dlog[i] = (uint8_t)c->keff[i];
    c->level = c->level + 1;
    return bad ? -4 : 0;
}

/* one RK step (Eq. rk1): every stage argument, then its right-hand side */
static int step(orc_ctx* c)
{
    for (int s = 0; s < c->S; ++s) {
        orc_stage_begin(c, s);
        orc_stage_rhs(c, s);
    }
    return orc_step_end(c);
}

int orc_get_edges(const orc_ctx* c, int64_t level, int s, double* out)
{
    if (s < 0 || s >= c->S || level > c->level || level < c->level - c->R + 1) return -1;
    const double* f = field(c, level, s);
    for (int side = 0; side < 2; ++side)
        for (int h = 0; h < c->H; ++h) {
            int64_t m = side == 0 ? h : c->N - c->H + h;
            for (int v = 0; v < c->nvar; ++v) out[((size_t)side * c->H + h) * c->nvar + v] = f[(size_t)v * c->N + m];
        }
    return 0;
}

void orc_set_ext(orc_ctx* c, int64_t level, int s, int side, const double* win)
{
    int64_t r = level % c->R;
    if (r < 0) r += c->R;
    memcpy(c->ext + (((size_t)r * c->S + s) * 2 + side) * c->H * c->nvar, win, (size_t)c->H * c->nvar * sizeof(double));
}

int orc_delay(const orc_ctx* c, int64_t level, int stage, int64_t pe, int side)
{
    return clamp_k(c, level, orc_draw(c, level, stage, pe, side));
}

int orc_halo(const orc_ctx* c) { return c->H; }

int orc_run(orc_ctx* c, int64_t nsteps)
{
    for (int64_t i = 0; i < nsteps; ++i) {
        int st = step(c);
        if (st) return st;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
orc_ctx* orc_create(const orc_problem* pb, const double* init)
{
    if (!pb || !init) return NULL;
    if (pb->pe_size <= 0 || pb->n <= 0 || pb->n % pb->pe_size) return NULL;
    if (pb->k_max < 0 || pb->k_max > 15) return NULL;
    if (pb->pde < 0 || pb->pde > 5) return NULL;
    if (pb->history < 0 || pb->history > 1 || (pb->history == 1 && pb->open_ends)) return NULL;
    orc_ctx* c = (orc_ctx*)calloc(1, sizeof *c);
    if (!c) return NULL;
    c->pb = *pb;
    c->nvar = nvar_of(pb->pde);
    int weno = (pb->pde == ORC_EULER || pb->pde == ORC_ADV_WENO || pb->pde == ORC_BURGERS);
    if (pb->weno_interp && !weno) {
        free(c);
        return NULL;
    }
    if (weno) {
        c->H = pb->weno_interp ? 4 : 3; /* edges j +- 3/2 reach two more points */
        c->q = 1;
    } else {
        if (pb->order != 2 && pb->order != 4 && pb->order != 6) {
            free(c);
            return NULL;
        }
        c->H = pb->order / 2;
        c->q = pb->order / 2;
    }
    c->nder = (pb->pde == ORC_ADVDIFF) ? 1
              : ((pb->pde == ORC_ADV_WENO || pb->pde == ORC_BURGERS) ? 2 : (pb->pde == ORC_RNS_CHAIN ? 6 : 8));
    if (pb->pe_size < 2 * c->H) {
        free(c);
        return NULL;
    }
    tableau(c);
    c->N = pb->n;
    c->B = pb->pe_size;
    c->P = pb->n / pb->pe_size;
    c->R = pb->k_max + c->q + 1;
    orc_thresholds(pb->k_max, pb->dist, pb->prob, c->thr);
    size_t nf = (size_t)c->nvar * c->N;
    c->u = (double*)malloc(nf * sizeof(double));
    c->hist = (double*)calloc(nf * c->R * c->S, sizeof(double));
    c->ext = (double*)calloc((size_t)c->R * c->S * 2 * c->H * c->nvar, sizeof(double));
    if (pb->history == 1) {
        orc_problem spb = *pb;
        spb.mode = ORC_SYNC;
        spb.history = 0;
        spb.open_ends = 0;
        c->shadow = orc_create(&spb, init);
        c->syncf = (double*)calloc(nf * c->R * c->S, sizeof(double));
        if (!c->shadow || !c->syncf) {
            orc_destroy(c);
            return NULL;
        }
    }
    c->K = (double*)calloc(nf * c->S, sizeof(double));
    c->keff = (int32_t*)calloc((size_t)c->S * c->P * 2, sizeof(int32_t));
    c->dlog = (uint8_t*)calloc((size_t)c->S * c->P * 2, 1);
    if (!c->u || !c->hist || !c->K || !c->keff || !c->dlog || !c->ext) {
        orc_destroy(c);
        return NULL;
    }
    memcpy(c->u, init, nf * sizeof(double));
    c->level = 0;
    return c;
}

void orc_destroy(orc_ctx* c)
{
    if (!c) return;
    free(c->kfix);
    free(c->trace);
    free(c->u);
    free(c->hist);
    free(c->ext);
    free(c->syncf);
    orc_destroy(c->shadow);
    free(c->K);
    free(c->keff);
    free(c->dlog);
    free(c);
}

/* Host threads of the OpenMP loops (n < 1: the OpenMP default, all cores);
 * returns the number of threads that the loops will use (1 without OpenMP). */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n >= 1 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_nvar(const orc_ctx* c) { return c->nvar; }
int orc_stages(const orc_ctx* c) { return c->S; }
int orc_q(const orc_ctx* c) { return c->q; }
int orc_ring_levels(const orc_ctx* c) { return c->R; }
int64_t orc_level(const orc_ctx* c) { return c->level; }

void orc_get_state(const orc_ctx* c, double* out)
{
    memcpy(out, c->u, (size_t)c->nvar * c->N * sizeof(double));
}

void orc_get_delays(const orc_ctx* c, uint8_t* out)
{
    memcpy(out, c->dlog, (size_t)c->S * c->P * 2);
}

int orc_get_history(const orc_ctx* c, int64_t level, int stage, double* out)
{
    /* kept: every stage of the last R completed steps, and the stage-0
     * argument of the current level (the state itself) */
    if (stage < 0 || stage >= c->S) return -1;
    if (level == c->level && stage == 0) {
        memcpy(out, c->u, (size_t)c->nvar * c->N * sizeof(double));
        return 0;
    }
    if (level >= c->level || level < c->level - c->R) return -1;
    memcpy(out, field(c, level, stage), (size_t)c->nvar * c->N * sizeof(double));
    return 0;
}

void orc_set_history(orc_ctx* c, int64_t level, int stage, const double* f)
{
    memcpy(field(c, level, stage), f, (size_t)c->nvar * c->N * sizeof(double));
}

/* numerical WENO flux at the edge between points i and i+1 as PE pe sees it
 * (exposed for the pins; kforce as in orc_rhs) */
void orc_edge_flux(orc_ctx* c, int64_t level, int stage, const int32_t* kforce, int64_t pe, int64_t i,
                   double* F)
{
    set_keff(c, level, stage, kforce);
    edge_flux(c, level, stage, pe, i, F);
}

/* pieces for the pins: place the run at a level with a given u^n, and use
 * fixed delays (clamped like drawn ones) instead of drawing them */
void orc_set_level(orc_ctx* c, int64_t level) { c->level = level; }

void orc_set_state(orc_ctx* c, const double* u)
{
    memcpy(c->u, u, (size_t)c->nvar * c->N * sizeof(double));
}

void orc_set_delay_trace(orc_ctx* c, const uint8_t* trace, int64_t n0, int64_t nsteps)
{
    free(c->trace);
    c->trace = NULL;
    if (!trace || nsteps <= 0) return;
    const size_t bytes = (size_t)nsteps * c->S * (size_t)c->P * 2;
    c->trace = (uint8_t*)malloc(bytes);
    memcpy(c->trace, trace, bytes);
    c->trace_n0 = n0;
    c->trace_steps = nsteps;
}

void orc_force_delays(orc_ctx* c, const int32_t* k)
{
    if (!k) {
        free(c->kfix);
        c->kfix = NULL;
        return;
    }
    if (!c->kfix) c->kfix = (int32_t*)malloc((size_t)c->P * 2 * sizeof(int32_t));
    memcpy(c->kfix, k, (size_t)c->P * 2 * sizeof(int32_t));
}
