/*
 * at_oracle.h -- plain FP64 CPU oracle for the asynchrony-tolerant (AT)
 * Runge-Kutta-stage right-hand side of Kumari, Aditya & Donzis,
 * "Evaluation of finite difference based asynchronous PDE solver for
 * reacting flows" (arXiv 2204.01133).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library; the two meet only through
 * the seeded input generators.
 *
 * Everything here is written for checkability, not speed: full stage-field
 * histories (not edge windows), Butcher-form Runge-Kutta, one point at a
 * time, coefficients written as the textbook/paper fractions.
 */
#ifndef AT_ORACLE_H
#define AT_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_ADVDIFF = 0, ORC_RNS = 1, ORC_EULER = 2, ORC_ADV_WENO = 3, ORC_BURGERS = 4, ORC_RNS_CHAIN = 5 };
enum { ORC_RK2 = 0, ORC_RK3TVD = 1, ORC_RK4 = 2 };
enum { ORC_SYNC = 0, ORC_AS = 1, ORC_AT = 2 };
enum { ORC_UNIFORM = 0, ORC_TABLE = 1, ORC_GEOMETRIC = 2 };

typedef struct {
    int pde;          /* ORC_ADVDIFF | ORC_RNS | ORC_EULER | ORC_ADV_WENO | ORC_BURGERS | ORC_RNS_CHAIN */
    int order;        /* central order 2|4|6 (ADVDIFF, RNS); ignored for WENO  */
    int rk;           /* ORC_RK2 | ORC_RK3TVD | ORC_RK4                        */
    int64_t n;        /* grid points (periodic), n % pe_size == 0              */
    int32_t pe_size;  /* points per processing element (PE)                    */
    double dx, dt;
    double prm[16];   /* physics constants, see at_oracle.c                    */
    int mode;         /* ORC_SYNC | ORC_AS | ORC_AT                            */
    int k_max;        /* largest delay (inclusive)                             */
    int dist;         /* ORC_UNIFORM | ORC_TABLE | ORC_GEOMETRIC               */
    double prob[16];
    uint64_t seed;
    int per_stage;    /* 1: one draw per (step, stage); 0: one per step        */
    uint32_t instance;
    int64_t pe_base;  /* global index of PE 0 when the problem is a window  */
    int64_t pe_total; /* of a larger domain of pe_total PEs (0: no window);
                         only the delay counter uses them                  */
    int open_ends;    /* 1: the window's outer PE edges are not periodic: their
                         buffer points read the edge windows of the PEs
                         beyond them, supplied with orc_set_ext (a PE range
                         of one domain split over ranks)                   */
    int history;      /* what a buffer point reads at a delayed level m and
                         stage s (Sec. 2.3): 0 (reading B) the neighbour's
                         stage argument U^{m,(s)} as the neighbour computed
                         it; 1 (reading A) the stage argument recomputed
                         synchronously from the neighbour's u^m            */
    int weno_interp;  /* WENO PDEs: 0 the flux-reconstruction form (Eqs.
                         atRecon, idRec); 1 the interpolation form (Eqs.
                         interpS, fullSten, omg: edge values of the split
                         fluxes, ideal weights {1/16, 5/8, 5/16}) with the
                         fourth-order staggered difference of edge values */
} orc_problem;

typedef struct orc_ctx orc_ctx;

/* returns NULL on invalid input */
orc_ctx* orc_create(const orc_problem* pb, const double* init /* [nvar][n] */);
void orc_destroy(orc_ctx* c);
int orc_nvar(const orc_ctx* c);
int orc_stages(const orc_ctx* c);
int orc_q(const orc_ctx* c);
int orc_ring_levels(const orc_ctx* c);
int64_t orc_level(const orc_ctx* c);
/* advance nsteps full RK steps; returns 0, or -4 if a non-finite value appeared */
int orc_run(orc_ctx* c, int64_t nsteps);
void orc_get_state(const orc_ctx* c, double* out /* [nvar][n] */);
/* k_eff of the last completed step, [stages][P][2] (side 0 = left, 1 = right) */
void orc_get_delays(const orc_ctx* c, uint8_t* out);
/* host threads for the loops over PEs and points (OpenMP; n < 1: all cores);
 * returns the thread count in effect.  Results do not depend on it. */
int orc_set_threads(int n);

/* ---- one RK step stage by stage (what a rank owning a PE range does
 * between exchanges); orc_run(c, 1) is exactly these calls in order ---- */
/* form the stage argument U^{n,(s)} of the current level n */
void orc_stage_begin(orc_ctx* c, int s);
/* K_s: the right-hand side of stage s (delays drawn, clamped, logged) */
void orc_stage_rhs(orc_ctx* c, int s);
/* u^{n+1} from the K_s, level n -> n+1; 0, or -4 on a non-finite value */
int orc_step_end(orc_ctx* c);
/* edge windows of U^{level,(s)} at the window's two outer ends:
 * out[0][h][v] = points 0..H-1, out[1][h][v] = points n-H..n-1; -1 if that
 * level and stage are not stored */
int orc_get_edges(const orc_ctx* c, int64_t level, int s, double* out);
/* open_ends: the edge window of U^{level,(s)} of the PE beyond side `side`
 * (0: left of point 0, the neighbour's right edge, points in increasing x;
 * 1: right of point n-1, the neighbour's left edge), [H][nvar] */
void orc_set_ext(orc_ctx* c, int64_t level, int s, int side, const double* win);
/* the delay PE `pe` uses at (level, stage, side): the draw through the
 * start-up clamp (0 in SYNC mode) */
int orc_delay(const orc_ctx* c, int64_t level, int stage, int64_t pe, int side);
int orc_halo(const orc_ctx* c);

/* ---- pieces exposed for the pins in tests/ ---- */
/* copy the stored stage argument U^{level,(stage)} (a full field [nvar][n]);
 * -1 if that level and stage are not in the kept history */
int orc_get_history(const orc_ctx* c, int64_t level, int stage, double* out);
/* overwrite the stored stage argument U^{level,(stage)} (a full field) */
void orc_set_history(orc_ctx* c, int64_t level, int stage, const double* field);
/* right-hand side K of stage `stage` at level `level`, reading U^{level,(stage)}
 * for own points and delayed levels for PE-boundary taps.  kforce: [P][2]
 * raw delays to use (clamped like a drawn delay), or NULL to draw them. */
void orc_rhs(orc_ctx* c, int64_t level, int stage, const int32_t* kforce, double* K);
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_thresholds(int k_max, int dist, const double* prob, uint64_t* thr);
int orc_draw(const orc_ctx* c, int64_t level, int stage, int64_t pe, int side);
void orc_lagrange_weights(int q, int k, double* w);
double orc_weno5_js(const double v[5], double eps);
/* WENO5 interpolation of the value at x_{j+1/2} from v = u_{j-2..j+2}
 * (Eqs. interpS, fullSten, omg; indicators of Eq. betaS) */
double orc_weno5_interp(const double v[5], double eps);
void orc_set_level(orc_ctx* c, int64_t level);
void orc_set_state(orc_ctx* c, const double* u /* [nvar][n] */);
/* fixed raw delays [P][2] for every following step (NULL: draw again) */
void orc_force_delays(orc_ctx* c, const int32_t* k);
/* replay recorded delays: trace[nsteps][stages][P][2] holds the delay of
 * every stage of levels n0 .. n0 + nsteps - 1 (copied; NULL clears) */
void orc_set_delay_trace(orc_ctx* c, const uint8_t* trace, int64_t n0, int64_t nsteps);
/* WENO flux F[nvar] at the edge between points i and i+1 as PE `pe` sees it */
void orc_edge_flux(orc_ctx* c, int64_t level, int stage, const int32_t* kforce, int64_t pe, int64_t i,
                   double* F);

#ifdef __cplusplus
}
#endif
#endif
