/*
 * at.h -- C ABI of libat_gb300.so: the asynchrony-tolerant (AT) Runge-Kutta
 * stage right-hand side of Kumari, Aditya & Donzis, "Evaluation of finite
 * difference based asynchronous PDE solver for reacting flows"
 * (arXiv 2204.01133), on one NVIDIA GB300 (sm_103a), FP64 throughout.
 *
 * The problem statement follows the paper's (Sec. 2.1 and Sec. 5): a
 * periodic 1-D domain of n points split into processing elements (PEs) of
 * pe_size points; a PDE (Sec. 4, Eqs. ge and convEq; Sec. 2.1 Eq. heat and
 * Sec. 3 advection); a stencil order (Sec. 2.2, Appendix A) or WENO5 (Sec. 3);
 * an explicit RK scheme (Sec. 2.3, Eq. rk1); a largest delay and the delay
 * probabilities (Sec. 2.1 and Table dels).  On one GPU the PEs are virtual:
 * every PE reads the values beyond its edges from a device history ring of
 * the neighbours' edge windows, at a delay drawn per (step, stage, PE,
 * side) from Philox4x32-10 keyed by the seed, so runs are reproducible.
 *
 * Ownership: the caller owns every device buffer (state and workspace) and
 * keeps it alive while the context uses it; the library owns only the opaque
 * context.  Host pointers are used only for the duration of the call.  The
 * CUDA stream is borrowed: every kernel and copy is enqueued on it.
 *
 * Errors: every call returns an at_status; nothing throws or aborts across
 * the ABI.  at_last_error() returns a message for the calling thread's last
 * failure.  Calls on one context are not thread-safe.
 */
#ifndef AT_GB300_H
#define AT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct at_ctx at_ctx;

typedef enum {
    AT_OK = 0,
    AT_EINVAL = -1,    /* an argument is out of range or inconsistent           */
    AT_ENOMEM = -2,    /* the workspace is smaller than at_workspace_bytes()    */
    AT_ECUDA = -3,     /* a CUDA call failed; at_last_error() has its message   */
    AT_EUNSTABLE = -4, /* a non-finite value appeared in the state              */
    AT_ETIMEOUT = -5,  /* a bounded device wait (persistent, fused path) ran out */
    AT_ESTATE = -6,    /* calls out of order (problem, then delays, then steps) */
    AT_ECORRUPT = -7   /* a canary zone of the workspace was overwritten         */
} at_status;

/* PDEs.  Physics constants prm[] for each (nondimensional, rho0 = T0 = 1,
 * gas constant 1 so p = rho T):
 *   AT_ADVDIFF  u_t + c u_x = a u_xx (Sec. 2.1 Eq. heat with advection)
 *               prm = {c, a}; central stencils of order 2, 4 or 6
 *   AT_RNS      reacting Navier-Stokes, Sec. 4 Eqs. ge / convEq with two
 *               species (fuel -> product), constant mu, Prandtl Pr, Lewis Le
 *               and a one-step Arrhenius rate A rho Y exp(-Ea/T);
 *               state (rho, rho u, rho E, rho Y),
 *               rho E = p/(gamma-1) + rho u^2/2 + q_c rho Y;
 *               prm = {gamma, mu, Pr, Le, A, Ea, q_c}; central order 2/4/6
 *   AT_EULER    reactive Euler (Sec. 5.6), WENO5 / AT-WENO5 fluxes with local
 *               Lax-Friedrichs splitting (Sec. 3, Eqs. Csplit, wender);
 *               prm = {gamma, A, Ea, Q, eps}
 *   AT_ADV_WENO u_t + c u_x = 0 with WENO5 (the order test of Sec. 3);
 *               prm = {c, eps}
 *   AT_BURGERS  u_t + (u^2/2)_x = 0 with WENO5 (the nonlinear order test of
 *               Sec. 3); prm = {0, eps}
 *   AT_RNS_CHAIN the AT_RNS equations with every product derivative
 *               expanded by the chain rule, as in the paper's 1-D solver
 *               (Sec. 4): only rho, u, p, rho E, Y and T are differentiated
 *               (and extrapolated at buffer points).  Not conservative.
 *               Same state and prm as AT_RNS; per-stage path only.        */
enum { AT_ADVDIFF = 0, AT_RNS = 1, AT_EULER = 2, AT_ADV_WENO = 3, AT_BURGERS = 4, AT_RNS_CHAIN = 5 };
/* RK schemes (Sec. 2.3): Heun RK2 (Eq. rk2), Shu-Osher TVD RK3, classic RK4 */
enum { AT_RK2 = 0, AT_RK3TVD = 1, AT_RK4 = 2 };
/* Boundary treatment (Sec. 2.1, 2.2, 3): synchronous; standard scheme on
 * delayed data (AS, Eq. async-fde / Eq. asweno); asynchrony-tolerant (AT,
 * Eq. geDer, Appendix A, Eq. atRecon)                                        */
enum { AT_SYNC = 0, AT_AS = 1, AT_AT = 2 };
/* Delay distributions on {0..k_max}: uniform; table p_0..p_kmax (normalised
 * by its sum); geometric p_k proportional to r (1-r)^k with r = prob[0]      */
enum { AT_UNIFORM = 0, AT_TABLE = 1, AT_GEOMETRIC = 2 };
/* at_read targets */
enum { AT_READ_STATE = 0, AT_READ_DELAYS = 1, AT_READ_RING = 2, AT_READ_STATS = 3 };
/* execution paths (at_set_option(AT_OPT_PATH)): AT_PATH_STAGE launches one
 * kernel per RK stage; AT_PATH_PERSISTENT runs all steps of an at_step call
 * in one cooperative launch with one CTA per PE that synchronises only with
 * its two neighbours (central PDEs, up to as many PEs as the GPU holds at
 * once; advection-diffusion on at most 64 PEs of 32..256 points runs instead
 * in one thread-block cluster of up to 16 CTAs with its ring in distributed
 * shared memory); AT_PATH_FUSED runs all RK stages of a step in one pass
 * over the state, recomputing the edge points of the neighbours beyond each
 * CTA: all steps of the call in one cooperative launch whose CTAs wait only
 * for their neighbour CTAs' previous step when they fit on the GPU at once,
 * else one launch per step (advection-diffusion, PEs of 32, 64, 128 or 256
 * points and at least stages x halo points; the reacting flow in flux form,
 * one launch per step over tiles of up to 8 PEs with recomputed strips of
 * the outer neighbours, PEs of at least stages x halo points; the WENO PDEs
 * in the reconstruction form, one launch per step over the per-stage
 * windows with recomputed strips; AT_EINVAL from at_step otherwise; u^{n+1} goes to workspace field A and back, so an odd
 * number of steps in one call ends with a device copy of the state); AT_PATH_AUTO
 * (default) takes the one-cluster kernel when it can, else for
 * advection-diffusion the fused path when it can, else the persistent path
 * when it can, else the per-stage path (delays by arrival order and
 * AT_OPT_WITHHOLD_PE keep the persistent path).  All paths compute the same
 * values in the same order.                                                */
enum { AT_PATH_AUTO = 0, AT_PATH_STAGE = 1, AT_PATH_PERSISTENT = 2, AT_PATH_FUSED = 3 };
/* at_set_option keys */
enum {
    AT_OPT_PATH = 0,        /* value: AT_PATH_*                                                  */
    AT_OPT_WAIT_LIMIT = 1,  /* polls (~0.2 us each) before a wait of the persistent or the
                               multi-step fused kernel gives up with AT_ETIMEOUT; default
                               4,000,000                                                         */
    AT_OPT_WITHHOLD_PE = 2, /* fault injection: this PE (on the fused path: the CTA holding it)
                               never announces its progress, so its neighbours' waits run out
                               (-1, the default: none)                                           */
    AT_OPT_ARRIVAL = 3,     /* 1: real asynchrony on the persistent path.  Instead of drawing a
                               delay, each PE boundary uses the freshest stage argument of the
                               neighbour that has arrived (never older than k_max, or than the
                               start-up clamp allows: it waits for that), as the CPU PEs of the
                               paper do.  Runs are then not reproducible; at_set_delay_trace
                               records the delays so that a run can be replayed (the oracle
                               does).  0 (default): Philox delays.  AT_EINVAL from at_step if
                               the persistent path cannot be taken.                             */
    AT_OPT_HISTORY = 4,     /* what a buffer point reads at a delayed level m and stage s
                               (Sec. 2.3; value AT_HIST_*).  AT_HIST_STAGE (default): the
                               neighbour's stage argument U^{m,(s)} as the neighbour computed it
                               (the per-step message carries every stage).  AT_HIST_RECOMPUTE:
                               the stage values formed again from the neighbour's u^m, as a
                               synchronous RK step from u^m would form them: after each step a
                               kernel recomputes them on a strip of 2 S H points around every PE
                               boundary and writes them into the history ring.  Takes
                               advection-diffusion and the reacting flow in flux form on the
                               per-stage path (AT_PATH_AUTO picks it); AT_EINVAL from at_step
                               otherwise.  Both readings give the same values bit for bit when
                               every delay is 0.  Set it before at_set_delays, which seeds the
                               ring of level 0 by the chosen reading.                           */
    AT_OPT_OPEN_ENDS = 5,   /* 1: the context owns a range of PEs of a larger domain split over
                               ranks (Sec. 2.1): the buffer points beyond its first and last PE
                               read windows supplied with at_put_ext instead of wrapping around
                               the range.  It then advances one stage at a time (at_stage; at_step
                               returns AT_EINVAL) on the per-stage path, reading B.  0: periodic */
    AT_OPT_PE_BASE = 6,     /* global index of the context's PE 0 in the whole domain (default 0) */
    AT_OPT_PE_TOTAL = 7     /* PEs of the whole domain (0, the default: the context's own P); the
                               delay draws use global PE indices (pe_base + p) mod pe_total, so a
                               range draws exactly the delays the whole domain draws there      */
};
enum { AT_HIST_STAGE = 0, AT_HIST_RECOMPUTE = 1 };

typedef struct {
    int32_t pde;      /* AT_ADVDIFF | AT_RNS | AT_EULER | AT_ADV_WENO | AT_BURGERS | AT_RNS_CHAIN */
    int32_t order;    /* 2 | 4 | 6 for central PDEs; ignored for WENO5                */
    int32_t rk;       /* AT_RK2 | AT_RK3TVD | AT_RK4                                  */
    int32_t pe_size;  /* points per PE, >= 2 x halo width (order/2; 3, or 4 for the
                         WENO interpolation form)                                    */
    int64_t n;        /* grid points, periodic, n % pe_size == 0, n < 2^31            */
    double dx, dt;    /* grid spacing and the fixed time step                         */
    double prm[16];   /* physics constants, see the PDE list above                    */
    int32_t weno;     /* WENO PDEs: AT_WENO_RECONSTRUCT (0) flux reconstruction, Sec. 3
                         Eq. atRecon (the default); AT_WENO_INTERPOLATE (1) edge values
                         of the split fluxes by interpolation, Eqs. interpS, fullSten,
                         omg (ideal weights 1/16, 5/8, 5/16), differenced by the
                         fourth-order staggered formula (9/8, -1/24), halo width 4,
                         per-stage path only (not in batches).  0 for central PDEs.   */
    int32_t reserved; /* 0                                                            */
} at_problem;
enum { AT_WENO_RECONSTRUCT = 0, AT_WENO_INTERPOLATE = 1 };

typedef struct {
    int32_t mode;      /* AT_SYNC | AT_AS | AT_AT                                     */
    int32_t k_max;     /* largest delay in steps, 0..15 (the paper's L - 1)           */
    int32_t dist;      /* AT_UNIFORM | AT_TABLE | AT_GEOMETRIC                        */
    int32_t per_stage; /* 1: one delay per (step, stage); 0: one per step (Sec. 2.3)  */
    double prob[16];   /* AT_TABLE: p_0..p_kmax; AT_GEOMETRIC: prob[0] = r            */
    uint64_t seed;     /* Philox key                                                  */
    uint32_t instance; /* fourth Philox counter word (independent instances)          */
    uint32_t pad_;
} at_delays;

typedef struct {
    int64_t level;     /* steps completed                                             */
    int32_t status;    /* 0, or AT_EUNSTABLE once a non-finite state value appeared   */
    int32_t stages;    /* RK stages per step                                          */
    int32_t nvar;      /* state variables                                             */
    int32_t halo;      /* halo width H                                                */
    int32_t q;         /* temporal extrapolation degree of the AT halo                */
    int32_t ring_levels;
    int32_t path;             /* AT_PATH_STAGE, _PERSISTENT or _FUSED: the last at_step */
    int32_t pad_;
    int64_t kernels_launched; /* kernels enqueued by this context so far             */
    int64_t launches_timed;   /* stage kernels timed since at_profile(ctx, 1)        */
    double stage_ms;          /* summed device time of those launches (CUDA events)  */
} at_stats;

/* Create a context on CUDA device `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out is set on AT_OK. */
int at_create(at_ctx** out, int device, void* cuda_stream);

/* Device workspace bytes the problem needs with the given delay model
 * (stage buffers, RK accumulator, history ring, delay log, status word).
 * Returns 0 for an invalid description. */
size_t at_workspace_bytes(const at_problem* pb, const at_delays* dl);

/* Validate and bind the problem.  state_dev: the caller's [nvar][n] FP64
 * device array that holds u^n (SoA, 16-byte aligned); init: initial state,
 * [nvar][n] FP64, host (init_on_device = 0) or device memory, copied into
 * state_dev on the stream (init may equal state_dev).  workspace_dev /
 * workspace_bytes: caller-owned device memory, 256-byte aligned, of at least
 * at_workspace_bytes(pb, dl) for every delay model used later.  Invalidates
 * any previous delay model (call at_set_delays next). */
int at_set_problem(at_ctx* ctx, const at_problem* pb, double* state_dev, const double* init,
                   int init_on_device, void* workspace_dev, size_t workspace_bytes);

/* Set the delay model, reset the step counter to 0 and seed the history ring
 * with the edge windows of the current state (level 0). */
int at_set_delays(at_ctx* ctx, const at_delays* dl);

/* Enqueue nsteps full RK steps (S stage kernels each) on the stream.  A
 * solve holds at most 2^31 - 2 steps in total (AT_EINVAL beyond). */
int at_step(at_ctx* ctx, int64_t nsteps);

/* at_step, then synchronise the stream and return AT_EUNSTABLE if a
 * non-finite value appeared, AT_ETIMEOUT if a persistent-path wait ran out
 * (the state is then incomplete; the context stays usable after at_set_delays). */
int at_run(at_ctx* ctx, int64_t nsteps);

/* Copy out: AT_READ_STATE the [nvar][n] state; AT_READ_DELAYS the delays of
 * the last completed step, [stages][P][2] uint8 (side 0 = left boundary of
 * the PE); AT_READ_RING the whole history ring [R][S][P][2][H][nvar] FP64;
 * AT_READ_STATS an at_stats (host only).  bytes must be at least the size of
 * the target; the copy is synchronous. */
int at_read(at_ctx* ctx, int what, void* dst, size_t bytes, int dst_on_device);

/* Checkpoint / resume.  The delays are counter-based (Philox of the seed,
 * level, stage, PE and side, Sec. 5), so between two steps a run is fully
 * described by the problem, the delay model, the level n, the state u^n, the
 * history ring (the edge windows of the stage arguments of the levels a
 * delayed buffer point can still read, Sec. 2.3), the delays of the last step
 * and, for a PE range (AT_OPT_OPEN_ENDS), its outside windows.
 * at_checkpoint_bytes gives the size of such a blob (0 without a problem and
 * a delay model); at_save copies it to dst (host or device memory, as
 * dst_on_device says; synchronous), between steps only (AT_ESTATE within a
 * step begun with at_stage); at_restore loads one into a context that has
 * the same problem, delay model and history / PE-range options (AT_EINVAL
 * otherwise, and for a truncated or foreign blob; nothing is changed then),
 * after which the run continues exactly, bit for bit, as the run that saved
 * it, on any path.  The blob's layout is private to the library (a header,
 * then the state, the delay log, the ring and the outside windows). */
size_t at_checkpoint_bytes(const at_ctx* ctx);
int at_save(at_ctx* ctx, void* dst, size_t bytes, int dst_on_device);
int at_restore(at_ctx* ctx, const void* src, size_t bytes, int src_on_device);

/* Canary zones: the workspace holds kGuardBytes = 256 bytes of 0xA5 after
 * each of its slices (stage buffers, RK accumulator, history ring, delay log,
 * status words, progress counters, placement, ring of derived quantities,
 * outside windows), written by at_set_delays.  at_check_guards reads them
 * back (synchronous): AT_OK while every zone is intact, AT_ECORRUPT naming
 * the first overwritten one otherwise, the evidence a kernel or a caller
 * wrote past a slice.  A check for tests and debugging; no kernel reads the
 * zones. */
int at_check_guards(at_ctx* ctx);

/* Options (AT_OPT_*); they apply from the next at_step on. */
int at_set_option(at_ctx* ctx, int key, int64_t value);

/* ---- a PE range of a domain split over ranks (AT_OPT_OPEN_ENDS) ----------
 * The host side of the split exchanges, for every stage, the edge windows of
 * the stage arguments between neighbouring ranks (the per-step message of S
 * stages, Sec. 2.3).  at_stage enqueues the next RK stage of the current
 * step (stage 0 of level n, then 1, ...; after the last one the level is
 * n + 1); at_step may not be mixed into a step begun with at_stage.
 * at_edges copies the range's two outer edge windows of U^{level,(stage)}
 * (the first PE's left window, then the last PE's right window; [2][H][nvar]
 * FP64, host memory, synchronous) once the stage before it has run: they are
 * what the neighbouring ranks' buffer points read.  at_put_ext copies a
 * neighbour's window beyond `side` of the range (0: left of PE 0, that PE's
 * right edge window; 1: right of PE P-1, its left edge window; [H][nvar] FP64
 * in host memory, points in increasing x) for (level, stage) into the
 * context's buffer of outside windows (kept for the ring's levels), to be
 * read by the stages launched afterwards; it synchronises the stream.
 * at_delay returns the delay PE `pe` of the context uses at (level, stage,
 * side): the Philox draw through the start-up clamp, computed on the host
 * (what the kernels draw), so that a rank knows which levels of a window it
 * must have before a stage.  AT_EINVAL for levels outside the ring or a
 * context without open ends where the call needs them. */
int at_stage(at_ctx* ctx);
int at_edges(at_ctx* ctx, int64_t level, int stage, double* out);
int at_put_ext(at_ctx* ctx, int64_t level, int stage, int side, const double* win);
int at_delay(at_ctx* ctx, int64_t level, int stage, int64_t pe, int side);

/* Delay trace: from the current level on, the kernels write the delay of
 * every (step, stage, PE, side) of the next max_steps steps into trace_dev,
 * uint8 [max_steps][stages][P][2] in caller-owned device memory (side 0 =
 * left boundary of the PE); steps beyond max_steps are not recorded.  NULL or
 * max_steps <= 0 detaches it.  The buffer is borrowed until it is detached
 * or the context is destroyed. */
int at_set_delay_trace(at_ctx* ctx, uint8_t* trace_dev, int64_t max_steps);

/* Tracing: with enable = 1, every kernel launch at_step enqueues afterwards is
 * bracketed by two CUDA events on the stream, and at_read(AT_READ_STATS)
 * reports their number and summed device time (it synchronises the stream).
 * enable = 0 stops timing; either call resets the totals.  At most 65,536
 * launches are timed between two reads; later ones run untimed. */
int at_profile(at_ctx* ctx, int enable);

int at_destroy(at_ctx* ctx);

/* ---- batched solves ------------------------------------------------------
 *
 * Many independent solves (instances) of possibly different PDEs, sizes, PE
 * sizes, delay models and step counts advance together.  Each instance owns
 * its state and workspace (caller-owned device memory, sized by
 * at_workspace_bytes for its own problem and delay model); the batch keeps a
 * device table of slots.  One launch per kernel variant advances every bound
 * slot: a persistent grid takes instances largest first from a device queue,
 * and one CTA runs all stages and steps of an instance.  Each instance's
 * result is bit-for-bit the one a context would compute for it alone
 * (instance = its Philox counter word, as for a context).                   */
typedef struct at_batch at_batch;

typedef struct {
    at_problem pb;
    at_delays dl;
    double* state_dev;      /* [nvar][n] FP64 device array; holds the initial state at bind  */
    void* workspace_dev;    /* at_workspace_bytes(&pb, &dl) bytes of device memory, 256-B aligned */
    size_t workspace_bytes;
    int64_t nsteps;         /* steps this instance is to run in total                         */
} at_instance;

typedef struct {
    int64_t level;      /* steps done                                                       */
    int64_t left;       /* steps still to run                                               */
    int32_t status;     /* 0 or AT_EUNSTABLE                                                */
    int32_t bound;      /* 1 while the slot holds an instance                               */
} at_slot_info;

/* Batch modes (at_batch_set_config): AT_BATCH_INSTANCE, a persistent grid
 * where one CTA runs all stages and steps of one instance (best for many
 * small instances); AT_BATCH_FLAT, one launch per stage over the windows of
 * all instances, so a large instance spreads over every SM (replayed from a
 * captured graph of chunk x stages launches).  Same results either way. */
enum { AT_BATCH_INSTANCE = 0, AT_BATCH_FLAT = 1 };

/* device bytes of the slot table for `capacity` slots and, for the flat
 * mode, a window map of `max_windows` windows (the sum over bound instances
 * of n / window length) */
size_t at_batch_table_bytes(int64_t capacity, int64_t max_windows);
/* table_dev: caller-owned device memory of at_batch_table_bytes(capacity,
 * max_windows), 256-B aligned */
int at_batch_create(at_batch** out, int device, void* cuda_stream, int64_t capacity, int64_t max_windows,
                    void* table_dev, size_t table_bytes);
/* Bind an instance to a free slot: validates it, seeds its history ring from
 * its state (level 0) and queues it.  Enqueued on the stream.  AT_ENOMEM when
 * the window map would overflow. */
int at_batch_bind(at_batch* b, int64_t slot, const at_instance* inst);
/* Free a slot (its instance's memory may be reused once the stream has passed). */
int at_batch_release(at_batch* b, int64_t slot);
/* Launch configuration: mode (AT_BATCH_*), threads per CTA (64..256,
 * multiple of 32), resident CTAs per SM in the instance mode (1..16, clamped
 * to what fits), and whether at_batch_step replays a captured CUDA graph (1)
 * or launches directly (0).  Default AT_BATCH_INSTANCE, 256, 3, 1. */
int at_batch_set_config(at_batch* b, int mode, int block, int ctas_per_sm, int use_graph);
/* Every bound slot with steps left advances min(chunk, steps left).  Enqueued. */
int at_batch_step(at_batch* b, int64_t chunk);
/* at_batch_step, then synchronise and return AT_EUNSTABLE if any bound
 * instance produced a non-finite value (at_batch_query tells which). */
int at_batch_run(at_batch* b, int64_t chunk);
/* state of one slot (synchronises the stream) */
int at_batch_query(at_batch* b, int64_t slot, at_slot_info* info);
int at_batch_destroy(at_batch* b);

/* ---- allocation-free entry point (no counterpart in the paper) ----------
 *
 * For callers that must not allocate device memory while they run: a host
 * application that sizes all device memory up front and hands libraries a
 * fixed budget, or code on a path where cudaMalloc is unwelcome (it can
 * synchronise the device and can fail under memory pressure partway through
 * a run).  at_run_noalloc performs one whole solve with no context and no
 * caller workspace: it binds the problem and the delay model, runs nsteps
 * steps on state_dev in place ([nvar][n] FP64, device memory, 16-byte
 * aligned: the initial state on entry, u^nsteps on return), synchronises
 * the stream and checks for non-finite values, exactly like at_set_problem
 * + at_set_delays + at_run on a fresh context.
 *
 * Its workspace (stage buffers, RK accumulator, history ring, delay log,
 * status word) lives in one file-scope device array of
 * AT_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until
 * the process exits.  Problems whose at_workspace_bytes() exceeds it are
 * rejected with AT_ENOMEM before anything is enqueued.  The call ends by
 * synchronising its stream, as at_run does, so it cannot be made inside a
 * stream capture.  The first call on a device looks the array's device
 * address up (cudaGetSymbolAddress).  The address is kept for the
 * life of the process: after cudaDeviceReset on a device the kept address is
 * stale, so do not call at_run_noalloc on that device again in that process.
 * Each call clears the parts of
 * the array that must start at zero; all calls share the one array, so calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller.  Nothing is allocated: no cudaMalloc, no
 * cudaFree, no host heap. */
#define AT_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)
int at_run_noalloc(const at_problem* pb, const at_delays* dl, double* state_dev, int64_t nsteps, int device,
                   void* cuda_stream);

/* message for the calling thread's last failed call ("" if none) */
const char* at_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
