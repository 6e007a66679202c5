// at_abi.cu -- the C ABI of libat_gb300.so (declared in include/at.h).
//
// Host-side only: argument validation, carving the caller's workspace, the
// delay threshold table, the temporal extrapolation weights, and the launch
// sequence of the stage kernels.  Every step of the computation itself runs
// in the kernels of at_stage.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/at.h"
#include "at_device.cuh"

size_t atk_stage_smem_bytes(int pde, int Tw, int H);
int atk_stage_block(int pde, int Tw);
cudaError_t atk_launch_stage(const atk::StageArgs& a, int pde, int order, cudaStream_t st);
cudaError_t atk_launch_ring_seed(const atk::StageArgs& a, cudaStream_t st);
cudaError_t atk_launch_ring_recompute(const atk::StageArgs& a, int pde, int order, int rk, const double* um,
                                      int64_t m, cudaStream_t st);
cudaError_t atk_set_smem_limits();
int64_t atk_persist_capacity(int pde, int order, int B, int device);
int atk_cluster_size(int pde, int order, int B, int64_t P, int R, int S, int device);
cudaError_t atk_launch_cluster(const atk::StageArgs& a, int order, int csize, int64_t level0, int64_t nsteps,
                               cudaStream_t st);
bool atk_fused_supported(int pde, int order, int B, int S);
int atk_fused_multi_w(int order, int rk, int B, int S, int64_t P, int device);
cudaError_t atk_launch_fused_steps(const atk::StageArgs& a, int order, int W, int64_t level0, int64_t nsteps,
                                   double* b0, double* b1, cudaStream_t st);
bool atk_tile_fused_supported(int pde, int order, int B, int rk, int q);
cudaError_t atk_launch_tile_fused(const atk::StageArgs& a, int pde, int order, int64_t n, const double* uin,
                                  double* uout, cudaStream_t st);
cudaError_t atk_launch_fused(const atk::StageArgs& a, int order, int64_t n, const double* uin, double* uout,
                             cudaStream_t st);
cudaError_t atk_launch_persist(const atk::StageArgs& a, int pde, int order, int64_t level0, int64_t nsteps,
                               cudaStream_t st);
int atk_batch_variant(int pde, int order);
cudaError_t atk_launch_batch(int variant, const atk::StageArgs* tab, int64_t* lvl, int64_t* left, const int* order,
                             int n_order, int* queue, int64_t chunk, int grid, int block, size_t smem, cudaStream_t st);
int atk_batch_max_ctas_per_sm(int variant, int block, size_t smem);
cudaError_t atk_launch_batch_stage(int variant, const atk::StageArgs* tab, const int64_t* lvl, const int64_t* left,
                                   const int* win_slot, const int* win_idx, int nwin, int stage, int block,
                                   size_t smem, int win_smem, cudaStream_t st);
cudaError_t atk_launch_batch_advance(int64_t* lvl, int64_t* left, const int* slots, int n, cudaStream_t st);
cudaError_t atk_launch_batch_status(const atk::StageArgs* tab, const int* slots, int n, int* out, cudaStream_t st);

// spare ring levels beyond k_max + q + 1: how far a PE of the persistent
// path may run ahead of a neighbour before it must wait to reuse a slot
static const int kRingSlack = 2;
// Levels stay below 2^31 so that the kernels take ring slots with 32-bit
// arithmetic (a solve of more steps is refused).
static const int64_t kMaxLevel = ((int64_t)1 << 31) - 2;
// the persistent path holds one CTA per PE on the GPU at once; its
// workspace (ring of derived quantities) is laid out for at most this many
static const int64_t kPersistMaxPE = 4096;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(AT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// canary zones: kGuardBytes of kGuardByte after each workspace slice,
// written by at_set_delays and checked by at_check_guards
const int kGuards = 10;
const size_t kGuardBytes = 256;
const unsigned char kGuardByte = 0xA5;

struct Layout {
    int nvar, H, q, S, R;
    int64_t P;
    int Tw, wpp;
    size_t off_A, off_B, off_acc, off_ring, off_dlog, off_status, off_done, off_place, off_gring, off_ext, total;
    size_t ring_elems, gring_elems, ext_elems;
    size_t guard[kGuards];  // a canary zone of kGuardBytes after every slice
    int nguard;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// element of the history ring [R][S][P][2][H][nvar] at (level, stage, PE, side), h = 0, v = 0
size_t host_ring_index(const Layout& L, int64_t level, int stage, int64_t pe, int side)
{
    const int64_t r = level % L.R;
    return ((((size_t)r * L.S + stage) * L.P + pe) * 2 + side) * L.H * L.nvar;
}

int nvar_of(int pde) { return (pde == AT_RNS || pde == AT_EULER || pde == AT_RNS_CHAIN) ? 4 : 1; }
bool is_weno(int pde) { return pde == AT_EULER || pde == AT_ADV_WENO || pde == AT_BURGERS; }
// stencil reach beyond a point: order/2 for central stencils; WENO5 reaches 3
// points, and the interpolation form's edges j +- 3/2 one more
int halo_of(const at_problem* pb)
{
    if (!is_weno(pb->pde)) return pb->order / 2;
    return pb->weno == AT_WENO_INTERPOLATE ? 4 : 3;
}
int stages_of(int rk) { return rk == AT_RK2 ? 2 : (rk == AT_RK3TVD ? 3 : 4); }

// window length: the largest divisor of the PE size in [2H, 256]; a PE size
// without one (a large prime, say) is one window when it is at most 1024.
// Returns 0 when neither holds.
int window_of(int B, int H)
{
    int best = 0;
    for (int t = 2 * H; t <= 256 && t <= B; ++t)
        if (B % t == 0) best = t;
    if (best == 0 && B <= 1024) best = B;
    return best;
}

int check_problem(const at_problem* pb)
{
    if (!pb) return fail(AT_EINVAL, "problem is NULL");
    if (pb->pde < 0 || pb->pde > 5) return fail(AT_EINVAL, "unknown pde %d", pb->pde);
    if (pb->rk < 0 || pb->rk > 2) return fail(AT_EINVAL, "unknown rk %d", pb->rk);
    if (!is_weno(pb->pde) && pb->order != 2 && pb->order != 4 && pb->order != 6)
        return fail(AT_EINVAL, "central order must be 2, 4 or 6 (got %d)", pb->order);
    if (pb->n <= 0 || pb->n >= ((int64_t)1 << 31)) return fail(AT_EINVAL, "n out of range");
    if (pb->pe_size <= 0 || pb->n % pb->pe_size) return fail(AT_EINVAL, "n must be a multiple of pe_size");
    if (pb->weno != AT_WENO_RECONSTRUCT && pb->weno != AT_WENO_INTERPOLATE)
        return fail(AT_EINVAL, "unknown weno form %d", pb->weno);
    if (pb->weno == AT_WENO_INTERPOLATE && !is_weno(pb->pde))
        return fail(AT_EINVAL, "the WENO interpolation form needs a WENO PDE");
    const int H = halo_of(pb);
    if (pb->pe_size < 2 * H) return fail(AT_EINVAL, "pe_size must be at least %d", 2 * H);
    if (window_of(pb->pe_size, H) == 0)
        return fail(AT_EINVAL, "pe_size above 1024 needs a divisor between %d and 256", 2 * H);
    if (!(pb->dx > 0.0) || !(pb->dt > 0.0)) return fail(AT_EINVAL, "dx and dt must be positive");
    return AT_OK;
}

int check_delays(const at_delays* dl)
{
    if (!dl) return fail(AT_EINVAL, "delays is NULL");
    if (dl->mode < 0 || dl->mode > 2) return fail(AT_EINVAL, "unknown mode %d", dl->mode);
    if (dl->k_max < 0 || dl->k_max > AT_KMAX_LIMIT) return fail(AT_EINVAL, "k_max must be 0..15");
    if (dl->dist < 0 || dl->dist > 2) return fail(AT_EINVAL, "unknown dist %d", dl->dist);
    if (dl->dist == AT_TABLE) {
        double s = 0.0;
        for (int i = 0; i <= dl->k_max; ++i) {
            if (!(dl->prob[i] >= 0.0)) return fail(AT_EINVAL, "negative probability");
            s += dl->prob[i];
        }
        if (!(s > 0.0)) return fail(AT_EINVAL, "probabilities sum to zero");
    }
    if (dl->dist == AT_GEOMETRIC && !(dl->prob[0] > 0.0 && dl->prob[0] <= 1.0))
        return fail(AT_EINVAL, "geometric parameter must be in (0, 1]");
    return AT_OK;
}



Layout layout(const at_problem* pb, const at_delays* dl)
{
    Layout L{};
    L.nvar = nvar_of(pb->pde);
    L.H = halo_of(pb);
    L.q = is_weno(pb->pde) ? 1 : pb->order / 2;
    L.S = stages_of(pb->rk);
    L.R = dl->k_max + L.q + 1 + kRingSlack;
    L.P = pb->n / pb->pe_size;
    L.Tw = window_of(pb->pe_size, L.H);
    L.wpp = pb->pe_size / L.Tw;
    const size_t field = sizeof(double) * (size_t)L.nvar * pb->n;
    size_t off = 0;
    L.nguard = 0;
    // a slice of `bytes` at the current offset, then its canary zone
    auto slice = [&](size_t bytes) -> size_t {
        const size_t at = off;
        off = align256(off + bytes);
        L.guard[L.nguard++] = off;
        off += kGuardBytes;
        return at;
    };
    L.off_A = slice(field);
    L.off_B = slice(field);
    L.off_acc = slice(pb->rk != AT_RK3TVD ? field : 0);
    L.ring_elems = (size_t)L.R * L.S * L.P * 2 * L.H * L.nvar;
    L.off_ring = slice(sizeof(double) * L.ring_elems);
    L.off_dlog = slice((size_t)L.S * L.P * 2);
    L.off_status = slice(256);  // status word, the abort flag and the placement count of the persistent path
    L.off_done = slice(sizeof(int64_t) * (size_t)L.P);  // per-PE progress counters of the persistent path
    // the persistent path's SM of every CTA (PE placement)
    L.off_place = slice(L.P <= kPersistMaxPE ? sizeof(int) * (size_t)L.P : 0);
    // the persistent path's ring of derived quantities of the edge windows
    // (central PDEs with few enough PEs to take that path)
    L.gring_elems = 0;
    if ((pb->pde == AT_ADVDIFF || pb->pde == AT_RNS) && L.P <= kPersistMaxPE)
        L.gring_elems = (size_t)L.R * L.S * L.P * 2 * L.H * (pb->pde == AT_RNS ? 8 : 1);
    L.off_gring = slice(sizeof(double) * L.gring_elems);
    // windows beyond the ends of a PE range (open ends): [R][S][2][H][nvar]
    L.ext_elems = (size_t)L.R * L.S * 2 * L.H * L.nvar;
    L.off_ext = slice(sizeof(double) * L.ext_elems);
    L.total = off;
    return L;
}

// thresholds: T_i = floor(2^32 CDF(i)), CDF accumulated in index order
void thresholds(const at_delays* dl, uint64_t* thr)
{
    double w[AT_KMAX_LIMIT + 1];
    for (int i = 0; i <= dl->k_max; ++i) {
        if (dl->dist == AT_UNIFORM) {
            w[i] = 1.0;
        } else if (dl->dist == AT_TABLE) {
            w[i] = dl->prob[i];
        } else {
            double t = dl->prob[0];
            for (int j = 0; j < i; ++j) t *= (1.0 - dl->prob[0]);
            w[i] = t;
        }
    }
    double total = 0.0;
    for (int i = 0; i <= dl->k_max; ++i) total += w[i];
    double cum = 0.0;
    for (int i = 0; i < dl->k_max; ++i) {
        cum += w[i];
        double t = std::floor((cum / total) * 4294967296.0);
        if (t < 0.0) t = 0.0;
        if (t > 4294967296.0) t = 4294967296.0;
        thr[i] = (uint64_t)t;
    }
}

// extrapolation weights from levels -k..-k-q to 0 (exact integer ratios)
void extrap_weights(int q, int k, double* w)
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

// The argument block of every kernel of one solve: layout of its workspace,
// delay thresholds, extrapolation weights, pre-scaled stencil coefficients.
atk::StageArgs build_args(const at_problem* pb, const at_delays* dl, const Layout& L, unsigned char* ws, double* state)
{
    atk::StageArgs a{};
    a.acc = (double*)(ws + L.off_acc);
    a.ring = (double*)(ws + L.off_ring);
    a.dlog = (uint8_t*)(ws + L.off_dlog);
    a.status = (int*)(ws + L.off_status);
    a.abort_flag = (int*)(ws + L.off_status + sizeof(int));
    a.place_count = (int*)(ws + L.off_status + 2 * sizeof(int));
    a.done = (int64_t*)(ws + L.off_done);
    a.place = L.P <= kPersistMaxPE ? (int*)(ws + L.off_place) : nullptr;
    a.gring = L.gring_elems ? (double*)(ws + L.off_gring) : nullptr;
    a.wait_limit = (int64_t)4000000;
    a.withhold_pe = (int64_t)-1;
    a.slack = kRingSlack;
    a.N = pb->n;
    a.P = L.P;
    a.B = pb->pe_size;
    a.Tw = L.Tw;
    a.wpp = L.wpp;
    a.S = L.S;
    a.R = L.R;
    a.H = L.H;
    a.q = L.q;
    a.nvar = L.nvar;
    a.mode = dl->mode;
    a.kmax = dl->k_max;
    a.per_stage = dl->per_stage ? 1 : 0;
    a.rk = pb->rk;
    a.instance = dl->instance;
    a.key0 = (uint32_t)(dl->seed & 0xffffffffu);
    a.key1 = (uint32_t)(dl->seed >> 32);
    a.dt = pb->dt;
    a.hdt = 0.5 * pb->dt;
    a.dt6 = pb->dt * (1.0 / 6.0);
    thresholds(dl, a.thr);
    for (int k = 0; k <= dl->k_max; ++k) {
        extrap_weights(L.q, k, a.w[k]);
        a.wnz[k] = 1;  // AS and SYNC read the delayed level only
        if (dl->mode == AT_AT) {
            a.wnz[k] = 0;
            for (int l = 0; l <= L.q; ++l)
                if (a.w[k][l] != 0.0) a.wnz[k] |= (uint8_t)(1u << l);
        }
    }
    for (int i = 0; i < 16; ++i) a.prm[i] = pb->prm[i];
    const double dx = pb->dx;
    if (!is_weno(pb->pde)) {
        static const double d1_2[3] = {-1, 0, 1}, d2_2[3] = {1, -2, 1};
        static const double d1_4[5] = {1, -8, 0, 8, -1}, d2_4[5] = {-1, 16, -30, 16, -1};
        static const double d1_6[7] = {-1, 9, -45, 0, 45, -9, 1}, d2_6[7] = {2, -27, 270, -490, 270, -27, 2};
        const double* d1 = pb->order == 2 ? d1_2 : (pb->order == 4 ? d1_4 : d1_6);
        const double* d2 = pb->order == 2 ? d2_2 : (pb->order == 4 ? d2_4 : d2_6);
        const double den1 = pb->order == 2 ? 2.0 : (pb->order == 4 ? 12.0 : 60.0);
        const double den2 = pb->order == 2 ? 1.0 : (pb->order == 4 ? 12.0 : 180.0);
        for (int o = 0; o <= 2 * L.H; ++o) {
            a.c1[o] = -d1[o] / (den1 * dx);
            a.c2[o] = d2[o] / (den2 * dx * dx);
        }
        if (pb->pde == AT_ADVDIFF) {
            const double cc = pb->prm[0], aa = pb->prm[1];
            for (int o = 0; o <= 2 * L.H; ++o)
                a.cm[o] = -cc * d1[o] / (den1 * dx) + aa * d2[o] / (den2 * dx * dx);
        } else {
            const double gam = pb->prm[0], mu = pb->prm[1], Pr = pb->prm[2], Le = pb->prm[3];
            const double cp = gam / (gam - 1.0);
            const double lam = mu * cp / Pr;
            a.k0 = 4.0 / 3.0 * mu;
            a.k1 = 2.0 / 3.0 * mu;
            a.k2 = lam;
            a.k3 = lam / (cp * Le);
            // the diffusion rows carry u, the energy term over lambda and Y; the
            // constants go into the taps (without viscosity every row term is 0)
            const bool visc = a.k2 != 0.0;
            for (int o = 0; o <= 2 * L.H; ++o) {
                a.c2v[0][o] = a.c2[o] * a.k0;
                a.c2v[1][o] = visc ? a.c2[o] * a.k2 : 0.0;
                a.c2v[2][o] = a.c2[o] * a.k3;
            }
            a.kd1 = visc ? a.k1 / a.k2 : 0.0;
            a.kd3 = visc ? pb->prm[6] * a.k3 / a.k2 : 0.0;
        }
    } else {
        a.k0 = 1.0 / dx;
        a.weno_interp = pb->weno == AT_WENO_INTERPOLATE ? 1 : 0;
    }
    a.ext = (double*)(ws + L.off_ext);
    a.bufA = (double*)(ws + L.off_A);
    a.bufB = (double*)(ws + L.off_B);
    a.state = state;
    a.u = state;
    return a;
}

} // namespace

namespace {
// An NVTX range over a scope: the library's calls, steps and persistent
// launches appear on the Nsight Systems timeline (a no-op without a tool).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

struct at_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool have_problem = false, have_delays = false;
    at_problem pb{};
    at_delays dl{};
    double* state = nullptr;
    unsigned char* ws = nullptr;
    size_t ws_bytes = 0;
    Layout L{};
    atk::StageArgs base{};
    int64_t level = 0;
    int64_t launched = 0;
    int path = AT_PATH_AUTO;       // at_set_option(AT_OPT_PATH)
    int last_path = 0;             // path of the last at_step
    int64_t persist_cap = 0;       // PEs one cooperative launch can hold (0: unavailable)
    int cluster_c = 0;             // CTAs of the one-cluster kernel for this problem (0: not used)
    int fused_multi_w = 0;         // PEs per CTA when the fused path's steps fit one cooperative launch
    int64_t wait_limit = 4000000;  // polls of a bounded wait
    int64_t withhold_pe = -1;
    int arrival = 0;               // at_set_option(AT_OPT_ARRIVAL)
    int hist = AT_HIST_STAGE;      // at_set_option(AT_OPT_HISTORY)
    int open_ends = 0;             // at_set_option(AT_OPT_OPEN_ENDS): a PE range of a split domain
    int64_t pe_base = 0, pe_total = 0;  // AT_OPT_PE_BASE, AT_OPT_PE_TOTAL
    int stage_pos = 0;             // at_stage: the next stage of the current level
    int64_t hist_level = -1;       // reading A: the level whose recomputed stage values the ring holds
    uint8_t* trace = nullptr;      // at_set_delay_trace: caller-owned device buffer
    int64_t trace_n0 = 0, trace_steps = 0;
    // tracing (at_profile)
    bool profile = false;
    std::vector<cudaEvent_t> ev;  // pairs: ev[2i] before, ev[2i+1] after launch i
    size_t ev_used = 0;
    int64_t timed = 0;
    double timed_ms = 0.0;
};

namespace {
const size_t kMaxTimed = 65536;

cudaError_t record(at_ctx* c, bool before)
{
    if (!c->profile) return cudaSuccess;
    if (before && c->ev_used / 2 >= kMaxTimed) return cudaSuccess;
    if (!before && (c->ev_used % 2) == 0) return cudaSuccess;  // the launch was not timed
    if (c->ev_used == c->ev.size()) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        c->ev.push_back(e);
    }
    return cudaEventRecord(c->ev[c->ev_used++], c->stream);
}

cudaError_t harvest(at_ctx* c)
{
    if (c->ev_used < 2) {
        c->ev_used = 0;
        return cudaSuccess;
    }
    cudaError_t e = cudaEventSynchronize(c->ev[c->ev_used - 1]);
    if (e != cudaSuccess) return e;
    for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]);
        if (e != cudaSuccess) return e;
        c->timed_ms += ms;
        ++c->timed;
    }
    c->ev_used = 0;
    return cudaSuccess;
}
} // namespace

extern "C" {

const char* at_last_error(void) { return g_err; }

int at_create(at_ctx** out, int device, void* cuda_stream)
{
    if (!out) return fail(AT_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(AT_EINVAL, "device %d out of range (%d devices)", device, ndev);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    e = atk_set_smem_limits();
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    at_ctx* c = new (std::nothrow) at_ctx;
    if (!c) return fail(AT_ENOMEM, "host allocation failed");
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    *out = c;
    g_err[0] = 0;
    return AT_OK;
}

size_t at_workspace_bytes(const at_problem* pb, const at_delays* dl)
{
    if (check_problem(pb) != AT_OK || check_delays(dl) != AT_OK) return 0;
    return layout(pb, dl).total;
}

int at_set_problem(at_ctx* c, const at_problem* pb, double* state_dev, const double* init, int init_on_device,
                   void* workspace_dev, size_t workspace_bytes)
{
    if (!c) return fail(AT_EINVAL, "context is NULL");
    int st = check_problem(pb);
    if (st != AT_OK) return st;
    if (!state_dev || !workspace_dev) return fail(AT_EINVAL, "state and workspace must be device pointers");
    if (((uintptr_t)state_dev & 15) || ((uintptr_t)workspace_dev & 255))
        return fail(AT_EINVAL, "state must be 16-byte and workspace 256-byte aligned");
    at_delays probe{};
    probe.mode = AT_SYNC;
    probe.k_max = 0;
    if (workspace_bytes < layout(pb, &probe).total)
        return fail(AT_ENOMEM, "workspace of %zu bytes is below the %zu bytes needed", workspace_bytes,
                    layout(pb, &probe).total);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    c->pb = *pb;
    c->state = state_dev;
    c->ws = (unsigned char*)workspace_dev;
    c->ws_bytes = workspace_bytes;
    c->have_problem = true;
    c->have_delays = false;
    const size_t bytes = sizeof(double) * (size_t)nvar_of(pb->pde) * pb->n;
    if (init && init != state_dev) {
        e = cudaMemcpyAsync(state_dev, init, bytes, init_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "copy of the initial state");
        if (!init_on_device) {
            e = cudaStreamSynchronize(c->stream);  // the host buffer is borrowed for this call only
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        }
    }
    g_err[0] = 0;
    return AT_OK;
}

int at_set_delays(at_ctx* c, const at_delays* dl)
{
    NvtxRange nvtx_range("at_set_delays");
    if (!c) return fail(AT_EINVAL, "context is NULL");
    if (!c->have_problem) return fail(AT_ESTATE, "at_set_problem must come first");
    int st = check_delays(dl);
    if (st != AT_OK) return st;
    Layout L = layout(&c->pb, dl);
    if (L.total > c->ws_bytes)
        return fail(AT_ENOMEM, "workspace of %zu bytes is below the %zu bytes this delay model needs", c->ws_bytes,
                    L.total);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    c->dl = *dl;
    c->L = L;
    c->base = build_args(&c->pb, dl, L, c->ws, c->state);
    c->base.wait_limit = c->wait_limit;
    c->base.withhold_pe = c->withhold_pe;
    atk::StageArgs& a = c->base;
    // reset the run: zero ring, delay log and status, then seed level 0
    e = cudaMemsetAsync(a.ring, 0, sizeof(double) * L.ring_elems, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.dlog, 0, (size_t)L.S * L.P * 2, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.status, 0, 2 * sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.ext, 0, sizeof(double) * L.ext_elems, c->stream);
    for (int g = 0; g < L.nguard && e == cudaSuccess; ++g)
        e = cudaMemsetAsync(c->ws + L.guard[g], kGuardByte, kGuardBytes, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "workspace reset");
    c->stage_pos = 0;
    atk::StageArgs s = a;
    s.u = c->state;
    e = atk_launch_ring_seed(s, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ring seed launch");
    c->level = 0;
    c->hist_level = -1;  // reading A recomputes level 0 at the first at_step
    c->persist_cap = (c->pb.pde == AT_ADVDIFF || c->pb.pde == AT_RNS)
                         ? atk_persist_capacity(c->pb.pde, c->pb.order, c->pb.pe_size, c->device)
                         : 0;
    if (c->persist_cap > kPersistMaxPE) c->persist_cap = kPersistMaxPE;
    c->cluster_c = c->pb.pde == AT_ADVDIFF
                       ? atk_cluster_size(c->pb.pde, c->pb.order, c->pb.pe_size, L.P, L.R, L.S, c->device)
                       : 0;
    c->fused_multi_w = atk_fused_supported(c->pb.pde, c->pb.order, c->pb.pe_size, L.S)
                           ? atk_fused_multi_w(c->pb.order, c->pb.rk, c->pb.pe_size, L.S, L.P, c->device)
                           : 0;
    cudaGetLastError();  // an unavailable persistent path is not an error
    c->have_delays = true;
    g_err[0] = 0;
    return AT_OK;
}

int at_step(at_ctx* c, int64_t nsteps)
{
    NvtxRange nvtx_range("at_step");
    if (!c) return fail(AT_EINVAL, "context is NULL");
    if (!c->have_problem || !c->have_delays) return fail(AT_ESTATE, "at_set_problem and at_set_delays must come first");
    if (nsteps < 0) return fail(AT_EINVAL, "nsteps must be >= 0");
    if (nsteps > kMaxLevel - c->level)
        return fail(AT_EINVAL, "a solve is limited to %lld steps (level %lld, %lld more asked)", (long long)kMaxLevel,
                    (long long)c->level, (long long)nsteps);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const Layout& L = c->L;
    double* A = (double*)(c->ws + L.off_A);
    double* Bf = (double*)(c->ws + L.off_B);
    double* u = c->state;
    if (c->open_ends) return fail(AT_EINVAL, "a PE range with open ends advances with at_stage");
    if (c->stage_pos != 0) return fail(AT_ESTATE, "a step begun with at_stage is not finished");
    c->base.pe_base = c->pe_base;
    c->base.pe_total = c->pe_total;
    const bool recompute = c->hist == AT_HIST_RECOMPUTE;
    if (recompute) {
        if (c->pb.pde != AT_ADVDIFF && c->pb.pde != AT_RNS)
            return fail(AT_EINVAL, "AT_HIST_RECOMPUTE takes advection-diffusion and the reacting flow in flux form");
        if (c->path == AT_PATH_PERSISTENT || c->path == AT_PATH_FUSED)
            return fail(AT_EINVAL, "AT_HIST_RECOMPUTE runs on the per-stage path");
        if (c->arrival) return fail(AT_EINVAL, "AT_HIST_RECOMPUTE uses drawn delays, not delays by arrival");
    }
    const bool can_persist = !recompute && c->persist_cap > 0 && L.P <= c->persist_cap;
    if (c->path == AT_PATH_PERSISTENT && !can_persist)
        return fail(AT_EINVAL, "the persistent path needs a central PDE and at most %lld PEs (have %lld)",
                    (long long)c->persist_cap, (long long)L.P);
    const bool fused_ok = !recompute && atk_fused_supported(c->pb.pde, c->pb.order, c->pb.pe_size, L.S);
    // the reacting flow and the WENO PDEs: the tile-fused kernels, on request
    // only (AT_PATH_FUSED); a WENO tile is one window plus strips of S H
    // points, which must stay inside the window's PE or its neighbour
    const bool tile_ok = !recompute && !fused_ok && c->pb.weno != AT_WENO_INTERPOLATE &&
                         atk_tile_fused_supported(c->pb.pde, c->pb.order, c->pb.pe_size, c->pb.rk, L.q) &&
                         (!is_weno(c->pb.pde) || L.wpp == 1 || L.Tw >= L.S * L.H);
    const bool cluster_ok = c->cluster_c > 0 && !c->arrival && c->withhold_pe < 0;
    bool persist = c->path == AT_PATH_PERSISTENT || (c->path == AT_PATH_AUTO && can_persist);
    // advection-diffusion beyond one thread-block cluster: the step-fused
    // kernel is faster than the neighbour-wait kernel (measured on GB300 at
    // 256 PEs of 64 points: 10.3 against 13.1 us per step); delays by arrival
    // and withheld progress need the neighbour waits
    if (c->path == AT_PATH_AUTO && persist && !cluster_ok && fused_ok && !c->arrival && c->withhold_pe < 0)
        persist = false;
    if (c->arrival && !persist)
        return fail(AT_EINVAL, "delays by arrival need the persistent path (a central PDE and at most %lld PEs)",
                    (long long)c->persist_cap);
    if (c->path == AT_PATH_FUSED || (c->path == AT_PATH_AUTO && !persist && !c->arrival && fused_ok)) {
        if (!fused_ok && !tile_ok)
            return fail(AT_EINVAL, "the fused path takes advection-diffusion with PEs of 32, 64, 128 or 256 points, "
                                   "the reacting flow in flux form or a WENO PDE in the reconstruction form, with at "
                                   "least stages x halo points per PE");
        if (c->arrival) return fail(AT_EINVAL, "delays by arrival need the persistent path");
        c->last_path = AT_PATH_FUSED;
        c->base.trace = c->trace;
        c->base.trace_n0 = c->trace_n0;
        c->base.trace_steps = c->trace_steps;
        // u^n and u^{n+1} alternate between the state and workspace field A;
        // after an odd number of steps the result is copied back
        const double* cur = u;
        double* nxt = A;
        if (c->fused_multi_w > 0 && nsteps > 0) {
            // every CTA resident: all steps in one cooperative launch
            atk::StageArgs a = c->base;
            a.level = c->level;
            a.wait_limit = c->wait_limit;
            a.withhold_pe = c->withhold_pe;
            e = record(c, true);
            if (e == cudaSuccess)
                e = atk_launch_fused_steps(a, c->pb.order, c->fused_multi_w, c->level, nsteps, u, A, c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "fused multi-step kernel launch");
            e = record(c, false);
            if (e != cudaSuccess) return cuda_fail(e, "profiling event");
            c->launched += 2;  // counter reset + the kernel
            c->level += nsteps;
            if (nsteps & 1) cur = A;  // the result's buffer
            nsteps = 0;               // nothing left for the per-step launches
        }
        for (int64_t i = 0; i < nsteps; ++i) {
            NvtxRange step_range("step (fused path)");
            atk::StageArgs a = c->base;
            a.level = c->level;
            e = record(c, true);
            if (e == cudaSuccess)
                e = fused_ok ? atk_launch_fused(a, c->pb.order, c->level, cur, nxt, c->stream)
                             : atk_launch_tile_fused(a, c->pb.pde, c->pb.order, c->level, cur, nxt, c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "fused step kernel launch");
            e = record(c, false);
            if (e != cudaSuccess) return cuda_fail(e, "profiling event");
            ++c->launched;
            ++c->level;
            double* t = (double*)cur;
            cur = nxt;
            nxt = t;
        }
        if (cur != u) {
            e = cudaMemcpyAsync(u, cur, sizeof(double) * (size_t)L.nvar * c->pb.n, cudaMemcpyDeviceToDevice,
                                c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "copy of the state after the fused steps");
        }
        g_err[0] = 0;
        return AT_OK;
    }
    c->last_path = persist ? AT_PATH_PERSISTENT : AT_PATH_STAGE;
    c->base.trace = c->trace;
    c->base.trace_n0 = c->trace_n0;
    c->base.trace_steps = c->trace_steps;
    if (persist) {
        if (nsteps == 0) return AT_OK;
        atk::StageArgs a = c->base;
        a.u = u;
        a.Y = u;
        a.wait_limit = c->wait_limit;
        a.withhold_pe = c->withhold_pe;
        a.arrival = c->arrival;
        // a small advection-diffusion problem runs in one thread-block cluster
        // (Philox delays only; fault injection needs the neighbour waits)
        const bool cluster = cluster_ok;
        e = record(c, true);
        if (e == cudaSuccess)
            e = cluster ? atk_launch_cluster(a, c->pb.order, c->cluster_c, c->level, nsteps, c->stream)
                        : atk_launch_persist(a, c->pb.pde, c->pb.order, c->level, nsteps, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "persistent kernel launch");
        e = record(c, false);
        if (e != cudaSuccess) return cuda_fail(e, "profiling event");
        c->launched += cluster ? 1 : 2;  // (counter reset +) the kernel
        c->level += nsteps;
        g_err[0] = 0;
        return AT_OK;
    }
    // reading A: the stage values of the current level, recomputed from its
    // u, must be in the ring before its first stage (once per at_set_delays,
    // then kept up to date after every step below)
    auto recompute_level = [&](int64_t m) -> cudaError_t {
        atk::StageArgs a = c->base;
        a.level = m;
        cudaError_t er = record(c, true);
        if (er == cudaSuccess)
            er = atk_launch_ring_recompute(a, c->pb.pde, c->pb.order, c->pb.rk, u, m, c->stream);
        if (er == cudaSuccess) er = record(c, false);
        ++c->launched;
        c->hist_level = m;
        return er;
    };
    if (recompute && nsteps > 0 && c->hist_level != c->level) {
        e = recompute_level(c->level);
        if (e != cudaSuccess) return cuda_fail(e, "stage-history recompute launch");
    }
    for (int64_t i = 0; i < nsteps; ++i) {
        NvtxRange step_range("step (per-stage path)");
        atk::StageArgs a = c->base;
        a.level = c->level;
        a.u = u;
        a.hist_recompute = recompute ? 1 : 0;
        for (int s = 0; s < L.S; ++s) {
            a.stage = s;
            // stencil source and output of each stage (ping-pong A/B, last stage in place)
            const double* X = (s == 0) ? u : ((s % 2 == 1) ? A : Bf);
            double* Y = (s == L.S - 1) ? u : ((s % 2 == 0) ? A : Bf);
            a.X = X;
            a.Y = Y;
            e = record(c, true);
            if (e == cudaSuccess) e = atk_launch_stage(a, c->pb.pde, c->pb.order, c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "stage kernel launch");
            e = record(c, false);
            if (e != cudaSuccess) return cuda_fail(e, "profiling event");
            ++c->launched;
        }
        ++c->level;
        if (recompute) {
            e = recompute_level(c->level);
            if (e != cudaSuccess) return cuda_fail(e, "stage-history recompute launch");
        }
    }
    g_err[0] = 0;
    return AT_OK;
}

int at_run(at_ctx* c, int64_t nsteps)
{
    int st = at_step(c, nsteps);
    if (st != AT_OK) return st;
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, c->base.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "at_run synchronisation");
    if (status & 2) return fail(AT_ETIMEOUT, "a bounded wait of the persistent kernel ran out");
    if (status) return fail(AT_EUNSTABLE, "a non-finite value appeared in the state");
    return AT_OK;
}

int at_read(at_ctx* c, int what, void* dst, size_t bytes, int dst_on_device)
{
    if (!c || !dst) return fail(AT_EINVAL, "context or destination is NULL");
    if (!c->have_problem) return fail(AT_ESTATE, "no problem is set");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    size_t need = 0;
    const void* src = nullptr;
    if (what == AT_READ_STATE) {
        need = sizeof(double) * (size_t)nvar_of(c->pb.pde) * c->pb.n;
        src = c->state;
    } else if (what == AT_READ_DELAYS || what == AT_READ_RING) {
        if (!c->have_delays) return fail(AT_ESTATE, "no delay model is set");
        if (what == AT_READ_DELAYS) {
            need = (size_t)c->L.S * c->L.P * 2;
            src = c->base.dlog;
        } else {
            need = sizeof(double) * c->L.ring_elems;
            src = c->base.ring;
        }
    } else if (what == AT_READ_STATS) {
        if (dst_on_device) return fail(AT_EINVAL, "stats are read to host memory");
        if (bytes < sizeof(at_stats)) return fail(AT_EINVAL, "destination too small");
        at_stats s{};
        int status = 0;
        if (c->have_delays) {
            e = cudaMemcpyAsync(&status, c->base.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "status read");
        }
        s.level = c->level;
        s.status = (status & 2) ? AT_ETIMEOUT : (status ? AT_EUNSTABLE : 0);
        s.path = c->last_path;
        s.stages = stages_of(c->pb.rk);
        s.nvar = nvar_of(c->pb.pde);
        s.halo = halo_of(&c->pb);
        s.q = is_weno(c->pb.pde) ? 1 : c->pb.order / 2;
        s.ring_levels = c->have_delays ? c->L.R : 0;
        s.kernels_launched = c->launched;
        e = harvest(c);
        if (e != cudaSuccess) return cuda_fail(e, "profiling events");
        s.launches_timed = c->timed;
        s.stage_ms = c->timed_ms;
        std::memcpy(dst, &s, sizeof s);
        return AT_OK;
    } else {
        return fail(AT_EINVAL, "unknown read target %d", what);
    }
    if (bytes < need) return fail(AT_EINVAL, "destination of %zu bytes is below the %zu bytes needed", bytes, need);
    e = cudaMemcpyAsync(dst, src, need, kind, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "at_read copy");
    return AT_OK;
}

int at_check_guards(at_ctx* c)
{
    if (!c) return fail(AT_EINVAL, "context is NULL");
    if (!c->have_problem || !c->have_delays) return fail(AT_ESTATE, "at_set_problem and at_set_delays must come first");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    static const char* const names[kGuards] = {"stage buffer A", "stage buffer B", "RK accumulator", "history ring",
                                               "delay log", "status words", "progress counters", "PE placement",
                                               "ring of derived quantities", "outside windows"};
    const Layout& L = c->L;
    std::vector<unsigned char> buf(kGuardBytes * (size_t)L.nguard);
    for (int g = 0; g < L.nguard && e == cudaSuccess; ++g)
        e = cudaMemcpyAsync(buf.data() + kGuardBytes * g, c->ws + L.guard[g], kGuardBytes, cudaMemcpyDeviceToHost,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "canary read");
    for (int g = 0; g < L.nguard; ++g)
        for (size_t b = 0; b < kGuardBytes; ++b)
            if (buf[kGuardBytes * g + b] != kGuardByte)
                return fail(AT_ECORRUPT, "the canary zone after the %s was overwritten (byte %zu of %zu)", names[g], b,
                            kGuardBytes);
    return AT_OK;
}

// ---------------------------------------------------------------------------
// checkpoint / resume.  The delays are counter-based (Philox of seed, level,
// stage, PE, side), so a run is determined by the problem, the delay model
// and, at a step boundary, the state, the history ring, the outside windows
// of a PE range and the level: a blob of those resumes bit for bit.
// ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];  // "AT-CKPT1"
    int64_t level, hist_level;
    at_problem pb;
    at_delays dl;
    int32_t hist, open_ends;
    int64_t pe_base, pe_total;
    int64_t state_bytes, dlog_bytes, ring_bytes, ext_bytes;
};
const char kCkptMagic[8] = {'A', 'T', '-', 'C', 'K', 'P', 'T', '1'};

bool same_problem(const at_problem& a, const at_problem& b)
{
    return a.pde == b.pde && a.order == b.order && a.rk == b.rk && a.pe_size == b.pe_size && a.n == b.n &&
           std::memcmp(&a.dx, &b.dx, sizeof(double)) == 0 && std::memcmp(&a.dt, &b.dt, sizeof(double)) == 0 &&
           std::memcmp(a.prm, b.prm, sizeof a.prm) == 0 && a.weno == b.weno;
}

bool same_delays(const at_delays& a, const at_delays& b)
{
    return a.mode == b.mode && a.k_max == b.k_max && a.dist == b.dist && a.per_stage == b.per_stage &&
           std::memcmp(a.prob, b.prob, sizeof a.prob) == 0 && a.seed == b.seed && a.instance == b.instance;
}

void ckpt_sizes(const at_ctx* c, CkptHeader& h)
{
    h.state_bytes = (int64_t)(sizeof(double) * (size_t)nvar_of(c->pb.pde) * c->pb.n);
    h.dlog_bytes = (int64_t)((size_t)c->L.S * c->L.P * 2);
    h.ring_bytes = (int64_t)(sizeof(double) * c->L.ring_elems);
    h.ext_bytes = (int64_t)(sizeof(double) * c->L.ext_elems);
}
}  // namespace

size_t at_checkpoint_bytes(const at_ctx* c)
{
    if (!c || !c->have_problem || !c->have_delays) return 0;
    CkptHeader h{};
    ckpt_sizes(c, h);
    return sizeof(CkptHeader) + (size_t)(h.state_bytes + h.dlog_bytes + h.ring_bytes + h.ext_bytes);
}

int at_save(at_ctx* c, void* dst, size_t bytes, int dst_on_device)
{
    NvtxRange nvtx_range("at_save");
    if (!c || !dst) return fail(AT_EINVAL, "context or destination is NULL");
    if (!c->have_problem || !c->have_delays) return fail(AT_ESTATE, "at_set_problem and at_set_delays must come first");
    if (c->stage_pos != 0) return fail(AT_ESTATE, "a checkpoint is taken between steps, not within a step begun with at_stage");
    const size_t need = at_checkpoint_bytes(c);
    if (bytes < need) return fail(AT_EINVAL, "destination of %zu bytes is below the %zu bytes needed", bytes, need);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, sizeof h.magic);
    h.level = c->level;
    h.hist_level = c->hist_level;
    h.pb = c->pb;
    h.dl = c->dl;
    h.hist = c->hist;
    h.open_ends = c->open_ends;
    h.pe_base = c->pe_base;
    h.pe_total = c->pe_total;
    ckpt_sizes(c, h);
    unsigned char* d = (unsigned char*)dst;
    const cudaMemcpyKind from_host = dst_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    const cudaMemcpyKind from_dev = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    size_t off = 0;
    e = cudaMemcpyAsync(d, &h, sizeof h, from_host, c->stream);
    off += sizeof h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + off, c->state, (size_t)h.state_bytes, from_dev, c->stream);
    off += (size_t)h.state_bytes;
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + off, c->base.dlog, (size_t)h.dlog_bytes, from_dev, c->stream);
    off += (size_t)h.dlog_bytes;
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + off, c->base.ring, (size_t)h.ring_bytes, from_dev, c->stream);
    off += (size_t)h.ring_bytes;
    if (e == cudaSuccess && h.ext_bytes)
        e = cudaMemcpyAsync(d + off, c->base.ext, (size_t)h.ext_bytes, from_dev, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // h lives on this frame
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint copy");
    return AT_OK;
}

int at_restore(at_ctx* c, const void* src, size_t bytes, int src_on_device)
{
    NvtxRange nvtx_range("at_restore");
    if (!c || !src) return fail(AT_EINVAL, "context or source is NULL");
    if (!c->have_problem || !c->have_delays) return fail(AT_ESTATE, "at_set_problem and at_set_delays must come first");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if (bytes < sizeof(CkptHeader)) return fail(AT_EINVAL, "a checkpoint of %zu bytes has no header", bytes);
    CkptHeader h{};
    e = cudaMemcpyAsync(&h, src, sizeof h, src_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint header read");
    if (std::memcmp(h.magic, kCkptMagic, sizeof h.magic) != 0) return fail(AT_EINVAL, "not a checkpoint of this library");
    CkptHeader want{};
    ckpt_sizes(c, want);
    if (!same_problem(h.pb, c->pb) || !same_delays(h.dl, c->dl))
        return fail(AT_EINVAL, "the checkpoint belongs to another problem or delay model");
    if (h.hist != c->hist || h.open_ends != c->open_ends || h.pe_base != c->pe_base || h.pe_total != c->pe_total)
        return fail(AT_EINVAL, "the checkpoint was taken with other history / PE-range options");
    if (h.state_bytes != want.state_bytes || h.dlog_bytes != want.dlog_bytes || h.ring_bytes != want.ring_bytes ||
        h.ext_bytes != want.ext_bytes || h.level < 0)
        return fail(AT_EINVAL, "the checkpoint's sizes do not match this context");
    const size_t need = at_checkpoint_bytes(c);
    if (bytes < need) return fail(AT_EINVAL, "a checkpoint of %zu bytes is below the %zu bytes it needs", bytes, need);
    const unsigned char* sp = (const unsigned char*)src;
    const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    size_t off = sizeof h;
    e = cudaMemcpyAsync(c->state, sp + off, (size_t)h.state_bytes, kind, c->stream);
    off += (size_t)h.state_bytes;
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->base.dlog, sp + off, (size_t)h.dlog_bytes, kind, c->stream);
    off += (size_t)h.dlog_bytes;
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->base.ring, sp + off, (size_t)h.ring_bytes, kind, c->stream);
    off += (size_t)h.ring_bytes;
    if (e == cudaSuccess && h.ext_bytes) e = cudaMemcpyAsync(c->base.ext, sp + off, (size_t)h.ext_bytes, kind, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->base.status, 0, 2 * sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint restore");
    c->level = h.level;
    c->hist_level = h.hist_level;
    c->stage_pos = 0;
    g_err[0] = 0;
    return AT_OK;
}

int at_set_option(at_ctx* c, int key, int64_t value)
{
    if (!c) return fail(AT_EINVAL, "context is NULL");
    switch (key) {
    case AT_OPT_PATH:
        if (value < AT_PATH_AUTO || value > AT_PATH_FUSED) return fail(AT_EINVAL, "unknown path %lld", (long long)value);
        c->path = (int)value;
        return AT_OK;
    case AT_OPT_WAIT_LIMIT:
        if (value < 1) return fail(AT_EINVAL, "wait limit must be positive");
        c->wait_limit = value;
        return AT_OK;
    case AT_OPT_WITHHOLD_PE:
        c->withhold_pe = value;
        return AT_OK;
    case AT_OPT_ARRIVAL:
        if (value != 0 && value != 1) return fail(AT_EINVAL, "AT_OPT_ARRIVAL takes 0 or 1");
        c->arrival = (int)value;
        return AT_OK;
    case AT_OPT_HISTORY:
        if (value != AT_HIST_STAGE && value != AT_HIST_RECOMPUTE)
            return fail(AT_EINVAL, "AT_OPT_HISTORY takes AT_HIST_STAGE or AT_HIST_RECOMPUTE");
        c->hist = (int)value;
        c->hist_level = -1;
        return AT_OK;
    case AT_OPT_OPEN_ENDS:
        if (value != 0 && value != 1) return fail(AT_EINVAL, "AT_OPT_OPEN_ENDS takes 0 or 1");
        c->open_ends = (int)value;
        return AT_OK;
    case AT_OPT_PE_BASE:
        if (value < 0) return fail(AT_EINVAL, "AT_OPT_PE_BASE must be >= 0");
        c->pe_base = value;
        return AT_OK;
    case AT_OPT_PE_TOTAL:
        if (value < 0 || value >= ((int64_t)1 << 32)) return fail(AT_EINVAL, "AT_OPT_PE_TOTAL out of range");
        c->pe_total = value;
        return AT_OK;
    default: return fail(AT_EINVAL, "unknown option %d", key);
    }
}

// ---------------------------------------------------------------------------
// a PE range of a domain split over ranks
// ---------------------------------------------------------------------------
namespace {
// Philox4x32-10 word 0 on the host, as the kernels compute it (Salmon et al.,
// SC'11: ten rounds of two 32x32->64 products, Weyl key increments)
uint32_t host_philox_w0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c0 = n0;
        c1 = (uint32_t)p1;
        c2 = n2;
        c3 = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c0;
}

// the range range checks shared by at_stage / at_edges / at_put_ext
int range_ready(at_ctx* c)
{
    if (!c) return fail(AT_EINVAL, "context is NULL");
    if (!c->have_problem || !c->have_delays) return fail(AT_ESTATE, "at_set_problem and at_set_delays must come first");
    return AT_OK;
}

bool level_in_ring(const at_ctx* c, int64_t level)
{
    // the current level and the older ones the ring still keeps
    return level >= 0 && level <= c->level && level > c->level - c->L.R;
}
} // namespace

int at_delay(at_ctx* c, int64_t level, int stage, int64_t pe, int side)
{
    int st = range_ready(c);
    if (st != AT_OK) return st;
    if (level < 0 || stage < 0 || stage >= c->L.S || pe < 0 || pe >= c->L.P || (side != 0 && side != 1))
        return fail(AT_EINVAL, "level, stage, PE or side out of range");
    const atk::StageArgs& a = c->base;
    if (a.mode == atk::SYNC) return 0;
    int64_t gpe = pe;
    if (c->pe_total > 0) {
        gpe += c->pe_base;
        if (gpe >= c->pe_total) gpe -= c->pe_total;
    }
    const uint32_t sc = a.per_stage ? (uint32_t)stage : 0u;
    const uint32_t x = host_philox_w0((uint32_t)level, (uint32_t)gpe, sc | (uint32_t)side << 8, a.instance, a.key0,
                                      a.key1);
    int k = 0;
    for (int i = 0; i < a.kmax; ++i) k += ((uint64_t)x >= a.thr[i]) ? 1 : 0;
    int64_t avail = level - ((a.mode == atk::AT) ? a.q : 0);
    if (avail < 0) avail = 0;
    return (int64_t)k < avail ? k : (int)avail;
}

int at_stage(at_ctx* c)
{
    NvtxRange nvtx_range("at_stage");
    int st = range_ready(c);
    if (st != AT_OK) return st;
    if (c->hist == AT_HIST_RECOMPUTE) return fail(AT_EINVAL, "at_stage runs reading B of the stage history");
    if (c->arrival) return fail(AT_EINVAL, "at_stage uses drawn delays");
    if (c->level >= kMaxLevel) return fail(AT_EINVAL, "a solve is limited to %lld steps", (long long)kMaxLevel);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const Layout& L = c->L;
    double* A = (double*)(c->ws + L.off_A);
    double* Bf = (double*)(c->ws + L.off_B);
    double* u = c->state;
    const int s = c->stage_pos;
    atk::StageArgs a = c->base;
    a.level = c->level;
    a.u = u;
    a.stage = s;
    a.open_ends = c->open_ends;
    a.pe_base = c->pe_base;
    a.pe_total = c->pe_total;
    a.trace = c->trace;
    a.trace_n0 = c->trace_n0;
    a.trace_steps = c->trace_steps;
    // the buffers of at_step's per-stage loop
    a.X = (s == 0) ? u : ((s % 2 == 1) ? A : Bf);
    a.Y = (s == L.S - 1) ? u : ((s % 2 == 0) ? A : Bf);
    e = record(c, true);
    if (e == cudaSuccess) e = atk_launch_stage(a, c->pb.pde, c->pb.order, c->stream);
    if (e == cudaSuccess) e = record(c, false);
    if (e != cudaSuccess) return cuda_fail(e, "stage kernel launch");
    ++c->launched;
    c->last_path = AT_PATH_STAGE;
    if (++c->stage_pos == L.S) {
        c->stage_pos = 0;
        ++c->level;
    }
    g_err[0] = 0;
    return AT_OK;
}

int at_edges(at_ctx* c, int64_t level, int stage, double* out)
{
    int st = range_ready(c);
    if (st != AT_OK) return st;
    if (!out) return fail(AT_EINVAL, "destination is NULL");
    if (stage < 0 || stage >= c->L.S || !level_in_ring(c, level))
        return fail(AT_EINVAL, "level %lld stage %d is not in the ring", (long long)level, stage);
    const Layout& L = c->L;
    const size_t win = (size_t)L.H * L.nvar;
    cudaError_t e = cudaSetDevice(c->device);
    const double* ring = c->base.ring;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, ring + host_ring_index(L, level, stage, 0, 0), sizeof(double) * win,
                            cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out + win, ring + host_ring_index(L, level, stage, L.P - 1, 1), sizeof(double) * win,
                            cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "edge window copy");
    return AT_OK;
}

int at_put_ext(at_ctx* c, int64_t level, int stage, int side, const double* win)
{
    int st = range_ready(c);
    if (st != AT_OK) return st;
    if (!win) return fail(AT_EINVAL, "window is NULL");
    if (!c->open_ends) return fail(AT_EINVAL, "outside windows need AT_OPT_OPEN_ENDS");
    if (stage < 0 || stage >= c->L.S || (side != 0 && side != 1) || level < 0)
        return fail(AT_EINVAL, "level, stage or side out of range");
    const Layout& L = c->L;
    const size_t n = (size_t)L.H * L.nvar;
    const int64_t r = level % L.R;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->base.ext + ((r * L.S + stage) * 2 + side) * n, win, sizeof(double) * n,
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "outside window copy");
    return AT_OK;
}

int at_set_delay_trace(at_ctx* c, uint8_t* trace_dev, int64_t max_steps)
{
    if (!c) return fail(AT_EINVAL, "context is NULL");
    if (!trace_dev || max_steps <= 0) {
        c->trace = nullptr;
        c->trace_steps = 0;
        return AT_OK;
    }
    if (!c->have_problem) return fail(AT_ESTATE, "at_set_problem must come first");
    c->trace = trace_dev;
    c->trace_n0 = c->level;
    c->trace_steps = max_steps;
    return AT_OK;
}

int at_profile(at_ctx* c, int enable)
{
    if (!c) return fail(AT_EINVAL, "context is NULL");
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = harvest(c);
    if (e != cudaSuccess) return cuda_fail(e, "profiling events");
    c->profile = enable != 0;
    c->timed = 0;
    c->timed_ms = 0.0;
    return AT_OK;
}

int at_destroy(at_ctx* c)
{
    if (!c) return AT_OK;
    cudaSetDevice(c->device);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    delete c;
    return AT_OK;
}

// ---------------------------------------------------------------------------
// batched solves
// ---------------------------------------------------------------------------
namespace {
const int kVariants = 12;

struct BatchTable {  // carving of the caller's table memory
    size_t off_args, off_lvl, off_left, off_order, off_slots, off_status, off_queue, off_wslot, off_widx, total;
    int64_t max_windows;
};

BatchTable batch_table(int64_t cap, int64_t max_windows)
{
    BatchTable t{};
    size_t off = 0;
    t.off_args = off;
    off = align256(off + sizeof(atk::StageArgs) * (size_t)cap);
    t.off_lvl = off;
    off = align256(off + sizeof(int64_t) * (size_t)cap);
    t.off_left = off;
    off = align256(off + sizeof(int64_t) * (size_t)cap);
    t.off_order = off;  // queue order, grouped by kernel variant
    off = align256(off + sizeof(int) * (size_t)cap);
    t.off_slots = off;  // bound slots, for the status gather
    off = align256(off + sizeof(int) * (size_t)cap);
    t.off_status = off;
    off = align256(off + sizeof(int) * (size_t)cap);
    t.off_queue = off;  // one queue counter per variant
    off = align256(off + sizeof(int) * kVariants);
    t.off_wslot = off;  // flat mode: slot and window index of every window, grouped by variant
    off = align256(off + sizeof(int) * (size_t)max_windows);
    t.off_widx = off;
    off = align256(off + sizeof(int) * (size_t)max_windows);
    t.max_windows = max_windows;
    t.total = off;
    return t;
}
} // namespace

// kernel variants of the WENO PDEs (one window per CTA in flat mode)
static bool variant_is_weno(int g) { return g == 6 || g == 7 || g == 8; }

struct at_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t cap = 0;
    unsigned char* tab = nullptr;
    BatchTable T{};
    int sms = 0;
    int mode = 0, block = 256, ctas_per_sm = 3, use_graph = 1;
    // host mirrors
    std::vector<atk::StageArgs> args;
    std::vector<int64_t> level, left, cost;
    std::vector<int> variant, bound;
    std::vector<size_t> smem;
    std::vector<int> order_h, slots_h, status_h;
    std::vector<int64_t> lvl_h, left_h;  // staging for uploads
    int group_begin[kVariants + 1] = {0};
    size_t group_smem[kVariants] = {0};
    std::vector<int> wslot_h, widx_h;
    std::vector<int64_t> windows;  // windows per slot
    int64_t bound_windows = 0;
    int64_t wbegin[kVariants + 1] = {0};
    int group_stages[kVariants] = {0};
    bool dirty = true;
    // graph of the last (chunk, order) configuration
    cudaGraphExec_t gexec = nullptr;
    int64_t gchunk = -1;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t branch[kVariants] = {nullptr};
    cudaEvent_t fork = nullptr, join[kVariants] = {nullptr};
};

namespace {
cudaError_t batch_upload_order(at_batch* b)
{
    std::vector<std::vector<int>> groups(kVariants);
    b->slots_h.clear();
    for (int64_t i = 0; i < b->cap; ++i)
        if (b->bound[i]) {
            groups[b->variant[i]].push_back((int)i);
            b->slots_h.push_back((int)i);
        }
    b->order_h.clear();
    for (int g = 0; g < kVariants; ++g) {
        // largest remaining work first (longest-processing-time order)
        std::stable_sort(groups[g].begin(), groups[g].end(),
                         [&](int x, int y) { return b->cost[x] * b->left[x] > b->cost[y] * b->left[y]; });
        b->group_begin[g] = (int)b->order_h.size();
        size_t sm = 0;
        for (int i : groups[g]) {
            b->order_h.push_back(i);
            sm = std::max(sm, b->smem[i]);
        }
        b->group_smem[g] = sm;
    }
    b->group_begin[kVariants] = (int)b->order_h.size();
    // flat-mode map of CTAs, in the same order: one window each, or (central
    // PDEs) two consecutive windows of one slot, marked by bit 30 of the
    // window index (a lone last window of a slot takes a CTA alone)
    b->wslot_h.clear();
    b->widx_h.clear();
    for (int g = 0; g < kVariants; ++g) {
        b->wbegin[g] = (int64_t)b->wslot_h.size();
        const bool pairs = !variant_is_weno(g);
        int smax = 0;
        for (int q = b->group_begin[g]; q < b->group_begin[g + 1]; ++q) {
            const int i = b->order_h[q];
            for (int64_t w = 0; w < b->windows[i];) {
                const bool two = pairs && w + 1 < b->windows[i];
                b->wslot_h.push_back(i);
                b->widx_h.push_back((int)w | (two ? (1 << 30) : 0));
                w += two ? 2 : 1;
            }
            smax = std::max(smax, b->args[i].S);
        }
        b->group_stages[g] = smax;
    }
    b->wbegin[kVariants] = (int64_t)b->wslot_h.size();
    cudaError_t e = cudaSuccess;
    if (!b->wslot_h.empty()) {
        e = cudaMemcpyAsync(b->tab + b->T.off_wslot, b->wslot_h.data(), sizeof(int) * b->wslot_h.size(),
                            cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->tab + b->T.off_widx, b->widx_h.data(), sizeof(int) * b->widx_h.size(),
                                cudaMemcpyHostToDevice, b->stream);
    }
    if (!b->order_h.empty())
        e = cudaMemcpyAsync(b->tab + b->T.off_order, b->order_h.data(), sizeof(int) * b->order_h.size(),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !b->slots_h.empty())
        e = cudaMemcpyAsync(b->tab + b->T.off_slots, b->slots_h.data(), sizeof(int) * b->slots_h.size(),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // host staging vectors change later
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    b->dirty = false;
    return e;
}

// queue reset, then one launch per non-empty kernel variant; variants run on
// branch streams forked from and joined back into `st`, so they overlap.
// Flat mode: per variant, `chunk` x (stages + level advance) launches.
cudaError_t batch_enqueue(at_batch* b, cudaStream_t st, int64_t chunk)
{
    cudaError_t e = cudaMemsetAsync(b->tab + b->T.off_queue, 0, sizeof(int) * kVariants, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, st);
    const atk::StageArgs* tab = (const atk::StageArgs*)(b->tab + b->T.off_args);
    int64_t* lvl = (int64_t*)(b->tab + b->T.off_lvl);
    int64_t* left = (int64_t*)(b->tab + b->T.off_left);
    for (int g = 0; g < kVariants && e == cudaSuccess; ++g) {
        const int n = b->group_begin[g + 1] - b->group_begin[g];
        if (n == 0) continue;
        const size_t smem = b->group_smem[g];
        const int* order = (const int*)(b->tab + b->T.off_order) + b->group_begin[g];
        e = cudaStreamWaitEvent(b->branch[g], b->fork, 0);
        if (e != cudaSuccess) break;
        if (b->mode == 0) {
            int per_sm = atk_batch_max_ctas_per_sm(g, b->block, smem);
            if (per_sm < 1) return cudaErrorInvalidConfiguration;
            per_sm = std::min(per_sm, b->ctas_per_sm);
            const int grid = std::min(n, per_sm * b->sms);
            e = atk_launch_batch(g, tab, lvl, left, order, n, (int*)(b->tab + b->T.off_queue) + g, chunk, grid,
                                 b->block, smem, b->branch[g]);
        } else {
            const int nwin = (int)(b->wbegin[g + 1] - b->wbegin[g]);
            const int* ws = (const int*)(b->tab + b->T.off_wslot) + b->wbegin[g];
            const int* wi = (const int*)(b->tab + b->T.off_widx) + b->wbegin[g];
            for (int64_t step = 0; step < chunk && e == cudaSuccess; ++step) {
                for (int stage = 0; stage < b->group_stages[g] && e == cudaSuccess; ++stage)
                    e = atk_launch_batch_stage(g, tab, lvl, left, ws, wi, nwin, stage, b->block,
                                               variant_is_weno(g) ? smem : 2 * smem, (int)(smem / sizeof(double)),
                                               b->branch[g]);
                if (e == cudaSuccess) e = atk_launch_batch_advance(lvl, left, order, n, b->branch[g]);
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(b->join[g], b->branch[g]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->join[g], 0);
    }
    return e;
}
} // namespace

size_t at_batch_table_bytes(int64_t capacity, int64_t max_windows)
{
    if (capacity <= 0 || capacity > (1 << 24) || max_windows < 0 || max_windows > ((int64_t)1 << 30)) return 0;
    return batch_table(capacity, max_windows).total;
}

int at_batch_create(at_batch** out, int device, void* cuda_stream, int64_t capacity, int64_t max_windows,
                    void* table_dev, size_t table_bytes)
{
    if (!out) return fail(AT_EINVAL, "out is NULL");
    *out = nullptr;
    if (capacity <= 0 || capacity > (1 << 24)) return fail(AT_EINVAL, "capacity must be 1..2^24");
    if (max_windows < 0 || max_windows > ((int64_t)1 << 30)) return fail(AT_EINVAL, "max_windows out of range");
    if (!table_dev || ((uintptr_t)table_dev & 255)) return fail(AT_EINVAL, "table must be 256-byte aligned device memory");
    if (table_bytes < batch_table(capacity, max_windows).total)
        return fail(AT_ENOMEM, "table of %zu bytes is below the %zu bytes needed", table_bytes,
                    batch_table(capacity, max_windows).total);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    at_batch* b = new (std::nothrow) at_batch;
    if (!b) return fail(AT_ENOMEM, "host allocation failed");
    b->device = device;
    b->stream = (cudaStream_t)cuda_stream;
    b->cap = capacity;
    b->tab = (unsigned char*)table_dev;
    b->T = batch_table(capacity, max_windows);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, device);
    b->args.resize(capacity);
    b->level.assign(capacity, 0);
    b->left.assign(capacity, 0);
    b->cost.assign(capacity, 0);
    b->variant.assign(capacity, 0);
    b->bound.assign(capacity, 0);
    b->smem.assign(capacity, 0);
    b->windows.assign(capacity, 0);
    b->lvl_h.assign(capacity, 0);
    b->left_h.assign(capacity, 0);
    e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int g = 0; g < kVariants && e == cudaSuccess; ++g) {
        e = cudaStreamCreateWithFlags(&b->branch[g], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[g], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = atk_set_smem_limits();
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "batch set-up");
    }
    *out = b;
    return AT_OK;
}

int at_batch_bind(at_batch* b, int64_t slot, const at_instance* in)
{
    if (!b || !in) return fail(AT_EINVAL, "batch or instance is NULL");
    if (slot < 0 || slot >= b->cap) return fail(AT_EINVAL, "slot %lld out of range", (long long)slot);
    if (b->bound[slot]) return fail(AT_ESTATE, "slot %lld is bound", (long long)slot);
    int st = check_problem(&in->pb);
    if (st == AT_OK) st = check_delays(&in->dl);
    if (st != AT_OK) return st;
    if (in->pb.weno == AT_WENO_INTERPOLATE)
        return fail(AT_EINVAL, "the WENO interpolation form runs on a context's per-stage path, not in batches");
    if (in->nsteps < 0) return fail(AT_EINVAL, "nsteps must be >= 0");
    if (in->nsteps > kMaxLevel) return fail(AT_EINVAL, "a solve is limited to %lld steps", (long long)kMaxLevel);
    if (!in->state_dev || !in->workspace_dev || ((uintptr_t)in->state_dev & 15) || ((uintptr_t)in->workspace_dev & 255))
        return fail(AT_EINVAL, "state (16-B aligned) and workspace (256-B aligned) must be device memory");
    const Layout L = layout(&in->pb, &in->dl);
    if (in->workspace_bytes < L.total)
        return fail(AT_ENOMEM, "workspace of %zu bytes is below the %zu bytes needed", in->workspace_bytes, L.total);
    const int64_t nwin = L.P * L.wpp;
    if (b->bound_windows + nwin > b->T.max_windows)
        return fail(AT_ENOMEM, "the batch's window map holds %lld windows; bound %lld + this %lld",
                    (long long)b->T.max_windows, (long long)b->bound_windows, (long long)nwin);
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    atk::StageArgs a = build_args(&in->pb, &in->dl, L, (unsigned char*)in->workspace_dev, in->state_dev);
    e = cudaMemsetAsync(a.ring, 0, sizeof(double) * L.ring_elems, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.dlog, 0, (size_t)L.S * L.P * 2, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.status, 0, 2 * sizeof(int), b->stream);
    if (e == cudaSuccess) e = atk_launch_ring_seed(a, b->stream);
    b->args[slot] = a;
    b->lvl_h[slot] = 0;
    b->left_h[slot] = in->nsteps;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tab + b->T.off_args + sizeof(atk::StageArgs) * slot, &b->args[slot],
                            sizeof(atk::StageArgs), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tab + b->T.off_lvl + sizeof(int64_t) * slot, &b->lvl_h[slot], sizeof(int64_t),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tab + b->T.off_left + sizeof(int64_t) * slot, &b->left_h[slot], sizeof(int64_t),
                            cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch bind");
    b->level[slot] = 0;
    b->left[slot] = in->nsteps;
    b->cost[slot] = (int64_t)L.nvar * in->pb.n * L.S * (is_weno(in->pb.pde) ? 8 : 1);
    b->variant[slot] = atk_batch_variant(in->pb.pde, in->pb.order);
    b->smem[slot] = atk_stage_smem_bytes(in->pb.pde, L.Tw, L.H);
    b->windows[slot] = nwin;
    b->bound_windows += nwin;
    b->bound[slot] = 1;
    b->dirty = true;
    return AT_OK;
}

int at_batch_release(at_batch* b, int64_t slot)
{
    if (!b) return fail(AT_EINVAL, "batch is NULL");
    if (slot < 0 || slot >= b->cap || !b->bound[slot]) return fail(AT_EINVAL, "slot %lld is not bound", (long long)slot);
    b->bound[slot] = 0;
    b->bound_windows -= b->windows[slot];
    b->windows[slot] = 0;
    b->dirty = true;
    return AT_OK;
}

int at_batch_set_config(at_batch* b, int mode, int block, int ctas_per_sm, int use_graph)
{
    if (!b) return fail(AT_EINVAL, "batch is NULL");
    if (mode != AT_BATCH_INSTANCE && mode != AT_BATCH_FLAT) return fail(AT_EINVAL, "unknown batch mode %d", mode);
    if (block < 64 || block > 256 || block % 32) return fail(AT_EINVAL, "block must be 64..256, a multiple of 32");
    if (ctas_per_sm < 1 || ctas_per_sm > 16) return fail(AT_EINVAL, "ctas_per_sm must be 1..16");
    b->mode = mode;
    b->block = block;
    b->ctas_per_sm = ctas_per_sm;
    b->use_graph = use_graph ? 1 : 0;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return AT_OK;
}

int at_batch_step(at_batch* b, int64_t chunk)
{
    NvtxRange nvtx_range("at_batch_step");
    if (!b) return fail(AT_EINVAL, "batch is NULL");
    if (chunk < 0) return fail(AT_EINVAL, "chunk must be >= 0");
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if (b->dirty) {
        e = batch_upload_order(b);
        if (e != cudaSuccess) return cuda_fail(e, "batch queue upload");
    }
    if (chunk == 0 || b->order_h.empty()) return AT_OK;
    if (b->use_graph) {
        if (!b->gexec || b->gchunk != chunk) {
            if (b->gexec) {
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t le = batch_enqueue(b, b->cap_stream, chunk);
                e = cudaStreamEndCapture(b->cap_stream, &g);
                if (le != cudaSuccess) e = le;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "batch graph capture");
            b->gchunk = chunk;
        }
        e = cudaGraphLaunch(b->gexec, b->stream);
    } else {
        e = batch_enqueue(b, b->stream, chunk);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    for (int64_t i = 0; i < b->cap; ++i)
        if (b->bound[i]) {
            const int64_t n = std::min(chunk, b->left[i]);
            b->level[i] += n;
            b->left[i] -= n;
        }
    return AT_OK;
}

int at_batch_run(at_batch* b, int64_t chunk)
{
    int st = at_batch_step(b, chunk);
    if (st != AT_OK) return st;
    const int n = (int)b->slots_h.size();
    b->status_h.assign(n, 0);
    cudaError_t e = atk_launch_batch_status((const atk::StageArgs*)(b->tab + b->T.off_args),
                                            (const int*)(b->tab + b->T.off_slots), n,
                                            (int*)(b->tab + b->T.off_status), b->stream);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(b->status_h.data(), b->tab + b->T.off_status, sizeof(int) * n, cudaMemcpyDeviceToHost,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch run");
    for (int i = 0; i < n; ++i)
        if (b->status_h[i]) return fail(AT_EUNSTABLE, "slot %d produced a non-finite value", b->slots_h[i]);
    return AT_OK;
}

int at_batch_query(at_batch* b, int64_t slot, at_slot_info* info)
{
    if (!b || !info) return fail(AT_EINVAL, "batch or info is NULL");
    if (slot < 0 || slot >= b->cap) return fail(AT_EINVAL, "slot out of range");
    at_slot_info r{};
    r.bound = b->bound[slot];
    if (r.bound) {
        int64_t dev[2] = {0, 0};
        int status = 0;
        cudaError_t e = cudaMemcpyAsync(&dev[0], b->tab + b->T.off_lvl + sizeof(int64_t) * slot, sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&dev[1], b->tab + b->T.off_left + sizeof(int64_t) * slot, sizeof(int64_t),
                                cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&status, b->args[slot].status, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "batch query");
        r.level = dev[0];
        r.left = dev[1];
        r.status = status ? AT_EUNSTABLE : 0;
    }
    *info = r;
    return AT_OK;
}

int at_batch_destroy(at_batch* b)
{
    if (!b) return AT_OK;
    cudaSetDevice(b->device);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (int g = 0; g < kVariants; ++g) {
        if (b->branch[g]) cudaStreamDestroy(b->branch[g]);
        if (b->join[g]) cudaEventDestroy(b->join[g]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
    return AT_OK;
}

// ---------------------------------------------------------------------------
// allocation-free entry point: the workspace is this file-scope device array
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[AT_NOALLOC_SCRATCH_BYTES];

namespace {
const int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices];  // device address of the array, per device (set up once)
} // namespace

int at_run_noalloc(const at_problem* pb, const at_delays* dl, double* state_dev, int64_t nsteps, int device,
                   void* cuda_stream)
{
    NvtxRange nvtx_range("at_run_noalloc");
    if (!state_dev) return fail(AT_EINVAL, "state must be a device pointer");
    if (nsteps < 0) return fail(AT_EINVAL, "nsteps must be >= 0");
    const size_t need = at_workspace_bytes(pb, dl);
    if (need == 0) return AT_EINVAL;  // at_last_error() names the invalid field
    if (need > AT_NOALLOC_SCRATCH_BYTES)
        return fail(AT_ENOMEM, "this problem needs %zu workspace bytes; at_run_noalloc has %zu", need,
                    (size_t)AT_NOALLOC_SCRATCH_BYTES);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev || device >= kMaxDevices) return fail(AT_EINVAL, "device %d out of range", device);
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        e = cudaSetDevice(device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
        if (!g_noalloc_ptr[device]) {
            // once per device, with the device current: the host-side name of a
            // __device__ array is not its device address
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the scratch array");
            e = atk_set_smem_limits();
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
            g_noalloc_ptr[device] = ptr;
        }
        scratch = g_noalloc_ptr[device];
    }
    at_ctx c;  // on the stack: no heap allocation (tracing stays off)
    c.device = device;
    c.stream = (cudaStream_t)cuda_stream;
    int st = at_set_problem(&c, pb, state_dev, nullptr, 1, scratch, AT_NOALLOC_SCRATCH_BYTES);
    if (st == AT_OK) st = at_set_delays(&c, dl);  // clears ring, delay log and status word
    if (st == AT_OK) st = at_run(&c, nsteps);
    return st;
}

} // extern "C"
