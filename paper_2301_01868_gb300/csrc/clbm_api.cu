// clbm_api.cu -- host side of the C ABI declared in include/clbm.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include <nvtx3/nvToolsExt.h>

#include "../../include/clbm.h"
#include "clbm_batch.cuh"
#include "clbm_internal.cuh"

using namespace clbm;

namespace {

// NVTX range over one API call (visible in Nsight timelines; free when no
// tool is attached).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

thread_local char g_err[512] = "";

clbm_status fail(clbm_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(CLBM_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                        __FILE__, __LINE__);                                            \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t stA, stB, tab, geo, wall_r, wall_u, ghost, pos, partial, red, prev, err, total;
};

}  // namespace

void clbm::set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

struct clbm_grid {
    int Q, prec, n1, n2, ld, h, kind, bc_lo, bc_hi, device;
    double dx;
    cudaStream_t stream;
    char* ws;
    bool owns_ws;
    Layout L;
    void *stA, *stB, *tab, *wall_r, *wall_u;
    double *geo, *ghost, *pos, *partial, *red, *prev;
    clbm_case cs;
    bool ghosts_ok;         // ghost rows / columns of the current state are filled
    bool have_case;
    long long t, t_prev, launches;
    bool have_prev;
    bool profiling;
    int prof_period;        // record every prof_period-th update launch
    long long prof_count;   // update launches since profiling was switched on
    std::vector<cudaEvent_t> ev;
    size_t ev_used;
    long long ev_launches;  // update launches the recorded event pairs span
    std::vector<double> edges;
    double step2;
    double* stage;          // lazily allocated FP64 staging buffer for host transfers
    struct HostPipe* pipe;  // asynchronous host copies (created on first use)
    int ncol;               // geometry columns: 1 (planar, polar) or n2 (general)
    int n2_period;          // columns of the whole ring (polar slabs), else n2
    double rest_mass;       // rho0 times the total volume (the rest part of the mass)
    std::vector<double> nodes;  // node positions of a general grid (for the no-flow clone)
    void* phys[2];          // the two state buffers (stA / stB alternate over them)
    TmaMaps* tma;           // tensor maps of the TMA-staged update (16/32-bit storage)
    int nsm;                // SM count of the device
    int variant;            // 0 auto, 1 per-cell loads, 2 TMA-staged tiles, ... (clbm_set_kernel)
    int* err;               // device error word of bounded waits
    unsigned long long* prog;  // progress words and tile counter of the multi-step runs (nsm + 1, device)
    unsigned run_epoch;        // tag of the last multi-step run on prog
    bool run_refused;          // a cooperative launch was refused: the automatic choice keeps to a launch per step
    // CUDA graph of GRAPH_STEPS update launches (an even count, so the two
    // state buffers end where they started), replayed by clbm_step; the key
    // is what the launches take, and a change of it rebuilds the graph
    cudaGraph_t graph;       // kept while gexec lives: its nodes address gexec's
    cudaGraphExec_t gexec;
    cudaGraphNode_t gev[2];  // event-record nodes before the first and after the last launch
    cudaEvent_t gdummy[2];   // their events while profiling is off
    StepArgs gargs;          // arguments of the first captured launch
    int gpath[4];            // use_tma, general, variant, nsm at capture
    bool graphs_off;         // capture failed once: plain launches from then on
};

namespace {

clbm_status layout_of(const clbm_grid_desc* d, Layout* L, int* ld_out, int* h_out) {
    if (!d) return fail(CLBM_EINVAL, "desc is NULL");
    if (d->lattice != 9 && d->lattice != 21) return fail(CLBM_EINVAL, "lattice must be 9 or 21");
    if (d->precision < 0 || d->precision > 3) return fail(CLBM_EINVAL, "bad precision");
    if (d->n1 < 4 || d->n2 < 1) return fail(CLBM_EINVAL, "need n1 >= 4 and n2 >= 1");
    if ((long long)d->n1 * d->n2 > (1LL << 31) / 32)
        return fail(CLBM_EINVAL, "grid too large for 32-bit cell indexing");
    if (d->kind < CLBM_GEOM_PLANAR || d->kind > CLBM_GEOM_GENERAL)
        return fail(CLBM_EINVAL, "kind must be PLANAR, POLAR or GENERAL");
    const int Q = d->lattice, h = Q == 9 ? 1 : 3;
    const int ld = (d->n2 + 2 * GC + 31) / 32 * 32;
    const size_t sb = storage_bytes(d->precision), cb = compute_bytes(d->precision);
    // general grids carry per-cell geometry and tables, the others one row each
    const int ncol = d->kind == CLBM_GEOM_GENERAL ? d->n2 : 1;
    const size_t tab_entries = ncol > 1 ? (size_t)(Q == 9 ? CellTabLayout<9>::S : CellTabLayout<21>::S) *
                                              d->n1 * d->n2
                                        : (size_t)(Q == 9 ? Tab<9>::S : Tab<21>::S) * d->n1;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    if ((long long)Q * (d->n1 + 2 * h) * ld >= (1LL << 31))
        return fail(CLBM_EINVAL, "grid too large: the Q population planes must hold fewer than 2^31 values");
    L->stA = take((size_t)Q * (d->n1 + 2 * h) * ld * sb);
    L->stB = take((size_t)Q * (d->n1 + 2 * h) * ld * sb);
    L->tab = take(tab_entries * cb);
    L->geo = take((size_t)d->n1 * ncol * Geo::stride(Q) * 8);
    L->wall_r = take((size_t)2 * h * d->n2 * cb);
    L->wall_u = take((size_t)2 * h * d->n2 * cb);
    L->ghost = take((size_t)2 * h * Q * 2 * ncol * 8);
    L->pos = take((size_t)(d->n1 + 8) * (ncol + 8) * 2 * 8);
    L->partial = take((size_t)moments_blocks(d->n1, d->n2) * NRED * 8);
    L->red = take(16 * 8);
    L->prev = take((size_t)2 * d->n1 * d->n2 * 8);
    L->err = take(16);
    L->total = o;
    *ld_out = ld;
    *h_out = h;
    return CLBM_OK;
}

// Wall-normal node coordinate of 1-based row i: edge midpoints inside, mirror
// images through the walls outside (App. B, App. C).
double node_coord(const std::vector<double>& e, int n1, int i) {
    auto mid = [&](int k) { return 0.5 * (e[k - 1] + e[k]); };
    if (i >= 1 && i <= n1) return mid(i);
    if (i < 1) return 2.0 * e[0] - mid(1 - i);
    return 2.0 * e[n1] - mid(2 * n1 + 1 - i);
}

StepScalars scalars(const clbm_case& c) {
    StepScalars k;
    k.rho0 = c.rho0;
    k.g1 = c.g_ext[0];
    k.g2 = c.g_ext[1];
    k.tau_inv = 1.0 / c.tau;
    k.omt = 1.0 - 1.0 / c.tau;
    k.pref = -0.5 * (1.0 - 0.5 / c.tau);
    k.frho0 = (float)k.rho0;
    k.fg1 = (float)k.g1;
    k.fg2 = (float)k.g2;
    k.ftau_inv = (float)k.tau_inv;
    k.fomt = (float)k.omt;
    k.fpref = (float)k.pref;
    return k;
}

StepArgs step_args(const clbm_grid* g, const void* src, void* dst) {
    StepArgs a{};   // zeroed padding: graph keys compare these bytes
    a.k = scalars(g->cs);
    a.src = src;
    a.dst = dst;
    a.tab = g->tab;
    a.wall_rho = g->wall_r;
    a.wall_ut2 = g->wall_u;
    a.ghost = g->ghost;
    a.n1 = g->n1;
    a.n2 = g->n2;
    a.ld = g->ld;
    a.h = g->h;
    a.plane = (long long)(g->n1 + 2 * g->h) * g->ld;
    a.tau = g->cs.tau;
    a.rho0 = g->cs.rho0;
    a.g1 = g->cs.g_ext[0];
    a.g2 = g->cs.g_ext[1];
    a.U0_lo = g->cs.u_wall_lo;
    a.U0_hi = g->cs.u_wall_hi;
    a.bc_lo = g->bc_lo;
    a.bc_hi = g->bc_hi;
    a.ncol = g->ncol;
    a.iters = g->cs.force_iterations;
    a.err = g->err;
    return a;
}

// General grids run the per-cell kernel (the automatic choice) or, asked
// for, the pipelined form with per-cell tables (kernel 3): with the 73 table
// planes read from global memory by 16 consumer warps per SM, and spilling
// at the pipeline's 96 registers, that form measured 0.474 ms against the
// per-cell kernel's 0.419 ms on the 1024 x 4096 wavy channel.  The TMA tiles
// of kernel 2 and the pipelined residual read row tables: planar and polar
// grids only.
bool general_grid(const clbm_grid* g) { return g->ncol > 1; }

// Which TMA-staged update a planar or polar grid runs: kernel 2 the tiles
// with a shared output tile, 3 the pipeline, 4 the pipeline with two cells
// per thread; automatic: the two-cell pipeline for 16-bit storage (bound by
// instruction issue there, it executes 29 % fewer instructions: 105.7 us
// against 110.9 us per launch on the 1024 x 4096 annulus) and the one-cell
// pipeline for FP32 (bound by HBM, where the two-cell form's fewer resident
// warps cost more than its instructions save: 133 us against 116 us).
int tma_mode(const clbm_grid* g) {
    if (g->variant == 2) return 0;
    if (g->variant == 4 || g->variant == 6 || (g->variant == 0 && g->prec >= 2)) return 2;
    return 1;
}

bool use_tma(const clbm_grid* g) {
    if (!g->tma || g->cs.force_iterations > 0) return false;
    if (general_grid(g)) return g->variant == 3;
    return g->variant != 1;
}

// Whether clbm_step runs the pipelined update as multi-step launches (kernels
// 5 and 6).  Automatic: 16-bit storage on planar and polar grids of at least
// RUN_TILES_PER_SM tiles per SM, where the update is bound by instruction
// issue and the run saves the per-launch ramp-up and tail (FP16 on the
// 1024 x 4096 annulus: 0.1006 ms per step against 0.1055 with a launch per
// step).  FP32 storage keeps a launch per step: bound by HBM, the run
// measured 0.119-0.139 ms per step against 0.116 (the CTAs spread their
// reads over more of the state than the CTAs of one launch, and every
// published progress word is a release at GPU scope).
constexpr int RUN_TILES_PER_SM = 8;
constexpr int RUN_MAX_STEPS = 1000;   // time steps per multi-step launch

bool use_run(const clbm_grid* g) {
    if (!use_tma(g) || general_grid(g)) return false;
    if (g->variant == 5 || g->variant == 6) return true;
    if (g->variant != 0 || g->prec < 2 || g->run_refused) return false;
    return run_tiles(g->Q, tma_mode(g), g->n1, g->n2) >= RUN_TILES_PER_SM * g->nsm;
}

// Device-side failures recorded by bounded waits since the last check.
clbm_status check_err(clbm_grid* g) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, g->err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (e != 0) {
        CK(cudaMemsetAsync(g->err, 0, sizeof(int), g->stream));
        return fail(CLBM_ETIMEOUT, "a bounded device wait gave up (code %d)", e);
    }
    return CLBM_OK;
}

MomArgs mom_args(const clbm_grid* g) {
    MomArgs m;
    memset(&m, 0, sizeof(m));
    m.k = scalars(g->cs);
    m.src = g->stA;
    m.tab = g->tab;
    m.geo = g->geo;
    m.n1 = g->n1;
    m.n2 = g->n2;
    m.ld = g->ld;
    m.h = g->h;
    m.plane = (long long)(g->n1 + 2 * g->h) * g->ld;
    m.tau = g->cs.tau;
    m.rho0 = g->cs.rho0;
    m.g1 = g->cs.g_ext[0];
    m.g2 = g->cs.g_ext[1];
    m.ncol = g->ncol;
    m.ut_prev = g->prev;
    m.partial = g->partial;
    m.err = g->err;
    return m;
}

clbm_status select(clbm_grid* g) {
    CK(cudaSetDevice(g->device));
    return CLBM_OK;
}

// FP64 device staging for host transfers: max(Q, 7) fields of n1*n2, kept
// for the grid's lifetime so repeated host calls do not allocate.
clbm_status staging(clbm_grid* g, double** out) {
    if (!g->stage) {
        const size_t n = (size_t)(g->Q > 7 ? g->Q : 7) * g->n1 * g->n2;
        cudaError_t e = cudaMalloc((void**)&g->stage, n * 8);
        if (e != cudaSuccess) {
            g->stage = nullptr;
            return fail(CLBM_ENOMEM, "host staging buffer: %s", cudaGetErrorString(e));
        }
    }
    *out = g->stage;
    return CLBM_OK;
}

// Asynchronous host copies of one grid: a copy stream of its own, two FP64
// state slots (uploads) and two moment slots (downloads), each slot with an
// event that marks it filled and one that marks it read, so that an upload
// for the next start overlaps the update of this one, and a download of
// these moments overlaps the next update.  (Outside the unnamed namespace:
// clbm_grid names it.)
}  // namespace

struct HostPipe {
    cudaStream_t copy = nullptr;
    double* in[2] = {nullptr, nullptr};    // Q n1 n2 FP64 each
    double* out[2] = {nullptr, nullptr};   // 3 n1 n2 FP64 each: rho, Ut^1, Ut^2
    cudaEvent_t in_ready[2] = {}, in_free[2] = {}, out_ready[2] = {}, out_free[2] = {};
    bool in_used[2] = {false, false}, out_used[2] = {false, false};
    int next_in = 0, next_set = 0, next_out = 0, staged = 0;
};

namespace {

void free_pipe(HostPipe* p) {
    if (!p) return;
    if (p->copy) cudaStreamSynchronize(p->copy);
    for (int k = 0; k < 2; ++k) {
        cudaFree(p->in[k]);
        cudaFree(p->out[k]);
        for (cudaEvent_t e : {p->in_ready[k], p->in_free[k], p->out_ready[k], p->out_free[k]})
            if (e) cudaEventDestroy(e);
    }
    if (p->copy) cudaStreamDestroy(p->copy);
    delete p;
}

clbm_status host_pipe(clbm_grid* g, HostPipe** out) {
    if (!g->pipe) {
        HostPipe* p = new (std::nothrow) HostPipe();
        if (!p) return fail(CLBM_ENOMEM, "host copy pipeline");
        const size_t nc = (size_t)g->n1 * g->n2;
        bool ok = cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking) == cudaSuccess;
        for (int k = 0; k < 2 && ok; ++k) {
            ok = cudaMalloc((void**)&p->in[k], (size_t)g->Q * nc * 8) == cudaSuccess &&
                 cudaMalloc((void**)&p->out[k], 3 * nc * 8) == cudaSuccess;
            for (cudaEvent_t* e : {&p->in_ready[k], &p->in_free[k], &p->out_ready[k], &p->out_free[k]})
                ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
        }
        if (!ok) {
            free_pipe(p);
            cudaGetLastError();
            return fail(CLBM_ENOMEM, "host copy pipeline: device buffers, stream or events");
        }
        g->pipe = p;
    }
    *out = g->pipe;
    return CLBM_OK;
}

// Ghost rows and columns of the current state (what the next collision
// pulls), rebuilt only after the state or the case was set from outside:
// every update fills those of the buffer it writes.
void fill_ghosts(clbm_grid* g) {
    if (g->ghosts_ok) return;
    StepArgs a = step_args(g, g->stA, g->stB);
    launch_boundary(g->Q, g->prec, a, g->stA, g->stream);
    g->launches++;
    g->ghosts_ok = true;
}

clbm_status rebuild_tables(clbm_grid* g) {
    launch_reference(g->Q, g->geo, g->n1 * g->ncol, g->cs.rho0, g->stream);
    launch_tables(g->Q, g->prec, g->geo, g->tab, g->ghost, g->n1, g->n2, g->ncol, g->bc_lo, g->bc_hi,
                  g->stream);
    launch_rest_mass(g->Q, g->geo, g->n1 * g->ncol, g->ncol == 1 ? g->n2 : 1, g->cs.rho0, g->red + NRED,
                     g->stream);
    g->launches += 4;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&g->rest_mass, g->red + NRED, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return CLBM_OK;
}

clbm_status check_case(const clbm_case* c) {
    if (!c) return fail(CLBM_EINVAL, "case is NULL");
    if (!(c->tau > 0.5) || !std::isfinite(c->tau)) return fail(CLBM_EINVAL, "tau must be > 1/2");
    if (!(c->rho0 > 0.0) || !std::isfinite(c->rho0)) return fail(CLBM_EINVAL, "rho0 must be > 0");
    if (!std::isfinite(c->u_wall_lo) || !std::isfinite(c->u_wall_hi) ||
        !std::isfinite(c->g_ext[0]) || !std::isfinite(c->g_ext[1]))
        return fail(CLBM_EINVAL, "non-finite wall speed or body force");
    if (c->force_iterations < 0 || c->force_iterations > 16)
        return fail(CLBM_EINVAL, "force_iterations must be in [0, 16]");
    return CLBM_OK;
}

}  // namespace

extern "C" {

const char* clbm_last_error(void) { return g_err; }

clbm_status clbm_workspace_bytes(const clbm_grid_desc* desc, size_t* bytes) {
    Layout L;
    int ld, h;
    clbm_status st = layout_of(desc, &L, &ld, &h);
    if (st != CLBM_OK) return st;
    if (!bytes) return fail(CLBM_EINVAL, "bytes is NULL");
    *bytes = L.total;
    return CLBM_OK;
}

clbm_status clbm_create_grid(const clbm_grid_desc* d, clbm_handle* out) {
    Range nvtx_range("clbm_create_grid");
    g_err[0] = 0;
    if (!out) return fail(CLBM_EINVAL, "out is NULL");
    *out = nullptr;
    Layout L;
    int ld, h;
    clbm_status st = layout_of(d, &L, &ld, &h);
    if (st != CLBM_OK) return st;
    if ((d->bc_lo != 0 && d->bc_lo != 1) || (d->bc_hi != 0 && d->bc_hi != 1))
        return fail(CLBM_EINVAL, "bad wall condition");
    const bool general = d->kind == CLBM_GEOM_GENERAL;
    const int ncol = general ? d->n2 : 1;
    std::vector<double> e, pos;
    double dx = d->dx;
    if (general) {
        if (!d->nodes) return fail(CLBM_EINVAL, "GENERAL needs nodes");
        if (!(d->dx > 0.0)) return fail(CLBM_EINVAL, "GENERAL needs dx > 0");
        pos.assign(d->nodes, d->nodes + (size_t)(d->n1 + 8) * (d->n2 + 8) * 2);
        for (double v : pos)
            if (!std::isfinite(v)) return fail(CLBM_EINVAL, "node positions must be finite");
    } else {
        if (!d->edges1) return fail(CLBM_EINVAL, "edges1 is NULL");
        e.assign(d->edges1, d->edges1 + d->n1 + 1);
        for (int k = 0; k < d->n1; ++k)
            if (!(e[k + 1] > e[k]) || !std::isfinite(e[k + 1]))
                return fail(CLBM_EINVAL, "edges1 must be finite and strictly increasing");
        if (d->kind == CLBM_GEOM_PLANAR && !(d->step2 > 0.0))
            return fail(CLBM_EINVAL, "step2 must be > 0");
        if (!(dx > 0.0)) dx = (e[d->n1] - e[0]) / d->n1;
        // node positions of rows -3..n1+4, columns -3..5 (1-based)
        pos.resize((size_t)(d->n1 + 8) * 9 * 2);
    }
    const double pi = 3.14159265358979323846;
    const int n2_period = d->n2_period > 0 ? d->n2_period : d->n2;
    if (d->kind == CLBM_GEOM_POLAR && n2_period < d->n2)
        return fail(CLBM_EINVAL, "n2_period (%d) < n2 (%d)", n2_period, d->n2);
    for (int i = -3; !general && i <= d->n1 + 4; ++i) {
        const double s = node_coord(e, d->n1, i);
        if (d->kind == CLBM_GEOM_POLAR && !(s > 0.0))
            return fail(CLBM_EINVAL, "mirrored ghost radius %g <= 0 at row %d: the annulus is "
                        "too thin at this resolution", s, i);
        for (int j = -3; j <= 5; ++j) {
            double* p = &pos[(((size_t)(i + 3)) * 9 + (j + 3)) * 2];
            if (d->kind == CLBM_GEOM_PLANAR) {
                p[0] = s;
                p[1] = (j - 0.5) * d->step2;
            } else {
                const double th = (j - 0.5) * (2.0 * pi / n2_period);
                p[0] = s * cos(th);
                p[1] = s * sin(th);
            }
        }
    }
    clbm_grid* g = new (std::nothrow) clbm_grid();
    if (!g) return fail(CLBM_ENOMEM, "host allocation failed");
    g->Q = d->lattice;
    g->prec = d->precision;
    g->n1 = d->n1;
    g->n2 = d->n2;
    g->n2_period = n2_period;
    g->ld = ld;
    g->h = h;
    g->kind = d->kind;
    g->bc_lo = d->bc_lo;
    g->bc_hi = d->bc_hi;
    g->device = d->device;
    g->dx = dx;
    g->stream = (cudaStream_t)d->stream;
    g->L = L;
    g->edges = e;
    g->step2 = d->step2;
    g->ncol = ncol;
    if (general) g->nodes = pos;
    cudaError_t ce = cudaSetDevice(d->device);
    if (ce != cudaSuccess) {
        delete g;
        return fail(CLBM_ECUDA, "cudaSetDevice(%d): %s", d->device, cudaGetErrorString(ce));
    }
    if (d->workspace) {
        if (d->workspace_bytes < L.total || ((uintptr_t)d->workspace & 255)) {
            delete g;
            return fail(CLBM_ENOMEM, "workspace needs %zu bytes aligned to 256, got %zu", L.total,
                        d->workspace_bytes);
        }
        g->ws = (char*)d->workspace;
        g->owns_ws = false;
    } else {
        ce = cudaMalloc((void**)&g->ws, L.total);
        if (ce != cudaSuccess) {
            delete g;
            return fail(CLBM_ENOMEM, "cudaMalloc(%zu): %s", L.total, cudaGetErrorString(ce));
        }
        g->owns_ws = true;
    }
    g->stA = g->ws + L.stA;
    g->stB = g->ws + L.stB;
    g->tab = g->ws + L.tab;
    g->geo = (double*)(g->ws + L.geo);
    g->wall_r = g->ws + L.wall_r;
    g->wall_u = g->ws + L.wall_u;
    g->ghost = (double*)(g->ws + L.ghost);
    g->pos = (double*)(g->ws + L.pos);
    g->partial = (double*)(g->ws + L.partial);
    g->red = (double*)(g->ws + L.red);
    g->prev = (double*)(g->ws + L.prev);
    g->err = (int*)(g->ws + L.err);
    g->phys[0] = g->stA;
    g->phys[1] = g->stB;
    cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, d->device);
    if (g->nsm <= 0) g->nsm = 1;
    ce = cudaMemsetAsync(g->ws, 0, L.total, g->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(g->pos, pos.data(), pos.size() * 8, cudaMemcpyHostToDevice, g->stream);
    if (ce == cudaSuccess) {
        launch_geometry(g->Q, g->pos, g->n1, ncol, dx, d->kind != CLBM_GEOM_PLANAR, g->geo, g->stream);
        g->launches++;
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(g->stream);
    if (ce != cudaSuccess) {
        clbm_destroy(g);
        return fail(CLBM_ECUDA, "geometry precompute: %s", cudaGetErrorString(ce));
    }
    if (g->prec != CLBM_FP64) {
        int major = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, d->device);
        if (major >= 9 && make_tma_maps(g->Q, g->prec, &g->tma, g->phys[0], g->phys[1], g->n1, g->n2,
                                        g->ld) != 0)
            g->tma = nullptr;
    }
    // every cell volume must be positive
    std::vector<double> geo((size_t)g->n1 * ncol * Geo::stride(g->Q));
    ce = cudaMemcpy(geo.data(), g->geo, geo.size() * 8, cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) {
        clbm_destroy(g);
        return fail(CLBM_ECUDA, "geometry readback: %s", cudaGetErrorString(ce));
    }
    for (size_t r = 0; r < (size_t)g->n1 * ncol; ++r)
        if (!(geo[r * Geo::stride(g->Q) + Geo::J] > 0.0)) {
            clbm_destroy(g);
            return fail(CLBM_EINVAL, "cell volume J <= 0 at row %d, column %d", (int)(r / ncol) + 1,
                        (int)(r % ncol) + 1);
        }
    *out = g;
    return CLBM_OK;
}

clbm_status clbm_set_case(clbm_handle g, const clbm_case* c) {
    Range nvtx_range("clbm_set_case");
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    clbm_status st = check_case(c);
    if (st != CLBM_OK) return st;
    st = select(g);
    if (st != CLBM_OK) return st;
    g->cs = *c;
    g->have_case = true;
    st = rebuild_tables(g);
    if (st != CLBM_OK) return st;
    launch_state_from_fp64(g->Q, g->prec, nullptr, g->geo, g->stA, g->n1, g->n2, g->ld, g->h, g->ncol,
                           g->stream);
    launch_wall_init(g->prec, g->wall_r, g->wall_u, nullptr, nullptr, g->n1, g->n2, g->h,
                     c->rho0, g->stream);
    g->launches += 2;
    CK(cudaGetLastError());
    g->t = 0;
    g->have_prev = false;
    g->ghosts_ok = false;
    return CLBM_OK;
}

clbm_status clbm_set_state(clbm_handle g, const double* Np, const double* rho_prev,
                           const double* ut2_prev, int src_is_device) {
    Range nvtx_range("clbm_set_state");
    if (!g || !Np) return fail(CLBM_EINVAL, "handle or Np is NULL");
    if (!g->have_case) return fail(CLBM_EINVAL, "call clbm_set_case first");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    const size_t nc = (size_t)g->n1 * g->n2, nq = nc * g->Q;
    const double *dN = Np, *dr = rho_prev, *du = ut2_prev;
    if (!src_is_device) {
        double* sb = nullptr;
        st = staging(g, &sb);
        if (st != CLBM_OK) return st;
        // the staging buffer holds max(Q, 7) fields: state, then the two moment fields
        CK(cudaMemcpyAsync(sb, Np, nq * 8, cudaMemcpyHostToDevice, g->stream));
        dN = sb;
        dr = du = nullptr;
        double* extra = nullptr;
        struct FreeOnExit {
            double** p;
            ~FreeOnExit() { cudaFree(*p); }
        } guard{&extra};
        if (rho_prev || ut2_prev) {
            CK(cudaMalloc((void**)&extra, 2 * nc * 8));
            if (rho_prev) {
                CK(cudaMemcpyAsync(extra, rho_prev, nc * 8, cudaMemcpyHostToDevice, g->stream));
                dr = extra;
            }
            if (ut2_prev) {
                CK(cudaMemcpyAsync(extra + nc, ut2_prev, nc * 8, cudaMemcpyHostToDevice, g->stream));
                du = extra + nc;
            }
        }
        launch_state_from_fp64(g->Q, g->prec, dN, g->geo, g->stA, g->n1, g->n2, g->ld, g->h, g->ncol,
                               g->stream);
        launch_wall_init(g->prec, g->wall_r, g->wall_u, dr, du, g->n1, g->n2, g->h, g->cs.rho0,
                         g->stream);
        g->launches += 2;
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(g->stream));
    } else {
        launch_state_from_fp64(g->Q, g->prec, dN, g->geo, g->stA, g->n1, g->n2, g->ld, g->h, g->ncol,
                               g->stream);
        launch_wall_init(g->prec, g->wall_r, g->wall_u, dr, du, g->n1, g->n2, g->h, g->cs.rho0,
                         g->stream);
        g->launches += 2;
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(g->stream));
    }
    g->have_prev = false;
    g->ghosts_ok = false;
    return CLBM_OK;
}

clbm_status clbm_set_equilibrium(clbm_handle g, const double* rho, const double* U1,
                                 const double* U2, int src_is_device) {
    Range nvtx_range("clbm_set_equilibrium");
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    if (!g->have_case) return fail(CLBM_EINVAL, "call clbm_set_case first");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    const size_t nc = (size_t)g->n1 * g->n2;
    double* sb = nullptr;
    st = staging(g, &sb);
    if (st != CLBM_OK) return st;
    const double *dr = rho, *d1 = U1, *d2 = U2;
    if (!src_is_device) {
        // host fields go to the last three staging fields, which the
        // equilibrium kernel overwrites cell by cell after reading them
        double* f = sb + (size_t)(g->Q - 3) * nc;
        const double* src[3] = {rho, U1, U2};
        const double** dst[3] = {&dr, &d1, &d2};
        for (int k = 0; k < 3; ++k) {
            if (!src[k]) continue;
            CK(cudaMemcpyAsync(f + k * nc, src[k], nc * 8, cudaMemcpyHostToDevice, g->stream));
            *dst[k] = f + k * nc;
        }
    }
    // wall moments of the "last collision": rho and Ut^2 of the start
    launch_wall_init(g->prec, g->wall_r, g->wall_u, dr, d2, g->n1, g->n2, g->h, g->cs.rho0, g->stream);
    launch_equilibrium(g->Q, dr, d1, d2, g->geo, sb, g->n1, g->n2, g->ncol, g->cs.rho0, g->stream);
    launch_state_from_fp64(g->Q, g->prec, sb, g->geo, g->stA, g->n1, g->n2, g->ld, g->h, g->ncol,
                           g->stream);
    g->launches += 3;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(g->stream));
    g->t = 0;
    g->have_prev = false;
    g->ghosts_ok = false;
    return check_err(g);
}

clbm_status clbm_get_state(clbm_handle g, double* Np, int dst_is_device) {
    Range nvtx_range("clbm_get_state");
    if (!g || !Np) return fail(CLBM_EINVAL, "handle or Np is NULL");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    const size_t nq = (size_t)g->n1 * g->n2 * g->Q;
    double* dN = Np;
    if (!dst_is_device) {
        st = staging(g, &dN);
        if (st != CLBM_OK) return st;
    }
    launch_state_to_fp64(g->Q, g->prec, g->stA, g->geo, dN, g->n1, g->n2, g->ld, g->h, g->ncol,
                         g->stream);
    g->launches++;
    CK(cudaGetLastError());
    if (!dst_is_device) {
        CK(cudaMemcpyAsync(Np, dN, nq * 8, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
    } else {
        CK(cudaStreamSynchronize(g->stream));
    }
    return CLBM_OK;
}

// One launch of the fused update from stA into stB (no bookkeeping).
static clbm_status launch_update(clbm_grid* g, const StepArgs& a) {
    if (use_tma(g)) {
        const int src = a.src == g->phys[0] ? 0 : 1;
        const int rc = general_grid(g)
                           ? launch_step_tma_general(g->Q, g->prec, *g->tma, a, src, g->nsm, g->stream)
                           : launch_step_tma(g->Q, g->prec, *g->tma, a, src, g->nsm, tma_mode(g), g->stream);
        if (rc != 0) return fail(CLBM_ECUDA, "TMA-staged update could not be launched");
    } else {
        launch_step(g->Q, g->prec, a, g->stream);
    }
    return CLBM_OK;
}

// step_run's answer when the cooperative launch was refused under the
// automatic choice (internal, never returned by the C ABI).
constexpr clbm_status CLBM_EAGAIN_RUN = (clbm_status)-100;

// nsteps time steps in one multi-step launch (recorded as a whole while
// profiling, counted as nsteps launches of the update).
static clbm_status step_run(clbm_grid* g, int nsteps) {
    if (!g->prog) {
        const size_t bytes = (size_t)(g->nsm + 1) * sizeof(unsigned long long);
        CK(cudaMalloc((void**)&g->prog, bytes));
        CK(cudaMemsetAsync(g->prog, 0, bytes, g->stream));
    }
    if (++g->run_epoch == 0) g->run_epoch = 1;   // 0 marks words no run wrote
    const StepArgs a = step_args(g, g->stA, g->stB);
    const int src = a.src == g->phys[0] ? 0 : 1;
    if (g->profiling) {
        if (g->ev_used + 2 > g->ev.size()) {
            for (int k = 0; k < 256; ++k) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                g->ev.push_back(e);
            }
        }
        CK(cudaEventRecord(g->ev[g->ev_used], g->stream));
    }
    const cudaError_t e = launch_step_tma_run(g->Q, g->prec, *g->tma, a, src, g->nsm, tma_mode(g), nsteps,
                                              g->prog, g->run_epoch, g->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (e == cudaErrorCooperativeLaunchTooLarge && g->variant == 0) {
            // not every CTA can be resident (another context holds SMs):
            // nothing was launched, the caller steps one launch at a time
            g->run_refused = true;
            return CLBM_EAGAIN_RUN;
        }
        return fail(CLBM_ECUDA, "multi-step update could not be launched: %s", cudaGetErrorString(e));
    }
    if (g->profiling) {
        CK(cudaEventRecord(g->ev[g->ev_used + 1], g->stream));
        g->ev_used += 2;
        g->ev_launches += nsteps;
        g->prof_count += nsteps;
    }
    g->launches += 1;
    if (nsteps & 1) std::swap(g->stA, g->stB);
    g->t += nsteps;
    return CLBM_OK;
}

// One time step with plain launches (and the sampled profiling events).
static clbm_status step_plain(clbm_grid* g) {
    const StepArgs a = step_args(g, g->stA, g->stB);
    const bool timed = g->profiling && g->prof_count++ % g->prof_period == 0;
    if (timed) {
        if (g->ev_used + 2 > g->ev.size()) {
            for (int k = 0; k < 256; ++k) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                g->ev.push_back(e);
            }
        }
        CK(cudaEventRecord(g->ev[g->ev_used], g->stream));
    }
    const clbm_status st = launch_update(g, a);
    if (st != CLBM_OK) return st;
    if (timed) {
        CK(cudaEventRecord(g->ev[g->ev_used + 1], g->stream));
        g->ev_used += 2;
        g->ev_launches += 1;
    }
    g->launches += 1;
    std::swap(g->stA, g->stB);
    g->t++;
    return CLBM_OK;
}

constexpr int GRAPH_STEPS = 10;

// Capture GRAPH_STEPS launches from the current stA into a graph; false (and
// plain launches from then on) if the capture or the instantiation fails.
static bool capture_graph(clbm_grid* g) {
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->graph) cudaGraphDestroy(g->graph);
    g->gexec = nullptr;
    g->graph = nullptr;
    // (the legacy default stream cannot be captured: such grids keep to
    // plain launches)
    if ((!g->gdummy[0] && (cudaEventCreate(&g->gdummy[0]) != cudaSuccess ||
                           cudaEventCreate(&g->gdummy[1]) != cudaSuccess)) ||
        cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        g->graphs_off = true;
        return false;
    }
    cudaGraph_t graph = nullptr;
    void* a = g->stA;
    void* b = g->stB;
    bool ok = true;
    ok = cudaEventRecordWithFlags(g->gdummy[0], g->stream, cudaEventRecordExternal) == cudaSuccess;
    for (int k = 0; k < GRAPH_STEPS && ok; ++k) {
        ok = launch_update(g, step_args(g, a, b)) == CLBM_OK;
        std::swap(a, b);
    }
    if (ok) ok = cudaEventRecordWithFlags(g->gdummy[1], g->stream, cudaEventRecordExternal) == cudaSuccess;
    const bool ended = cudaStreamEndCapture(g->stream, &graph) == cudaSuccess;
    ok = ok && ended && graph;
    if (ok) {
        // the two event-record nodes, to be pointed at the profiling events
        size_t nn = 0;
        ok = cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess;
        std::vector<cudaGraphNode_t> nodes(nn);
        if (ok) ok = cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess;
        g->gev[0] = g->gev[1] = nullptr;
        for (size_t k = 0; ok && k < nn; ++k) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nodes[k], &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t e;
            if (cudaGraphEventRecordNodeGetEvent(nodes[k], &e) != cudaSuccess) continue;
            if (e == g->gdummy[0]) g->gev[0] = nodes[k];
            if (e == g->gdummy[1]) g->gev[1] = nodes[k];
        }
        ok = ok && g->gev[0] && g->gev[1] &&
             cudaGraphInstantiate(&g->gexec, graph, 0) == cudaSuccess;
    }
    cudaGetLastError();   // a failed capture leaves its error behind; plain launches report their own
    if (!ok) {
        if (g->gexec) cudaGraphExecDestroy(g->gexec);
        if (graph) cudaGraphDestroy(graph);
        g->gexec = nullptr;
        g->graphs_off = true;
        return false;
    }
    g->graph = graph;
    g->gargs = step_args(g, g->stA, g->stB);
    g->gpath[0] = use_tma(g);
    g->gpath[1] = general_grid(g);
    g->gpath[2] = g->variant;
    g->gpath[3] = g->nsm;
    return true;
}

// Whether the graph replays exactly what plain launches from stA would do.
static bool graph_matches(const clbm_grid* g) {
    if (!g->gexec) return false;
    const StepArgs a = step_args(g, g->stA, g->stB);
    return memcmp(&a, &g->gargs, sizeof a) == 0 && g->gpath[0] == (int)use_tma(g) &&
           g->gpath[1] == (int)general_grid(g) && g->gpath[2] == g->variant && g->gpath[3] == g->nsm;
}

// One replay of the graph: GRAPH_STEPS time steps.
static clbm_status step_graph(clbm_grid* g) {
    cudaEvent_t e0 = g->gdummy[0], e1 = g->gdummy[1];
    if (g->profiling) {
        // a replay is timed as a whole: its GRAPH_STEPS back-to-back launches
        if (g->ev_used + 2 > g->ev.size()) {
            for (int k = 0; k < 256; ++k) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                g->ev.push_back(e);
            }
        }
        e0 = g->ev[g->ev_used];
        e1 = g->ev[g->ev_used + 1];
        g->ev_used += 2;
        g->ev_launches += GRAPH_STEPS;
        g->prof_count += GRAPH_STEPS;
    }
    if (cudaGraphExecEventRecordNodeSetEvent(g->gexec, g->gev[0], e0) != cudaSuccess ||
        cudaGraphExecEventRecordNodeSetEvent(g->gexec, g->gev[1], e1) != cudaSuccess) {
        // not expected; keep to plain launches rather than fail the step
        cudaGetLastError();
        if (g->profiling) {
            g->ev_used -= 2;
            g->ev_launches -= GRAPH_STEPS;
            g->prof_count -= GRAPH_STEPS;
        }
        g->graphs_off = true;
        for (int k = 0; k < GRAPH_STEPS; ++k) {
            const clbm_status st = step_plain(g);
            if (st != CLBM_OK) return st;
        }
        return CLBM_OK;
    }
    CK(cudaGraphLaunch(g->gexec, g->stream));
    g->launches += GRAPH_STEPS;
    g->t += GRAPH_STEPS;
    return CLBM_OK;
}

clbm_status clbm_step(clbm_handle g, long long n) {
    Range nvtx_range("clbm_step");
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    if (!g->have_case) return fail(CLBM_EINVAL, "call clbm_set_case first");
    if (n < 0) return fail(CLBM_EINVAL, "n < 0");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    fill_ghosts(g);
    long long s = 0;
    if (use_run(g)) {
        for (; s < n; s += RUN_MAX_STEPS) {
            st = step_run(g, (int)std::min<long long>(n - s, RUN_MAX_STEPS));
            if (st == CLBM_EAGAIN_RUN) break;   // refused: the rest with a launch per step
            if (st != CLBM_OK) return st;
        }
        if (s >= n) {
            CK(cudaGetLastError());
            return CLBM_OK;
        }
    }
    // long runs replay a captured graph of GRAPH_STEPS launches: one host call
    // per replay instead of one per launch, so the device never waits on the
    // host.  Before a capture two plain launches set the kernels up
    // (attributes) and bring the buffers back to the parity they started
    // from, so that runs of an even number of steps replay from their start
    if (!g->graphs_off && n >= 2 * GRAPH_STEPS + 2) {
        if (!graph_matches(g)) {
            std::swap(g->stA, g->stB);   // the graph as seen from the other parity
            const bool other = graph_matches(g);
            std::swap(g->stA, g->stB);
            for (const long long k = other ? 1 : 2; s < k; ++s) {
                st = step_plain(g);
                if (st != CLBM_OK) return st;
            }
            if (!other) capture_graph(g);
        }
        if (graph_matches(g)) {
            for (; n - s >= GRAPH_STEPS; s += GRAPH_STEPS) {
                st = step_graph(g);
                if (st != CLBM_OK) return st;
            }
        }
    }
    for (; s < n; ++s) {
        st = step_plain(g);
        if (st != CLBM_OK) return st;
    }
    CK(cudaGetLastError());
    return CLBM_OK;
}

clbm_status clbm_moments(clbm_handle g, double* rho, double* U1, double* U2, double* Ut1,
                         double* Ut2, double* F1, double* F2, int dst_is_device) {
    Range nvtx_range("clbm_moments");
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    if (!g->have_case) return fail(CLBM_EINVAL, "call clbm_set_case first");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    const size_t nc = (size_t)g->n1 * g->n2;
    double* outs[7] = {rho, U1, U2, Ut1, Ut2, F1, F2};
    double* dev[7] = {nullptr};
    double* tmp = nullptr;
    if (!dst_is_device) {
        st = staging(g, &tmp);
        if (st != CLBM_OK) return st;
        int at = 0;
        for (int k = 0; k < 7; ++k)
            if (outs[k]) dev[k] = tmp + (at++) * nc;
    } else {
        for (int k = 0; k < 7; ++k) dev[k] = outs[k];
    }
    fill_ghosts(g);
    MomArgs m = mom_args(g);
    m.rho = dev[0];
    m.U1 = dev[1];
    m.U2 = dev[2];
    m.Ut1 = dev[3];
    m.Ut2 = dev[4];
    m.F1 = dev[5];
    m.F2 = dev[6];
    launch_moments(g->Q, g->prec, m, g->cs.force_iterations, 0, g->stream);
    g->launches++;
    CK(cudaGetLastError());
    if (!dst_is_device)
        for (int k = 0; k < 7; ++k)
            if (outs[k]) CK(cudaMemcpyAsync(outs[k], dev[k], nc * 8, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return check_err(g);
}

clbm_status clbm_upload_state_async(clbm_handle g, const double* Np) {
    Range nvtx_range("clbm_upload_state_async");
    if (!g || !Np) return fail(CLBM_EINVAL, "handle or Np is NULL");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    HostPipe* p = nullptr;
    st = host_pipe(g, &p);
    if (st != CLBM_OK) return st;
    if (p->staged == 2) return fail(CLBM_EBUSY, "two uploads wait already: set one first");
    const int s = p->next_in;
    // the slot is free once the conversion that read it last has run
    if (p->in_used[s]) CK(cudaStreamWaitEvent(p->copy, p->in_free[s], 0));
    CK(cudaMemcpyAsync(p->in[s], Np, (size_t)g->Q * g->n1 * g->n2 * 8, cudaMemcpyHostToDevice, p->copy));
    CK(cudaEventRecord(p->in_ready[s], p->copy));
    p->in_used[s] = true;
    p->next_in ^= 1;
    p->staged++;
    return CLBM_OK;
}

clbm_status clbm_set_uploaded_state(clbm_handle g) {
    Range nvtx_range("clbm_set_uploaded_state");
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    if (!g->have_case) return fail(CLBM_EINVAL, "call clbm_set_case first");
    if (!g->pipe || g->pipe->staged == 0) return fail(CLBM_EINVAL, "no upload waits to be set");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    HostPipe* p = g->pipe;
    const int s = p->next_set;
    CK(cudaStreamWaitEvent(g->stream, p->in_ready[s], 0));
    launch_state_from_fp64(g->Q, g->prec, p->in[s], g->geo, g->stA, g->n1, g->n2, g->ld, g->h, g->ncol,
                           g->stream);
    launch_wall_init(g->prec, g->wall_r, g->wall_u, nullptr, nullptr, g->n1, g->n2, g->h, g->cs.rho0,
                     g->stream);
    g->launches += 2;
    CK(cudaGetLastError());
    CK(cudaEventRecord(p->in_free[s], g->stream));
    p->next_set ^= 1;
    p->staged--;
    g->have_prev = false;
    g->ghosts_ok = false;
    return CLBM_OK;
}

clbm_status clbm_download_moments_async(clbm_handle g, double* rho, double* Ut1, double* Ut2) {
    Range nvtx_range("clbm_download_moments_async");
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    if (!g->have_case) return fail(CLBM_EINVAL, "call clbm_set_case first");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    HostPipe* p = nullptr;
    st = host_pipe(g, &p);
    if (st != CLBM_OK) return st;
    const size_t nc = (size_t)g->n1 * g->n2;
    const int s = p->next_out;
    // the slot is free once the copies that read it last have landed
    if (p->out_used[s]) CK(cudaStreamWaitEvent(g->stream, p->out_free[s], 0));
    fill_ghosts(g);
    MomArgs m = mom_args(g);
    m.rho = p->out[s];
    m.Ut1 = p->out[s] + nc;
    m.Ut2 = p->out[s] + 2 * nc;
    launch_moments(g->Q, g->prec, m, g->cs.force_iterations, 0, g->stream);
    g->launches++;
    CK(cudaGetLastError());
    CK(cudaEventRecord(p->out_ready[s], g->stream));
    CK(cudaStreamWaitEvent(p->copy, p->out_ready[s], 0));
    double* dst[3] = {rho, Ut1, Ut2};
    for (int k = 0; k < 3; ++k)
        if (dst[k]) CK(cudaMemcpyAsync(dst[k], p->out[s] + k * nc, nc * 8, cudaMemcpyDeviceToHost, p->copy));
    CK(cudaEventRecord(p->out_free[s], p->copy));
    p->out_used[s] = true;
    p->next_out ^= 1;
    return CLBM_OK;
}

clbm_status clbm_wait_copies(clbm_handle g) {
    Range nvtx_range("clbm_wait_copies");
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    if (g->pipe) CK(cudaStreamSynchronize(g->pipe->copy));
    return check_err(g);
}

clbm_status clbm_fill_ghosts(clbm_handle g) {
    Range nvtx_range("clbm_fill_ghosts");
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    if (!g->have_case) return fail(CLBM_EINVAL, "call clbm_set_case first");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    fill_ghosts(g);
    CK(cudaGetLastError());
    return CLBM_OK;
}

clbm_status clbm_halo_values(clbm_handle g, size_t* values) {
    if (!g || !values) return fail(CLBM_EINVAL, "NULL argument");
    *values = (size_t)halo_entries(g->Q) * (g->n1 + 2 * g->h);
    return CLBM_OK;
}

clbm_status clbm_halo_pack(clbm_handle g, int side, void* buf) {
    Range nvtx_range("clbm_halo_pack");
    if (!g || !buf) return fail(CLBM_EINVAL, "handle or buf is NULL");
    if (side != 0 && side != 1) return fail(CLBM_EINVAL, "side must be 0 or 1");
    if (g->n2 < g->h) return fail(CLBM_EINVAL, "a slab needs n2 >= %d columns", g->h);
    if (g->ncol != 1) return fail(CLBM_EINVAL, "halo strips need a planar or polar grid");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    launch_halo(g->Q, g->prec, g->stA, buf, (long long)(g->n1 + 2 * g->h) * g->ld, g->ld, g->n1 + 2 * g->h,
                g->n2, side, 0, g->stream);
    g->launches++;
    CK(cudaGetLastError());
    return CLBM_OK;
}

clbm_status clbm_halo_unpack(clbm_handle g, int side, const void* buf) {
    Range nvtx_range("clbm_halo_unpack");
    if (!g || !buf) return fail(CLBM_EINVAL, "handle or buf is NULL");
    if (side != 0 && side != 1) return fail(CLBM_EINVAL, "side must be 0 or 1");
    if (g->n2 < g->h) return fail(CLBM_EINVAL, "a slab needs n2 >= %d columns", g->h);
    if (g->ncol != 1) return fail(CLBM_EINVAL, "halo strips need a planar or polar grid");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    launch_halo(g->Q, g->prec, g->stA, const_cast<void*>(buf), (long long)(g->n1 + 2 * g->h) * g->ld, g->ld,
                g->n1 + 2 * g->h, g->n2, side, 1, g->stream);
    g->launches++;
    CK(cudaGetLastError());
    return CLBM_OK;
}

}  // extern "C"

namespace {

// The residual / conservation sums of the current state (slots of NRED, the
// rest part of the mass added) and the steps since the last call (0 on the
// first); moves the snapshot to this state.
clbm_status residual_sums(clbm_grid* g, double (&v)[NRED], long long* dt_out) {
    if (!g->have_case) return fail(CLBM_EINVAL, "call clbm_set_case first");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    fill_ghosts(g);
    MomArgs m = mom_args(g);
    m.have_prev = g->have_prev ? 1 : 0;
    // the pipelined pass where the update runs pipelined, else one thread
    // per cell loading from global memory
    int nb = -1;
    if (use_tma(g) && !general_grid(g))
        nb = launch_residual_tma(g->Q, g->prec, *g->tma, m, g->stA == g->phys[0] ? 0 : 1, g->nsm, g->stream);
    if (nb < 0) {
        launch_moments(g->Q, g->prec, m, g->cs.force_iterations, 1, g->stream);
        nb = moments_blocks(g->n1, g->n2);
    }
    launch_reduce_final(g->partial, nb, g->red, g->stream);
    g->launches += 2;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(v, g->red, sizeof(v), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    st = check_err(g);
    if (st != CLBM_OK) return st;
    *dt_out = g->have_prev ? g->t - g->t_prev : 0;
    v[2] += g->rest_mass;
    g->have_prev = true;
    g->t_prev = g->t;
    return CLBM_OK;
}

clbm_status unstable_status(const clbm_grid* g, const double (&v)[NRED]) {
    if (v[8] > 0.0 || !std::isfinite(v[2]))
        return fail(CLBM_EUNSTABLE, "%g cells with a non-finite or non-positive density at t=%lld",
                    v[8], g->t);
    return CLBM_OK;
}

}  // namespace

extern "C" {

clbm_status clbm_residual(clbm_handle g, double* res, double cons[6]) {
    Range nvtx_range("clbm_residual");
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    double v[NRED];
    long long dt = 0;
    clbm_status st = residual_sums(g, v, &dt);
    if (st != CLBM_OK) return st;
    double r = INFINITY;
    if (dt > 0) r = v[1] > 0.0 ? sqrt(v[0]) / (dt * sqrt(v[1])) : (v[0] > 0 ? INFINITY : 0.0);
    if (res) *res = r;
    if (cons)
        for (int k = 0; k < 6; ++k) cons[k] = v[2 + k];
    return unstable_status(g, v);
}

clbm_status clbm_residual_parts(clbm_handle g, double parts[9], long long* dt) {
    Range nvtx_range("clbm_residual_parts");
    if (!g || !parts || !dt) return fail(CLBM_EINVAL, "NULL argument");
    double v[NRED];
    clbm_status st = residual_sums(g, v, dt);
    if (st != CLBM_OK) return st;
    for (int k = 0; k < 9; ++k) parts[k] = v[k];
    return unstable_status(g, v);
}


clbm_status clbm_no_flow_adjust(clbm_handle g, long long nsteps, double* rho_nf) {
    Range nvtx_range("clbm_no_flow_adjust");
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    if (!g->have_case) return fail(CLBM_EINVAL, "call clbm_set_case first");
    if (nsteps < 0) return fail(CLBM_EINVAL, "nsteps < 0");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    // FP64 clone of the grid with the walls at rest and no body force.
    clbm_grid_desc d;
    memset(&d, 0, sizeof(d));
    d.lattice = g->Q;
    d.precision = CLBM_FP64;
    d.n1 = g->n1;
    d.n2 = g->n2;
    d.kind = g->kind;
    d.edges1 = g->edges.empty() ? nullptr : g->edges.data();
    d.nodes = g->nodes.empty() ? nullptr : g->nodes.data();
    d.step2 = g->step2;
    d.dx = g->dx;
    d.bc_lo = g->bc_lo;
    d.bc_hi = g->bc_hi;
    d.device = g->device;
    d.stream = g->stream;
    d.n2_period = g->n2_period;
    clbm_handle nf = nullptr;
    st = clbm_create_grid(&d, &nf);
    if (st != CLBM_OK) return st;
    clbm_case c0 = g->cs;
    c0.u_wall_lo = c0.u_wall_hi = 0.0;
    c0.g_ext[0] = c0.g_ext[1] = 0.0;
    const size_t nc = (size_t)g->n1 * g->n2, nq = nc * g->Q;
    double *rho = nullptr, *rowm = nullptr, *Np = nullptr;
    st = clbm_set_case(nf, &c0);
    if (st == CLBM_OK) st = clbm_step(nf, nsteps);
    if (st == CLBM_OK && (cudaMalloc((void**)&rho, nc * 8) != cudaSuccess ||
                          cudaMalloc((void**)&rowm, g->n1 * 8) != cudaSuccess ||
                          cudaMalloc((void**)&Np, nq * 8) != cudaSuccess))
        st = fail(CLBM_ENOMEM, "no-flow scratch allocation failed");
    if (st == CLBM_OK) st = clbm_moments(nf, rho, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 1);
    if (st == CLBM_OK) st = clbm_get_state(nf, Np, 1);
    if (st == CLBM_OK) {
        // Eq. 23: J <- J rho_nf / rho0 (the row mean of rho_nf where one
        // geometry row serves the whole row), then references and tables anew
        if (g->ncol == 1) {
            launch_row_mean(rho, g->n1, g->n2, rowm, g->stream);
            g->launches++;
        }
        launch_scale_volume(g->Q, g->geo, g->ncol == 1 ? rowm : rho, g->n1 * g->ncol, g->cs.rho0,
                            g->stream);
        g->launches++;
        st = rebuild_tables(g);
    }
    if (st == CLBM_OK) {
        // keep the no-flow state; its last-collision densities scale by rho0/rho_nf
        launch_state_from_fp64(g->Q, g->prec, Np, g->geo, g->stA, g->n1, g->n2, g->ld, g->h, g->ncol,
                               g->stream);
        launch_wall_copy(g->prec, g->wall_r, g->wall_u, (const double*)nf->wall_r,
                         (const double*)nf->wall_u, g->ncol == 1 ? rowm : rho, g->n1, g->n2, g->h,
                         g->cs.rho0, g->ncol, g->stream);
        g->launches += 2;
        if (cudaGetLastError() != cudaSuccess) st = fail(CLBM_ECUDA, "no-flow state transfer failed");
    }
    if (st == CLBM_OK && rho_nf &&
        cudaMemcpyAsync(rho_nf, rho, nc * 8, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
        st = fail(CLBM_ECUDA, "rho_nf copy failed");
    if (st == CLBM_OK && cudaStreamSynchronize(g->stream) != cudaSuccess)
        st = fail(CLBM_ECUDA, "no-flow synchronise failed");
    g->launches += nf->launches;
    cudaFree(rho);
    cudaFree(rowm);
    cudaFree(Np);
    clbm_destroy(nf);
    g->t = 0;
    g->have_prev = false;
    g->ghosts_ok = false;
    return st;
}

clbm_status clbm_time(clbm_handle g, long long* t) {
    if (!g || !t) return fail(CLBM_EINVAL, "NULL argument");
    *t = g->t;
    return CLBM_OK;
}

clbm_status clbm_set_stream(clbm_handle g, void* stream) {
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    g->stream = (cudaStream_t)stream;
    return CLBM_OK;
}

clbm_status clbm_set_profiling(clbm_handle g, int period) {
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    if (period < 0) return fail(CLBM_EINVAL, "period < 0");
    g->profiling = period > 0;
    g->prof_period = period > 0 ? period : 1;
    g->prof_count = 0;
    g->ev_used = 0;
    g->ev_launches = 0;
    return CLBM_OK;
}

clbm_status clbm_kernel_time(clbm_handle g, double* ms, long long* launches) {
    if (!g || !ms || !launches) return fail(CLBM_EINVAL, "NULL argument");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    CK(cudaStreamSynchronize(g->stream));
    double tot = 0.0;
    for (size_t k = 0; k + 1 < g->ev_used; k += 2) {
        float x = 0.f;
        CK(cudaEventElapsedTime(&x, g->ev[k], g->ev[k + 1]));
        tot += x;
    }
    *ms = tot;
    *launches = g->ev_launches;
    g->ev_used = 0;
    g->ev_launches = 0;
    return CLBM_OK;
}

clbm_status clbm_set_kernel(clbm_handle g, int variant) {
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    if (variant < 0 || variant > 6) return fail(CLBM_EINVAL, "variant must be 0 .. 6");
    if (variant >= 2 && !g->tma)
        return fail(CLBM_EINVAL, "the TMA-staged update needs 16/32-bit storage on sm_90 or newer");
    if ((variant == 2 || variant >= 4) && general_grid(g))
        return fail(CLBM_EINVAL, "general grids run kernel 1 or 3 (kernels 2, 4, 5 and 6 read row tables)");
    g->variant = variant;
    return CLBM_OK;
}

clbm_status clbm_launch_count(clbm_handle g, long long* launches) {
    if (!g || !launches) return fail(CLBM_EINVAL, "NULL argument");
    *launches = g->launches;
    return CLBM_OK;
}

// Checkpoint: header (sizes, case, time counters), then the raw current state
// buffer (ghosts included), the wall moments of the last collision, the
// residual snapshot and the geometry (which carries a no-flow adjustment of J).
struct CkptHeader {
    char magic[8];
    int Q, prec, n1, n2, ld, ncol;
    long long t, t_prev;
    int have_prev;
    clbm_case cs;
    size_t state_bytes, wall_bytes, prev_bytes, geo_bytes;
};

static void ckpt_sizes(const clbm_grid* g, CkptHeader* h) {
    memset(h, 0, sizeof(*h));
    memcpy(h->magic, "CLBMCKP1", 8);
    h->Q = g->Q;
    h->prec = g->prec;
    h->n1 = g->n1;
    h->n2 = g->n2;
    h->ld = g->ld;
    h->ncol = g->ncol;
    h->t = g->t;
    h->t_prev = g->t_prev;
    h->have_prev = g->have_prev ? 1 : 0;
    h->cs = g->cs;
    h->state_bytes = g->L.stB - g->L.stA;
    h->wall_bytes = g->L.wall_u - g->L.wall_r;
    h->prev_bytes = (size_t)2 * g->n1 * g->n2 * 8;
    h->geo_bytes = (size_t)g->n1 * g->ncol * Geo::stride(g->Q) * 8;
}

clbm_status clbm_checkpoint_bytes(clbm_handle g, size_t* bytes) {
    if (!g || !bytes) return fail(CLBM_EINVAL, "NULL argument");
    CkptHeader h;
    ckpt_sizes(g, &h);
    *bytes = sizeof(h) + h.state_bytes + 2 * h.wall_bytes + h.prev_bytes + h.geo_bytes;
    return CLBM_OK;
}

clbm_status clbm_checkpoint(clbm_handle g, void* buf) {
    Range nvtx_range("clbm_checkpoint");
    if (!g || !buf) return fail(CLBM_EINVAL, "NULL argument");
    if (!g->have_case) return fail(CLBM_EINVAL, "call clbm_set_case first");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    fill_ghosts(g);  // the saved buffer is complete, ghosts included
    CkptHeader h;
    ckpt_sizes(g, &h);
    char* p = (char*)buf;
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    CK(cudaMemcpyAsync(p, g->stA, h.state_bytes, cudaMemcpyDeviceToHost, g->stream));
    p += h.state_bytes;
    CK(cudaMemcpyAsync(p, g->wall_r, h.wall_bytes, cudaMemcpyDeviceToHost, g->stream));
    p += h.wall_bytes;
    CK(cudaMemcpyAsync(p, g->wall_u, h.wall_bytes, cudaMemcpyDeviceToHost, g->stream));
    p += h.wall_bytes;
    CK(cudaMemcpyAsync(p, g->prev, h.prev_bytes, cudaMemcpyDeviceToHost, g->stream));
    p += h.prev_bytes;
    CK(cudaMemcpyAsync(p, g->geo, h.geo_bytes, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return check_err(g);
}

clbm_status clbm_restore(clbm_handle g, const void* buf) {
    Range nvtx_range("clbm_restore");
    if (!g || !buf) return fail(CLBM_EINVAL, "NULL argument");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    CkptHeader h, mine;
    memcpy(&h, buf, sizeof(h));
    ckpt_sizes(g, &mine);
    if (memcmp(h.magic, mine.magic, 8) != 0 || h.Q != mine.Q || h.prec != mine.prec || h.n1 != mine.n1 ||
        h.n2 != mine.n2 || h.ld != mine.ld || h.ncol != mine.ncol || h.state_bytes != mine.state_bytes ||
        h.wall_bytes != mine.wall_bytes || h.prev_bytes != mine.prev_bytes || h.geo_bytes != mine.geo_bytes)
        return fail(CLBM_EINVAL, "checkpoint does not match this grid (lattice, precision or size)");
    st = check_case(&h.cs);
    if (st != CLBM_OK) return st;
    const char* p = (const char*)buf + sizeof(h);
    // the state goes into the first physical buffer, which becomes current
    g->stA = g->phys[0];
    g->stB = g->phys[1];
    CK(cudaMemcpyAsync(g->stA, p, h.state_bytes, cudaMemcpyHostToDevice, g->stream));
    p += h.state_bytes;
    CK(cudaMemcpyAsync(g->wall_r, p, h.wall_bytes, cudaMemcpyHostToDevice, g->stream));
    p += h.wall_bytes;
    CK(cudaMemcpyAsync(g->wall_u, p, h.wall_bytes, cudaMemcpyHostToDevice, g->stream));
    p += h.wall_bytes;
    CK(cudaMemcpyAsync(g->prev, p, h.prev_bytes, cudaMemcpyHostToDevice, g->stream));
    p += h.prev_bytes;
    CK(cudaMemcpyAsync(g->geo, p, h.geo_bytes, cudaMemcpyHostToDevice, g->stream));
    g->cs = h.cs;
    g->have_case = true;
    st = rebuild_tables(g);  // tables and rest mass of the restored geometry and case (synchronises)
    if (st != CLBM_OK) return st;
    g->t = h.t;
    g->t_prev = h.t_prev;
    g->have_prev = h.have_prev != 0;
    g->ghosts_ok = true;
    return CLBM_OK;
}

clbm_status clbm_destroy(clbm_handle g) {
    if (!g) return CLBM_OK;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    else cudaDeviceSynchronize();
    for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->graph) cudaGraphDestroy(g->graph);
    for (cudaEvent_t e : g->gdummy)
        if (e) cudaEventDestroy(e);
    if (g->stage) cudaFree(g->stage);
    if (g->prog) cudaFree(g->prog);
    free_pipe(g->pipe);
    if (g->tma) free_tma_maps(g->tma);
    if (g->owns_ws) cudaFree(g->ws);
    delete g;
    return CLBM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches

struct clbm_batch {
    std::vector<clbm_grid*> g;
    int Q, prec, device;
    cudaStream_t stream;
    int variant;
    bool cached;                     // variant taken from the tuner's cache at creation
    int phase;                       // time steps taken through the batch, mod 2
    BatchGrid* d_grids;
    std::vector<BatchGrid> h_grids;
    int4* d_step[BATCH_ALL];         // update tiles of lagged-force lattices, per variant
    int nstep[BATCH_ALL];
    std::vector<int2> wave[BATCH_ALL];  // (first tile, tiles) of each launch of a time step
    std::vector<int4> hws[BATCH_ALL];   // the tile lists on the host (waves are cut from them)
    size_t wave_bytes;                  // workspace bytes of lattices per wave
    void* d_maps;                    // TMA load maps of every lattice (variant BATCH_WS)
    bool ws_ok;                      // every lattice has TMA maps
    int4* d_iter;                    // update tiles of lattices that iterate the force
    int niter;
    int4* d_bnd;
    int nbnd;
    int4* d_mom;                     // diagnostics items: lagged-force lattices first
    int nmom, nmom_lag;
    int2* d_range;
    double* d_partial;
    double* d_out;
    int nblk;
    cudaGraphExec_t graph[2];
    long long launches;
};

namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tune_cache;  // (Q, prec, width class, size class)

std::tuple<int, int, int, int> shape_class(const clbm_batch* b) {
    std::vector<int> w;
    long long cells = 0;
    for (clbm_grid* g : b->g) {
        w.push_back(g->n2);
        cells += (long long)g->n1 * g->n2;
    }
    std::sort(w.begin(), w.end());
    int wc = 0, sc = 0;
    for (int m = w[w.size() / 2]; m > 32; m >>= 1) ++wc;
    for (long long c = cells; c > 65536; c >>= 2) ++sc;
    return std::make_tuple(b->Q, b->prec, wc, sc);
}

void fill_desc(clbm_batch* b) {
    b->h_grids.resize(b->g.size());
    for (size_t k = 0; k < b->g.size(); ++k) {
        clbm_grid* g = b->g[k];
        BatchGrid& d = b->h_grids[k];
        d.phys[0] = g->phys[0];
        d.phys[1] = g->phys[1];
        d.tab = g->tab;
        d.wall_rho = g->wall_r;
        d.wall_ut2 = g->wall_u;
        d.ghost = g->ghost;
        d.geo = g->geo;
        d.prev = g->prev;
        d.k = scalars(g->cs);
        d.U0_lo = g->cs.u_wall_lo;
        d.U0_hi = g->cs.u_wall_hi;
        d.plane = (long long)(g->n1 + 2 * g->h) * g->ld;
        d.n1 = g->n1;
        d.n2 = g->n2;
        d.ld = g->ld;
        // source buffer at batch phase 0 given the grid's current source now
        const int cur = g->stA == g->phys[0] ? 0 : 1;
        d.parity = cur ^ b->phase;
        d.bc_lo = g->bc_lo;
        d.bc_hi = g->bc_hi;
        d.have_prev = g->have_prev ? 1 : 0;
        d.iters = g->cs.force_iterations;
    }
}

clbm_status upload_desc(clbm_batch* b) {
    fill_desc(b);
    CK(cudaMemcpyAsync(b->d_grids, b->h_grids.data(), b->h_grids.size() * sizeof(BatchGrid),
                       cudaMemcpyHostToDevice, b->stream));
    return CLBM_OK;
}

void drop_graphs(clbm_batch* b) {
    for (int p = 0; p < 2; ++p)
        if (b->graph[p]) {
            cudaGraphExecDestroy(b->graph[p]);
            b->graph[p] = nullptr;
        }
}

// One time step of every lattice at batch phase p: the update tiles of the
// current variant, then those of iterated-force lattices (each update fills
// the ghost rows and columns of the buffer it writes).  Returns the number of
// kernels launched.
int batch_one(clbm_batch* b, int p) {
    const int v = b->variant;
    for (const int2& w : b->wave[v]) {
        if (v == BATCH_WS)
            launch_batch_ws(b->Q, b->prec, b->d_grids, b->d_maps, b->d_step[v] + w.x, w.y, p, b->g[0]->nsm,
                            b->g[0]->err, b->stream);
        else
            launch_batch(b->Q, b->prec, 1, v, b->d_grids, b->d_step[v] + w.x, w.y, p, b->nblk, nullptr,
                         b->stream);
    }
    launch_batch(b->Q, b->prec, 3, 0, b->d_grids, b->d_iter, b->niter, p, b->nblk, nullptr, b->stream);
    return (int)b->wave[v].size() + (b->niter > 0);
}

// Split each variant's tile list into waves, one launch each per time step,
// of at most wave_bytes of lattice workspace (whole lattices; the list is
// lattice by lattice): the update slows as the state it sweeps in one launch
// grows into tens of GB.  512 lattices (39.5 GB), pipelined update: 72 % of
// the copy rate in one launch per step, 76.2 / 77.0 / 74.8 % in waves of
// 8 / 4 / 2 GiB (smaller waves pay more launch tails).
constexpr size_t WAVE_BYTES = size_t(4) << 30;

void make_waves(clbm_batch* b) {
    const std::vector<int4>* ws = b->hws;
    const size_t WAVE = b->wave_bytes;
    for (int v = 0; v < BATCH_ALL; ++v) {
        b->wave[v].clear();
        int start = 0, last = -1;
        size_t bytes = 0;
        for (int e = 0; e < (int)ws[v].size(); ++e) {
            const int k = ws[v][e].x;
            if (k == last) continue;
            const size_t lb = b->g[k]->L.total;
            if (e > start && bytes + lb > WAVE) {
                b->wave[v].push_back(make_int2(start, e - start));
                start = e;
                bytes = 0;
            }
            bytes += lb;
            last = k;
        }
        if ((int)ws[v].size() > start) b->wave[v].push_back(make_int2(start, (int)ws[v].size() - start));
    }
}

// Lattices stepped on their own since the last batch call: new descriptors.
clbm_status refresh(clbm_batch* b) {
    bool stale = false;
    for (size_t k = 0; k < b->g.size(); ++k) {
        const int cur = b->g[k]->stA == b->g[k]->phys[0] ? 0 : 1;
        if ((b->h_grids[k].parity ^ b->phase) != cur) stale = true;
    }
    if (!stale) return CLBM_OK;
    clbm_status st = upload_desc(b);
    if (st == CLBM_OK) drop_graphs(b);
    return st;
}

// Ghost rows and columns of every lattice's current state, when some
// lattice's state or case was set from outside since its last update.
void batch_ghosts(clbm_batch* b) {
    bool stale = false;
    for (clbm_grid* g : b->g) stale = stale || !g->ghosts_ok;
    if (!stale) return;
    launch_batch(b->Q, b->prec, 0, 0, b->d_grids, b->d_bnd, b->nbnd, b->phase, b->nblk, nullptr, b->stream);
    b->launches++;
    for (clbm_grid* g : b->g) g->ghosts_ok = true;
}

clbm_status batch_graph(clbm_batch* b, int p) {
    if (b->graph[p]) return CLBM_OK;
    cudaGraph_t gr = nullptr;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    batch_one(b, p);
    batch_one(b, p ^ 1);
    cudaError_t e = cudaStreamEndCapture(b->stream, &gr);
    if (e != cudaSuccess) return fail(CLBM_ECUDA, "batch graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph[p], gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
        b->graph[p] = nullptr;
        return fail(CLBM_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
    }
    return CLBM_OK;
}

// Advance every lattice's host-side bookkeeping by n steps.
void batch_advance(clbm_batch* b, long long n) {
    for (clbm_grid* g : b->g) {
        if (n & 1) std::swap(g->stA, g->stB);
        g->t += n;
    }
    b->phase = (int)((b->phase + n) & 1);
}

}  // namespace

extern "C" {

clbm_status clbm_batch_create(const clbm_handle* grids, int n, clbm_batch_handle* out) {
    Range nvtx_range("clbm_batch_create");
    if (!grids || n < 1 || !out) return fail(CLBM_EINVAL, "need grids, n >= 1 and out");
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        if (!grids[k]) return fail(CLBM_EINVAL, "grid %d is NULL", k);
        if (!grids[k]->have_case) return fail(CLBM_EINVAL, "grid %d has no case", k);
        if (grids[k]->ncol != 1)
            return fail(CLBM_EINVAL, "grid %d is a general grid: batches take planar and polar grids", k);
        if (grids[k]->Q != grids[0]->Q || grids[k]->prec != grids[0]->prec ||
            grids[k]->device != grids[0]->device || grids[k]->stream != grids[0]->stream)
            return fail(CLBM_EINVAL, "grids of a batch share lattice, precision, device and stream");
    }
    clbm_batch* b = new (std::nothrow) clbm_batch();
    if (!b) return fail(CLBM_ENOMEM, "host allocation failed");
    b->g.assign(grids, grids + n);
    b->Q = grids[0]->Q;
    b->prec = grids[0]->prec;
    b->device = grids[0]->device;
    b->stream = grids[0]->stream;
    b->variant = 0;
    b->phase = 0;
    clbm_status st = select(grids[0]);
    if (st != CLBM_OK) {
        delete b;
        return st;
    }
    // work-lists
    std::vector<int4> wb, wm;
    std::vector<int2> range;
    std::vector<int4> ws[BATCH_ALL], wi;
    b->ws_ok = true;
    for (int k = 0; k < n; ++k) b->ws_ok = b->ws_ok && grids[k]->tma != nullptr;
    int tj0, tr0;
    batch_tile_shape(0, &tj0, &tr0);
    for (int k = 0; k < n; ++k) {
        clbm_grid* g = grids[k];
        for (int j = 0; j < g->n2; j += 128) {
            wb.push_back(make_int4(k, 0, j, 0));
            wb.push_back(make_int4(k, 1, j, 0));
        }
        for (int t = 0; t < g->n1 * b->Q; t += 128 / (2 * GC)) wb.push_back(make_int4(k, 2, t, 0));
        if (g->cs.force_iterations > 0) {
            for (int i = 0; i < g->n1; i += tr0)
                for (int j = 0; j < g->n2; j += tj0) wi.push_back(make_int4(k, i, j, 0));
            continue;
        }
        for (int v = 0; v < BATCH_ALL; ++v) {
            if (v == BATCH_WS && !b->ws_ok) continue;
            int tj, tr;
            batch_tile_shape(v, &tj, &tr);
            for (int i = 0; i < g->n1; i += tr)
                for (int j = 0; j < g->n2; j += tj) ws[v].push_back(make_int4(k, i, j, 0));
        }
    }
    // diagnostics items, lattice by lattice: lagged-force lattices first
    range.resize(n);
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) b->nmom_lag = (int)wm.size();
        for (int k = 0; k < n; ++k) {
            clbm_grid* g = grids[k];
            if ((g->cs.force_iterations > 0) != (pass == 1)) continue;
            const int r0 = (int)wm.size();
            for (int i = 0; i < g->n1; ++i)
                for (int j = 0; j < g->n2; j += 128) wm.push_back(make_int4(k, i, j, 0));
            range[k] = make_int2(r0, (int)wm.size());
        }
    }
    b->nbnd = (int)wb.size();
    b->nmom = (int)wm.size();
    size_t bytes = n * sizeof(BatchGrid) + wb.size() * sizeof(int4) + wm.size() * sizeof(int4) +
                   range.size() * sizeof(int2) + wm.size() * NRED * 8 + (size_t)n * NRED * 8;
    for (int v = 0; v < BATCH_ALL; ++v) {
        b->nstep[v] = (int)ws[v].size();
        bytes += ws[v].size() * sizeof(int4);
    }
    b->wave_bytes = WAVE_BYTES;
    for (int v = 0; v < BATCH_ALL; ++v) b->hws[v] = ws[v];
    make_waves(b);
    std::vector<unsigned char> maps;
    if (b->ws_ok) {
        const size_t mb = tma_load_maps(grids[0]->tma, nullptr);
        maps.resize(mb * n);
        for (int k = 0; k < n; ++k) tma_load_maps(grids[k]->tma, maps.data() + mb * k);
        bytes += maps.size();
    }
    b->niter = (int)wi.size();
    bytes += wi.size() * sizeof(int4);
    cudaError_t e = cudaSuccess;
    e = cudaMalloc((void**)&b->d_grids, n * sizeof(BatchGrid));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_bnd, wb.size() * sizeof(int4));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_mom, wm.size() * sizeof(int4));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_range, range.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_partial, wm.size() * NRED * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_out, (size_t)n * NRED * 8);
    for (int v = 0; v < BATCH_ALL && e == cudaSuccess; ++v)
        if (!ws[v].empty()) e = cudaMalloc((void**)&b->d_step[v], ws[v].size() * sizeof(int4));
    if (e == cudaSuccess && !maps.empty()) e = cudaMalloc(&b->d_maps, maps.size());
    if (e == cudaSuccess && !wi.empty()) e = cudaMalloc((void**)&b->d_iter, wi.size() * sizeof(int4));
    if (e != cudaSuccess) {
        clbm_batch_destroy(b);
        return fail(CLBM_ENOMEM, "batch work-lists (%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    cudaMemcpyAsync(b->d_bnd, wb.data(), wb.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream);
    cudaMemcpyAsync(b->d_mom, wm.data(), wm.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream);
    cudaMemcpyAsync(b->d_range, range.data(), range.size() * sizeof(int2), cudaMemcpyHostToDevice,
                    b->stream);
    if (!maps.empty())
        cudaMemcpyAsync(b->d_maps, maps.data(), maps.size(), cudaMemcpyHostToDevice, b->stream);
    for (int v = 0; v < BATCH_ALL; ++v)
        if (!ws[v].empty())
            cudaMemcpyAsync(b->d_step[v], ws[v].data(), ws[v].size() * sizeof(int4), cudaMemcpyHostToDevice,
                            b->stream);
    if (!wi.empty())
        cudaMemcpyAsync(b->d_iter, wi.data(), wi.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream);
    st = upload_desc(b);
    if (st == CLBM_OK && cudaStreamSynchronize(b->stream) != cudaSuccess)
        st = fail(CLBM_ECUDA, "batch set-up failed");
    if (st != CLBM_OK) {
        clbm_batch_destroy(b);
        return st;
    }
    int nsm = grids[0]->nsm;
    b->nblk = nsm * 8;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(shape_class(b));
        if (it != g_tune_cache.end()) {
            b->variant = it->second;
            b->cached = true;
        }
    }
    *out = b;
    return CLBM_OK;
}

clbm_status clbm_batch_step(clbm_batch_handle b, long long n) {
    Range nvtx_range("clbm_batch_step");
    if (!b) return fail(CLBM_EINVAL, "batch is NULL");
    if (n < 0) return fail(CLBM_EINVAL, "n < 0");
    clbm_status st = select(b->g[0]);
    if (st != CLBM_OK) return st;
    st = refresh(b);
    if (st != CLBM_OK) return st;
    batch_ghosts(b);
    const bool graphs = b->stream != nullptr;
    long long left = n;
    while (left >= 2 && graphs) {
        st = batch_graph(b, b->phase);
        if (st != CLBM_OK) return st;
        CK(cudaGraphLaunch(b->graph[b->phase], b->stream));
        b->launches += 2 * ((int)b->wave[b->variant].size() + (b->niter > 0));
        batch_advance(b, 2);
        left -= 2;
    }
    while (left > 0) {
        b->launches += batch_one(b, b->phase);
        batch_advance(b, 1);
        --left;
    }
    CK(cudaGetLastError());
    return CLBM_OK;
}

clbm_status clbm_batch_residual(clbm_batch_handle b, double* res, double* cons) {
    Range nvtx_range("clbm_batch_residual");
    if (!b) return fail(CLBM_EINVAL, "batch is NULL");
    clbm_status st = select(b->g[0]);
    if (st != CLBM_OK) return st;
    // the per-cell sums over the current buffers, then one reduction per lattice
    st = refresh(b);
    if (st != CLBM_OK) return st;
    batch_ghosts(b);
    launch_batch(b->Q, b->prec, 2, 0, b->d_grids, b->d_mom, b->nmom_lag, b->phase, b->nblk, b->d_partial,
                 b->stream);
    launch_batch(b->Q, b->prec, 4, 0, b->d_grids, b->d_mom + b->nmom_lag, b->nmom - b->nmom_lag, b->phase,
                 b->nblk, b->d_partial + (size_t)b->nmom_lag * NRED, b->stream);
    launch_batch_reduce(b->d_partial, b->d_range, (int)b->g.size(), b->d_out, b->stream);
    b->launches += 2 + (b->nmom_lag > 0 && b->nmom > b->nmom_lag ? 1 : 0);
    CK(cudaGetLastError());
    std::vector<double> v(b->g.size() * NRED);
    CK(cudaMemcpyAsync(v.data(), b->d_out, v.size() * 8, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    bool unstable = false, changed = false;
    for (size_t k = 0; k < b->g.size(); ++k) {
        clbm_grid* g = b->g[k];
        const double* x = &v[k * NRED];
        const long long dt = g->t - g->t_prev;
        double r = INFINITY;
        if (g->have_prev && dt > 0) r = x[1] > 0.0 ? sqrt(x[0]) / (dt * sqrt(x[1])) : (x[0] > 0 ? INFINITY : 0.0);
        if (x[8] > 0.0 || !std::isfinite(x[2])) r = NAN;
        if (res) res[k] = r;
        if (cons)
            for (int q = 0; q < 6; ++q) cons[k * 6 + q] = x[2 + q] + (q == 0 ? g->rest_mass : 0.0);
        if (!g->have_prev) changed = true;
        g->have_prev = true;
        g->t_prev = g->t;
        if (x[8] > 0.0 || !std::isfinite(x[2])) unstable = true;
    }
    if (changed) {
        st = upload_desc(b);
        if (st != CLBM_OK) return st;
    }
    st = check_err(b->g[0]);  // bounded waits of the pipelined variant
    if (st != CLBM_OK) return st;
    if (unstable) return fail(CLBM_EUNSTABLE, "a lattice of the batch has a non-finite or non-positive density");
    return CLBM_OK;
}

clbm_status clbm_batch_set_variant(clbm_batch_handle b, int variant) {
    if (!b) return fail(CLBM_EINVAL, "batch is NULL");
    if (variant < 0 || variant > BATCH_WS) return fail(CLBM_EINVAL, "variant out of range");
    if (variant == BATCH_WS && !b->ws_ok)
        return fail(CLBM_EINVAL, "the pipelined TMA variant needs 16/32-bit storage and TMA maps on every grid");
    if (variant != b->variant) drop_graphs(b);
    b->variant = variant;
    return CLBM_OK;
}

clbm_status clbm_batch_tune(clbm_batch_handle b, int steps, int* best, double* ms_per_step) {
    Range nvtx_range("clbm_batch_tune");
    if (!b || steps < 1) return fail(CLBM_EINVAL, "batch is NULL or steps < 1");
    clbm_status st = select(b->g[0]);
    if (st != CLBM_OK) return st;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double bestms = INFINITY;
    int bestv = 0;
    const int keep = b->variant;
    st = refresh(b);
    if (st != CLBM_OK) return st;
    batch_ghosts(b);
    for (int v = 0; v < BATCH_ALL; ++v) {
        if (v == BATCH_WS && !b->ws_ok) {
            if (ms_per_step) ms_per_step[v] = -1.0;
            continue;
        }
        b->variant = v;
        b->launches += batch_one(b, b->phase);  // warm-up step
        batch_advance(b, 1);
        CK(cudaEventRecord(e0, b->stream));
        for (int s = 0; s < steps; ++s) {
            b->launches += batch_one(b, b->phase);
            batch_advance(b, 1);
        }
        CK(cudaEventRecord(e1, b->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        const double per = ms / steps;
        if (ms_per_step) ms_per_step[v] = per;
        if (per < bestms) {
            bestms = per;
            bestv = v;
        }
    }
    (void)keep;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    if (bestv != b->variant) drop_graphs(b);
    b->variant = bestv;
    drop_graphs(b);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[shape_class(b)] = bestv;
    }
    if (best) *best = bestv;
    return CLBM_OK;
}

clbm_status clbm_batch_set_wave_bytes(clbm_batch_handle b, size_t bytes) {
    if (!b || bytes < 1) return fail(CLBM_EINVAL, "batch is NULL or bytes < 1");
    b->wave_bytes = bytes;
    make_waves(b);
    drop_graphs(b);
    return CLBM_OK;
}

clbm_status clbm_batch_get_variant(clbm_batch_handle b, int* variant, int* cached) {
    if (!b) return fail(CLBM_EINVAL, "batch is NULL");
    if (variant) *variant = b->variant;
    if (cached) *cached = b->cached ? 1 : 0;
    return CLBM_OK;
}

clbm_status clbm_batch_launch_count(clbm_batch_handle b, long long* launches) {
    if (!b || !launches) return fail(CLBM_EINVAL, "NULL argument");
    *launches = b->launches;
    return CLBM_OK;
}

clbm_status clbm_batch_destroy(clbm_batch_handle b) {
    if (!b) return CLBM_OK;
    // the batch's own copy of the device: its grids may already be gone
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    cudaFree(b->d_grids);
    cudaFree(b->d_bnd);
    cudaFree(b->d_mom);
    cudaFree(b->d_range);
    cudaFree(b->d_partial);
    cudaFree(b->d_out);
    for (int v = 0; v < BATCH_ALL; ++v) cudaFree(b->d_step[v]);
    cudaFree(b->d_maps);
    cudaFree(b->d_iter);
    delete b;
    return CLBM_OK;
}

}  // extern "C"
