// clbm_api.cu -- host side of the C ABI declared in include/clbm.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/clbm.h"
#include "clbm_internal.cuh"

using namespace clbm;

namespace {

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
    float inv_scale;
    clbm_case cs;
    bool have_case;
    long long t, t_prev, launches;
    bool have_prev;
    bool profiling;
    std::vector<cudaEvent_t> ev;
    size_t ev_used;
    std::vector<double> edges;
    double step2;
    double* stage;          // lazily allocated FP64 staging buffer for host transfers
    void* phys[2];          // the two state buffers (stA / stB alternate over them)
    TmaMaps* tma;           // tensor maps of the TMA-staged update (16/32-bit storage)
    int nsm;                // SM count of the device
    int variant;            // 0 auto, 1 per-cell loads, 2 TMA-staged tiles
    int* err;               // device error word of bounded waits
};

namespace {

clbm_status layout_of(const clbm_grid_desc* d, Layout* L, int* ld_out, int* h_out) {
    if (!d) return fail(CLBM_EINVAL, "desc is NULL");
    if (d->lattice != 9 && d->lattice != 21) return fail(CLBM_EINVAL, "lattice must be 9 or 21");
    if (d->precision < 0 || d->precision > 3) return fail(CLBM_EINVAL, "bad precision");
    if (d->n1 < 4 || d->n2 < 1) return fail(CLBM_EINVAL, "need n1 >= 4 and n2 >= 1");
    if ((long long)d->n1 * d->n2 > (1LL << 31) / 32)
        return fail(CLBM_EINVAL, "grid too large for 32-bit cell indexing");
    const int Q = d->lattice, h = Q == 9 ? 1 : 3;
    const int ld = (d->n2 + 2 * GC + 31) / 32 * 32;
    const size_t sb = storage_bytes(d->precision), cb = compute_bytes(d->precision);
    const int TS = Q == 9 ? Tab<9>::S : Tab<21>::S;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    L->stA = take((size_t)Q * (d->n1 + 2 * h) * ld * sb);
    L->stB = take((size_t)Q * (d->n1 + 2 * h) * ld * sb);
    L->tab = take((size_t)d->n1 * TS * cb);
    L->geo = take((size_t)d->n1 * Geo::stride(Q) * 8);
    L->wall_r = take((size_t)2 * h * d->n2 * cb);
    L->wall_u = take((size_t)2 * h * d->n2 * cb);
    L->ghost = take((size_t)2 * h * Q * 2 * 8);
    L->pos = take((size_t)(d->n1 + 8) * 9 * 2 * 8);
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
    StepArgs a;
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
    a.inv_scale = g->inv_scale;
    a.bc_lo = g->bc_lo;
    a.bc_hi = g->bc_hi;
    a.iters = g->cs.force_iterations;
    a.err = g->err;
    return a;
}

bool use_tma(const clbm_grid* g) {
    if (!g->tma || g->cs.force_iterations > 0) return false;
    return g->variant != 1;
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
    m.inv_scale = g->inv_scale;
    m.ut_prev = g->prev;
    m.partial = g->partial;
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

// Ghost rows of the current state (what the next collision pulls).
void fill_ghosts(clbm_grid* g) {
    StepArgs a = step_args(g, g->stA, g->stB);
    launch_boundary(g->Q, g->prec, a, g->stA, g->stream);
    g->launches++;
}

clbm_status rebuild_tables(clbm_grid* g) {
    launch_reference(g->Q, g->geo, g->n1, g->cs.rho0, g->stream);
    launch_tables(g->Q, g->prec, g->geo, g->tab, g->ghost, g->n1, g->cs.tau, g->bc_lo, g->bc_hi,
                  g->stream);
    g->launches += 3;
    CK(cudaGetLastError());
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
    g_err[0] = 0;
    if (!out) return fail(CLBM_EINVAL, "out is NULL");
    *out = nullptr;
    Layout L;
    int ld, h;
    clbm_status st = layout_of(d, &L, &ld, &h);
    if (st != CLBM_OK) return st;
    if (d->kind != CLBM_GEOM_PLANAR && d->kind != CLBM_GEOM_POLAR)
        return fail(CLBM_EINVAL, "kind must be PLANAR or POLAR");
    if ((d->bc_lo != 0 && d->bc_lo != 1) || (d->bc_hi != 0 && d->bc_hi != 1))
        return fail(CLBM_EINVAL, "bad wall condition");
    if (!d->edges1) return fail(CLBM_EINVAL, "edges1 is NULL");
    std::vector<double> e(d->edges1, d->edges1 + d->n1 + 1);
    for (int k = 0; k < d->n1; ++k)
        if (!(e[k + 1] > e[k]) || !std::isfinite(e[k + 1]))
            return fail(CLBM_EINVAL, "edges1 must be finite and strictly increasing");
    if (d->kind == CLBM_GEOM_PLANAR && !(d->step2 > 0.0))
        return fail(CLBM_EINVAL, "step2 must be > 0");
    const double dx = d->dx > 0.0 ? d->dx : (e[d->n1] - e[0]) / d->n1;
    // node positions of rows -3..n1+4, columns -3..5 (1-based)
    std::vector<double> pos((size_t)(d->n1 + 8) * 9 * 2);
    const double pi = 3.14159265358979323846;
    for (int i = -3; i <= d->n1 + 4; ++i) {
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
                const double th = (j - 0.5) * (2.0 * pi / d->n2);
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
    g->ld = ld;
    g->h = h;
    g->kind = d->kind;
    g->bc_lo = d->bc_lo;
    g->bc_hi = d->bc_hi;
    g->device = d->device;
    g->dx = dx;
    g->stream = (cudaStream_t)d->stream;
    g->L = L;
    g->inv_scale = d->precision == CLBM_FP32_F16STORE ? 1.0f / 4096.0f : 1.0f;
    g->edges = e;
    g->step2 = d->step2;
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
        launch_geometry(g->Q, g->pos, g->n1, dx, d->kind == CLBM_GEOM_POLAR, g->geo, g->stream);
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
    std::vector<double> geo((size_t)g->n1 * Geo::stride(g->Q));
    ce = cudaMemcpy(geo.data(), g->geo, geo.size() * 8, cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) {
        clbm_destroy(g);
        return fail(CLBM_ECUDA, "geometry readback: %s", cudaGetErrorString(ce));
    }
    for (int r = 0; r < g->n1; ++r)
        if (!(geo[(size_t)r * Geo::stride(g->Q) + Geo::J] > 0.0)) {
            clbm_destroy(g);
            return fail(CLBM_EINVAL, "cell volume J <= 0 at row %d", r + 1);
        }
    *out = g;
    return CLBM_OK;
}

clbm_status clbm_set_case(clbm_handle g, const clbm_case* c) {
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    clbm_status st = check_case(c);
    if (st != CLBM_OK) return st;
    st = select(g);
    if (st != CLBM_OK) return st;
    g->cs = *c;
    g->have_case = true;
    st = rebuild_tables(g);
    if (st != CLBM_OK) return st;
    launch_state_from_fp64(g->Q, g->prec, nullptr, g->geo, g->stA, g->n1, g->n2, g->ld, g->h,
                           g->inv_scale, g->stream);
    launch_wall_init(g->prec, g->wall_r, g->wall_u, nullptr, nullptr, g->n1, g->n2, g->h,
                     c->rho0, g->stream);
    g->launches += 2;
    CK(cudaGetLastError());
    g->t = 0;
    g->have_prev = false;
    return CLBM_OK;
}

clbm_status clbm_set_state(clbm_handle g, const double* Np, const double* rho_prev,
                           const double* ut2_prev, int src_is_device) {
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
        launch_state_from_fp64(g->Q, g->prec, dN, g->geo, g->stA, g->n1, g->n2, g->ld, g->h,
                               g->inv_scale, g->stream);
        launch_wall_init(g->prec, g->wall_r, g->wall_u, dr, du, g->n1, g->n2, g->h, g->cs.rho0,
                         g->stream);
        g->launches += 2;
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(g->stream));
        cudaFree(extra);
    } else {
        launch_state_from_fp64(g->Q, g->prec, dN, g->geo, g->stA, g->n1, g->n2, g->ld, g->h,
                               g->inv_scale, g->stream);
        launch_wall_init(g->prec, g->wall_r, g->wall_u, dr, du, g->n1, g->n2, g->h, g->cs.rho0,
                         g->stream);
        g->launches += 2;
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(g->stream));
    }
    g->have_prev = false;
    return CLBM_OK;
}

clbm_status clbm_get_state(clbm_handle g, double* Np, int dst_is_device) {
    if (!g || !Np) return fail(CLBM_EINVAL, "handle or Np is NULL");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    const size_t nq = (size_t)g->n1 * g->n2 * g->Q;
    double* dN = Np;
    if (!dst_is_device) {
        st = staging(g, &dN);
        if (st != CLBM_OK) return st;
    }
    launch_state_to_fp64(g->Q, g->prec, g->stA, g->geo, dN, g->n1, g->n2, g->ld, g->h,
                         g->inv_scale, g->stream);
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

clbm_status clbm_step(clbm_handle g, long long n) {
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    if (!g->have_case) return fail(CLBM_EINVAL, "call clbm_set_case first");
    if (n < 0) return fail(CLBM_EINVAL, "n < 0");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    for (long long s = 0; s < n; ++s) {
        StepArgs a = step_args(g, g->stA, g->stB);
        launch_boundary(g->Q, g->prec, a, g->stA, g->stream);
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
        if (use_tma(g)) {
            const int src = g->stA == g->phys[0] ? 0 : 1;
            if (launch_step_tma(g->Q, g->prec, *g->tma, a, src, g->nsm, g->stream) != 0)
                return fail(CLBM_ECUDA, "TMA-staged update could not be launched");
        } else {
            launch_step(g->Q, g->prec, a, g->stream);
        }
        if (g->profiling) {
            CK(cudaEventRecord(g->ev[g->ev_used + 1], g->stream));
            g->ev_used += 2;
        }
        g->launches += 2;
        void* t = g->stA;
        g->stA = g->stB;
        g->stB = t;
        g->t++;
    }
    CK(cudaGetLastError());
    return CLBM_OK;
}

clbm_status clbm_moments(clbm_handle g, double* rho, double* U1, double* U2, double* Ut1,
                         double* Ut2, double* F1, double* F2, int dst_is_device) {
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

clbm_status clbm_residual(clbm_handle g, double* res, double cons[6]) {
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    if (!g->have_case) return fail(CLBM_EINVAL, "call clbm_set_case first");
    clbm_status st = select(g);
    if (st != CLBM_OK) return st;
    fill_ghosts(g);
    MomArgs m = mom_args(g);
    m.have_prev = g->have_prev ? 1 : 0;
    launch_moments(g->Q, g->prec, m, g->cs.force_iterations, 1, g->stream);
    launch_reduce_final(g->partial, moments_blocks(g->n1, g->n2), g->red, g->stream);
    g->launches += 2;
    CK(cudaGetLastError());
    double v[NRED];
    CK(cudaMemcpyAsync(v, g->red, sizeof(v), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    st = check_err(g);
    if (st != CLBM_OK) return st;
    const long long dt = g->t - g->t_prev;
    double r = INFINITY;
    if (g->have_prev && dt > 0) r = v[1] > 0.0 ? sqrt(v[0]) / (dt * sqrt(v[1])) : (v[0] > 0 ? INFINITY : 0.0);
    if (res) *res = r;
    if (cons)
        for (int k = 0; k < 6; ++k) cons[k] = v[2 + k];
    g->have_prev = true;
    g->t_prev = g->t;
    if (v[8] > 0.0 || !std::isfinite(v[2]))
        return fail(CLBM_EUNSTABLE, "%g cells with a non-finite or non-positive density at t=%lld",
                    v[8], g->t);
    return CLBM_OK;
}

clbm_status clbm_no_flow_adjust(clbm_handle g, long long nsteps, double* rho_nf) {
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
    d.edges1 = g->edges.data();
    d.step2 = g->step2;
    d.dx = g->dx;
    d.bc_lo = g->bc_lo;
    d.bc_hi = g->bc_hi;
    d.device = g->device;
    d.stream = g->stream;
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
        launch_row_mean(rho, g->n1, g->n2, rowm, g->stream);
        // Eq. 23: J <- J rho_nf / rho0, then references and tables anew
        launch_scale_volume(g->Q, g->geo, rowm, g->n1, g->cs.rho0, g->stream);
        g->launches += 2;
        st = rebuild_tables(g);
    }
    if (st == CLBM_OK) {
        // keep the no-flow state; its last-collision densities scale by rho0/rho_nf
        launch_state_from_fp64(g->Q, g->prec, Np, g->geo, g->stA, g->n1, g->n2, g->ld, g->h,
                               g->inv_scale, g->stream);
        launch_wall_copy(g->prec, g->wall_r, g->wall_u, (const double*)nf->wall_r,
                         (const double*)nf->wall_u, rowm, g->n1, g->n2, g->h, g->cs.rho0, g->stream);
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

clbm_status clbm_set_profiling(clbm_handle g, int on) {
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    g->profiling = on != 0;
    g->ev_used = 0;
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
    *launches = (long long)(g->ev_used / 2);
    g->ev_used = 0;
    return CLBM_OK;
}

clbm_status clbm_set_kernel(clbm_handle g, int variant) {
    if (!g) return fail(CLBM_EINVAL, "handle is NULL");
    if (variant < 0 || variant > 2) return fail(CLBM_EINVAL, "variant must be 0, 1 or 2");
    if (variant == 2 && !g->tma)
        return fail(CLBM_EINVAL, "the TMA-staged update needs 16/32-bit storage on sm_90 or newer");
    g->variant = variant;
    return CLBM_OK;
}

clbm_status clbm_launch_count(clbm_handle g, long long* launches) {
    if (!g || !launches) return fail(CLBM_EINVAL, "NULL argument");
    *launches = g->launches;
    return CLBM_OK;
}

clbm_status clbm_destroy(clbm_handle g) {
    if (!g) return CLBM_OK;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    else cudaDeviceSynchronize();
    for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
    if (g->stage) cudaFree(g->stage);
    if (g->tma) free_tma_maps(g->tma);
    if (g->owns_ws) cudaFree(g->ws);
    delete g;
    return CLBM_OK;
}

}  // extern "C"
