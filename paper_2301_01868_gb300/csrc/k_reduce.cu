// k_reduce.cu -- diagnostics (moments, residual and conservation sums with a
// warp-shuffle reduction in a fixed order) and the state conversions between
// FP64 populations and the stored deviations.
#include "clbm_cell.cuh"

namespace clbm {

namespace {

constexpr int RB = 128;  // threads per block of the diagnostics kernels

// Persistent blocks of the residual reduction: eight per SM of a GB300,
// never more than there are (row, 128-column) items.  Each thread then sums
// many cells before the warp and block reductions, whose shuffles would
// otherwise cost as much as the cells themselves.
int residual_blocks(int n1, int n2) {
    const int items = n1 * ((n2 + RB - 1) / RB);
    return items < 1216 ? items : 1216;
}

// Geometry row / cell of cell (i, j).
__device__ __forceinline__ const double* geo_of(const double* geo, int Q, int ncol, int i, int j) {
    return geo + ((size_t)i * ncol + (ncol > 1 ? j : 0)) * Geo::stride(Q);
}

template <int Q, typename S, typename C, bool ITER, bool GEN>
__device__ __forceinline__ void cell_moments(const MomArgs& a, int iters, int i, int j,
                                             Cell<Q, C>& c) {
    constexpr int H = Lat<Q>::H;
    const auto tb = TabOf<Q, C, GEN>::at(a.tab, i, j, a.n1, a.n2);
    const Consts<C> kc = Consts<C>::make(a.k);
    const long long off = (long long)(i + H) * a.ld + j + GC;
    pull_cell<Q, C>(GlobalLoad<S>{(const S*)a.src + off, (int)a.plane, a.ld}, tb, kc, c);
    if (ITER) {
        C out[Q];
        collide_emit<Q, C>(tb, c, kc, [&](int al, C x) { out[al] = x; });
        for (int it = 0; it < iters; ++it) {
            force_again<Q, C>(tb, out, kc, c);
            collide_emit<Q, C>(tb, c, kc, [&](int al, C x) { out[al] = x; });
        }
    } else {
        collide_emit<Q, C>(tb, c, kc, [](int, C) {});
    }
}

// Field output of the moments: one thread per cell.
template <int Q, typename S, typename C, bool ITER, bool GEN>
__global__ void __launch_bounds__(RB) k_moments(const MomArgs a, int iters) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= a.n2) return;
    Cell<Q, C> c;
    cell_moments<Q, S, C, ITER, GEN>(a, iters, i, j, c);
    const size_t m = (size_t)i * a.n2 + j;
    if (a.rho) a.rho[m] = double(c.rho);
    if (a.U1) a.U1[m] = double(c.U1);
    if (a.U2) a.U2[m] = double(c.U2);
    if (a.Ut1) a.Ut1[m] = double(c.Ut1);
    if (a.Ut2) a.Ut2[m] = double(c.Ut2);
    if (a.F1) a.F1[m] = double(c.F1);
    if (a.F2) a.F2[m] = double(c.F2);
}

// Residual and conservation sums: persistent blocks stride over (row,
// 128-column) items; each thread accumulates its cells in a fixed order
// (ResAcc), then a warp-shuffle and block reduction in FP64 in a fixed tree
// writes one partial per block, so repeated runs give identical bits.  The
// rest parts of the totals are exact per row: sum_a ref_a(i) = J rho0 and
// sum_a c_a ref_a(i) = 0.  The largest |u| is tracked as the largest |u|^2
// and rooted once per block.
template <int Q, typename S, typename C, bool ITER, bool GEN>
__global__ void __launch_bounds__(RB, ITER ? 2 : 4) k_residual(const MomArgs a, int iters) {
    const int bx = (a.n2 + RB - 1) / RB;
    const int items = a.n1 * bx;
    const size_t nc = (size_t)a.n1 * a.n2;
    ResAcc<C> acc;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int i = it / bx, j = (it % bx) * RB + threadIdx.x;
        if (j >= a.n2) continue;
        const size_t m = (size_t)i * a.n2 + j;
        C* prev = (C*)a.ut_prev;
        const bool hp = a.have_prev != 0;
        // the snapshot first: its load overlaps the pull
        const C p1 = hp ? prev[m] : C(0), p2 = hp ? prev[nc + m] : C(0);
        Cell<Q, C> c;
        cell_moments<Q, S, C, ITER, GEN>(a, iters, i, j, c);
        acc.add(residual_terms<Q, C>(c, TabOf<Q, C, GEN>::at(a.tab, i, j, a.n1, a.n2), p1, p2, hp));
        prev[m] = c.Ut1;
        prev[nc + m] = c.Ut2;
    }
    double v[NRED];
    acc.out(v);
    block_partial<RB>(v, a.partial + (size_t)blockIdx.x * NRED);
}

// Final reduction: block k reduces quantity k over all block partials, each
// thread a fixed strided subset, then a fixed tree (repeatable bits).
__global__ void __launch_bounds__(1024) k_reduce_final(const double* __restrict__ partial,
                                                       int nblocks, double* __restrict__ out) {
    __shared__ double sh[1024];
    const int k = blockIdx.x;
    double x = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 1024) {
        const double y = partial[(size_t)b * NRED + k];
        x = (k == 7) ? fmax(x, y) : x + y;
    }
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int st = 512; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            sh[threadIdx.x] = (k == 7) ? fmax(sh[threadIdx.x], sh[threadIdx.x + st])
                                       : sh[threadIdx.x] + sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
}

template <int Q, typename S>
__global__ void k_from_fp64(const double* __restrict__ Np, const double* __restrict__ geo,
                            S* __restrict__ st, int n1, int n2, int ld, int h, int ncol) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= n2) return;
    const long long P = (long long)(n1 + 2 * h) * ld;
    const double* ge = geo_of(geo, Q, ncol, i, j);
#pragma unroll
    for (int al = 0; al < Q; ++al) {
        // Np == nullptr: the rest state N' = J f^eq(rho0, 0) of this cell.
        const double Nv = Np ? Np[((size_t)al * n1 + i) * n2 + j] : ge[Geo::ref(Q, al)];
        const double v = Nv - ge[Geo::ref(Q, al)];
        using CT = typename Store<S>::C;
        store_periodic<S, CT>(st + al * P + (long long)(i + h) * ld, j, n2, CT(v));
    }
}

// Equilibrium start N(q, 0) = J f^eq(rho, U, Ut = U; g^{ij}(q)) in FP64
// (Eq. 19: the third-order Hermite polynomial whose second moment is
// T0 g^{ij} + Ut^i Ut^j and whose third is built from Ut, U and g^{ij}; with
// no force known at the start Ut = U).  Absent fields are rho0 and 0.  The
// inputs may alias fields of the output: each thread reads its own cell's
// rho, U before it writes that cell's Q values.
template <int Q>
__global__ void k_equilibrium(const double* rho, const double* U1, const double* U2,
                              const double* __restrict__ geo, double* Np, int n1, int n2, int ncol,
                              double rho0) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= n2) return;
    const size_t m = (size_t)i * n2 + j;
    const double r = rho ? rho[m] : rho0;
    const double u1 = U1 ? U1[m] : 0.0, u2 = U2 ? U2[m] : 0.0;
    const double* ge = geo_of(geo, Q, ncol, i, j);
    const double T0 = Lat<Q>::T0, J = ge[Geo::J];
    const double e11 = ge[Geo::GI11] - 1.0, e12 = ge[Geo::GI12], e22 = ge[Geo::GI22] - 1.0;
    // second- and third-order Hermite coefficients (symmetric)
    const double A11 = u1 * u1 + T0 * e11, A12 = u1 * u2 + T0 * e12, A22 = u2 * u2 + T0 * e22;
    const double C111 = u1 * u1 * u1 + 3.0 * T0 * e11 * u1;
    const double C112 = u1 * u1 * u2 + T0 * (e11 * u2 + 2.0 * e12 * u1);
    const double C122 = u1 * u2 * u2 + T0 * (2.0 * e12 * u2 + e22 * u1);
    const double C222 = u2 * u2 * u2 + 3.0 * T0 * e22 * u2;
    double out[Q];
#pragma unroll
    for (int al = 0; al < Q; ++al) {
        const double c1 = c1_of(al), c2 = c2_of(al);
        const double h1 = c1 * u1 + c2 * u2;
        const double h2 = c1 * c1 * A11 + 2.0 * c1 * c2 * A12 + c2 * c2 * A22 - T0 * (A11 + A22);
        const double h3 = c1 * c1 * c1 * C111 + 3.0 * c1 * c1 * c2 * C112 + 3.0 * c1 * c2 * c2 * C122 +
                          c2 * c2 * c2 * C222 - 3.0 * T0 * (c1 * (C111 + C122) + c2 * (C112 + C222));
        const double P = 1.0 + h1 / T0 + h2 / (2.0 * T0 * T0) + h3 / (6.0 * T0 * T0 * T0);
        out[al] = J * Lat<Q>::w(al) * r * P;
    }
#pragma unroll
    for (int al = 0; al < Q; ++al) Np[((size_t)al * n1 + i) * n2 + j] = out[al];
}

template <int Q, typename S>
__global__ void k_to_fp64(const S* __restrict__ st, const double* __restrict__ geo,
                          double* __restrict__ Np, int n1, int n2, int ld, int h, int ncol) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= n2) return;
    const long long P = (long long)(n1 + 2 * h) * ld;
    const double* ge = geo_of(geo, Q, ncol, i, j);
#pragma unroll
    for (int al = 0; al < Q; ++al) {
        const double s = double(Store<S>::ld(st + al * P + (long long)(i + h) * ld + j + GC));
        Np[((size_t)al * n1 + i) * n2 + j] = s + ge[Geo::ref(Q, al)];
    }
}

template <typename C>
__global__ void k_wall_init(C* __restrict__ wr, C* __restrict__ wu, const double* __restrict__ rho,
                            const double* __restrict__ ut2, int n1, int n2, int h, double rho0) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int wk = blockIdx.y;  // wall * h + (k - 1)
    if (j >= n2) return;
    const int wall = wk / h, k = wk % h + 1;
    const int row = wall == 0 ? k - 1 : n1 - k;  // 0-based fluid row
    const size_t m = (size_t)row * n2 + j;
    wr[(size_t)wk * n2 + j] = C(rho ? rho[m] : rho0);
    wu[(size_t)wk * n2 + j] = C(ut2 ? ut2[m] : 0.0);
}

template <typename C>
__global__ void k_wall_copy(C* __restrict__ wr, C* __restrict__ wu, const double* __restrict__ sr,
                            const double* __restrict__ su, const double* __restrict__ rnf, int n1,
                            int n2, int h, double rho0, int ncol) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int wk = blockIdx.y;
    if (j >= n2) return;
    const int wall = wk / h, k = wk % h + 1;
    const int row = wall == 0 ? k - 1 : n1 - k;
    const size_t m = (size_t)wk * n2 + j;
    wr[m] = C(sr[m] * (rnf ? rho0 / rnf[(size_t)row * ncol + (ncol > 1 ? j : 0)] : 1.0));
    wu[m] = C(su[m]);
}

// Rest part of the total mass, rho0 times the total volume: FP64, one block,
// fixed order; each geometry entry covers `mult` cells (n2 for row geometry).
__global__ void __launch_bounds__(256) k_rest_mass(const double* __restrict__ geo, int stride, int count,
                                                   double mult, double rho0, double* __restrict__ out) {
    __shared__ double sh[256];
    double x = 0.0;
    for (int e = threadIdx.x; e < count; e += 256) x += geo[(size_t)e * stride + Geo::J];
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] * mult * rho0;
}

// Eq. 23, J <- J rho_nf / rho0, for every geometry entry (rows, or cells of a
// general grid) with its no-flow density rnf.
__global__ void k_scale_volume(double* __restrict__ geo, int stride, const double* __restrict__ rnf,
                               int count, double rho0) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= count) return;
    geo[(size_t)r * stride + Geo::J] *= rnf[r] / rho0;
}

__global__ void __launch_bounds__(256) k_row_mean(const double* __restrict__ f, int n2,
                                                  double* __restrict__ out) {
    __shared__ double sh[256];
    const int i = blockIdx.x;
    double x = 0.0;
    for (int j = threadIdx.x; j < n2; j += 256) x += f[(size_t)i * n2 + j];
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = sh[0] / n2;
}

template <int Q, typename S, typename C, bool GEN>
void run_moments_g(const MomArgs& a, int iters, int reduce, cudaStream_t s) {
    if (reduce) {
        const int nb = residual_blocks(a.n1, a.n2);
        if (iters > 0) k_residual<Q, S, C, true, GEN><<<nb, RB, 0, s>>>(a, iters);
        else k_residual<Q, S, C, false, GEN><<<nb, RB, 0, s>>>(a, iters);
    } else {
        dim3 b(RB), g((a.n2 + RB - 1) / RB, a.n1);
        if (iters > 0) k_moments<Q, S, C, true, GEN><<<g, b, 0, s>>>(a, iters);
        else k_moments<Q, S, C, false, GEN><<<g, b, 0, s>>>(a, iters);
    }
}

template <int Q, typename S, typename C>
void run_moments(const MomArgs& a, int iters, int reduce, cudaStream_t s) {
    if (a.ncol > 1) run_moments_g<Q, S, C, true>(a, iters, reduce, s);
    else run_moments_g<Q, S, C, false>(a, iters, reduce, s);
}

}  // namespace

int moments_blocks(int n1, int n2) { return residual_blocks(n1, n2); }

void launch_moments(int Q, int prec, const MomArgs& a, int iters, int reduce, cudaStream_t s) {
    if (Q == 9) {
        switch (prec) {
            case 0: run_moments<9, double, double>(a, iters, reduce, s); break;
            case 1: run_moments<9, float, float>(a, iters, reduce, s); break;
            case 2: run_moments<9, __half, float>(a, iters, reduce, s); break;
            default: run_moments<9, __nv_bfloat16, float>(a, iters, reduce, s); break;
        }
    } else {
        switch (prec) {
            case 0: run_moments<21, double, double>(a, iters, reduce, s); break;
            case 1: run_moments<21, float, float>(a, iters, reduce, s); break;
            case 2: run_moments<21, __half, float>(a, iters, reduce, s); break;
            default: run_moments<21, __nv_bfloat16, float>(a, iters, reduce, s); break;
        }
    }
}

void launch_reduce_final(const double* partial, int nblocks, double* out, cudaStream_t s) {
    k_reduce_final<<<NRED, 1024, 0, s>>>(partial, nblocks, out);
}

template <int Q>
static void from64(int prec, const double* Np, const double* geo, void* st, int n1, int n2, int ld,
                   int h, int ncol, cudaStream_t s) {
    dim3 b(128), g((n2 + 127) / 128, n1);
    switch (prec) {
        case 0: k_from_fp64<Q, double><<<g, b, 0, s>>>(Np, geo, (double*)st, n1, n2, ld, h, ncol); break;
        case 1: k_from_fp64<Q, float><<<g, b, 0, s>>>(Np, geo, (float*)st, n1, n2, ld, h, ncol); break;
        case 2: k_from_fp64<Q, __half><<<g, b, 0, s>>>(Np, geo, (__half*)st, n1, n2, ld, h, ncol); break;
        default: k_from_fp64<Q, __nv_bfloat16><<<g, b, 0, s>>>(Np, geo, (__nv_bfloat16*)st, n1, n2, ld, h, ncol); break;
    }
}

template <int Q>
static void to64(int prec, const void* st, const double* geo, double* Np, int n1, int n2, int ld,
                 int h, int ncol, cudaStream_t s) {
    dim3 b(128), g((n2 + 127) / 128, n1);
    switch (prec) {
        case 0: k_to_fp64<Q, double><<<g, b, 0, s>>>((const double*)st, geo, Np, n1, n2, ld, h, ncol); break;
        case 1: k_to_fp64<Q, float><<<g, b, 0, s>>>((const float*)st, geo, Np, n1, n2, ld, h, ncol); break;
        case 2: k_to_fp64<Q, __half><<<g, b, 0, s>>>((const __half*)st, geo, Np, n1, n2, ld, h, ncol); break;
        default: k_to_fp64<Q, __nv_bfloat16><<<g, b, 0, s>>>((const __nv_bfloat16*)st, geo, Np, n1, n2, ld, h, ncol); break;
    }
}

void launch_state_from_fp64(int Q, int prec, const double* Np, const double* geo, void* state,
                            int n1, int n2, int ld, int h, int ncol, cudaStream_t s) {
    if (Q == 9) from64<9>(prec, Np, geo, state, n1, n2, ld, h, ncol, s);
    else from64<21>(prec, Np, geo, state, n1, n2, ld, h, ncol, s);
}

void launch_state_to_fp64(int Q, int prec, const void* state, const double* geo, double* Np,
                          int n1, int n2, int ld, int h, int ncol, cudaStream_t s) {
    if (Q == 9) to64<9>(prec, state, geo, Np, n1, n2, ld, h, ncol, s);
    else to64<21>(prec, state, geo, Np, n1, n2, ld, h, ncol, s);
}

void launch_equilibrium(int Q, const double* rho, const double* U1, const double* U2,
                        const double* geo, double* Np, int n1, int n2, int ncol, double rho0,
                        cudaStream_t s) {
    dim3 b(128), g((n2 + 127) / 128, n1);
    if (Q == 9) k_equilibrium<9><<<g, b, 0, s>>>(rho, U1, U2, geo, Np, n1, n2, ncol, rho0);
    else k_equilibrium<21><<<g, b, 0, s>>>(rho, U1, U2, geo, Np, n1, n2, ncol, rho0);
}

void launch_wall_init(int prec, void* wr, void* wu, const double* rho, const double* ut2, int n1,
                      int n2, int h, double rho0, cudaStream_t s) {
    dim3 b(128), g((n2 + 127) / 128, 2 * h);
    if (prec == 0) k_wall_init<double><<<g, b, 0, s>>>((double*)wr, (double*)wu, rho, ut2, n1, n2, h, rho0);
    else k_wall_init<float><<<g, b, 0, s>>>((float*)wr, (float*)wu, rho, ut2, n1, n2, h, rho0);
}

void launch_wall_copy(int prec, void* wr, void* wu, const double* sr, const double* su,
                      const double* rnf, int n1, int n2, int h, double rho0, int ncol, cudaStream_t s) {
    dim3 b(128), g((n2 + 127) / 128, 2 * h);
    if (prec == 0) k_wall_copy<double><<<g, b, 0, s>>>((double*)wr, (double*)wu, sr, su, rnf, n1, n2, h, rho0, ncol);
    else k_wall_copy<float><<<g, b, 0, s>>>((float*)wr, (float*)wu, sr, su, rnf, n1, n2, h, rho0, ncol);
}

void launch_rest_mass(int Q, const double* geo, int count, int mult, double rho0, double* out,
                      cudaStream_t s) {
    k_rest_mass<<<1, 256, 0, s>>>(geo, Geo::stride(Q), count, double(mult), rho0, out);
}

void launch_scale_volume(int Q, double* geo, const double* rnf, int count, double rho0, cudaStream_t s) {
    k_scale_volume<<<(count + 127) / 128, 128, 0, s>>>(geo, Geo::stride(Q), rnf, count, rho0);
}

void launch_row_mean(const double* f, int n1, int n2, double* out, cudaStream_t s) {
    k_row_mean<<<n1, 256, 0, s>>>(f, n2, out);
}

}  // namespace clbm
