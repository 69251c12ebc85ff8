// k_batch.cu -- many lattices of uneven shapes advanced by one persistent
// launch per phase over a tile work-list.
//
// Every lattice keeps its own state, tables and walls (a clbm_grid); the
// batch holds a device array of their descriptors and three work-lists:
// boundary items (ghost rows of both walls, periodic ghost columns), update
// tiles and diagnostics tiles.  Persistent CTAs stride over the work-list, so
// one launch covers all lattices whatever their sizes.  The per-cell
// arithmetic is the same code as the single-lattice kernels
// (clbm_cell.cuh).  Tile shape and cells per thread are template parameters;
// the host autotuner times the compiled variants on the batch.
#include "clbm_batch.cuh"
#include "clbm_cell.cuh"

namespace clbm {
namespace {

// Update tile of variant V: TJ columns x TR rows, CPT cells per thread
// along the row (cells j and j + TJ / CPT).
template <int V> struct Var;
template <> struct Var<0> { static constexpr int TJ = 128, TR = 1, CPT = 1, NT = 128; };
template <> struct Var<1> { static constexpr int TJ = 256, TR = 1, CPT = 2, NT = 128; };
template <> struct Var<2> { static constexpr int TJ = 32, TR = 4, CPT = 1, NT = 128; };
template <> struct Var<3> { static constexpr int TJ = 64, TR = 1, CPT = 1, NT = 64; };

template <int Q, typename S, typename C, bool ITER>
__device__ __forceinline__ void batch_cell(const BatchGrid& g, int src, int i, int j) {
    using T = Tab<Q>;
    constexpr int H = Lat<Q>::H;
    const RowTab<Q, C> tb{(const C*)g.tab + (size_t)i * T::S};
    const Consts<C> k = Consts<C>::make(g.k);
    const long long off = (long long)(i + H) * g.ld + j + GC;
    Cell<Q, C> c;
    pull_cell<Q, C>(GlobalLoad<S>{(const S*)g.phys[src] + off, (int)g.plane, g.ld}, tb, k, c);
    S* dst = (S*)g.phys[src ^ 1] + off;
    const int dw = wrap_offset(j, g.n2);
    auto put = [&](int al, C v) {
        Store<S>::st(dst + al * g.plane, v);
        if (dw != 0) Store<S>::st(dst + al * g.plane + dw, v);
    };
    if (!ITER) {
        collide_emit<Q, C>(tb, c, k, put);
    } else {
        C out[Q];
        collide_emit<Q, C>(tb, c, k, [&](int al, C v) { out[al] = v; });
        for (int it = 0; it < g.iters; ++it) {
            force_again<Q, C>(tb, out, k, c);
            collide_emit<Q, C>(tb, c, k, [&](int al, C v) { out[al] = v; });
        }
#pragma unroll
        for (int al = 0; al < Q; ++al) put(al, out[al]);
    }
    if (EdgeFill<Q, S>::needed(i, g.n1, g.n2)) {
        const EdgeFill<Q, S> ef{(S*)g.phys[src ^ 1], (const C*)g.ghost, g.plane, g.ld, g.n1, g.n2, g.bc_lo,
                                g.bc_hi, C(g.U0_lo), C(g.U0_hi), g.n2 < 2 * GC, 1};
        ef.fill(i, j, dst, g.plane, c.rho, c.Ut2);
    }
    if (i < H) {
        const int idx = i * g.n2 + j;
        ((C*)g.wall_rho)[idx] = c.rho;
        ((C*)g.wall_ut2)[idx] = c.Ut2;
    }
    if (i >= g.n1 - H) {
        const int idx = (H + (g.n1 - 1 - i)) * g.n2 + j;
        ((C*)g.wall_rho)[idx] = c.rho;
        ((C*)g.wall_ut2)[idx] = c.Ut2;
    }
}

template <int Q, typename S, typename C, int V, bool ITER>
__global__ void __launch_bounds__(Var<V>::NT, ITER ? 2 : 4) k_batch_step(const BatchGrid* __restrict__ grids,
                                                          const int4* __restrict__ work, int nwork,
                                                          int parity) {
    using W = Var<V>;
    for (int e = blockIdx.x; e < nwork; e += gridDim.x) {
        const int4 w = work[e];  // (grid, row0, col0, -)
        const BatchGrid& g = grids[w.x];
        const int src = g.parity ^ parity;
        const int tr = threadIdx.x / (W::TJ / W::CPT), tc = threadIdx.x % (W::TJ / W::CPT);
        const int i = w.y + tr;
        if (i >= g.n1) continue;
#pragma unroll
        for (int q = 0; q < W::CPT; ++q) {
            const int j = w.z + tc + q * (W::TJ / W::CPT);
            if (j < g.n2) batch_cell<Q, S, C, ITER>(g, src, i, j);
        }
    }
}

// Boundary items: w = (grid, kind, start, -); kind 0 / 1 ghost rows of the
// low / high wall for columns start..start+127, kind 2 periodic ghost columns
// of (population, row) pairs start..start+7, a half-warp per pair.  Needed
// only when a lattice's state or case was set from outside: the update keeps
// ghost rows and columns current.
template <int Q, typename S, typename C>
__global__ void __launch_bounds__(128) k_batch_boundary(const BatchGrid* __restrict__ grids,
                                                       const int4* __restrict__ work, int nwork,
                                                       int parity) {
    constexpr int H = Lat<Q>::H;
    for (int e = blockIdx.x; e < nwork; e += gridDim.x) {
        const int4 w = work[e];
        const BatchGrid& g = grids[w.x];
        S* st = (S*)g.phys[g.parity ^ parity];
        const long long P = g.plane;
        if (w.y == 2) {
            const int pr = w.z + threadIdx.x / (2 * GC), x = threadIdx.x % (2 * GC);
            if (pr >= g.n1 * Q) continue;
            const int al = pr / g.n1, i = pr % g.n1;
            S* rowp = st + al * P + (long long)(i + H) * g.ld;
            const int cs = x < GC ? x : g.n2 + x;
            int jw = (cs - GC) % g.n2;
            if (jw < 0) jw += g.n2;
            rowp[cs] = rowp[jw + GC];
            continue;
        }
        const int t = w.z + threadIdx.x;
        const int j = t, wall = w.y;
        if (j >= g.n2) continue;
        const int bc = wall == 0 ? g.bc_lo : g.bc_hi;
        const C U0 = C(wall == 0 ? g.U0_lo : g.U0_hi);
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            const int gr = wall == 0 ? H - k : g.n1 + H + k - 1;
            const int mr = wall == 0 ? H + k - 1 : g.n1 + H - k;
            const int widx = (wall * H + (k - 1)) * g.n2 + j;
            const C wr = ((const C*)g.wall_rho)[widx];
            const C wu = ((const C*)g.wall_ut2)[widx];
#pragma unroll
            for (int al = 1; al < Q; ++al) {
                const int c1 = c1_of(al);
                if (wall == 0 ? (c1 < k) : (c1 > -k)) continue;
                const int b = bc == 0 ? opp_of(al) : hat_of(al);
                const C* gt = (const C*)g.ghost + 2 * ((wall * H + (k - 1)) * Q + al);
                const C x = C(Store<S>::ld(st + b * P + (long long)mr * g.ld + j + GC));
                store_periodic<S, C>(st + al * P + (long long)gr * g.ld, j, g.n2,
                                     ghost_value<C>(x, gt, wr, U0, wu));
            }
        }
    }
}

// Diagnostics tiles (128 cells of one row): the per-lattice residual and
// conservation sums of clbm_residual, one partial per work item (the same
// per-cell terms as k_residual).  ITER: lattices that iterate the force.
template <int Q, typename S, typename C, bool ITER>
__global__ void __launch_bounds__(128, ITER ? 2 : 4) k_batch_moments(const BatchGrid* __restrict__ grids,
                                                      const int4* __restrict__ work, int nwork,
                                                      int parity, double* __restrict__ partial) {
    using T = Tab<Q>;
    constexpr int H = Lat<Q>::H;
    __shared__ double sh[4][NRED];
    for (int e = blockIdx.x; e < nwork; e += gridDim.x) {
        const int4 w = work[e];
        const BatchGrid& g = grids[w.x];
        const int src = g.parity ^ parity;
        const int i = w.y, j = w.z + threadIdx.x;
        double v[NRED];
#pragma unroll
        for (int q = 0; q < NRED; ++q) v[q] = 0.0;
        if (j < g.n2) {
            const RowTab<Q, C> tb{(const C*)g.tab + (size_t)i * T::S};
            const Consts<C> kc = Consts<C>::make(g.k);
            const long long off = (long long)(i + H) * g.ld + j + GC;
            const S* p = (const S*)g.phys[src] + off;
            Cell<Q, C> c;
            pull_cell<Q, C>(GlobalLoad<S>{p, (int)g.plane, g.ld}, tb, kc, c);
            if (ITER) {
                C out[Q];
                collide_emit<Q, C>(tb, c, kc, [&](int al, C x) { out[al] = x; });
                for (int it = 0; it < g.iters; ++it) {
                    force_again<Q, C>(tb, out, kc, c);
                    collide_emit<Q, C>(tb, c, kc, [&](int al, C x) { out[al] = x; });
                }
            } else {
                collide_emit<Q, C>(tb, c, kc, [](int, C) {});
            }
            const size_t m = (size_t)i * g.n2 + j, nc = (size_t)g.n1 * g.n2;
            C* prev = (C*)g.prev;
            ResAcc<C> acc;
            acc.add(residual_terms<Q, C>(c, tb, prev + m, prev + nc + m, g.have_prev != 0));
            acc.out(v);
        }
#pragma unroll
        for (int q = 0; q < NRED; ++q) {
            double x = v[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double y = __shfl_down_sync(0xffffffffu, x, o);
                x = q == 7 ? fmax(x, y) : x + y;
            }
            if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][q] = x;
        }
        __syncthreads();
        if (threadIdx.x < NRED) {
            const int q = threadIdx.x;
            double x = sh[0][q];
            for (int ww = 1; ww < 4; ++ww) x = q == 7 ? fmax(x, sh[ww][q]) : x + sh[ww][q];
            partial[(size_t)e * NRED + q] = q == 7 ? sqrt(x) : x;
        }
        __syncthreads();
    }
}

// One block per lattice: its contiguous range of diagnostics items, in order.
__global__ void __launch_bounds__(256) k_batch_reduce(const double* __restrict__ partial,
                                                     const int2* __restrict__ range,
                                                     double* __restrict__ out) {
    __shared__ double sh[256];
    const int2 rg = range[blockIdx.x];
    for (int q = 0; q < NRED; ++q) {
        double x = 0.0;
        for (int e = rg.x + threadIdx.x; e < rg.y; e += 256) {
            const double y = partial[(size_t)e * NRED + q];
            x = q == 7 ? fmax(x, y) : x + y;
        }
        sh[threadIdx.x] = x;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s)
                sh[threadIdx.x] = q == 7 ? fmax(sh[threadIdx.x], sh[threadIdx.x + s])
                                         : sh[threadIdx.x] + sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[(size_t)blockIdx.x * NRED + q] = sh[0];
        __syncthreads();
    }
}

template <int Q, typename S, typename C>
void step_variant(int v, const BatchGrid* grids, const int4* work, int nwork, int parity, int nblk,
                  cudaStream_t s) {
    switch (v) {
        case 0: k_batch_step<Q, S, C, 0, false><<<nblk, Var<0>::NT, 0, s>>>(grids, work, nwork, parity); break;
        case 1: k_batch_step<Q, S, C, 1, false><<<nblk, Var<1>::NT, 0, s>>>(grids, work, nwork, parity); break;
        case 2: k_batch_step<Q, S, C, 2, false><<<nblk, Var<2>::NT, 0, s>>>(grids, work, nwork, parity); break;
        default: k_batch_step<Q, S, C, 3, false><<<nblk, Var<3>::NT, 0, s>>>(grids, work, nwork, parity); break;
    }
}

template <int Q, typename S, typename C>
void run_all(int what, int v, const BatchGrid* grids, const int4* work, int nwork, int parity,
             int nblk, double* partial, cudaStream_t s) {
    if (what == 0) k_batch_boundary<Q, S, C><<<nblk, 128, 0, s>>>(grids, work, nwork, parity);
    else if (what == 1) step_variant<Q, S, C>(v, grids, work, nwork, parity, nblk, s);
    else if (what == 3) k_batch_step<Q, S, C, 0, true><<<nblk, Var<0>::NT, 0, s>>>(grids, work, nwork, parity);
    else if (what == 4) k_batch_moments<Q, S, C, true><<<nblk, 128, 0, s>>>(grids, work, nwork, parity, partial);
    else k_batch_moments<Q, S, C, false><<<nblk, 128, 0, s>>>(grids, work, nwork, parity, partial);
}

}  // namespace

void batch_tile_shape(int variant, int* tj, int* tr) {
    switch (variant) {
        case 0: *tj = Var<0>::TJ; *tr = Var<0>::TR; break;
        case 1: *tj = Var<1>::TJ; *tr = Var<1>::TR; break;
        case 2: *tj = Var<2>::TJ; *tr = Var<2>::TR; break;
        case 3: *tj = Var<3>::TJ; *tr = Var<3>::TR; break;
        default: *tj = 64; *tr = 8; break;  // BATCH_WS: the TMA tile of k_step_tma.cu
    }
}

void launch_batch(int Q, int prec, int what, int variant, const BatchGrid* grids, const int4* work,
                  int nwork, int parity, int nblk, double* partial, cudaStream_t s) {
    if (nwork <= 0) return;
    if (Q == 9) {
        switch (prec) {
            case 0: run_all<9, double, double>(what, variant, grids, work, nwork, parity, nblk, partial, s); break;
            case 1: run_all<9, float, float>(what, variant, grids, work, nwork, parity, nblk, partial, s); break;
            case 2: run_all<9, __half, float>(what, variant, grids, work, nwork, parity, nblk, partial, s); break;
            default: run_all<9, __nv_bfloat16, float>(what, variant, grids, work, nwork, parity, nblk, partial, s); break;
        }
    } else {
        switch (prec) {
            case 0: run_all<21, double, double>(what, variant, grids, work, nwork, parity, nblk, partial, s); break;
            case 1: run_all<21, float, float>(what, variant, grids, work, nwork, parity, nblk, partial, s); break;
            case 2: run_all<21, __half, float>(what, variant, grids, work, nwork, parity, nblk, partial, s); break;
            default: run_all<21, __nv_bfloat16, float>(what, variant, grids, work, nwork, parity, nblk, partial, s); break;
        }
    }
}

void launch_batch_reduce(const double* partial, const int2* range, int ngrids, double* out,
                         cudaStream_t s) {
    k_batch_reduce<<<ngrids, 256, 0, s>>>(partial, range, out);
}

}  // namespace clbm
