// k_step.cu -- the fused stream-collide-force update (Sec. 2, Eqs. 6-19)
// and the boundary ghost fill (App. B).
//
// One thread per cell; a warp covers 32 consecutive cells of one row, so every
// per-row coefficient is a warp-uniform load and every population access is a
// coalesced row segment at a constant offset (ghost rows and periodic ghost
// columns surround the interior).  Cells next to a periodic end also store
// their value's periodic copy, and cells next to a wall the ghost values they
// supply (EdgeFill), so one launch per time step leaves the written buffer
// ready to be pulled from.  Lagged values are consumed as they are
// loaded and new populations are stored as they are produced, so a thread
// holds only the Q pulled deviations and the pair odd parts.  Populations are
// deviations from the rest equilibrium of their own row (zero at rest), so
// the large rest part never enters a rounding-sensitive difference.
#include "clbm_cell.cuh"

namespace clbm {

namespace {

template <int Q, typename S, typename C, bool ITER, bool GEN>
__global__ void __launch_bounds__(128, ITER ? 2 : (GEN ? 3 : 4)) k_fused_step(const StepArgs a) {
    using L = Lat<Q>;
    constexpr int H = L::H;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= a.n2) return;
    const auto tb = TabOf<Q, C, GEN>::at(a.tab, i, j, a.n1, a.n2);
    const Consts<C> k = Consts<C>::make(a.k);
    const int row = i + H;
    const long long off = (long long)row * a.ld + j + GC;
    Cell<Q, C> c;
    const int pl = (int)a.plane;
    pull_cell<Q, C>(GlobalLoad<S>{(const S*)a.src + off, pl, a.ld}, tb, k, c);
    S* dst = (S*)a.dst + off;
    const int dw = wrap_offset(j, a.n2);
    auto put = [&](int al, C v) {
        StStream<S>::st(dst + al * pl, v);
        if (dw != 0) StStream<S>::st(dst + (al * pl + dw), v);
    };
    if (!ITER) {
        collide_emit<Q, C>(tb, c, k, put);
    } else {
        C out[Q];
        collide_emit<Q, C>(tb, c, k, [&](int al, C v) { out[al] = v; });
        for (int it = 0; it < a.iters; ++it) {
            force_again<Q, C>(tb, out, k, c);
            collide_emit<Q, C>(tb, c, k, [&](int al, C v) { out[al] = v; });
        }
#pragma unroll
        for (int al = 0; al < Q; ++al) put(al, out[al]);
    }
    if (EdgeFill<Q, S>::needed(i, a.n1, a.n2)) {
        const EdgeFill<Q, S> ef{(S*)a.dst, (const C*)a.ghost, a.plane, a.ld, a.n1, a.n2, a.bc_lo, a.bc_hi,
                                C(a.U0_lo), C(a.U0_hi), a.n2 < 2 * GC, a.ncol};
        ef.fill(i, j, dst, a.plane, c.rho, c.Ut2);
    }
    // Near-wall rows keep rho and Ut^2 for the moving-wall correction (App. B).
    if (i < H) {
        const int idx = (0 * H + i) * a.n2 + j;
        ((C*)a.wall_rho)[idx] = c.rho;
        ((C*)a.wall_ut2)[idx] = c.Ut2;
    }
    if (i >= a.n1 - H) {
        const int idx = (1 * H + (a.n1 - 1 - i)) * a.n2 + j;
        ((C*)a.wall_rho)[idx] = c.rho;
        ((C*)a.wall_ut2)[idx] = c.Ut2;
    }
}

// Ghost rows of both walls (App. B), blockIdx.y = 0 / 1: for every direction
// that enters the fluid through a wall, the ghost value is the mirrored
// fluid node's N' of the reversed (no-slip) or reflected (moving wall)
// direction, plus the moving-wall correction; one thread per column.
// blockIdx.y = 2: periodic ghost columns of the interior rows; a half-warp
// copies the 2 GC ghost columns of one (population, row).  Together they make
// a buffer whose state was set from outside ready to be pulled from (the
// update keeps them current afterwards).
template <int Q, typename S, typename C>
__global__ void __launch_bounds__(128) k_boundary(const StepArgs a, S* __restrict__ st) {
    constexpr int H = Lat<Q>::H;
    const long long P = a.plane;
    if (blockIdx.y == 2) {
        const int t = blockIdx.x * blockDim.x + threadIdx.x;
        const int pr = t / (2 * GC), e = t % (2 * GC);
        if (pr >= a.n1 * Q) return;
        const int al = pr / a.n1, i = pr % a.n1;
        S* rowp = st + al * P + (long long)(i + H) * a.ld;
        const int cs = e < GC ? e : a.n2 + e;  // ghost state column
        int jw = (cs - GC) % a.n2;
        if (jw < 0) jw += a.n2;
        rowp[cs] = rowp[jw + GC];
        return;
    }
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int wall = blockIdx.y;
    if (j >= a.n2) return;
    const int bc = wall == 0 ? a.bc_lo : a.bc_hi;
    const C U0 = C(wall == 0 ? a.U0_lo : a.U0_hi);
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        const int gr = wall == 0 ? H - k : a.n1 + H + k - 1;    // ghost state row
        const int mr = wall == 0 ? H + k - 1 : a.n1 + H - k;    // mirrored fluid state row
        const int widx = (wall * H + (k - 1)) * a.n2 + j;
        const C wr = ((const C*)a.wall_rho)[widx];
        const C wu = ((const C*)a.wall_ut2)[widx];
#pragma unroll
        for (int al = 1; al < Q; ++al) {
            const int c1 = c1_of(al);
            if (wall == 0 ? (c1 < k) : (c1 > -k)) continue;
            const int b = bc == 0 ? opp_of(al) : hat_of(al);
            const C* gt = (const C*)a.ghost + 2 * (((wall * H + (k - 1)) * Q + al) * a.ncol + (a.ncol > 1 ? j : 0));
            const C x = C(Store<S>::ld(st + b * P + (long long)mr * a.ld + j + GC));
            store_periodic<S, C>(st + al * P + (long long)gr * a.ld, j, a.n2,
                                 ghost_value<C>(x, gt, wr, U0, wu));
        }
    }
}

template <int Q, typename S, typename C>
void run_step(const StepArgs& a, cudaStream_t s) {
    dim3 b(128), g((a.n2 + 127) / 128, a.n1);
    if (a.ncol > 1) {
        if (a.iters > 0) k_fused_step<Q, S, C, true, true><<<g, b, 0, s>>>(a);
        else k_fused_step<Q, S, C, false, true><<<g, b, 0, s>>>(a);
    } else {
        if (a.iters > 0) k_fused_step<Q, S, C, true, false><<<g, b, 0, s>>>(a);
        else k_fused_step<Q, S, C, false, false><<<g, b, 0, s>>>(a);
    }
}

template <int Q, typename S, typename C>
void run_boundary(const StepArgs& a, void* st, cudaStream_t s) {
    const int nx = (a.n2 + 127) / 128, ny = (a.n1 * Q * 2 * GC + 127) / 128;
    dim3 b(128), g(nx > ny ? nx : ny, 3);
    k_boundary<Q, S, C><<<g, b, 0, s>>>(a, (S*)st);
}

}  // namespace

void launch_step(int Q, int prec, const StepArgs& a, cudaStream_t s) {
    if (Q == 9) {
        switch (prec) {
            case 0: run_step<9, double, double>(a, s); break;
            case 1: run_step<9, float, float>(a, s); break;
            case 2: run_step<9, __half, float>(a, s); break;
            default: run_step<9, __nv_bfloat16, float>(a, s); break;
        }
    } else {
        switch (prec) {
            case 0: run_step<21, double, double>(a, s); break;
            case 1: run_step<21, float, float>(a, s); break;
            case 2: run_step<21, __half, float>(a, s); break;
            default: run_step<21, __nv_bfloat16, float>(a, s); break;
        }
    }
}

void launch_boundary(int Q, int prec, const StepArgs& a, void* st, cudaStream_t s) {
    if (Q == 9) {
        switch (prec) {
            case 0: run_boundary<9, double, double>(a, st, s); break;
            case 1: run_boundary<9, float, float>(a, st, s); break;
            case 2: run_boundary<9, __half, float>(a, st, s); break;
            default: run_boundary<9, __nv_bfloat16, float>(a, st, s); break;
        }
    } else {
        switch (prec) {
            case 0: run_boundary<21, double, double>(a, st, s); break;
            case 1: run_boundary<21, float, float>(a, st, s); break;
            case 2: run_boundary<21, __half, float>(a, st, s); break;
            default: run_boundary<21, __nv_bfloat16, float>(a, st, s); break;
        }
    }
}

}  // namespace clbm
