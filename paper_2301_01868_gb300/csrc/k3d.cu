// k3d.cu -- the three-dimensional update on D3Q39 (Sec. 2 in three
// coordinates) and its C ABI (clbm3.h).
//
// Layout: deviations sigma_a = N'_a - ref_a(i) in the storage type, one
// plane per population of (n1 + 2H) x n2 x n3 values, rows 0..H-1 and
// n1+H..n1+2H-1 the ghost rows of App. B (written by the update itself for
// the buffer it writes, from the mirrored cells' new values and moments;
// by k3_boundary, from the stored state, after a new state or case),
// q^2 and q^3 periodic by index wrap.  The geometry of a row (the grids are
// invariant along q^2 and q^3) is evaluated once in FP64 (k3_geometry,
// k3_reference) and condensed into a per-row table in the compute type
// (k3_tables).  One thread per cell (k3_step): pull with the lagged read,
// moments, lagged force, Ut, the odd part of f^eq for the momentum-flux
// correction, dN and BGK, written in deviations as the 2-D kernels are.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include "clbm3.cuh"
#include "clbm3.h"
#include "clbm_cell.cuh"

namespace clbm {
namespace d3 {
namespace {

constexpr int TB = 128;  // threads per block of the cell kernels

__device__ __forceinline__ int wrapm(int x, int n) {
    while (x < 0) x += n;
    while (x >= n) x -= n;
    return x;
}

// x in [-3, n + 3) mapped into [0, n): one conditional correction when the
// extent is at least 4 (every shift of the lattice is at most 3), the loop
// of wrapm for the narrower extents.
__device__ __forceinline__ int wrap3(int x, int n) {
    if (n < 4) return wrapm(x, n);
    x = x < 0 ? x + n : x;
    return x >= n ? x - n : x;
}

// ------------------------------------------------------------- geometry

struct Shape {
    int kind, n1, n2;
    const double* edges;    // device, n1 + 1
    double step2, step3, dx;
};

// Wall-normal node coordinate of 1-based row i: midpoints of the edges
// inside (App. C), mirror images through the walls outside (App. B).
__device__ double node_coord(const Shape& s, int i) {
    const double* e = s.edges;
    if (i >= 1 && i <= s.n1) return 0.5 * (e[i - 1] + e[i]);
    if (i < 1) {
        const int m = 1 - i;
        return 2.0 * e[0] - 0.5 * (e[m - 1] + e[m]);
    }
    const int m = s.n1 + 1 - (i - s.n1);
    return 2.0 * e[s.n1] - 0.5 * (e[m - 1] + e[m]);
}

__device__ void node_pos(const Shape& s, int i, int j, int k, double x[3]) {
    const double r = node_coord(s, i);
    if (s.kind == CLBM3_CHANNEL) {
        x[0] = r;
        x[1] = (j - 0.5) * s.step2;
    } else {
        const double th = (j - 0.5) * (2.0 * 3.14159265358979323846 / s.n2);
        x[0] = r * cos(th);
        x[1] = r * sin(th);
    }
    x[2] = (k - 0.5) * s.step3;
}

// Tangent vector g_m at node (i, j, k): central difference of the node
// positions over the grid step, divided by 2 Delta x (Eq. 1 and below).
__device__ void tangent(const Shape& s, int m, int i, int j, int k, double t[3]) {
    double xp[3], xm[3];
    node_pos(s, i + (m == 0), j + (m == 1), k + (m == 2), xp);
    node_pos(s, i - (m == 0), j - (m == 1), k - (m == 2), xm);
    for (int r = 0; r < 3; ++r) t[r] = (xp[r] - xm[r]) / (2.0 * s.dx);
}

__device__ void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Row i: J = g_1 . (g_2 x g_3), g^1 = g_2 x g_3 / J and cyclic, g^{pq}, g_pq
// (Eqs. 2, 3), and a^k_a = sum_m c^m_a (g_m(q + c_a) - g_m(q)) . g^k (Eq. 5).
__global__ void k3_geometry(Shape s, double* __restrict__ geo) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= s.n1) return;
    const int i = r + 1;
    double t[3][3], u[3][3];
    for (int m = 0; m < 3; ++m) tangent(s, m, i, 1, 1, t[m]);
    double c12[3];
    cross3(t[1], t[2], c12);
    const double J = dot3(t[0], c12);
    for (int m = 0; m < 3; ++m) {
        double c[3];
        cross3(t[(m + 1) % 3], t[(m + 2) % 3], c);
        for (int q = 0; q < 3; ++q) u[m][q] = c[q] / J;
    }
    double* o = geo + (size_t)r * Geo3::S;
    o[Geo3::J] = J;
    const int P[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int q = 0; q < 6; ++q) {
        o[Geo3::GI + q] = dot3(u[P[q][0]], u[P[q][1]]);
        o[Geo3::GC + q] = dot3(t[P[q][0]], t[P[q][1]]);
    }
    for (int a = 0; a < Q; ++a) {
        const int c[3] = {c1_3(a), c2_3(a), c3_3(a)};
        double acc[3] = {0.0, 0.0, 0.0};
        for (int m = 0; m < 3; ++m) {
            if (c[m] == 0) continue;
            double tn[3], d[3];
            tangent(s, m, i + c[0], 1 + c[1], 1 + c[2], tn);
            for (int q = 0; q < 3; ++q) d[q] = tn[q] - t[m][q];
            for (int kk = 0; kk < 3; ++kk) acc[kk] += c[m] * dot3(d, u[kk]);
        }
        for (int kk = 0; kk < 3; ++kk) o[Geo3::A + 3 * a + kk] = acc[kk];
    }
}

// Rest polynomial of Eq. 19 at U = Ut = 0: 1 + [c.(g - 1).c / T0 - tr(g - 1)] / 2.
__device__ double rest_poly3(int a, const double* gi) {
    const double c[3] = {(double)c1_3(a), (double)c2_3(a), (double)c3_3(a)};
    const double e11 = gi[0] - 1.0, e12 = gi[1], e13 = gi[2], e22 = gi[3] - 1.0, e23 = gi[4],
                 e33 = gi[5] - 1.0;
    const double q = c[0] * c[0] * e11 + c[1] * c[1] * e22 + c[2] * c[2] * e33 +
                     2.0 * (c[0] * c[1] * e12 + c[0] * c[2] * e13 + c[1] * c[2] * e23);
    return 1.0 + 0.5 * (q / T0 - (e11 + e22 + e33));
}

__global__ void k3_reference(double* __restrict__ geo, int n1, double rho0) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n1) return;
    double* o = geo + (size_t)r * Geo3::S;
    for (int a = 0; a < Q; ++a) o[Geo3::REF + a] = o[Geo3::J] * w3(a) * rho0 * rest_poly3(a, o + Geo3::GI);
}

// Reference of direction a at 1-based row i; rows beyond a wall are the
// mirror images of the rows inside, which flips c^1.
__device__ double ref_row(const double* geo, int n1, int a, int i) {
    if (i < 1) return geo[(size_t)(-i) * Geo3::S + Geo3::REF + hat3(a)];
    if (i > n1) return geo[(size_t)(2 * n1 - i) * Geo3::S + Geo3::REF + hat3(a)];
    return geo[(size_t)(i - 1) * Geo3::S + Geo3::REF + a];
}

template <typename C>
__global__ void k3_tables(const double* __restrict__ geo, C* __restrict__ tab, int n1) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n1) return;
    const int i = r + 1;
    const double* g = geo + (size_t)r * Geo3::S;
    C* t = tab + (size_t)r * Tab3::S;
    for (int q = 0; q < Tab3::S; ++q) t[q] = C(0);
    const double J = g[Geo3::J];
    t[Tab3::INVJ] = C(1.0 / J);
    t[Tab3::J] = C(J);
    for (int q = 0; q < 6; ++q) {
        t[Tab3::G11 + q] = C(g[Geo3::GI + q]);
        t[Tab3::C11 + q] = C(g[Geo3::GC + q]);
    }
    double F0[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < Q; ++a) {
        const int b = opp3(a);
        const double ref = g[Geo3::REF + a];
        for (int k = 0; k < 3; ++k) F0[k] += (g[Geo3::A + 3 * a + k] + g[Geo3::A + 3 * b + k]) * ref;
        t[Tab3::P0 + a] = C(rest_poly3(a, g + Geo3::GI));
    }
    for (int p = 0; p < NP; ++p) {
        const int a = plus3(p), b = opp3(a);
        for (int k = 0; k < 3; ++k) {
            t[Tab3::PA(p) + 2 * k] = C(g[Geo3::A + 3 * b + k]);
            t[Tab3::PA(p) + 2 * k + 1] = C(g[Geo3::A + 3 * a + k]);
        }
        t[Tab3::PA(p) + 6] = C(ref_row(geo, n1, a, i - c1_3(a)) - g[Geo3::REF + a]);
        t[Tab3::PA(p) + 7] = C(ref_row(geo, n1, b, i - c1_3(b)) - g[Geo3::REF + b]);
    }
    for (int k = 0; k < 3; ++k) t[Tab3::F0 + k] = C(F0[k]);
    const int P[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int p = 0; p < NP; ++p) {
        const int a = plus3(p), b = opp3(a);
        const double c[3] = {(double)c1_3(a), (double)c2_3(a), (double)c3_3(a)};
        double D[3];
        for (int k = 0; k < 3; ++k) D[k] = g[Geo3::A + 3 * a + k] + g[Geo3::A + 3 * b + k];
        for (int q = 0; q < 6; ++q) {
            const int x = P[q][0], y = P[q][1];
            t[Tab3::E(p) + q] = C(w3(a) * (c[x] * D[y] + c[y] * D[x]));
        }
    }
}

// ------------------------------------------------------------- kernels

template <typename C>
__device__ __forceinline__ C* wall_ptr(void* wall, int field, int w, int m, int n23) {
    return (C*)wall + ((size_t)(field * 2 + w) * H + (m - 1)) * n23;
}

// Ghost rows of App. B for the buffer the next update reads: at depth m of
// the low wall the directions with c^1 >= m (high wall: <= -m) take the
// mirrored fluid node's N'_{a*} (no-slip) or N'_{a-hat} plus the moving-wall
// term (2/T0) w J rho [c^2 (U0 - Ut^2) + c^3 (0 - Ut^3)] from the last
// collision's moments there; stored as deviations from the ghost row's
// reference (the mirrored row's reference of a-hat).
template <typename S, typename C>
__global__ void __launch_bounds__(TB) k3_boundary(Args3 A, S* __restrict__ st) {
    const int n23 = A.n2 * A.n3;
    const int jk = blockIdx.x * blockDim.x + threadIdx.x;
    if (jk >= n23) return;
    const int wall = blockIdx.y / H, m = blockIdx.y % H + 1;
    const int gi = wall == 0 ? 1 - m : A.n1 + m;       // ghost row (1-based)
    const int mi = wall == 0 ? m : A.n1 + 1 - m;       // mirrored fluid row
    const bool moving = (wall == 0 ? A.bc_lo : A.bc_hi) == CLBM_BC_MOVING;
    const C U0 = C(wall == 0 ? A.U0_lo : A.U0_hi);
    const double* g = A.geo + (size_t)(mi - 1) * Geo3::S;
    const C rho = wall_ptr<C>(A.wall, 0, wall, m, n23)[jk];
    const C u2 = wall_ptr<C>(A.wall, 1, wall, m, n23)[jk];
    const C u3 = wall_ptr<C>(A.wall, 2, wall, m, n23)[jk];
    const C coef = C(2.0 / T0) * C(g[Geo3::J]) * rho;
    const S* src = st + (size_t)(mi - 1 + H) * n23 + jk;
    S* dst = st + (size_t)(gi - 1 + H) * n23 + jk;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int c1 = c1_3(a);
        if (wall == 0 ? c1 < m : c1 > -m) continue;
        const int h = hat3(a);
        C v;
        if (moving) {
            v = Store<S>::ld(src + (size_t)h * A.plane) +
                coef * C(w3(h)) * (C(c2_3(h)) * (U0 - u2) + C(c3_3(h)) * (C(0) - u3));
        } else {
            const int b = opp3(a);
            v = Store<S>::ld(src + (size_t)b * A.plane) + C(g[Geo3::REF + b] - g[Geo3::REF + h]);
        }
        Store<S>::st(dst + (size_t)a * A.plane, v);
    }
}

// The ghost populations of depth m of one wall in column jk of the buffer
// the update writes, from the mirrored fluid cell's new values (its row is
// m, or n1 + 1 - m at the high wall) and moments -- what k3_boundary
// computes from the stored state, with the same arithmetic, so that the
// update leaves the next step's ghost rows filled.  own: the cell's offset
// in its population plane.  The values were just stored by this thread and
// are read back through the coherent path.
template <typename S, typename C>
__device__ __forceinline__ void ghost_column(const Args3& A, int wall, int m, int jk, unsigned own, C rho,
                                             C u2, C u3) {
    const int n23 = A.n2 * A.n3;
    const int gi = wall == 0 ? 1 - m : A.n1 + m;           // ghost row (1-based)
    const int mi = wall == 0 ? m : A.n1 + 1 - m;           // mirrored fluid row
    const bool moving = (wall == 0 ? A.bc_lo : A.bc_hi) == CLBM_BC_MOVING;
    const C U0 = C(wall == 0 ? A.U0_lo : A.U0_hi);
    const double* g = A.geo + (size_t)(mi - 1) * Geo3::S;
    const C coef = C(2.0 / T0) * C(g[Geo3::J]) * rho;
    const S* src = (const S*)A.dst + own;
    S* dst = (S*)A.dst + (size_t)(gi - 1 + H) * n23 + jk;
    const size_t pl = (size_t)A.plane;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int c1 = c1_3(a);
        if (wall == 0 ? c1 < m : c1 > -m) continue;
        const int h = hat3(a);
        C v;
        if (moving) {
            v = Store<S>::lds(src + (size_t)h * pl) +
                coef * C(w3(h)) * (C(c2_3(h)) * (U0 - u2) + C(c3_3(h)) * (C(0) - u3));
        } else {
            const int b = opp3(a);
            v = Store<S>::lds(src + (size_t)b * pl) + C(g[Geo3::REF + b] - g[Geo3::REF + h]);
        }
        Store<S>::st(dst + (size_t)a * pl, v);
    }
}

template <typename C>
__device__ __forceinline__ C ldt(const C* p) { return *p; }

// One cell (i, j, k) of the update; MOM: write rho and Ut instead.  A block
// covers 128 cells of one row, so the row's table is staged in shared
// memory once per block and every coefficient is a shared-memory read.  Six
// blocks per SM (FP32 compute: 80 registers, a few bytes spilled) measured
// 8 % faster than four (128 registers, no spills); seven and eight spill more.
// With the pulled pairs in shared memory (SPAIRS, the default for FP32
// compute) seven blocks fit in 72 registers: on the 128 x 804 x 32 annulus
// 14,702 MLUPS against 13,914 (FP32 storage) and 15,862 against 14,841 (FP16);
// eight blocks (64 registers) 13,107.  Two cells per thread in packed FP32
// (168 registers, three blocks) measured 11,617, and all 78 reads issued as
// asynchronous 4-byte copies into shared memory 12,419: the update is bound
// by the latency of its loads, which wants resident warps.
template <typename S, typename C, bool MOM, int MINB = (sizeof(C) == 4 ? 6 : 2), bool SPAIRS = false>
__global__ void __launch_bounds__(TB, MINB)
    k3_step(Args3 A, double* __restrict__ mrho, double* __restrict__ mut) {
    static_assert(!SPAIRS || (!MOM && sizeof(C) == 4), "shared-memory pairs: FP32-compute update only");
    __shared__ __align__(16) C ts[Tab3::S];
    using P = typename PairOf<C>::T;
    // SPAIRS: the pulled pairs wait for the collision in shared memory (one
    // 8-byte slot per pair and thread, conflict-free) instead of 38
    // registers, which makes room for seven blocks per SM instead of six
    __shared__ P sdd[SPAIRS ? NP : 1][TB];
    const int n23 = A.n2 * A.n3;
    const int jk = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y, i = r + 1;
    {
        const C* tg = (const C*)A.tab + (size_t)r * Tab3::S;
        for (int q = threadIdx.x; q < Tab3::S; q += TB) ts[q] = tg[q];
    }
    __syncthreads();
    if (jk >= n23) return;
    const int j = jk / A.n3, k = jk - j * A.n3;
    const C* t = ts;
    const S* src = (const S*)A.src;
    int jo[7], ko[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        jo[q] = wrap3(j - (q - 3), A.n2) * A.n3;
        ko[q] = wrap3(k - (q - 3), A.n3);
    }
    // 32-bit element offsets (the grid's 39 planes hold fewer than 2^31
    // values, which clbm3_create_grid checks)
    const unsigned pl = (unsigned)A.plane;
    const unsigned own = (unsigned)(i - 1 + H) * (unsigned)n23 + (unsigned)jk;

    // pull (Eq. 12) with the lagged read, moments (Eqs. 7-10), lagged force
    // (Eq. 15), two directions a, b = -a at a time in the two lanes of a pair.
    // The arithmetic carries the storage scale SC (values as stored, a power
    // of two: exactly SC times the unscaled sums) up to the moments.
    constexpr int SC = Store<S>::SCALE;
    P dd[SPAIRS ? 1 : NP];
    const C d0 = Store<S>::ldr(src + own);
    P sd = mkp(d0, C(0)), s1 = mkp(C(0), C(0)), s2 = s1, s3 = s1;
    P f1 = mkp(ldt(t + Tab3::F0) * C(SC), C(0)), f2 = mkp(ldt(t + Tab3::F0 + 1) * C(SC), C(0)),
      f3 = mkp(ldt(t + Tab3::F0 + 2) * C(SC), C(0));
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int a = plus3(p), b = opp3(a);
        const int c1 = c1_3(a), c2 = c2_3(a), c3 = c3_3(a);
        // N_a from q - c_a, N_b from q + c_a; the lagged values are the cell's own
        const unsigned ia = (unsigned)(i - c1 - 1 + H) * (unsigned)n23 + (unsigned)(jo[c2 + 3] + ko[c3 + 3]);
        const unsigned ib = (unsigned)(i + c1 - 1 + H) * (unsigned)n23 + (unsigned)(jo[3 - c2] + ko[3 - c3]);
        const P pp = mkp(Store<S>::ldr(src + (a * pl + ia)), Store<S>::ldr(src + (b * pl + ib)));
        const P lg = mkp(Store<S>::ldr(src + (b * pl + own)), Store<S>::ldr(src + (a * pl + own)));
        const V4<C> w0 = ld4(t + Tab3::PA(p)), w1 = ld4(t + Tab3::PA(p) + 4);
        const P d = c1 == 0 ? pp
                    : SC == 1 ? padd(pp, mkp(w1.z, w1.w))
                              : pfma(mkp(w1.z, w1.w), mkp(C(SC), C(SC)), pp);
        if constexpr (SPAIRS) sdd[p][threadIdx.x] = d;
        else dd[p] = d;
        sd = padd(sd, d);
        if (c1) s1 = pfma(mkp(C(c1), C(-c1)), d, s1);
        if (c2) s2 = pfma(mkp(C(c2), C(-c2)), d, s2);
        if (c3) s3 = pfma(mkp(C(c3), C(-c3)), d, s3);
        // (N'_b + N_a, N'_a + N_b), weighed by (a^k_b, a^k_a)
        const P tt = padd(lg, d);
        f1 = pfma(mkp(w0.x, w0.y), tt, f1);
        f2 = pfma(mkp(w0.z, w0.w), tt, f2);
        f3 = pfma(mkp(w1.x, w1.y), tt, f3);
    }
    const C invJ = ldt(t + Tab3::INVJ) * C(1.0 / SC), J = ldt(t + Tab3::J) * C(SC);
    const C drho = (sd.x + sd.y) * invJ, rho = C(A.rho0) + drho, irho = C(1) / rho;
    const C U1 = (s1.x + s1.y) * invJ * irho, U2 = (s2.x + s2.y) * invJ * irho, U3 = (s3.x + s3.y) * invJ * irho;
    const C F1 = C(-0.5) * invJ * (f1.x + f1.y) + rho * C(A.g1);
    const C F2 = C(-0.5) * invJ * (f2.x + f2.y) + rho * C(A.g2);
    const C F3 = C(-0.5) * invJ * (f3.x + f3.y) + rho * C(A.g3);
    const C V1 = U1 + C(0.5) * F1 * irho, V2 = U2 + C(0.5) * F2 * irho, V3 = U3 + C(0.5) * F3 * irho;
    if (MOM) {
        const size_t m = (size_t)r * n23 + jk, nc = (size_t)A.n1 * n23;
        if (mrho) mrho[m] = double(rho);
        if (mut) {
            mut[m] = double(V1);
            mut[nc + m] = double(V2);
            mut[2 * nc + m] = double(V3);
        }
        return;
    }

    // Eq. 19: third-order coefficients C^{pqr} = Ut Ut Ut + T0 (g Ut - delta U)
    // (symmetrised), their contraction with the first Hermite term, and the
    // odd part O_a = c.U / T0 + H3(c) : C / (6 T0^3) of f^eq / (rho w)
    constexpr C iT0 = C(1.0 / T0), i2T02 = C(0.5 / (T0 * T0)), i6T03 = C(1.0 / (6.0 * T0 * T0 * T0));
    const C g11 = ldt(t + Tab3::G11), g12 = ldt(t + Tab3::G12), g13 = ldt(t + Tab3::G13);
    const C g22 = ldt(t + Tab3::G22), g23 = ldt(t + Tab3::G23), g33 = ldt(t + Tab3::G33);
    const C T = C(T0);
    const C C111 = V1 * V1 * V1 + T * (C(3) * g11 * V1 - C(3) * U1);
    const C C222 = V2 * V2 * V2 + T * (C(3) * g22 * V2 - C(3) * U2);
    const C C333 = V3 * V3 * V3 + T * (C(3) * g33 * V3 - C(3) * U3);
    const C C112 = V1 * V1 * V2 + T * (g11 * V2 + C(2) * g12 * V1 - U2);
    const C C113 = V1 * V1 * V3 + T * (g11 * V3 + C(2) * g13 * V1 - U3);
    const C C122 = V1 * V2 * V2 + T * (g22 * V1 + C(2) * g12 * V2 - U1);
    const C C133 = V1 * V3 * V3 + T * (g33 * V1 + C(2) * g13 * V3 - U1);
    const C C223 = V2 * V2 * V3 + T * (g22 * V3 + C(2) * g23 * V2 - U3);
    const C C233 = V2 * V3 * V3 + T * (g33 * V2 + C(2) * g23 * V3 - U2);
    const C C123 = V1 * V2 * V3 + T * (g12 * V3 + g23 * V1 + g13 * V2);
    const C K1 = U1 * iT0 - (C111 + C122 + C133) * i2T02;
    const C K2 = U2 * iT0 - (C112 + C222 + C233) * i2T02;
    const C K3 = U3 * iT0 - (C113 + C223 + C333) * i2T02;
    const C k111 = C111 * i6T03, k222 = C222 * i6T03, k333 = C333 * i6T03;
    const C k112 = C(3) * C112 * i6T03, k113 = C(3) * C113 * i6T03, k122 = C(3) * C122 * i6T03;
    const C k133 = C(3) * C133 * i6T03, k223 = C(3) * C223 * i6T03, k233 = C(3) * C233 * i6T03;
    const C k123 = C(6) * C123 * i6T03;

    // symmetric momentum-flux correction (Eq. 16): only the odd part of f^eq
    // survives the pair sums, weighed by w (c^p D^r + c^r D^p)
    C O[NP];
    C P11 = C(0), P22 = C(0), P33 = C(0), P12 = C(0), P13 = C(0), P23 = C(0);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int a = plus3(p);
        const double x = c1_3(a), y = c2_3(a), z = c3_3(a);
        KSum<C> os;
        os.add(K1, x);
        os.add(K2, y);
        os.add(K3, z);
        os.add(k111, x * x * x);
        os.add(k222, y * y * y);
        os.add(k333, z * z * z);
        os.add(k112, x * x * y);
        os.add(k113, x * x * z);
        os.add(k122, x * y * y);
        os.add(k133, x * z * z);
        os.add(k223, y * y * z);
        os.add(k233, y * z * z);
        os.add(k123, x * y * z);
        const C o = os.s;
        O[p] = o;
        // E_kl = w (c^k D^l + c^l D^k) vanishes exactly where c^k = c^l = 0
        const V4<C> e0 = ld4(t + Tab3::E(p)), e1 = ld4(t + Tab3::E(p) + 4);
        if (x != 0.0) P11 += e0.x * o;
        if (y != 0.0) P22 += e0.y * o;
        if (z != 0.0) P33 += e0.z * o;
        if (x != 0.0 || y != 0.0) P12 += e0.w * o;
        if (x != 0.0 || z != 0.0) P13 += e1.x * o;
        if (y != 0.0 || z != 0.0) P23 += e1.y * o;
    }
    const C pr = C(A.pref) * rho;
    P11 *= pr;
    P22 *= pr;
    P33 *= pr;
    P12 *= pr;
    P13 *= pr;
    P23 *= pr;
    const C trP = P11 + P22 + P33;

    // BGK (Eqs. 6, 11) with dN (Eq. 17), in deviations:
    // sigma'_a = (1 - 1/tau) d_a + J w [(drho P0_a + rho Pi_a) / tau + c.F / T0
    //            + (c.dPi.c / T0 - tr dPi) / T0],  Pi_a = f^eq_a / (rho w) - P0_a
    const C tinv = C(A.tau_inv), omt = C(A.omt);
    const C uu = V1 * V1 + V2 * V2 + V3 * V3;
    const C base = C(-0.5) * iT0 * uu * rho * tinv - trP * iT0;
    S* dst = (S*)A.dst + own;
    // the even part of the bracket is quadratic in c: c.M.c with
    // M = rho (Ut Ut) / (2 T0^2 tau) + dPi / T0^2, formed once per cell
    const C P0 = ldt(t + Tab3::P0);
    const C drt = drho * tinv, rt = rho * tinv, A1 = rt * i2T02, iT02 = iT0 * iT0;
    const C M11 = A1 * V1 * V1 + P11 * iT02, M22 = A1 * V2 * V2 + P22 * iT02, M33 = A1 * V3 * V3 + P33 * iT02;
    const C M12 = A1 * V1 * V2 + P12 * iT02, M13 = A1 * V1 * V3 + P13 * iT02, M23 = A1 * V2 * V3 + P23 * iT02;
    const C Fa = F1 * iT0, Fb = F2 * iT0, Fc = F3 * iT0;
    StStream<S>::str(dst, omt * d0 + J * C(w3(0)) * (drt * P0 + base));   // read only by the next launch
    const P omt2 = mkp(omt, omt), J2 = mkp(J, J);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int a = plus3(p), b = opp3(a);
        const double x = c1_3(a), y = c2_3(a), z = c3_3(a);
        KSum<C> xs(drt * ldt(t + Tab3::P0 + a) + base), ys(rt * O[p]);
        xs.add(M11, x * x);
        xs.add(M22, y * y);
        xs.add(M33, z * z);
        xs.add(M12, 2.0 * x * y);
        xs.add(M13, 2.0 * x * z);
        xs.add(M23, 2.0 * y * z);
        ys.add(Fa, x);
        ys.add(Fb, y);
        ys.add(Fc, z);
        const C X = xs.s, Y = ys.s;
        const C w = C(w3(a));
        // (N'_a, N'_b) = (1 - 1/tau)(d_a, d_b) + J w (X + Y, X - Y)
        const P o = pfma(pmul(J2, mkp(w, w)), mkp(X + Y, X - Y), pmul(SPAIRS ? sdd[p][threadIdx.x] : dd[SPAIRS ? 0 : p], omt2));
        StStream<S>::str(dst + a * pl, o.x);
        StStream<S>::str(dst + b * pl, o.y);
    }
    // the moments the walls read next (rows within H of a wall)
    if (i <= H) {
        wall_ptr<C>(A.wall, 0, 0, i, n23)[jk] = rho;
        wall_ptr<C>(A.wall, 1, 0, i, n23)[jk] = V2;
        wall_ptr<C>(A.wall, 2, 0, i, n23)[jk] = V3;
    }
    if (i > A.n1 - H) {
        const int m = A.n1 + 1 - i;
        wall_ptr<C>(A.wall, 0, 1, m, n23)[jk] = rho;
        wall_ptr<C>(A.wall, 1, 1, m, n23)[jk] = V2;
        wall_ptr<C>(A.wall, 2, 1, m, n23)[jk] = V3;
    }
    // and the ghost rows of the buffer written, which this cell mirrors
    // (a block is one row: the branch is uniform)
    if (i <= H) ghost_column<S, C>(A, 0, i, jk, own, rho, V2, V3);
    if (i > A.n1 - H) ghost_column<S, C>(A, 1, A.n1 + 1 - i, jk, own, rho, V2, V3);
}

// State conversions between FP64 N' ([a][cell]) and stored deviations.
template <typename S>
__global__ void k3_from64(const double* __restrict__ Np, const double* __restrict__ geo, S* __restrict__ st,
                          int n1, int n23, long long plane) {
    const int jk = blockIdx.x * blockDim.x + threadIdx.x;
    if (jk >= n23) return;
    const int r = blockIdx.y;
    const size_t nc = (size_t)n1 * n23, m = (size_t)r * n23 + jk, own = (size_t)(r + H) * n23 + jk;
    const double* g = geo + (size_t)r * Geo3::S;
    using C = typename Store<S>::C;
    for (int a = 0; a < Q; ++a)
        Store<S>::st(st + (size_t)a * plane + own, C(Np ? Np[a * nc + m] - g[Geo3::REF + a] : 0.0));
}

// Equilibrium start N(q, 0) = J f^eq(rho, U, Ut = U; g^{ij}(q)) in FP64 (Eq.
// 19 in three coordinates: second moment T0 g^{ij} + Ut^i Ut^j, third built
// from Ut, U and g^{ij}; Ut = U with no force known yet), written as FP64
// N' ([a][cell]) for k3_from64.  Absent fields are rho0 and 0.
__global__ void k3_equilibrium(const double* __restrict__ rho, const double* __restrict__ U,
                               const double* __restrict__ geo, double* __restrict__ Np, int n1, int n23,
                               double rho0) {
    const int jk = blockIdx.x * blockDim.x + threadIdx.x;
    if (jk >= n23) return;
    const int r = blockIdx.y;
    const size_t nc = (size_t)n1 * n23, m = (size_t)r * n23 + jk;
    const double* g = geo + (size_t)r * Geo3::S;
    const double R = rho ? rho[m] : rho0;
    const double u[3] = {U ? U[m] : 0.0, U ? U[nc + m] : 0.0, U ? U[2 * nc + m] : 0.0};
    const int P[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    double e[3][3];   // g^{ij} - delta^{ij}
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) e[p][q] = g[Geo3::GI + P[p][q]] - (p == q ? 1.0 : 0.0);
    for (int a = 0; a < Q; ++a) {
        const double c[3] = {(double)c1_3(a), (double)c2_3(a), (double)c3_3(a)};
        double h1 = 0.0, h2 = 0.0, h3 = 0.0;
        for (int p = 0; p < 3; ++p) h1 += c[p] * u[p];
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) {
                const double A = u[p] * u[q] + T0 * e[p][q];
                h2 += (c[p] * c[q] - (p == q ? T0 : 0.0)) * A;
                for (int k = 0; k < 3; ++k) {
                    // C^{pqk} = Ut Ut Ut + T0 ((g - delta)^{pq} U^k + cyclic), Ut = U
                    const double C3 = u[p] * u[q] * u[k] + T0 * (e[p][q] * u[k] + e[q][k] * u[p] + e[k][p] * u[q]);
                    const double H3 = c[p] * c[q] * c[k] - T0 * (c[p] * (q == k) + c[q] * (k == p) + c[k] * (p == q));
                    h3 += H3 * C3;
                }
            }
        const double Pa = 1.0 + h1 / T0 + h2 / (2.0 * T0 * T0) + h3 / (6.0 * T0 * T0 * T0);
        Np[(size_t)a * nc + m] = g[Geo3::J] * w3(a) * R * Pa;
    }
}

template <typename S>
__global__ void k3_to64(const S* __restrict__ st, const double* __restrict__ geo, double* __restrict__ Np, int n1,
                        int n23, long long plane) {
    const int jk = blockIdx.x * blockDim.x + threadIdx.x;
    if (jk >= n23) return;
    const int r = blockIdx.y;
    const size_t nc = (size_t)n1 * n23, m = (size_t)r * n23 + jk, own = (size_t)(r + H) * n23 + jk;
    const double* g = geo + (size_t)r * Geo3::S;
    for (int a = 0; a < Q; ++a) Np[a * nc + m] = double(Store<S>::ld(st + (size_t)a * plane + own)) + g[Geo3::REF + a];
}

// Wall moments of rows 1..H and n1-H+1..n1 from cell fields (NULL: rho0, 0).
template <typename C>
__global__ void k3_wall_init(void* wall, const double* rho, const double* u2, const double* u3, int n1, int n23,
                             double rho0) {
    const int jk = blockIdx.x * blockDim.x + threadIdx.x;
    if (jk >= n23) return;
    const int w = blockIdx.y / H, m = blockIdx.y % H + 1;
    const int row = w == 0 ? m - 1 : n1 - m;          // 0-based fluid row
    const size_t c = (size_t)row * n23 + jk;
    wall_ptr<C>(wall, 0, w, m, n23)[jk] = C(rho ? rho[c] : rho0);
    wall_ptr<C>(wall, 1, w, m, n23)[jk] = C(u2 ? u2[c] : 0.0);
    wall_ptr<C>(wall, 2, w, m, n23)[jk] = C(u3 ? u3[c] : 0.0);
}

// Totals of the stored deviations per block (sum sigma, sum c sigma), fixed
// order; the rest part sum ref = rho0 J per cell is added on the host.
template <typename S>
__global__ void __launch_bounds__(TB) k3_totals(const S* __restrict__ st, int n1, int n23, long long plane,
                                                double* __restrict__ partial) {
    const int jk = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (jk < n23) {
        const size_t own = (size_t)(r + H) * n23 + jk;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const double s = double(Store<S>::ld(st + (size_t)a * plane + own));
            v[0] += s;
            v[1] += c1_3(a) * s;
            v[2] += c2_3(a) * s;
            v[3] += c3_3(a) * s;
        }
    }
    __shared__ double sh[4][TB];
    for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int w = TB / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) partial[((size_t)r * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k3_totals_final(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    __shared__ double sh[256];
    const int q = blockIdx.x;
    double x = 0.0;
    for (int b = threadIdx.x; b < nb; b += 256) x += partial[(size_t)b * 4 + q];
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
}

}  // namespace
}  // namespace d3
}  // namespace clbm

// ------------------------------------------------------------------ C ABI

using namespace clbm::d3;
using clbm::Store;

struct clbm3_grid {
    int prec, n1, n2, n3, kind, bc_lo, bc_hi, device;
    double step2, step3, dx;
    cudaStream_t stream;
    double *edges, *geo, *partial, *red, *stage;
    void *tab, *st[2], *wall;
    int cur;                  // index of the buffer holding N'(t-1)
    clbm3_case cs;
    bool have_case;
    long long t;
    std::vector<double> hedges;
    // CUDA graph of GRAPH3_STEPS time steps (one update launch each; an
    // even count, so cur ends where it started), keyed by the launch
    // arguments of its first step
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    Args3 gargs;
    bool graphs_off;         // capture failed once (e.g. the legacy default stream)
    int kernel;              // update: 0 automatic, 1 pulled pairs in registers, 2 in shared memory
    bool ghosts_ok;          // the current buffer's ghost rows are filled (the update fills the next one's)
};

namespace k3api {

clbm_status fail3(clbm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    clbm::set_last_error(buf);
    return s;
}

#define CK3(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail3(CLBM_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                         __LINE__);                                                           \
    } while (0)

size_t sbytes(const clbm3_grid* g) { return g->prec == CLBM_FP64 ? 8 : g->prec == CLBM_FP32 ? 4 : 2; }
size_t cbytes(const clbm3_grid* g) { return g->prec == CLBM_FP64 ? 8 : 4; }  // tables, wall moments

template <typename T> struct Tag { using type = T; };

// Call f(Tag<S>{}) for the storage type S of precision prec.
template <typename F>
void by_storage(int prec, F&& f) {
    switch (prec) {
        case CLBM_FP64: f(Tag<double>{}); break;
        case CLBM_FP32: f(Tag<float>{}); break;
        case CLBM_FP32_F16STORE: f(Tag<__half>{}); break;
        default: f(Tag<__nv_bfloat16>{}); break;
    }
}
int n23(const clbm3_grid* g) { return g->n2 * g->n3; }
long long plane(const clbm3_grid* g) { return (long long)(g->n1 + 2 * H) * g->n2 * g->n3; }
size_t ncells(const clbm3_grid* g) { return (size_t)g->n1 * g->n2 * g->n3; }
dim3 cell_grid(const clbm3_grid* g) { return dim3((n23(g) + TB - 1) / TB, g->n1); }

Args3 args(const clbm3_grid* g) {
    Args3 A;
    memset(&A, 0, sizeof(A));
    A.src = g->st[g->cur];
    A.dst = g->st[g->cur ^ 1];
    A.tab = g->tab;
    A.geo = g->geo;
    A.wall = g->wall;
    A.n1 = g->n1;
    A.n2 = g->n2;
    A.n3 = g->n3;
    A.plane = plane(g);
    A.bc_lo = g->bc_lo;
    A.bc_hi = g->bc_hi;
    A.rho0 = g->cs.rho0;
    A.tau_inv = 1.0 / g->cs.tau;
    A.omt = 1.0 - 1.0 / g->cs.tau;
    A.pref = -0.5 * (1.0 - 1.0 / (2.0 * g->cs.tau));
    A.g1 = g->cs.g_ext[0];
    A.g2 = g->cs.g_ext[1];
    A.g3 = g->cs.g_ext[2];
    A.U0_lo = g->cs.u_wall_lo;
    A.U0_hi = g->cs.u_wall_hi;
    return A;
}

void launch_boundary(const clbm3_grid* g, const Args3& A) {
    dim3 grid((n23(g) + TB - 1) / TB, 2 * H);
    by_storage(g->prec, [&](auto tag) {
        using S = typename decltype(tag)::type;
        k3_boundary<S, typename Store<S>::C><<<grid, TB, 0, g->stream>>>(A, (S*)A.src);
    });
}

template <bool MOM>
void launch_cells(const clbm3_grid* g, const Args3& A, double* rho, double* ut) {
    by_storage(g->prec, [&](auto tag) {
        using S = typename decltype(tag)::type;
        using C = typename Store<S>::C;
        if constexpr (!MOM && !std::is_same<S, double>::value) {
            if (g->kernel != 1) {
                k3_step<S, C, false, 7, true><<<cell_grid(g), TB, 0, g->stream>>>(A, nullptr, nullptr);
                return;
            }
        }
        k3_step<S, C, MOM><<<cell_grid(g), TB, 0, g->stream>>>(A, rho, ut);
    });
}

constexpr int GRAPH3_STEPS = 10;

// One time step with plain launches.
void step3_plain(clbm3_grid* g) {
    const Args3 A = args(g);
    launch_cells<false>(g, A, nullptr, nullptr);
    g->cur ^= 1;
    g->t++;
}

// Whether the graph replays what plain launches from the current buffer do.
bool graph3_matches(const clbm3_grid* g) {
    if (!g->gexec) return false;
    const Args3 A = args(g);
    return memcmp(&A, &g->gargs, sizeof A) == 0;
}

// Capture GRAPH3_STEPS steps from the current buffer; on failure the grid
// keeps to plain launches.
void capture3(clbm3_grid* g) {
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->graph) cudaGraphDestroy(g->graph);
    g->gexec = nullptr;
    g->graph = nullptr;
    if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        g->graphs_off = true;
        return;
    }
    const Args3 first = args(g);
    for (int k = 0; k < GRAPH3_STEPS; ++k) {
        const Args3 A = args(g);
        launch_cells<false>(g, A, nullptr, nullptr);
        g->cur ^= 1;
    }
    cudaGraph_t graph = nullptr;
    const bool ok = cudaStreamEndCapture(g->stream, &graph) == cudaSuccess && graph &&
                    cudaGraphInstantiate(&g->gexec, graph, 0) == cudaSuccess;
    cudaGetLastError();
    if (!ok) {
        if (g->gexec) cudaGraphExecDestroy(g->gexec);
        if (graph) cudaGraphDestroy(graph);
        g->gexec = nullptr;
        g->graphs_off = true;
        return;
    }
    g->graph = graph;
    g->gargs = first;
}

clbm_status staging(clbm3_grid* g, double** out) {
    if (!g->stage) {
        const size_t n = (size_t)Q * ncells(g);
        if (cudaMalloc((void**)&g->stage, n * 8) != cudaSuccess) {
            g->stage = nullptr;
            cudaGetLastError();
            return fail3(CLBM_ENOMEM, "no device memory for the FP64 staging buffer (%zu bytes)", n * 8);
        }
    }
    *out = g->stage;
    return CLBM_OK;
}

// Checkpoint header: the grid's identity, case and time; the raw state
// buffer (ghost rows included, in the storage type) and the wall moments
// follow it.
struct Ckpt3 {
    char magic[8];
    int prec, n1, n2, n3, kind;
    long long t;
    clbm3_case cs;
};

Ckpt3 ckpt_header(const clbm3_grid* g) {
    Ckpt3 h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "CLBM3CK1", 8);
    h.prec = g->prec;
    h.n1 = g->n1;
    h.n2 = g->n2;
    h.n3 = g->n3;
    h.kind = g->kind;
    h.t = g->t;
    h.cs = g->cs;
    return h;
}

}  // namespace k3api

using namespace k3api;

extern "C" {

clbm_status clbm3_create_grid(const clbm3_grid_desc* d, clbm3_handle* out) {
    if (!d || !out) return fail3(CLBM_EINVAL, "NULL argument");
    *out = nullptr;
    if (d->precision < CLBM_FP64 || d->precision > CLBM_FP32_BF16STORE)
        return fail3(CLBM_EINVAL, "bad precision");
    if (d->n1 < 4 || d->n2 < 1 || d->n3 < 1) return fail3(CLBM_EINVAL, "need n1 >= 4 and n2, n3 >= 1");
    if ((long long)Q * (d->n1 + 2 * H) * d->n2 * d->n3 >= (1LL << 31))
        return fail3(CLBM_EINVAL, "grid too large: 39 (n1 + 6) n2 n3 must stay below 2^31");
    if (d->kind != CLBM3_CHANNEL && d->kind != CLBM3_ANNULUS) return fail3(CLBM_EINVAL, "bad kind");
    if (!d->edges) return fail3(CLBM_EINVAL, "edges is NULL");
    for (int i = 0; i < d->n1; ++i)
        if (!(d->edges[i + 1] > d->edges[i])) return fail3(CLBM_EINVAL, "edges must increase");
    if (d->kind == CLBM3_ANNULUS && !(d->edges[0] > 0.0)) return fail3(CLBM_EINVAL, "radii must be > 0");
    if (!(d->step3 > 0.0) || (d->kind == CLBM3_CHANNEL && !(d->step2 > 0.0)))
        return fail3(CLBM_EINVAL, "node spacings must be > 0");
    if ((d->bc_lo != CLBM_BC_NOSLIP && d->bc_lo != CLBM_BC_MOVING) ||
        (d->bc_hi != CLBM_BC_NOSLIP && d->bc_hi != CLBM_BC_MOVING))
        return fail3(CLBM_EINVAL, "bad wall condition");
    CK3(cudaSetDevice(d->device));
    clbm3_grid* g = new clbm3_grid();
    g->prec = d->precision;
    g->n1 = d->n1;
    g->n2 = d->n2;
    g->n3 = d->n3;
    g->kind = d->kind;
    g->bc_lo = d->bc_lo;
    g->bc_hi = d->bc_hi;
    g->device = d->device;
    g->step2 = d->step2;
    g->step3 = d->step3;
    g->dx = d->dx > 0.0 ? d->dx : (d->edges[d->n1] - d->edges[0]) / d->n1;
    g->stream = (cudaStream_t)d->stream;
    g->hedges.assign(d->edges, d->edges + d->n1 + 1);
    const size_t sb = sbytes(g), cb = cbytes(g);
    const size_t nb = (size_t)((n23(g) + TB - 1) / TB) * g->n1;
    bool ok = cudaMalloc((void**)&g->edges, (g->n1 + 1) * 8) == cudaSuccess &&
              cudaMalloc((void**)&g->geo, (size_t)g->n1 * Geo3::S * 8) == cudaSuccess &&
              cudaMalloc(&g->tab, (size_t)g->n1 * Tab3::S * cb) == cudaSuccess &&
              cudaMalloc(&g->st[0], (size_t)Q * plane(g) * sb) == cudaSuccess &&
              cudaMalloc(&g->st[1], (size_t)Q * plane(g) * sb) == cudaSuccess &&
              cudaMalloc(&g->wall, (size_t)3 * 2 * H * n23(g) * cb) == cudaSuccess &&
              cudaMalloc((void**)&g->partial, nb * 4 * 8) == cudaSuccess &&
              cudaMalloc((void**)&g->red, 4 * 8) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        clbm3_destroy(g);
        return fail3(CLBM_ENOMEM, "device allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(g->edges, d->edges, (g->n1 + 1) * 8, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->st[0], 0, (size_t)Q * plane(g) * sb, g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->st[1], 0, (size_t)Q * plane(g) * sb, g->stream);
    if (e == cudaSuccess) {
        Shape s{g->kind, g->n1, g->n2, g->edges, g->step2, g->step3, g->dx};
        k3_geometry<<<(g->n1 + 63) / 64, 64, 0, g->stream>>>(s, g->geo);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        clbm3_destroy(g);
        return fail3(CLBM_ECUDA, "geometry precompute failed: %s", cudaGetErrorString(e));
    }
    *out = g;
    return CLBM_OK;
}

clbm_status clbm3_set_case(clbm3_handle g, const clbm3_case* c) {
    if (!g || !c) return fail3(CLBM_EINVAL, "NULL argument");
    if (!(c->tau > 0.5) || !std::isfinite(c->tau)) return fail3(CLBM_EINVAL, "tau must be > 1/2");
    if (!(c->rho0 > 0.0) || !std::isfinite(c->rho0)) return fail3(CLBM_EINVAL, "rho0 must be > 0");
    CK3(cudaSetDevice(g->device));
    g->cs = *c;
    g->have_case = true;
    k3_reference<<<(g->n1 + 63) / 64, 64, 0, g->stream>>>(g->geo, g->n1, c->rho0);
    if (g->prec == CLBM_FP64)
        k3_tables<double><<<(g->n1 + 63) / 64, 64, 0, g->stream>>>(g->geo, (double*)g->tab, g->n1);
    else  // FP32 compute for FP32 and 16-bit storage
        k3_tables<float><<<(g->n1 + 63) / 64, 64, 0, g->stream>>>(g->geo, (float*)g->tab, g->n1);
    g->cur = 0;
    CK3(cudaMemsetAsync(g->st[0], 0, (size_t)Q * plane(g) * sbytes(g), g->stream));
    dim3 wg((n23(g) + TB - 1) / TB, 2 * H);
    if (g->prec == CLBM_FP64)
        k3_wall_init<double><<<wg, TB, 0, g->stream>>>(g->wall, nullptr, nullptr, nullptr, g->n1, n23(g), c->rho0);
    else
        k3_wall_init<float><<<wg, TB, 0, g->stream>>>(g->wall, nullptr, nullptr, nullptr, g->n1, n23(g), c->rho0);
    CK3(cudaGetLastError());
    CK3(cudaStreamSynchronize(g->stream));
    g->t = 0;
    g->ghosts_ok = false;
    return CLBM_OK;
}

clbm_status clbm3_set_state(clbm3_handle g, const double* Np, const double* rho, const double* u2,
                            const double* u3, int src_is_device) {
    if (!g || !Np) return fail3(CLBM_EINVAL, "NULL argument");
    if (!g->have_case) return fail3(CLBM_EINVAL, "call clbm3_set_case first");
    CK3(cudaSetDevice(g->device));
    const size_t nc = ncells(g);
    const double *dN = Np, *dr = rho, *d2 = u2, *d3 = u3;
    double* extra = nullptr;
    struct FreeOnExit {
        double** p;
        ~FreeOnExit() { cudaFree(*p); }
    } guard{&extra};
    if (!src_is_device) {
        double* sb = nullptr;
        clbm_status st = staging(g, &sb);
        if (st != CLBM_OK) return st;
        CK3(cudaMemcpyAsync(sb, Np, (size_t)Q * nc * 8, cudaMemcpyHostToDevice, g->stream));
        dN = sb;
        dr = d2 = d3 = nullptr;
        if (rho || u2 || u3) {
            CK3(cudaMalloc((void**)&extra, 3 * nc * 8));
            const double* h[3] = {rho, u2, u3};
            const double** dd[3] = {&dr, &d2, &d3};
            for (int q = 0; q < 3; ++q)
                if (h[q]) {
                    CK3(cudaMemcpyAsync(extra + q * nc, h[q], nc * 8, cudaMemcpyHostToDevice, g->stream));
                    *dd[q] = extra + q * nc;
                }
        }
    }
    dim3 cg((n23(g) + TB - 1) / TB, g->n1), wg((n23(g) + TB - 1) / TB, 2 * H);
    g->cur = 0;
    by_storage(g->prec, [&](auto tag) {
        using S = typename decltype(tag)::type;
        k3_from64<S><<<cg, TB, 0, g->stream>>>(dN, g->geo, (S*)g->st[0], g->n1, n23(g), plane(g));
        k3_wall_init<typename Store<S>::C><<<wg, TB, 0, g->stream>>>(g->wall, dr, d2, d3, g->n1, n23(g),
                                                                    g->cs.rho0);
    });
    CK3(cudaGetLastError());
    CK3(cudaStreamSynchronize(g->stream));
    g->ghosts_ok = false;
    return CLBM_OK;
}

clbm_status clbm3_set_equilibrium(clbm3_handle g, const double* rho, const double* U, int src_is_device) {
    if (!g) return fail3(CLBM_EINVAL, "handle is NULL");
    if (!g->have_case) return fail3(CLBM_EINVAL, "call clbm3_set_case first");
    CK3(cudaSetDevice(g->device));
    const size_t nc = ncells(g);
    double* sb = nullptr;
    clbm_status st = staging(g, &sb);
    if (st != CLBM_OK) return st;
    const double *dr = rho, *du = U;
    double* extra = nullptr;
    struct FreeOnExit {
        double** p;
        ~FreeOnExit() { cudaFree(*p); }
    } guard{&extra};
    if (!src_is_device && (rho || U)) {
        CK3(cudaMalloc((void**)&extra, 4 * nc * 8));
        if (rho) CK3(cudaMemcpyAsync(extra, rho, nc * 8, cudaMemcpyHostToDevice, g->stream));
        if (U) CK3(cudaMemcpyAsync(extra + nc, U, 3 * nc * 8, cudaMemcpyHostToDevice, g->stream));
        dr = rho ? extra : nullptr;
        du = U ? extra + nc : nullptr;
    }
    dim3 cg((n23(g) + TB - 1) / TB, g->n1), wg((n23(g) + TB - 1) / TB, 2 * H);
    k3_equilibrium<<<cg, TB, 0, g->stream>>>(dr, du, g->geo, sb, g->n1, n23(g), g->cs.rho0);
    g->cur = 0;
    by_storage(g->prec, [&](auto tag) {
        using S = typename decltype(tag)::type;
        k3_from64<S><<<cg, TB, 0, g->stream>>>(sb, g->geo, (S*)g->st[0], g->n1, n23(g), plane(g));
        k3_wall_init<typename Store<S>::C><<<wg, TB, 0, g->stream>>>(g->wall, dr, du ? du + nc : nullptr,
                                                                    du ? du + 2 * nc : nullptr, g->n1,
                                                                    n23(g), g->cs.rho0);
    });
    CK3(cudaGetLastError());
    CK3(cudaStreamSynchronize(g->stream));
    g->t = 0;
    g->ghosts_ok = false;
    return CLBM_OK;
}

clbm_status clbm3_checkpoint_bytes(clbm3_handle g, size_t* bytes) {
    if (!g || !bytes) return fail3(CLBM_EINVAL, "NULL argument");
    *bytes = sizeof(Ckpt3) + (size_t)Q * plane(g) * sbytes(g) + (size_t)3 * 2 * H * n23(g) * cbytes(g);
    return CLBM_OK;
}

clbm_status clbm3_checkpoint(clbm3_handle g, void* buf) {
    if (!g || !buf) return fail3(CLBM_EINVAL, "NULL argument");
    if (!g->have_case) return fail3(CLBM_EINVAL, "call clbm3_set_case first");
    CK3(cudaSetDevice(g->device));
    Ckpt3 h = ckpt_header(g);
    char* p = (char*)buf;
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    const size_t sbb = (size_t)Q * plane(g) * sbytes(g), wb = (size_t)3 * 2 * H * n23(g) * cbytes(g);
    CK3(cudaMemcpyAsync(p, g->st[g->cur], sbb, cudaMemcpyDeviceToHost, g->stream));
    CK3(cudaMemcpyAsync(p + sbb, g->wall, wb, cudaMemcpyDeviceToHost, g->stream));
    CK3(cudaStreamSynchronize(g->stream));
    return CLBM_OK;
}

clbm_status clbm3_restore(clbm3_handle g, const void* buf) {
    if (!g || !buf) return fail3(CLBM_EINVAL, "NULL argument");
    CK3(cudaSetDevice(g->device));
    Ckpt3 h, mine = ckpt_header(g);
    memcpy(&h, buf, sizeof(h));
    if (memcmp(h.magic, mine.magic, 8) != 0 || h.prec != mine.prec || h.n1 != mine.n1 || h.n2 != mine.n2 ||
        h.n3 != mine.n3 || h.kind != mine.kind)
        return fail3(CLBM_EINVAL, "checkpoint does not match this grid (precision, size or kind)");
    if (!(h.cs.tau > 0.5) || !(h.cs.rho0 > 0.0)) return fail3(CLBM_EINVAL, "checkpoint holds a bad case");
    clbm_status st = clbm3_set_case(g, &h.cs);     // tables of the saved case
    if (st != CLBM_OK) return st;
    const char* p = (const char*)buf + sizeof(h);
    const size_t sbb = (size_t)Q * plane(g) * sbytes(g), wb = (size_t)3 * 2 * H * n23(g) * cbytes(g);
    g->cur = 0;
    CK3(cudaMemcpyAsync(g->st[0], p, sbb, cudaMemcpyHostToDevice, g->stream));
    CK3(cudaMemcpyAsync(g->wall, p + sbb, wb, cudaMemcpyHostToDevice, g->stream));
    CK3(cudaStreamSynchronize(g->stream));
    g->t = h.t;
    g->ghosts_ok = false;
    return CLBM_OK;
}

clbm_status clbm3_get_state(clbm3_handle g, double* Np, int dst_is_device) {
    if (!g || !Np) return fail3(CLBM_EINVAL, "NULL argument");
    if (!g->have_case) return fail3(CLBM_EINVAL, "call clbm3_set_case first");
    CK3(cudaSetDevice(g->device));
    double* dN = Np;
    if (!dst_is_device) {
        clbm_status st = staging(g, &dN);
        if (st != CLBM_OK) return st;
    }
    dim3 cg((n23(g) + TB - 1) / TB, g->n1);
    by_storage(g->prec, [&](auto tag) {
        using S = typename decltype(tag)::type;
        k3_to64<S><<<cg, TB, 0, g->stream>>>((const S*)g->st[g->cur], g->geo, dN, g->n1, n23(g), plane(g));
    });
    CK3(cudaGetLastError());
    if (!dst_is_device)
        CK3(cudaMemcpyAsync(Np, dN, (size_t)Q * ncells(g) * 8, cudaMemcpyDeviceToHost, g->stream));
    CK3(cudaStreamSynchronize(g->stream));
    return CLBM_OK;
}

clbm_status clbm3_step(clbm3_handle g, long long n) {
    if (!g) return fail3(CLBM_EINVAL, "handle is NULL");
    if (n < 0) return fail3(CLBM_EINVAL, "n < 0");
    if (!g->have_case) return fail3(CLBM_EINVAL, "call clbm3_set_case first");
    CK3(cudaSetDevice(g->device));
    // the update fills the ghost rows of the buffer it writes; those of the
    // current buffer come from the boundary kernel after a new state or case
    // (before any replay: a graph holds update launches only)
    if (n > 0 && !g->ghosts_ok) {
        launch_boundary(g, args(g));
        g->ghosts_ok = true;
    }
    long long s = 0;
    // long runs replay a captured graph (one host call per GRAPH3_STEPS
    // steps); two plain steps first set the kernels up and bring cur back
    if (!g->graphs_off && n >= 2 * GRAPH3_STEPS + 2) {
        if (!graph3_matches(g)) {
            g->cur ^= 1;
            const bool other = graph3_matches(g);
            g->cur ^= 1;
            for (const long long k = other ? 1 : 2; s < k; ++s) step3_plain(g);
            if (!other) capture3(g);
        }
        if (graph3_matches(g)) {
            for (; n - s >= GRAPH3_STEPS; s += GRAPH3_STEPS) {
                CK3(cudaGraphLaunch(g->gexec, g->stream));
                g->t += GRAPH3_STEPS;
            }
        }
    }
    for (; s < n; ++s) step3_plain(g);
    CK3(cudaGetLastError());
    return CLBM_OK;
}

clbm_status clbm3_moments(clbm3_handle g, double* rho, double* ut, int dst_is_device) {
    if (!g) return fail3(CLBM_EINVAL, "handle is NULL");
    if (!g->have_case) return fail3(CLBM_EINVAL, "call clbm3_set_case first");
    CK3(cudaSetDevice(g->device));
    const size_t nc = ncells(g);
    double *dr = rho, *du = ut;
    if (!dst_is_device) {
        double* sb = nullptr;
        clbm_status st = staging(g, &sb);
        if (st != CLBM_OK) return st;
        dr = rho ? sb : nullptr;
        du = ut ? sb + nc : nullptr;
    }
    const Args3 A = args(g);
    launch_boundary(g, A);
    launch_cells<true>(g, A, dr, du);
    CK3(cudaGetLastError());
    if (!dst_is_device) {
        if (rho) CK3(cudaMemcpyAsync(rho, dr, nc * 8, cudaMemcpyDeviceToHost, g->stream));
        if (ut) CK3(cudaMemcpyAsync(ut, du, 3 * nc * 8, cudaMemcpyDeviceToHost, g->stream));
    }
    CK3(cudaStreamSynchronize(g->stream));
    return CLBM_OK;
}

clbm_status clbm3_totals(clbm3_handle g, double out[4]) {
    if (!g || !out) return fail3(CLBM_EINVAL, "NULL argument");
    if (!g->have_case) return fail3(CLBM_EINVAL, "call clbm3_set_case first");
    CK3(cudaSetDevice(g->device));
    dim3 cg((n23(g) + TB - 1) / TB, g->n1);
    const int nb = (int)(cg.x * cg.y);
    by_storage(g->prec, [&](auto tag) {
        using S = typename decltype(tag)::type;
        k3_totals<S><<<cg, TB, 0, g->stream>>>((const S*)g->st[g->cur], g->n1, n23(g), plane(g), g->partial);
    });
    k3_totals_final<<<4, 256, 0, g->stream>>>(g->partial, nb, g->red);
    CK3(cudaGetLastError());
    double v[4];
    std::vector<double> geo((size_t)g->n1 * Geo3::S);
    CK3(cudaMemcpyAsync(v, g->red, sizeof(v), cudaMemcpyDeviceToHost, g->stream));
    CK3(cudaMemcpyAsync(geo.data(), g->geo, geo.size() * 8, cudaMemcpyDeviceToHost, g->stream));
    CK3(cudaStreamSynchronize(g->stream));
    double rest = 0.0;  // sum of ref over the cells: rho0 J per cell
    for (int r = 0; r < g->n1; ++r) rest += g->cs.rho0 * geo[(size_t)r * Geo3::S + Geo3::J];
    out[0] = v[0] + rest * n23(g);
    for (int q = 1; q < 4; ++q) out[q] = v[q];
    return CLBM_OK;
}

clbm_status clbm3_set_kernel(clbm3_handle g, int kernel) {
    if (!g) return fail3(CLBM_EINVAL, "handle is NULL");
    if (kernel < 0 || kernel > 2) return fail3(CLBM_EINVAL, "kernel %d is not 0, 1 or 2", kernel);
    if (kernel == 2 && g->prec == CLBM_FP64)
        return fail3(CLBM_EINVAL, "kernel 2 is an FP32-compute update; FP64 grids run kernel 1");
    CK3(cudaSetDevice(g->device));
    CK3(cudaStreamSynchronize(g->stream));
    if (g->gexec) cudaGraphExecDestroy(g->gexec);   // the captured steps launch the old kernel
    if (g->graph) cudaGraphDestroy(g->graph);
    g->gexec = nullptr;
    g->graph = nullptr;
    g->kernel = kernel;
    return CLBM_OK;
}

clbm_status clbm3_time(clbm3_handle g, long long* t) {
    if (!g || !t) return fail3(CLBM_EINVAL, "NULL argument");
    *t = g->t;
    return CLBM_OK;
}

clbm_status clbm3_destroy(clbm3_handle g) {
    if (!g) return CLBM_OK;
    cudaSetDevice(g->device);
    cudaStreamSynchronize(g->stream);
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->graph) cudaGraphDestroy(g->graph);
    cudaFree(g->edges);
    cudaFree(g->geo);
    cudaFree(g->tab);
    cudaFree(g->st[0]);
    cudaFree(g->st[1]);
    cudaFree(g->wall);
    cudaFree(g->partial);
    cudaFree(g->red);
    cudaFree(g->stage);
    delete g;
    return CLBM_OK;
}

}  // extern "C"
