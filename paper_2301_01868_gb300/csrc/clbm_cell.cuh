// clbm_cell.cuh -- per-cell pieces of the update shared by the fused step
// and the diagnostics kernels: pull with the lagged read, moments and force
// (Eqs. 7-15), and the collision of Sec. 2 (Eqs. 16-19, 11), written in
// deviations from the rest equilibrium.
//
// The state buffer holds sigma_a(r) = N'_a(r) - ref_a(r), zero at rest, with
// ghost rows (walls) and ghost columns (periodic copies) around the interior,
// so a pull is a load at a constant offset from the cell.  A pulled value
// becomes a deviation from the cell's own reference by adding
// Delta_a = ref_a(i - c1) - ref_a(i); the rest parts of every sum are
// FP64-evaluated per-row constants of the table.
#pragma once

#include "clbm_internal.cuh"

namespace clbm {

// Per-launch scalars in the compute type (converted once on the host).
template <typename C> struct Consts;
template <> struct Consts<double> {
    double rho0, g1, g2, tau_inv, omt, pref;
    __device__ static Consts make(const StepScalars& s) {
        return {s.rho0, s.g1, s.g2, s.tau_inv, s.omt, s.pref};
    }
};
template <> struct Consts<float> {
    float rho0, g1, g2, tau_inv, omt, pref;
    __device__ static Consts make(const StepScalars& s) {
        return {s.frho0, s.fg1, s.fg2, s.ftau_inv, s.fomt, s.fpref};
    }
};

// Two compute values operated on together.  An FP32 pair is a float2, and
// pfma / padd / pmul issue one packed FP32 instruction (sm_100 and later)
// for both lanes, each lane rounded exactly as the scalar operation; an FP64
// pair is two scalar operations.  The update keeps the two directions of a
// +/- pair (and the two lanes of its sums) in one pair wherever the same
// operation applies to both, so the packed form halves those instructions.
template <typename C> struct PairOf;
template <> struct PairOf<float> { using T = float2; };
template <> struct PairOf<double> { using T = double2; };

__device__ __forceinline__ float2 mkp(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 mkp(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }

template <int Q, typename C>
struct Cell {
    C d[Q];                                   // pulled deviations from this row's reference
    C drho, rho, irho, U1, U2, F1, F2, Ut1, Ut2;
    C ls, ls1, ls2;                           // sums of the lagged sigma: 1, c^1, c^2 weighted
};

// Coefficient tables as the update reads them.  s(k): header value k of
// Tab<Q> (INVJ .. M2); pair q = (a, b = -a): pa(q) the Christoffel
// contractions (a^1_b, a^1_a, a^2_b, a^2_a), pd(q) the pull offsets
// (Delta_a, Delta_b), pb(q) the dPi weights and rest polynomial
// (E11, E22, E12, P0_a); p0(q): P0_a alone.
//
// RowTab: one Tab<Q> block per row (planar and polar grids), read as
// aligned vectors (global or shared memory).
template <int Q, typename C>
struct RowTab {
    // the pull offset vanishes for directions with c^1 = 0 (same row)
    static constexpr bool ALL_OFFSETS = false;
    const C* p;
    __device__ __forceinline__ C s(int k) const { return p[k]; }
    __device__ __forceinline__ V4<C> pa(int q) const { return ld4(p + Tab<Q>::pa(q)); }
    __device__ __forceinline__ V4<C> pb(int q) const { return ld4(p + Tab<Q>::pb(q)); }
    __device__ __forceinline__ C p0(int q) const { return p[Tab<Q>::pb(q) + 3]; }
    __device__ __forceinline__ V4<C> pd(int q) const { return ld4(p + Tab<Q>::pd(q)); }
};

// A sum of products v * k whose coefficients k are lattice constants
// (compile-time after unrolling), accumulated in the order of the terms.  A
// term with k = 0 is left out: IEEE rules forbid a compiler to drop a
// product with a literal zero (it would be NaN for an infinite v), but adding
// an exact zero leaves the sum unchanged, so leaving it out saves the
// instruction and keeps every rounding.
template <typename C>
struct KSum {
    C s = C(0);
    bool any = false;
    __device__ __forceinline__ KSum() {}
    __device__ __forceinline__ explicit KSum(C first) : s(first), any(true) {}
    __device__ __forceinline__ void add(C v, double k) {
        if (k != 0.0) {
            s = any ? fma(v, C(k), s) : v * C(k);
            any = true;
        }
    }
};

// Rest polynomial of Eq. 19 at U = Ut = 0 in the compute type:
// 1 + [c.(g - 1).c / T0 - tr(g - 1)] / 2 for direction a.
template <int Q, typename C>
__device__ __forceinline__ C rest_poly_c(int a, C gi11, C gi12, C gi22) {
    const double c1 = c1_of(a), c2 = c2_of(a);
    KSum<C> q;
    q.add(gi11 - C(1), c1 * c1);
    q.add(gi12, 2.0 * c1 * c2);
    q.add(gi22 - C(1), c2 * c2);
    return C(1) + C(0.5) * (q.s * C(1.0 / Lat<Q>::T0) - (gi11 - C(1)) - (gi22 - C(1)));
}

// CellTab: per-cell tables of general grids, one plane of n1 n2 values per
// entry (CellTabLayout), so a warp's loads are coalesced.  The dPi weights
// and P0 are formed from the metric and the contractions instead of stored.
template <int Q, typename C>
struct CellTab {
    using L = CellTabLayout<Q>;
    // every direction pulls from a cell with its own reference
    static constexpr bool ALL_OFFSETS = true;
    const C* p;             // entry 0 of this cell
    size_t st;              // plane stride (cells)
    C gi11, gi12, gi22;     // inverse metric of the cell (read once)
    __device__ __forceinline__ CellTab(const C* p_, size_t st_) : p(p_), st(st_) {
        gi11 = ld(Tab<Q>::G11);
        gi12 = ld(Tab<Q>::G12);
        gi22 = ld(Tab<Q>::G22);
    }
    __device__ __forceinline__ C ld(int k) const { return __ldg(p + (size_t)k * st); }
    __device__ __forceinline__ C s(int k) const {
        return k == Tab<Q>::G11 ? gi11 : k == Tab<Q>::G12 ? gi12 : k == Tab<Q>::G22 ? gi22 : ld(k);
    }
    __device__ __forceinline__ V4<C> pa(int q) const {
        return {ld(L::pa(q)), ld(L::pa(q) + 1), ld(L::pa(q) + 2), ld(L::pa(q) + 3)};
    }
    __device__ __forceinline__ V4<C> pd(int q) const { return {ld(L::pd(q)), ld(L::pd(q) + 1), C(0), C(0)}; }
    __device__ __forceinline__ C p0(int q) const { return rest_poly_c<Q, C>(Lat<Q>::plus(q), gi11, gi12, gi22); }
    __device__ __forceinline__ V4<C> pb(int q) const {
        const int a = Lat<Q>::plus(q);
        const double w = Lat<Q>::w(a), c1 = c1_of(a), c2 = c2_of(a);
        const V4<C> A = pa(q);
        const C D1 = A.x + A.y, D2 = A.z + A.w;
        KSum<C> e11, e22, e12;
        e11.add(D1, 2.0 * w * c1);
        e22.add(D2, 2.0 * w * c2);
        e12.add(D2, w * c1);
        e12.add(D1, w * c2);
        return {e11.s, e22.s, e12.s, p0(q)};
    }
};

// The table of cell (i, j): RowTab for planar / polar grids (GEN = false),
// CellTab for general grids.
template <int Q, typename C, bool GEN> struct TabOf;
template <int Q, typename C> struct TabOf<Q, C, false> {
    __device__ static __forceinline__ RowTab<Q, C> at(const void* tab, int i, int, int, int) {
        return {(const C*)tab + (size_t)i * Tab<Q>::S};
    }
};
template <int Q, typename C> struct TabOf<Q, C, true> {
    __device__ static __forceinline__ CellTab<Q, C> at(const void* tab, int i, int j, int n1, int n2) {
        return CellTab<Q, C>((const C*)tab + (size_t)i * n2 + j, (size_t)n1 * n2);
    }
};

// Advection (Eq. 12) with the lagged read of N'(q, t-1), moments (Eqs. 7, 8,
// 10) and the lagged inertial force (Eq. 15 with N'(q, t-1)):
//   F^k = -1/(2J) sum_b a^k_b [N'_b(q, t-1) + N_{opp b}(q, t)] + rho g^k.
// ld(alpha, dr, dc) returns the stored value of population alpha at the cell
// offset by (dr, dc) rows / columns; dr and dc are compile-time after unrolling.
// SC: the values ld returns are SC times the deviations (a power of two, so
// every sum is exactly SC times the unscaled one); c.d and the lagged sums
// keep the scale, the moments and the force are unscaled.
template <int Q, typename C, int SC = 1, typename LD, typename TB>
__device__ __forceinline__ void pull_cell(LD&& ld, const TB& tb, const Consts<C>& k, Cell<Q, C>& c) {
    using L = Lat<Q>;
    using T = Tab<Q>;
    using P = typename PairOf<C>::T;
    // two-lane sums: lane x collects direction a of each pair, lane y b
    // the rest parts of the sums (table constants) join at the same scale
    P sd = mkp(tb.s(T::D0) * C(SC), C(0));
    P s1 = mkp(tb.s(T::M1) * C(SC), C(0)), s2 = mkp(tb.s(T::M2) * C(SC), C(0));
    P f1 = mkp(tb.s(T::F01) * C(SC), C(0)), f2 = mkp(tb.s(T::F02) * C(SC), C(0));
    P ls = mkp(C(0), C(0)), ls1 = mkp(C(0), C(0)), ls2 = mkp(C(0), C(0));
    c.d[0] = ld(0, 0, 0);
#pragma unroll
    for (int q = 0; q < L::NP; ++q) {
        const int a = L::plus(q), b = opp_of(a);
        const int c1 = c1_of(a), c2 = c2_of(a);
        const V4<C> A = tb.pa(q);
        // pulled: N_a(q) from q - c_a, N_b(q) from q + c_a; lagged: own values
        const P pp = mkp(ld(a, -c1, -c2), ld(b, c1, c2));
        const P lg = mkp(ld(b, 0, 0), ld(a, 0, 0));        // (lagged b, lagged a)
        sd = padd(sd, pp);
        // momentum: c_b = -c_a, so the pair adds c_a (N_a - N_b).  With row
        // tables (the pipelined update, FMA-pipe bound) the scalar form is
        // faster: fewer lane operations than the packed one with its
        // constant pairs; with per-cell tables (general grids, bound by the
        // table loads) the packed form measured faster
        if (TB::ALL_OFFSETS) {
            if (c1 != 0) s1 = pfma(mkp(C(c1), C(-c1)), pp, s1);
            if (c2 != 0) s2 = pfma(mkp(C(c2), C(-c2)), pp, s2);
        } else if (c1 != 0 || c2 != 0) {
            const C df = pp.x - pp.y;
            if (c1 != 0) s1.x = fma(C(c1), df, s1.x);
            if (c2 != 0) s2.x = fma(C(c2), df, s2.x);
        }
        // (N'_b + N_a, N'_a + N_b): the two sums the contractions of a and b weigh
        const P t = padd(lg, pp);
        f1 = pfma(mkp(A.x, A.y), t, f1);
        f2 = pfma(mkp(A.z, A.w), t, f2);
        ls = padd(ls, lg);
        if (c1 != 0) ls1 = pfma(mkp(C(-c1), C(c1)), lg, ls1);
        if (c2 != 0) ls2 = pfma(mkp(C(-c2), C(c2)), lg, ls2);
        if (c1 != 0 || TB::ALL_OFFSETS) {
            const V4<C> D = tb.pd(q);
            const P dd = SC == 1 ? padd(pp, mkp(D.x, D.y)) : pfma(mkp(D.x, D.y), mkp(C(SC), C(SC)), pp);
            c.d[a] = dd.x;
            c.d[b] = dd.y;
        } else {
            c.d[a] = pp.x;
            c.d[b] = pp.y;
        }
    }
    c.ls = c.d[0] + (ls.x + ls.y);
    c.ls1 = ls1.x + ls1.y;
    c.ls2 = ls2.x + ls2.y;
    const C invJ = tb.s(T::INVJ) * C(1.0 / SC);
    c.drho = (c.d[0] + sd.x + sd.y) * invJ;
    c.rho = k.rho0 + c.drho;
    c.irho = C(1) / c.rho;
    c.U1 = (s1.x + s1.y) * invJ * c.irho;
    c.U2 = (s2.x + s2.y) * invJ * c.irho;
    c.F1 = -C(0.5) * invJ * (f1.x + f1.y) + c.rho * k.g1;
    c.F2 = -C(0.5) * invJ * (f2.x + f2.y) + c.rho * k.g2;
}

// Loader of the global buffer: p points at the cell in population plane 0,
// P is the plane stride and ld the row stride (elements).  Offsets are
// 32-bit: a grid's Q planes hold fewer than 2^31 values (checked when the
// grid is created).
template <typename S>
struct GlobalLoad {
    const S* p;
    int P;
    int ld;
    __device__ __forceinline__ typename Store<S>::C operator()(int al, int dr, int dc) const {
        return Store<S>::ld(p + (al * P + dr * ld + dc));
    }
};

// The force of Eq. 15 re-evaluated with the newest N'(q, t) (own-row
// deviations out[]) for one fixed-point pass of the implicit relation.
template <int Q, typename C, typename TB>
__device__ __forceinline__ void force_again(const TB& tb, const C (&out)[Q], const Consts<C>& k,
                                            Cell<Q, C>& c) {
    using T = Tab<Q>;
    using L = Lat<Q>;
    using P = typename PairOf<C>::T;
    P f1 = mkp(tb.s(T::FI1), C(0)), f2 = mkp(tb.s(T::FI2), C(0));
#pragma unroll
    for (int q = 0; q < L::NP; ++q) {
        const int a = L::plus(q), b = opp_of(a);
        const V4<C> A = tb.pa(q);
        const P t = padd(mkp(out[b], out[a]), mkp(c.d[a], c.d[b]));
        f1 = pfma(mkp(A.x, A.y), t, f1);
        f2 = pfma(mkp(A.z, A.w), t, f2);
    }
    const C invJ = tb.s(T::INVJ);
    c.F1 = -C(0.5) * invJ * (f1.x + f1.y) + c.rho * k.g1;
    c.F2 = -C(0.5) * invJ * (f2.x + f2.y) + c.rho * k.g2;
}

// Ut (Eq. 18), equilibrium coefficients (Eq. 19), odd parts, the momentum-flux
// correction (Eq. 16, symmetric part), source (Eq. 17) and BGK (Eqs. 6, 11).
// emit(alpha, value) receives every new post-collision deviation, times SC
// when pull_cell ran with that scale.
template <int Q, typename C, int SC = 1, typename TB, typename Emit>
__device__ __forceinline__ void collide_emit(const TB& tb, Cell<Q, C>& c, const Consts<C>& k,
                                             Emit&& emit) {
    using L = Lat<Q>;
    using T = Tab<Q>;
    constexpr C T0 = C(L::T0);
    constexpr C iT0 = C(1.0 / L::T0);
    constexpr C i2T02 = C(0.5 / (L::T0 * L::T0));
    constexpr C i6T03 = C(1.0 / (6.0 * L::T0 * L::T0 * L::T0));
    const C U1 = c.U1, U2 = c.U2;
    const C Ut1 = U1 + C(0.5) * c.F1 * c.irho;
    const C Ut2 = U2 + C(0.5) * c.F2 * c.irho;
    c.Ut1 = Ut1;
    c.Ut2 = Ut2;
    const C gi11 = tb.s(T::G11), gi12 = tb.s(T::G12), gi22 = tb.s(T::G22);
    // Third-order Hermite coefficients C^{ijk} of Eq. 19 (symmetric).
    const C C111 = T0 * (C(3) * gi11 * Ut1 - C(3) * U1) + Ut1 * Ut1 * Ut1;
    const C C112 = T0 * (gi11 * Ut2 + C(2) * gi12 * Ut1 - U2) + Ut1 * Ut1 * Ut2;
    const C C122 = T0 * (C(2) * gi12 * Ut2 + gi22 * Ut1 - U1) + Ut1 * Ut2 * Ut2;
    const C C222 = T0 * (C(3) * gi22 * Ut2 - C(3) * U2) + Ut2 * Ut2 * Ut2;
    const C K11 = U1 * iT0 - (C111 + C122) * i2T02;
    const C K12 = U2 * iT0 - (C112 + C222) * i2T02;
    const C K111 = C111 * i6T03, K112 = C(3) * C112 * i6T03;
    const C K122 = C(3) * C122 * i6T03, K222 = C222 * i6T03;
    const C dK0 = -(Ut1 * Ut1 + Ut2 * Ut2) * (C(0.5) * iT0);
    const C dK11 = Ut1 * Ut1 * i2T02, dK12 = C(2) * Ut1 * Ut2 * i2T02, dK22 = Ut2 * Ut2 * i2T02;

    // Odd part of f^eq / (rho w) per +/- pair; only odd parts survive the pair
    // sums of the momentum-flux correction.
    C O[L::NP];
    C S11 = C(0), S22 = C(0), S12 = C(0);
#pragma unroll
    for (int q = 0; q < L::NP; ++q) {
        const int a = L::plus(q);
        const double c1 = c1_of(a), c2 = c2_of(a);
        KSum<C> o;
        o.add(K11, c1);
        o.add(K12, c2);
        o.add(K111, c1 * c1 * c1);
        o.add(K112, c1 * c1 * c2);
        o.add(K122, c1 * c2 * c2);
        o.add(K222, c2 * c2 * c2);
        O[q] = o.s;
        // the weights vanish exactly with the velocity components they carry
        // (E11 = 2 w c1 D1, E22 = 2 w c2 D2)
        const V4<C> B = tb.pb(q);
        if (c1 != 0.0) S11 += B.x * O[q];
        if (c2 != 0.0) S22 += B.y * O[q];
        S12 += B.z * O[q];
    }
    const C pr = k.pref * c.rho;
    S11 *= pr;
    S22 *= pr;
    S12 *= pr;
    const C trS = S11 + S22;
    const C J = tb.s(T::J) * C(SC);
    const C omt = k.omt;
    const C drt = c.drho * k.tau_inv, rt = c.rho * k.tau_inv;
    const C Fa = c.F1 * iT0, Fb = c.F2 * iT0;
    const C base = rt * dK0 - trS * iT0;
    const C Ea = rt * dK11 + S11 * (iT0 * iT0);
    const C Eb = rt * dK12 + C(2) * S12 * (iT0 * iT0);
    const C Ec = rt * dK22 + S22 * (iT0 * iT0);
    using P = typename PairOf<C>::T;
    emit(0, c.d[0] * omt + J * C(L::w(0)) * (drt * tb.s(T::P00) + base));
    const P omt2 = mkp(omt, omt), J2 = mkp(J, J);
#pragma unroll
    for (int q = 0; q < L::NP; ++q) {
        const int a = L::plus(q), b = opp_of(a);
        const double c1 = c1_of(a), c2 = c2_of(a);
        KSum<C> x(drt * tb.p0(q) + base), y(rt * O[q]);
        x.add(Ea, c1 * c1);
        x.add(Eb, c1 * c2);
        x.add(Ec, c2 * c2);
        y.add(Fa, c1);
        y.add(Fb, c2);
        const C X = x.s, Y = y.s;
        const C w = C(L::w(a));
        // (N'_a, N'_b) = (d_a, d_b) (1 - 1/tau) + J w (X + Y, X - Y)
        const P o = pfma(pmul(J2, mkp(w, w)), mkp(X + Y, X - Y), pmul(mkp(c.d[a], c.d[b]), omt2));
        emit(a, o.x);
        emit(b, o.y);
    }
}

// Per-cell terms of the residual and conservation sums (clbm_residual):
// J |u(t) - u(t')|^2, J |u|^2 (physical u = Ut^k g_k), the deviation part of
// the mass (the rest part, rho0 times the total volume, is added on the
// host) and the momentum sum c N' (2), kinetic energy J rho |u|^2 / 2,
// angular momentum J rho (M1 Ut^1 + M2 Ut^2), |u|^2, and a flag for a
// non-finite or non-positive density.  Everything is formed in the compute
// type from the coefficient table (no FP64 work per cell in FP32 compute).
// prev holds Ut of the last call in the compute type.
template <typename C>
struct CellTerms {
    C dd, uu_j, ls, ls1, ls2, ke, am, uu;
    bool bad;
};

// p1, p2: Ut of the last call (read only when have_prev).
template <int Q, typename C, typename TB>
__device__ __forceinline__ CellTerms<C> residual_terms(const Cell<Q, C>& c, const TB& tb, C p1, C p2,
                                                       bool have_prev) {
    using T = Tab<Q>;
    const C g11 = tb.s(T::C11), g12 = tb.s(T::C12), g22 = tb.s(T::C22);
    const C J = tb.s(T::J);
    const C u1 = c.Ut1, u2 = c.Ut2;
    CellTerms<C> t;
    t.uu = g11 * u1 * u1 + C(2) * g12 * u1 * u2 + g22 * u2 * u2;
    t.dd = C(0);
    if (have_prev) {
        const C e1 = u1 - p1, e2 = u2 - p2;
        t.dd = J * (g11 * e1 * e1 + C(2) * g12 * e1 * e2 + g22 * e2 * e2);
    }
    t.uu_j = J * t.uu;
    t.ls = c.ls;
    t.ls1 = c.ls1;
    t.ls2 = c.ls2;
    t.ke = C(0.5) * J * c.rho * t.uu;
    t.am = J * c.rho * (tb.s(T::AM1) * u1 + tb.s(T::AM2) * u2);
    t.bad = !(c.rho > C(0) && isfinite(c.rho) && isfinite(t.uu));
    return t;
}

// The same with the snapshot in memory: reads the last Ut, writes this one.
template <int Q, typename C, typename TB>
__device__ __forceinline__ CellTerms<C> residual_terms(const Cell<Q, C>& c, const TB& tb, C* prev1, C* prev2,
                                                       bool have_prev) {
    const CellTerms<C> t = residual_terms<Q, C, TB>(c, tb, have_prev ? *prev1 : C(0),
                                                    have_prev ? *prev2 : C(0), have_prev);
    *prev1 = c.Ut1;
    *prev2 = c.Ut2;
    return t;
}

// A thread's running sums of CellTerms, reduced in FP64 afterwards (slots of
// NRED: 0 dd, 1 |u|^2, 2 mass, 3-4 momentum, 5 kinetic energy, 6 angular
// momentum, 7 largest |u|^2, 8 unstable cells).  FP64 compute sums in FP64;
// FP32 compute sums with Kahan compensation in FP32 (the FP64 pipe is far
// slower).
template <typename C> struct ResAcc;
template <> struct ResAcc<double> {
    double v[NRED] = {};
    __device__ __forceinline__ void add(const CellTerms<double>& t) {
        v[0] += t.dd;
        v[1] += t.uu_j;
        v[2] += t.ls;
        v[3] += t.ls1;
        v[4] += t.ls2;
        v[5] += t.ke;
        v[6] += t.am;
        v[7] = fmax(v[7], t.uu);
        v[8] += t.bad ? 1.0 : 0.0;
    }
    __device__ __forceinline__ void out(double (&o)[NRED]) const {
        for (int k = 0; k < NRED; ++k) o[k] = v[k];
    }
};
template <> struct ResAcc<float> {
    float s[7] = {}, e[7] = {};
    float umax = 0.f, bad = 0.f;
    __device__ __forceinline__ void kahan(int k, float x) {
        const float y = x - e[k];
        const float t = s[k] + y;
        e[k] = (t - s[k]) - y;
        s[k] = t;
    }
    __device__ __forceinline__ void add(const CellTerms<float>& t) {
        kahan(0, t.dd);
        kahan(1, t.uu_j);
        kahan(2, t.ls);
        kahan(3, t.ls1);
        kahan(4, t.ls2);
        kahan(5, t.ke);
        kahan(6, t.am);
        umax = fmaxf(umax, t.uu);
        bad += t.bad ? 1.f : 0.f;
    }
    __device__ __forceinline__ void out(double (&o)[NRED]) const {
        for (int k = 0; k < 7; ++k) o[k] = double(s[k]) - double(e[k]);
        o[7] = umax;
        o[8] = bad;
        o[9] = 0.0;
    }
};

// One CTA's partial of the residual sums: warp shuffles, then the warps in
// order (a fixed tree, so repeated runs give identical bits); slot 7 is the
// largest |u|^2, reduced by max and rooted here.  Every thread of the CTA
// calls it with its own sums.
template <int NT>
__device__ __forceinline__ void block_partial(double (&v)[NRED], double* out) {
#pragma unroll
    for (int k = 0; k < NRED; ++k) {
        double x = v[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double y = __shfl_down_sync(0xffffffffu, x, off);
            x = (k == 7) ? fmax(x, y) : x + y;
        }
        v[k] = x;
    }
    __shared__ double sh[NT / 32][NRED];
    const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
    if (ln == 0)
        for (int k = 0; k < NRED; ++k) sh[w][k] = v[k];
    __syncthreads();
    if (threadIdx.x < NRED) {
        const int k = threadIdx.x;
        double x = sh[0][k];
        for (int q = 1; q < NT / 32; ++q) x = (k == 7) ? fmax(x, sh[q][k]) : x + sh[q][k];
        out[k] = k == 7 ? sqrt(x) : x;
    }
}

// Reference N of direction a at 1-based row r and geometry column jc (FP64
// geometry table of ncol columns); rows beyond a wall are the mirror image
// of the row inside, which flips c^1.
template <int Q>
__device__ __forceinline__ double ref_at(const double* geo, int n1, int ncol, int a, int r, int jc) {
    int m = r, b = a;
    if (r < 1) { m = 1 - r; b = hat_of(a); }
    else if (r > n1) { m = 2 * n1 + 1 - r; b = hat_of(a); }
    return geo[((size_t)(m - 1) * ncol + jc) * Geo::stride(Q) + Geo::ref(Q, b)];
}

// The periodic copies of interior column j (0..n2-1) in the ghost columns
// (state column = j + GC), and the value with its copies.
template <typename S, typename C>
__device__ __forceinline__ void store_wrap(S* __restrict__ rowp, int j, int n2, C v) {
    if (j < GC)
        for (int jj = j + n2; jj < n2 + GC; jj += n2) Store<S>::st(rowp + jj + GC, v);
    if (j >= n2 - GC)
        for (int jj = j - n2; jj >= -GC; jj -= n2) Store<S>::st(rowp + jj + GC, v);
}
template <typename S, typename C>
__device__ __forceinline__ void store_periodic(S* __restrict__ rowp, int j, int n2, C v) {
    Store<S>::st(rowp + j + GC, v);
    store_wrap<S, C>(rowp, j, n2, v);
}

// Ghost value of App. B from the stored N' of the mirrored fluid node (x):
// the offset between the two rows' references plus, at a moving wall, the
// correction (2/T0) w J rho c^2 (U0^2 - Ut^2) of the mirrored node, whose
// per-direction factor is coef.
template <typename C>
__device__ __forceinline__ C ghost_value(C x, const C* __restrict__ gt, C rho, C U0, C ut2) {
    return x + (gt[0] + gt[1] * rho * (U0 - ut2));
}

// Periodic ghost column of interior column j when a row has at least 2 GC
// columns: one copy, at column j + n2 (j < GC) or j - n2 (j >= n2 - GC), as
// an offset from j; 0 when the cell has none.  Updates store it next to the
// cell's own value as it is produced (a read-back after the stores would
// hold the warp for a round trip).  Shorter rows need several copies:
// EdgeFill makes them.
__device__ __forceinline__ int wrap_offset(int j, int n2) {
    if (n2 < 2 * GC) return 0;
    return j < GC ? n2 : (j >= n2 - GC ? -n2 : 0);
}

// Fills, from the cell that supplies them, the ghost rows of App. B that the
// next update pulls from the buffer being written: at the first / last H rows
// (depth k = i + 1 / n1 - i) the new N'_b of the mirrored node feeds ghost
// population a = b* (no-slip) or a = b-hat (moving wall) of depth k when a
// crosses the wall that deep (c^1_a >= k at the low wall, <= -k at the high
// wall; * and hat are involutions), with the moving-wall correction from the
// cell's own rho and Ut^2.  The values are those the boundary kernel would
// compute from the stored state.  With own_wrap (rows shorter than 2 GC in
// the kernels that store cells one by one) it also makes the periodic ghost
// columns of the cell's own row.  needed(): the cells that have something
// to fill.
//
// Called once per edge cell after the collision with vp pointing at the
// cell's new stored N'_0 (N'_b at vp + b vstride, in global or shared
// memory), in a function of its own, since edge rows are few and the
// interior update should keep its registers and code small.
template <int Q, typename S>
struct EdgeFill {
    using C = typename Store<S>::C;
    S* st;                   // state buffer being written (row 0, column 0)
    const C* ghost;          // [2][H][Q] x {offset, coefficient}, compute type
    long long plane;
    int ld, n1, n2, bc_lo, bc_hi;
    C U0_lo, U0_hi;
    bool own_wrap;
    int gcols;               // ghost-table columns: 1 (planar, polar) or n2 (general)

    __device__ static __forceinline__ bool needed(int i, int n1, int n2) {
        return i < Lat<Q>::H || i >= n1 - Lat<Q>::H || n2 < 2 * GC;
    }

    __device__ __noinline__ void fill(int i, int j, const S* vp, long long vstride, C rho, C ut2) const {
        fill_inline(i, j, vp, vstride, rho, ut2);
    }
    // the same in line, for the kernels whose registers hold it without
    // spilling (the one-cell pipeline: no out-of-line call on its wall rows)
    __device__ __forceinline__ void fill_inline(int i, int j, const S* vp, long long vstride, C rho,
                                                C ut2) const {
        constexpr int H = Lat<Q>::H;
        // all read-backs first (independent loads in flight together), then
        // the stores; unrolled so that every direction's maps fold
        C vb[Q];
#pragma unroll
        for (int b = 0; b < Q; ++b) vb[b] = Store<S>::lds(vp + b * vstride);
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            const C v = vb[b];
            if (own_wrap) store_wrap<S, C>(st + b * plane + (long long)(i + H) * ld, j, n2, v);
            if (i < H) {
                const int k = i + 1;
                const int a = bc_lo == 0 ? opp_of(b) : hat_of(b);
                if (c1_of(a) >= k) {
                    const C* gt = ghost + 2 * (((k - 1) * Q + a) * gcols + (gcols > 1 ? j : 0));
                    store_periodic<S, C>(st + a * plane + (long long)(H - k) * ld, j, n2,
                                         ghost_value<C>(v, gt, rho, U0_lo, ut2));
                }
            }
            if (i >= n1 - H) {
                const int k = n1 - i;
                const int a = bc_hi == 0 ? opp_of(b) : hat_of(b);
                if (c1_of(a) <= -k) {
                    const C* gt = ghost + 2 * (((H + k - 1) * Q + a) * gcols + (gcols > 1 ? j : 0));
                    store_periodic<S, C>(st + a * plane + (long long)(n1 + H + k - 1) * ld, j, n2,
                                         ghost_value<C>(v, gt, rho, U0_hi, ut2));
                }
            }
        }
    }
};

}  // namespace clbm
