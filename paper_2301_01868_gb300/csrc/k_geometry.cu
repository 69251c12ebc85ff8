// k_geometry.cu -- geometry / metric / Christoffel precompute (Sec. 2,
// Eqs. 1-5) and the per-row coefficient tables of the fused update.
//
// Planar and polar grids are invariant under a shift along q^2 (translation,
// rotation), so every quantity is evaluated once per row, at column 1, from
// the node positions around it; a state that does not depend on j then stays
// exactly independent of j under the update, as in the paper's runs.
#include "clbm_cell.cuh"

namespace clbm {

namespace {

// Node positions (n1+8) x 9 columns: rows i = -3..n1+4, columns j = -3..5
// (1-based), x and y interleaved.
struct Pos {
    const double* p;
    __device__ double2 at(int i, int j) const {
        const double* q = p + (((size_t)(i + 3) * 9 + (size_t)(j + 3)) * 2);
        return make_double2(q[0], q[1]);
    }
};

// Tangent vector g_m at node (i, j): [D_m - D_-m] / (2 dx) (Sec. 2).
__device__ double2 tangent(const Pos& P, int m, int i, int j, double dx) {
    double2 xp = (m == 0) ? P.at(i + 1, j) : P.at(i, j + 1);
    double2 xm = (m == 0) ? P.at(i - 1, j) : P.at(i, j - 1);
    double2 x0 = P.at(i, j);
    double2 dp = make_double2(xp.x - x0.x, xp.y - x0.y);
    double2 dm = make_double2(xm.x - x0.x, xm.y - x0.y);
    return make_double2((dp.x - dm.x) / (2.0 * dx), (dp.y - dm.y) / (2.0 * dx));
}

template <int Q>
__global__ void k_geometry(const double* __restrict__ pos, int n1, double dx, int polar,
                           double* __restrict__ geo) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n1) return;
    const int i = r + 1;  // 1-based row
    Pos P{pos};
    double2 g1 = tangent(P, 0, i, 1, dx), g2 = tangent(P, 1, i, 1, dx);
    double J = g1.x * g2.y - g1.y * g2.x;                       // Eq. 2, g_3 = z
    double2 G1 = make_double2(g2.y / J, -g2.x / J);             // Eq. 3
    double2 G2 = make_double2(-g1.y / J, g1.x / J);
    double* o = geo + (size_t)r * Geo::stride(Q);
    o[Geo::J] = J;
    o[Geo::JGEO] = J;
    o[Geo::GI11] = G1.x * G1.x + G1.y * G1.y;
    o[Geo::GI12] = G1.x * G2.x + G1.y * G2.y;
    o[Geo::GI22] = G2.x * G2.x + G2.y * G2.y;
    o[Geo::G11] = g1.x * g1.x + g1.y * g1.y;
    o[Geo::G12] = g1.x * g2.x + g1.y * g2.y;
    o[Geo::G22] = g2.x * g2.x + g2.y * g2.y;
    double2 x = P.at(i, 1);
    o[Geo::M1] = polar ? (x.x * g1.y - x.y * g1.x) : 0.0;
    o[Geo::M2] = polar ? (x.x * g2.y - x.y * g2.x) : 0.0;
    o[Geo::G2N] = sqrt(o[Geo::G22]);
    o[Geo::R] = sqrt(x.x * x.x + x.y * x.y);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int c1 = c1_of(a), c2 = c2_of(a);
        double a1 = 0.0, a2 = 0.0;
        if (a != 0) {
            // Eq. 5: Theta^k_m(q + c, q) = [g_m(q + c) - g_m(q)] . g^k(q),
            // contracted with c^m.
            double2 h1 = tangent(P, 0, i + c1, 1 + c2, dx);
            double2 h2 = tangent(P, 1, i + c1, 1 + c2, dx);
            double2 d1 = make_double2(h1.x - g1.x, h1.y - g1.y);
            double2 d2 = make_double2(h2.x - g2.x, h2.y - g2.y);
            double t11 = d1.x * G1.x + d1.y * G1.y, t12 = d2.x * G1.x + d2.y * G1.y;
            double t21 = d1.x * G2.x + d1.y * G2.y, t22 = d2.x * G2.x + d2.y * G2.y;
            a1 = c1 * t11 + c2 * t12;
            a2 = c1 * t21 + c2 * t22;
        }
        o[Geo::a1(a)] = a1;
        o[Geo::a2(a)] = a2;
    }
}

// Rest-equilibrium polynomial P0(c) = 1 + 1/2 [c.(g - 1).c / T0 - tr(g - 1)]
// (the second-order term of Eq. 19 at U = Ut = 0).
template <int Q>
__host__ __device__ double rest_poly(int a, double gi11, double gi12, double gi22) {
    const double T0 = Lat<Q>::T0;
    const double c1 = c1_of(a), c2 = c2_of(a);
    double q = c1 * c1 * (gi11 - 1.0) + 2.0 * c1 * c2 * gi12 + c2 * c2 * (gi22 - 1.0);
    return 1.0 + 0.5 * (q / T0 - (gi11 - 1.0) - (gi22 - 1.0));
}

template <int Q>
__global__ void k_reference(double* __restrict__ geo, int n1, double rho0) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n1) return;
    double* o = geo + (size_t)r * Geo::stride(Q);
#pragma unroll
    for (int a = 0; a < Q; ++a)
        o[Geo::ref(Q, a)] = o[Geo::J] * Lat<Q>::w(a) * rho0 *
                            rest_poly<Q>(a, o[Geo::GI11], o[Geo::GI12], o[Geo::GI22]);
}

template <int Q, typename C>
__global__ void k_tables(const double* __restrict__ geo, C* __restrict__ tab, int n1) {
    using T = Tab<Q>;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n1) return;
    const int i = r + 1;
    const double* g = geo + (size_t)r * Geo::stride(Q);
    C* t = tab + (size_t)r * T::S;
    for (int k = 0; k < T::S; ++k) t[k] = C(0);
    const double J = g[Geo::J];
    t[T::INVJ] = C(1.0 / J);
    t[T::J] = C(J);
    t[T::G11] = C(g[Geo::GI11]);
    t[T::G12] = C(g[Geo::GI12]);
    t[T::G22] = C(g[Geo::GI22]);
    t[T::P00] = C(rest_poly<Q>(0, g[Geo::GI11], g[Geo::GI12], g[Geo::GI22]));
    // Pull offsets and the rest-state sums (FP64, rounded once).
    double dl[Q];
    double D0 = 0.0, M1 = 0.0, M2 = 0.0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        dl[a] = ref_at<Q>(geo, n1, a, i - c1_of(a)) - g[Geo::ref(Q, a)];
        D0 += dl[a];
        M1 += c1_of(a) * dl[a];
        M2 += c2_of(a) * dl[a];
    }
    t[T::D0] = C(D0);
    t[T::M1] = C(M1);
    t[T::M2] = C(M2);
    // Force of the rest parts: with the stored sigma (lagged) and the pulled
    // sigma, sum_b a_b [ref_b(i) + ref_{opp b}(i - c1_{opp b})]; with own-row
    // deviations d (implicit passes), sum_b a_b [ref_b(i) + ref_{opp b}(i)].
    double F01 = 0.0, F02 = 0.0, FI1 = 0.0, FI2 = 0.0;
#pragma unroll
    for (int b = 1; b < Q; ++b) {
        const int ob = opp_of(b);
        const double ab1 = g[Geo::a1(b)], ab2 = g[Geo::a2(b)];
        const double own = g[Geo::ref(Q, b)];
        const double in = g[Geo::ref(Q, ob)] + dl[ob];
        F01 += ab1 * (own + in);
        F02 += ab2 * (own + in);
        FI1 += ab1 * (own + in - dl[ob]);
        FI2 += ab2 * (own + in - dl[ob]);
    }
    t[T::F01] = C(F01);
    t[T::F02] = C(F02);
    t[T::FI1] = C(FI1);
    t[T::FI2] = C(FI2);
#pragma unroll
    for (int p = 0; p < Lat<Q>::NP; ++p) {
        const int a = Lat<Q>::plus(p), ab = opp_of(a);
        const double w = Lat<Q>::w(a);
        const double c1 = c1_of(a), c2 = c2_of(a);
        const double D1 = g[Geo::a1(a)] + g[Geo::a1(ab)];
        const double D2 = g[Geo::a2(a)] + g[Geo::a2(ab)];
        t[T::pa(p) + 0] = C(g[Geo::a1(a)]);
        t[T::pa(p) + 1] = C(g[Geo::a2(a)]);
        t[T::pa(p) + 2] = C(g[Geo::a1(ab)]);
        t[T::pa(p) + 3] = C(g[Geo::a2(ab)]);
        t[T::pb(p) + 0] = C(rest_poly<Q>(a, g[Geo::GI11], g[Geo::GI12], g[Geo::GI22]));
        t[T::pb(p) + 1] = C(2.0 * w * c1 * D1);
        t[T::pb(p) + 2] = C(2.0 * w * c2 * D2);
        t[T::pb(p) + 3] = C(w * (c1 * D2 + c2 * D1));
        t[T::pd(p) + 0] = C(dl[a]);
        t[T::pd(p) + 1] = C(dl[ab]);
    }
}

// Ghost table [wall][k-1][alpha] x {offset, coefficient}: the stored ghost
// value of direction a at depth k is sigma_b(m) + offset + coefficient * rho
// (U0 - Ut^2) with b = a* (no-slip) or a-hat (moving wall) and m the mirrored
// row; the offset converts between the two rows' references.
template <int Q>
__global__ void k_ghost(const double* __restrict__ geo, double* __restrict__ ghost, int n1,
                        int bc_lo, int bc_hi) {
    constexpr int H = Lat<Q>::H;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * H * Q) return;
    const int wall = t / (H * Q), k = (t / Q) % H + 1, a = t % Q;
    const int bc = wall == 0 ? bc_lo : bc_hi;
    const int b = bc == 0 ? opp_of(a) : hat_of(a);
    const int gr = wall == 0 ? 1 - k : n1 + k;          // ghost row (1-based)
    const int m = wall == 0 ? k : n1 + 1 - k;           // mirrored fluid row
    const double off = ref_at<Q>(geo, n1, b, m) - ref_at<Q>(geo, n1, a, gr);
    double coef = 0.0;
    if (bc == 1)  // App. B moving wall, reading (2/T0) w J rho c^2 (U0^2 - Ut^2)
        coef = 2.0 / Lat<Q>::T0 * Lat<Q>::w(b) * geo[(size_t)(m - 1) * Geo::stride(Q) + Geo::J] *
               c2_of(b);
    ghost[2 * t] = off;
    ghost[2 * t + 1] = coef;
}

}  // namespace

void launch_geometry(int Q, const double* pos, int n1, double dx, int polar, double* geo,
                     cudaStream_t s) {
    dim3 b(128), g((n1 + 127) / 128);
    if (Q == 9) k_geometry<9><<<g, b, 0, s>>>(pos, n1, dx, polar, geo);
    else k_geometry<21><<<g, b, 0, s>>>(pos, n1, dx, polar, geo);
}

void launch_reference(int Q, double* geo, int n1, double rho0, cudaStream_t s) {
    dim3 b(128), g((n1 + 127) / 128);
    if (Q == 9) k_reference<9><<<g, b, 0, s>>>(geo, n1, rho0);
    else k_reference<21><<<g, b, 0, s>>>(geo, n1, rho0);
}

void launch_tables(int Q, int prec, const double* geo, void* tab, double* ghost, int n1,
                   double, int bc_lo, int bc_hi, cudaStream_t s) {
    dim3 b(128), g((n1 + 127) / 128);
    if (Q == 9) {
        if (prec == 0) k_tables<9, double><<<g, b, 0, s>>>(geo, (double*)tab, n1);
        else k_tables<9, float><<<g, b, 0, s>>>(geo, (float*)tab, n1);
        k_ghost<9><<<1, 2 * 1 * 9, 0, s>>>(geo, ghost, n1, bc_lo, bc_hi);
    } else {
        if (prec == 0) k_tables<21, double><<<g, b, 0, s>>>(geo, (double*)tab, n1);
        else k_tables<21, float><<<g, b, 0, s>>>(geo, (float*)tab, n1);
        k_ghost<21><<<1, 2 * 3 * 21, 0, s>>>(geo, ghost, n1, bc_lo, bc_hi);
    }
}

}  // namespace clbm
