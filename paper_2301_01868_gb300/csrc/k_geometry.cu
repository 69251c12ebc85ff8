// k_geometry.cu -- geometry / metric / Christoffel precompute (Sec. 2,
// Eqs. 1-5) and the coefficient tables of the fused update.
//
// Planar and polar grids are invariant under a shift along q^2 (translation,
// rotation), so every quantity is evaluated once per row, at column 1, from
// the node positions around it (ncol = 1); a state that does not depend on j
// then stays exactly independent of j under the update, as in the paper's
// runs.  General grids evaluate every cell (ncol = n2) from the node
// positions the caller supplies, ghosts included.
#include "clbm_cell.cuh"

namespace clbm {

namespace {

// Node positions (n1+8) x (ncol+8): rows i = -3..n1+4, columns j = -3..ncol+4
// (1-based), x and y interleaved.
struct Pos {
    const double* p;
    int ncp;                // ncol + 8
    __device__ double2 at(int i, int j) const {
        const double* q = p + (((size_t)(i + 3) * ncp + (size_t)(j + 3)) * 2);
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

// One thread per (row, geometry column); moments: the angular momentum
// weights x cross g_k (about the origin) unless planar.
template <int Q>
__global__ void k_geometry(const double* __restrict__ pos, int n1, int ncol, double dx, int moments,
                           double* __restrict__ geo) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int jc = blockIdx.y;
    if (r >= n1) return;
    const int i = r + 1, j = jc + 1;  // 1-based node
    Pos P{pos, ncol + 8};
    double2 g1 = tangent(P, 0, i, j, dx), g2 = tangent(P, 1, i, j, dx);
    double J = g1.x * g2.y - g1.y * g2.x;                       // Eq. 2, g_3 = z
    double2 G1 = make_double2(g2.y / J, -g2.x / J);             // Eq. 3
    double2 G2 = make_double2(-g1.y / J, g1.x / J);
    double* o = geo + ((size_t)r * ncol + jc) * Geo::stride(Q);
    o[Geo::J] = J;
    o[Geo::JGEO] = J;
    o[Geo::GI11] = G1.x * G1.x + G1.y * G1.y;
    o[Geo::GI12] = G1.x * G2.x + G1.y * G2.y;
    o[Geo::GI22] = G2.x * G2.x + G2.y * G2.y;
    o[Geo::G11] = g1.x * g1.x + g1.y * g1.y;
    o[Geo::G12] = g1.x * g2.x + g1.y * g2.y;
    o[Geo::G22] = g2.x * g2.x + g2.y * g2.y;
    double2 x = P.at(i, j);
    o[Geo::M1] = moments ? (x.x * g1.y - x.y * g1.x) : 0.0;
    o[Geo::M2] = moments ? (x.x * g2.y - x.y * g2.x) : 0.0;
    o[Geo::G2N] = sqrt(o[Geo::G22]);
    o[Geo::R] = sqrt(x.x * x.x + x.y * x.y);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int c1 = c1_of(a), c2 = c2_of(a);
        double a1 = 0.0, a2 = 0.0;
        if (a != 0) {
            // Eq. 5: Theta^k_m(q + c, q) = [g_m(q + c) - g_m(q)] . g^k(q),
            // contracted with c^m.
            double2 h1 = tangent(P, 0, i + c1, j + c2, dx);
            double2 h2 = tangent(P, 1, i + c1, j + c2, dx);
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
__global__ void k_reference(double* __restrict__ geo, int count, double rho0) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= count) return;
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
    t[T::C11] = C(g[Geo::G11]);
    t[T::C12] = C(g[Geo::G12]);
    t[T::C22] = C(g[Geo::G22]);
    t[T::AM1] = C(g[Geo::M1]);
    t[T::AM2] = C(g[Geo::M2]);
    // Pull offsets and the rest-state sums (FP64, rounded once).
    double dl[Q];
    double D0 = 0.0, M1 = 0.0, M2 = 0.0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        dl[a] = ref_at<Q>(geo, n1, 1, a, i - c1_of(a), 0) - g[Geo::ref(Q, a)];
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
        // pair order of the update: (b, a) contractions, then the dPi weights
        t[T::pa(p) + 0] = C(g[Geo::a1(ab)]);
        t[T::pa(p) + 1] = C(g[Geo::a1(a)]);
        t[T::pa(p) + 2] = C(g[Geo::a2(ab)]);
        t[T::pa(p) + 3] = C(g[Geo::a2(a)]);
        t[T::pb(p) + 0] = C(2.0 * w * c1 * D1);
        t[T::pb(p) + 1] = C(2.0 * w * c2 * D2);
        t[T::pb(p) + 2] = C(w * (c1 * D2 + c2 * D1));
        t[T::pb(p) + 3] = C(rest_poly<Q>(a, g[Geo::GI11], g[Geo::GI12], g[Geo::GI22]));
        t[T::pd(p) + 0] = C(dl[a]);
        t[T::pd(p) + 1] = C(dl[ab]);
    }
}

// Per-cell tables of general grids (CellTabLayout, one plane per entry): the
// header values and, per +/- pair, the contractions a^k and the pull offsets,
// with Delta_a = ref_a(source cell) - ref_a(cell), the source cell being
// (i - c1, j - c2) with j periodic and rows beyond a wall mirrored.
template <int Q, typename C>
__global__ void k_tables_cell(const double* __restrict__ geo, C* __restrict__ tab, int n1, int n2) {
    using T = Tab<Q>;
    using L = CellTabLayout<Q>;
    const int jc = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (jc >= n2) return;
    const int i = r + 1;
    const size_t st = (size_t)n1 * n2, m = (size_t)r * n2 + jc;
    const double* g = geo + m * Geo::stride(Q);
    auto put = [&](int k, double v) { tab[(size_t)k * st + m] = C(v); };
    const double J = g[Geo::J];
    put(T::INVJ, 1.0 / J);
    put(T::J, J);
    put(T::G11, g[Geo::GI11]);
    put(T::G12, g[Geo::GI12]);
    put(T::G22, g[Geo::GI22]);
    put(T::P00, rest_poly<Q>(0, g[Geo::GI11], g[Geo::GI12], g[Geo::GI22]));
    put(T::C11, g[Geo::G11]);
    put(T::C12, g[Geo::G12]);
    put(T::C22, g[Geo::G22]);
    put(T::AM1, g[Geo::M1]);
    put(T::AM2, g[Geo::M2]);
    double dl[Q];
    double D0 = 0.0, M1 = 0.0, M2 = 0.0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        int js = (jc - c2_of(a)) % n2;
        if (js < 0) js += n2;
        dl[a] = ref_at<Q>(geo, n1, n2, a, i - c1_of(a), js) - g[Geo::ref(Q, a)];
        D0 += dl[a];
        M1 += c1_of(a) * dl[a];
        M2 += c2_of(a) * dl[a];
    }
    put(T::D0, D0);
    put(T::M1, M1);
    put(T::M2, M2);
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
    put(T::F01, F01);
    put(T::F02, F02);
    put(T::FI1, FI1);
    put(T::FI2, FI2);
#pragma unroll
    for (int p = 0; p < Lat<Q>::NP; ++p) {
        const int a = Lat<Q>::plus(p), ab = opp_of(a);
        put(L::pa(p) + 0, g[Geo::a1(ab)]);
        put(L::pa(p) + 1, g[Geo::a1(a)]);
        put(L::pa(p) + 2, g[Geo::a2(ab)]);
        put(L::pa(p) + 3, g[Geo::a2(a)]);
        put(L::pd(p) + 0, dl[a]);
        put(L::pd(p) + 1, dl[ab]);
    }
}

// Ghost table [wall][k-1][alpha][column] x {offset, coefficient} (one column
// unless the grid is general): the stored ghost value of direction a at
// depth k is sigma_b(m) + offset + coefficient * rho (U0 - Ut^2) with
// b = a* (no-slip) or a-hat (moving wall) and m the mirrored row of the same
// column; the offset converts between the two cells' references.  Stored in
// the compute type C (formed in FP64, rounded once here rather than at every
// use by the update's ghost fill).
template <int Q, typename C>
__global__ void k_ghost(const double* __restrict__ geo, C* __restrict__ ghost, int n1, int ncol,
                        int bc_lo, int bc_hi) {
    constexpr int H = Lat<Q>::H;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * H * Q * ncol) return;
    const int jc = t % ncol, u = t / ncol;
    const int wall = u / (H * Q), k = (u / Q) % H + 1, a = u % Q;
    const int bc = wall == 0 ? bc_lo : bc_hi;
    const int b = bc == 0 ? opp_of(a) : hat_of(a);
    const int gr = wall == 0 ? 1 - k : n1 + k;          // ghost row (1-based)
    const int m = wall == 0 ? k : n1 + 1 - k;           // mirrored fluid row
    const double off = ref_at<Q>(geo, n1, ncol, b, m, jc) - ref_at<Q>(geo, n1, ncol, a, gr, jc);
    double coef = 0.0;
    if (bc == 1)  // App. B moving wall, reading (2/T0) w J rho c^2 (U0^2 - Ut^2)
        coef = 2.0 / Lat<Q>::T0 * Lat<Q>::w(b) *
               geo[((size_t)(m - 1) * ncol + jc) * Geo::stride(Q) + Geo::J] * c2_of(b);
    ghost[2 * t] = C(off);
    ghost[2 * t + 1] = C(coef);
}

}  // namespace

void launch_geometry(int Q, const double* pos, int n1, int ncol, double dx, int moments, double* geo,
                     cudaStream_t s) {
    dim3 b(128), g((n1 + 127) / 128, ncol);
    if (Q == 9) k_geometry<9><<<g, b, 0, s>>>(pos, n1, ncol, dx, moments, geo);
    else k_geometry<21><<<g, b, 0, s>>>(pos, n1, ncol, dx, moments, geo);
}

void launch_reference(int Q, double* geo, int count, double rho0, cudaStream_t s) {
    dim3 b(128), g((count + 127) / 128);
    if (Q == 9) k_reference<9><<<g, b, 0, s>>>(geo, count, rho0);
    else k_reference<21><<<g, b, 0, s>>>(geo, count, rho0);
}

template <int Q>
static void tables(int prec, const double* geo, void* tab, void* ghost, int n1, int n2, int ncol,
                   int bc_lo, int bc_hi, cudaStream_t s) {
    constexpr int H = Lat<Q>::H;
    if (ncol > 1) {
        dim3 b(128), g((n2 + 127) / 128, n1);
        if (prec == 0) k_tables_cell<Q, double><<<g, b, 0, s>>>(geo, (double*)tab, n1, n2);
        else k_tables_cell<Q, float><<<g, b, 0, s>>>(geo, (float*)tab, n1, n2);
    } else {
        dim3 b(128), g((n1 + 127) / 128);
        if (prec == 0) k_tables<Q, double><<<g, b, 0, s>>>(geo, (double*)tab, n1);
        else k_tables<Q, float><<<g, b, 0, s>>>(geo, (float*)tab, n1);
    }
    const int nt = 2 * H * Q * ncol;
    if (prec == 0) k_ghost<Q, double><<<(nt + 127) / 128, 128, 0, s>>>(geo, (double*)ghost, n1, ncol, bc_lo, bc_hi);
    else k_ghost<Q, float><<<(nt + 127) / 128, 128, 0, s>>>(geo, (float*)ghost, n1, ncol, bc_lo, bc_hi);
}

void launch_tables(int Q, int prec, const double* geo, void* tab, void* ghost, int n1, int n2,
                   int ncol, int bc_lo, int bc_hi, cudaStream_t s) {
    if (Q == 9) tables<9>(prec, geo, tab, ghost, n1, n2, ncol, bc_lo, bc_hi, s);
    else tables<21>(prec, geo, tab, ghost, n1, n2, ncol, bc_lo, bc_hi, s);
}

}  // namespace clbm
