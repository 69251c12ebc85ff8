// clbm3.cuh -- the three-dimensional form of the update (Sec. 2 is written
// for three coordinates) on the D3Q39 lattice: constants, table layouts and
// launch arguments of k3d.cu.
//
// D3Q39: shells (0,0,0), (1,0,0), (1,1,1), (2,0,0), (2,2,0), (3,0,0) with
// weights 1/12, 1/12, 1/27, 2/135, 1/432, 1/1620 and T0 = 2/3, isotropic
// through the sixth order (the 3-D counterpart of D2Q21; the paper prints no
// 3-D set).  Velocity order: shell by shell, each shell in lexicographic
// order of (c1, c2, c3); reversal maps index s + e - a within shell [s, e].
// The order is part of the interface (populations cross it in this order).
#pragma once

#include "clbm_internal.cuh"

namespace clbm {
namespace d3 {

constexpr int Q = 39;          // velocities
constexpr int NP = 19;         // +/- pairs
constexpr int H = 3;           // ghost rows per wall (largest |c1|)
constexpr double T0 = 2.0 / 3.0;

__host__ __device__ __forceinline__ constexpr int c1_3(int a) {
    constexpr int v[39] = {0, -1, 0, 0, 0, 0, 1, -1, -1, -1, -1, 1, 1, 1, 1, -2, 0, 0, 0, 0, 2, -2, -2, -2, -2, 0, 0, 0, 0, 2, 2, 2, 2, -3, 0, 0, 0, 0, 3};
    return v[a];
}
__host__ __device__ __forceinline__ constexpr int c2_3(int a) {
    constexpr int v[39] = {0, 0, -1, 0, 0, 1, 0, -1, -1, 1, 1, -1, -1, 1, 1, 0, -2, 0, 0, 2, 0, -2, 0, 0, 2, -2, -2, 2, 2, -2, 0, 0, 2, 0, -3, 0, 0, 3, 0};
    return v[a];
}
__host__ __device__ __forceinline__ constexpr int c3_3(int a) {
    constexpr int v[39] = {0, 0, 0, -1, 1, 0, 0, -1, 1, -1, 1, -1, 1, -1, 1, 0, 0, -2, 2, 0, 0, 0, -2, 2, 0, -2, 2, -2, 2, 0, -2, 2, 0, 0, 0, -3, 3, 0, 0};
    return v[a];
}
__host__ __device__ __forceinline__ constexpr int hat3(int a) {
    constexpr int v[39] = {0, 6, 2, 3, 4, 5, 1, 11, 12, 13, 14, 7, 8, 9, 10, 20, 16, 17, 18, 19, 15, 29, 30, 31, 32, 25, 26, 27, 28, 21, 22, 23, 24, 38, 34, 35, 36, 37, 33};
    return v[a];
}

__host__ __device__ __forceinline__ constexpr int opp3(int a) {
    return a == 0 ? 0 : a <= 6 ? 7 - a : a <= 14 ? 21 - a : a <= 20 ? 35 - a : a <= 32 ? 53 - a : 71 - a;
}
__host__ __device__ __forceinline__ constexpr double w3(int a) {
    return a <= 6 ? 1.0 / 12.0 : a <= 14 ? 1.0 / 27.0 : a <= 20 ? 2.0 / 135.0 : a <= 32 ? 1.0 / 432.0
                                                                                       : 1.0 / 1620.0;
}
// "+" member of pair p (the one listed first); its partner is opp3.
__host__ __device__ __forceinline__ constexpr int plus3(int p) {
    constexpr int v[NP] = {1, 2, 3, 7, 8, 9, 10, 15, 16, 17, 21, 22, 23, 24, 25, 26, 33, 34, 35};
    return v[p];
}

// FP64 geometry of one interior row (k3_geometry): volume, inverse and
// covariant metric (11, 12, 13, 22, 23, 33), a^k_alpha = c^m Theta^k_m(q + c, q)
// (Eq. 5) and the rest reference ref_alpha = J w rho0 P0_alpha (case).
struct Geo3 {
    static constexpr int J = 0, GI = 1, GC = 7, A = 13, REF = 13 + 3 * Q, S = 13 + 4 * Q;
};

// Per-row table of the update in the compute type: header, then per pair
// (a = plus3(p), b = opp3(a)) the contractions and pull offsets in the lane
// order of the paired arithmetic, (a^1_b, a^1_a, a^2_b, a^2_a, a^3_b, a^3_a,
// Delta_a, Delta_b) with Delta_alpha = ref_alpha(i - c1) - ref_alpha(i), the
// rest polynomial P0 per direction, and per pair the symmetric dPi weights
// w (c^p D^r + c^r D^p), D = a_alpha + a_opp(alpha), in the order 11, 22, 33,
// 12, 13, 23.  (The rest direction has a = 0 and Delta = 0.)
struct Tab3 {
    static constexpr int INVJ = 0, J = 1, G11 = 2, G12 = 3, G13 = 4, G22 = 5, G23 = 6, G33 = 7;
    static constexpr int F0 = 8;                         // 3 values
    static constexpr int C11 = 11, C12 = 12, C13 = 13, C22 = 14, C23 = 15, C33 = 16;
    static constexpr int HDR = 20;
    __host__ __device__ static constexpr int PA(int p) { return HDR + 8 * p; }
    static constexpr int P0 = HDR + 8 * NP;              // 39 values
    __host__ __device__ static constexpr int E(int p) { return P0 + 40 + 8 * p; }
    static constexpr int S = P0 + 40 + 8 * NP;           // stride, a multiple of 4
};

struct Args3 {
    const void* src;        // state read (row 0 = first ghost row)
    void* dst;              // state written
    const void* tab;        // Tab3 rows (compute type)
    const double* geo;      // Geo3 rows
    void* wall;             // [3 fields][2 walls][H depths][n2 n3], compute type
    int n1, n2, n3;
    long long plane;        // elements per population plane: (n1 + 2H) n2 n3
    int bc_lo, bc_hi;
    double rho0, tau_inv, omt, pref, g1, g2, g3, U0_lo, U0_hi;
};

}  // namespace d3
}  // namespace clbm
