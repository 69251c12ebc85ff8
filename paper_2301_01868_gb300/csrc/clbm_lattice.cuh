// clbm_lattice.cuh -- D2Q9 / D2Q21 constants of the CUDA path (App. A).
//
// Velocity order follows the index maps of App. B (first component is the
// wall-normal one); the two outer D2Q21 shells carry 1/432 and 1/1620, the
// values that make the App. A isotropy conditions hold exactly (the printed
// 7/432 and 7/1620 do not sum to one).  Everything is constexpr so that, in
// unrolled loops, every c_alpha folds into the arithmetic.
#pragma once

namespace clbm {

__host__ __device__ __forceinline__ constexpr int c1_of(int a) {
    return (a == 1 || a == 5 || a == 8) ? 1
         : (a == 3 || a == 6 || a == 7) ? -1
         : (a == 9 || a == 13 || a == 16) ? 2
         : (a == 11 || a == 14 || a == 15) ? -2
         : (a == 17) ? 3
         : (a == 19) ? -3 : 0;
}

__host__ __device__ __forceinline__ constexpr int c2_of(int a) {
    return (a == 2 || a == 5 || a == 6) ? 1
         : (a == 4 || a == 7 || a == 8) ? -1
         : (a == 10 || a == 13 || a == 14) ? 2
         : (a == 12 || a == 15 || a == 16) ? -2
         : (a == 18) ? 3
         : (a == 20) ? -3 : 0;
}

// Reverse direction (bounce-back map alpha*).
__host__ __device__ __forceinline__ constexpr int opp_of(int a) {
    return a == 0 ? 0
         : (a <= 4) ? ((a + 1) % 4 + 1)                 // 1<->3, 2<->4
         : (a <= 8) ? ((a - 5 + 2) % 4 + 5)             // 5<->7, 6<->8
         : (a <= 12) ? ((a - 9 + 2) % 4 + 9)            // 9<->11, 10<->12
         : (a <= 16) ? ((a - 13 + 2) % 4 + 13)          // 13<->15, 14<->16
         : ((a - 17 + 2) % 4 + 17);                     // 17<->19, 18<->20
}

// Direction with the wall-normal component flipped (specular map alpha-hat).
__host__ __device__ __forceinline__ constexpr int hat_of(int a) {
    return (a == 1) ? 3 : (a == 3) ? 1 : (a == 5) ? 6 : (a == 6) ? 5
         : (a == 7) ? 8 : (a == 8) ? 7 : (a == 9) ? 11 : (a == 11) ? 9
         : (a == 13) ? 14 : (a == 14) ? 13 : (a == 15) ? 16 : (a == 16) ? 15
         : (a == 17) ? 19 : (a == 19) ? 17 : a;
}

template <int Q> struct Lat;

template <> struct Lat<9> {
    static constexpr int H = 1;          // stencil reach = ghost depth
    static constexpr int NP = 4;         // +/- pairs
    static constexpr double T0 = 1.0 / 3.0;
    __host__ __device__ static constexpr double w(int a) {
        return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    // "+" member of pair p; its partner is opp_of(plus(p)).
    __host__ __device__ static constexpr int plus(int p) { return p == 0 ? 1 : p == 1 ? 2 : p == 2 ? 5 : 6; }
};

template <> struct Lat<21> {
    static constexpr int H = 3;
    static constexpr int NP = 10;
    static constexpr double T0 = 2.0 / 3.0;
    __host__ __device__ static constexpr double w(int a) {
        return a == 0 ? 91.0 / 324.0
             : a <= 4 ? 1.0 / 12.0
             : a <= 8 ? 2.0 / 27.0
             : a <= 12 ? 7.0 / 360.0
             : a <= 16 ? 1.0 / 432.0
             : 1.0 / 1620.0;
    }
    __host__ __device__ static constexpr int plus(int p) {
        return p == 0 ? 1 : p == 1 ? 2 : p == 2 ? 5 : p == 3 ? 6 : p == 4 ? 9
             : p == 5 ? 10 : p == 6 ? 13 : p == 7 ? 14 : p == 8 ? 17 : 18;
    }
};

// Per-row coefficient table of the fused update, in the compute type.
// Slots: a 16-value header (metric, rest-state sums evaluated in FP64), then
// 12 values per +/- pair (a = plus(p), b = opp(a)), each group of four read
// as one vector, in the lane order of the update's paired arithmetic:
//   A = (a^1_b, a^1_a, a^2_b, a^2_a)          Christoffel contractions
//   B = (E11, E22, E12, P0_a)                  dPi weights, rest polynomial
//   D = (Delta_a, Delta_b, 0, 0)               pull offsets ref(i - c1) - ref(i)
template <int Q> struct Tab {
    static constexpr int INVJ = 0, J = 1, G11 = 2, G12 = 3, G22 = 4;
    static constexpr int F01 = 5, F02 = 6, P00 = 7, FI1 = 8, FI2 = 9;
    static constexpr int D0 = 10, M1 = 11, M2 = 12;
    // diagnostics only: covariant metric g_ij and angular-momentum weights
    static constexpr int C11 = 13, C12 = 14, C22 = 15, AM1 = 16, AM2 = 17;
    static constexpr int PB = 20;
    static constexpr int S = PB + 12 * Lat<Q>::NP;              // stride (multiple of 4)
    __host__ __device__ static constexpr int pa(int p) { return PB + 12 * p; }
    __host__ __device__ static constexpr int pb(int p) { return PB + 12 * p + 4; }
    __host__ __device__ static constexpr int pd(int p) { return PB + 12 * p + 8; }
};

// Per-cell table of a general grid, one plane of n1 n2 values per entry:
// the Tab<Q> header values INVJ .. AM2 at the same indices, then per pair the
// contractions (a^1_b, a^1_a, a^2_b, a^2_a) and the pull offsets
// (Delta_a, Delta_b); P0 and the dPi weights are formed when read.
template <int Q>
struct CellTabLayout {
    static constexpr int NS = Tab<Q>::AM2 + 1;                  // header values
    __host__ __device__ static constexpr int pa(int q) { return NS + 6 * q; }
    __host__ __device__ static constexpr int pd(int q) { return NS + 6 * q + 4; }
    static constexpr int S = NS + 6 * Lat<Q>::NP;               // entries per cell
};

// Four table values read with one vector load.
template <typename C> struct V4 { C x, y, z, w; };
__device__ __forceinline__ V4<float> ld4(const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
    const double2 u = reinterpret_cast<const double2*>(p)[0];
    const double2 v = reinterpret_cast<const double2*>(p)[1];
    return {u.x, u.y, v.x, v.y};
}

// Per-row FP64 geometry (geometry precompute output, plus the deviation
// reference).  a^k_alpha = c^m_alpha Theta^k_m(q + c_alpha, q) (Eq. 5).
struct Geo {
    static constexpr int J = 0, JGEO = 1, GI11 = 2, GI12 = 3, GI22 = 4;
    static constexpr int G11 = 5, G12 = 6, G22 = 7, M1 = 8, M2 = 9, G2N = 10, R = 11;
    static constexpr int A0 = 12;                       // a1, a2 per alpha (2Q)
    __host__ __device__ static constexpr int a1(int a) { return A0 + 2 * a; }
    __host__ __device__ static constexpr int a2(int a) { return A0 + 2 * a + 1; }
    __host__ __device__ static constexpr int ref(int Q, int a) { return A0 + 2 * Q + a; }
    __host__ __device__ static constexpr int stride(int Q) { return A0 + 3 * Q; }
};

}  // namespace clbm
