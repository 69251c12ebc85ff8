// clbm_f2.cuh -- two cells of one row computed together: a compute type F2
// whose every operation acts on both cells with one packed FP32 instruction
// (sm_100 and later: __ffma2_rn / __fadd2_rn / __fmul2_rn, each lane rounded
// exactly as the scalar operation), so that the update's arithmetic
// (pull_cell, collide_emit) compiles unchanged for a pair of neighbouring
// cells.  The two cells share their row's coefficient table, read once.
//
// A product is kept unevaluated (F2Prod) until it is added to something,
// where it becomes one fused multiply-add -- the contraction the compiler
// performs on the scalar form -- or until it is used as a value.
#pragma once

#include "clbm_cell.cuh"

namespace clbm {

struct F2 {
    float2 v;
    F2() = default;
    __host__ __device__ constexpr F2(float2 a) : v(a) {}
    __host__ __device__ constexpr F2(double d) : v{float(d), float(d)} {}
    __host__ __device__ constexpr F2(float d) : v{d, d} {}
    __host__ __device__ constexpr F2(int d) : v{float(d), float(d)} {}
    __host__ __device__ constexpr F2(float x, float y) : v{x, y} {}
};

struct F2Prod {
    float2 a, b;
    __device__ __forceinline__ operator F2() const { return F2(__fmul2_rn(a, b)); }
};

__device__ __forceinline__ F2 neg(F2 x) { return F2(-x.v.x, -x.v.y); }
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }

__device__ __forceinline__ F2Prod operator*(F2 a, F2 b) { return {a.v, b.v}; }
__device__ __forceinline__ F2Prod operator*(F2Prod p, F2 b) { return {F2(p).v, b.v}; }
__device__ __forceinline__ F2Prod operator*(F2 a, F2Prod p) { return {a.v, F2(p).v}; }
__device__ __forceinline__ F2Prod operator*(F2Prod p, F2Prod q) { return {F2(p).v, F2(q).v}; }

__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator+(F2Prod p, F2 c) { return F2(__ffma2_rn(p.a, p.b, c.v)); }
__device__ __forceinline__ F2 operator+(F2 c, F2Prod p) { return F2(__ffma2_rn(p.a, p.b, c.v)); }
__device__ __forceinline__ F2 operator+(F2Prod p, F2Prod q) { return F2(__ffma2_rn(p.a, p.b, F2(q).v)); }

// a - b as b (-1) + a: one packed instruction, exact as the subtraction
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
    return F2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v));
}
__device__ __forceinline__ F2 operator-(F2Prod p, F2 c) { return F2(p) - c; }
__device__ __forceinline__ F2 operator-(F2 c, F2Prod p) { return F2(__ffma2_rn(neg(F2(p.a)).v, p.b, c.v)); }
__device__ __forceinline__ F2 operator-(F2Prod p, F2Prod q) {
    return F2(__ffma2_rn(neg(F2(q.a)).v, q.b, F2(p).v));
}
__device__ __forceinline__ F2 operator-(F2 a) { return neg(a); }
__device__ __forceinline__ F2 operator-(F2Prod p) { return neg(F2(p)); }

__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2(a.v.x / b.v.x, a.v.y / b.v.y); }

__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator+=(F2& a, F2Prod p) { return a = a + p; }
__device__ __forceinline__ F2& operator*=(F2& a, F2 b) { return a = F2(a * b); }

// Two directions of a +/- pair for the two cells: four lanes.
struct F2P {
    F2 x, y;
};
template <> struct PairOf<F2> { using T = F2P; };
__device__ __forceinline__ F2P mkp(F2 x, F2 y) { return {x, y}; }
__device__ __forceinline__ F2P pfma(F2P a, F2P b, F2P c) { return {fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)}; }
__device__ __forceinline__ F2P padd(F2P a, F2P b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ F2P pmul(F2P a, F2P b) { return {F2(a.x * b.x), F2(a.y * b.y)}; }

template <> struct Consts<F2> {
    F2 rho0, g1, g2, tau_inv, omt, pref;
    __device__ static Consts make(const StepScalars& s) {
        return {F2(s.frho0), F2(s.fg1), F2(s.fg2), F2(s.ftau_inv), F2(s.fomt), F2(s.fpref)};
    }
};

// The row's table (FP32, shared memory) as both cells read it.
template <int Q>
struct RowTab2 {
    static constexpr bool ALL_OFFSETS = false;
    const float* p;
    __device__ __forceinline__ F2 s(int k) const { return F2(p[k]); }
    __device__ __forceinline__ static V4<F2> b4(const V4<float>& v) { return {F2(v.x), F2(v.y), F2(v.z), F2(v.w)}; }
    __device__ __forceinline__ V4<F2> pa(int q) const { return b4(ld4(p + Tab<Q>::pa(q))); }
    __device__ __forceinline__ V4<F2> pb(int q) const { return b4(ld4(p + Tab<Q>::pb(q))); }
    __device__ __forceinline__ F2 p0(int q) const { return F2(p[Tab<Q>::pb(q) + 3]); }
    __device__ __forceinline__ V4<F2> pd(int q) const { return b4(ld4(p + Tab<Q>::pd(q))); }
};

// Two neighbouring stored values (cells j, j + 1) as floats, from shared
// memory; EVEN: the first sits at an even element, so both come in one
// aligned load.
template <typename S, bool EVEN> struct Ld2;
template <bool EVEN> struct Ld2<float, EVEN> {
    __device__ static __forceinline__ float2 ld(const float* p) {
        if (EVEN) return *reinterpret_cast<const float2*>(p);
        return make_float2(p[0], p[1]);
    }
};
template <bool EVEN> struct Ld2<__half, EVEN> {
    __device__ static __forceinline__ float2 ld(const __half* p) {
        if (EVEN) return __half22float2(*reinterpret_cast<const __half2*>(p));
        return make_float2(__half2float(p[0]), __half2float(p[1]));
    }
};
template <bool EVEN> struct Ld2<__nv_bfloat16, EVEN> {
    __device__ static __forceinline__ float2 ld(const __nv_bfloat16* p) {
        if (EVEN) return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
        return make_float2(__bfloat162float(p[0]), __bfloat162float(p[1]));
    }
};

// Store of both cells' values (already in the storage scale) at an even
// element of global memory with the streaming hint; one only when the
// second cell lies past the row's end.
template <typename S> struct St2;
template <> struct St2<float> {
    __device__ static __forceinline__ void st(float* p, F2 v, bool both) {
        if (both) __stcs(reinterpret_cast<float2*>(p), v.v);
        else __stcs(p, v.v.x);
    }
};
template <> struct St2<__half> {
    __device__ static __forceinline__ void st(__half* p, F2 v, bool both) {
        if (both) __stcs(reinterpret_cast<__half2*>(p), __float22half2_rn(v.v));
        else __stcs(p, __float2half_rn(v.v.x));
    }
};
template <> struct St2<__nv_bfloat16> {
    __device__ static __forceinline__ void st(__nv_bfloat16* p, F2 v, bool both) {
        if (both) __stcs(reinterpret_cast<__nv_bfloat162*>(p), __float22bfloat162_rn(v.v));
        else __stcs(p, __float2bfloat16_rn(v.v.x));
    }
};

}  // namespace clbm
