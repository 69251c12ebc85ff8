// clbm_internal.cuh -- device-side data layout and kernel launchers shared by
// the translation units of the CUDA library (not part of the C ABI).
//
// Layout in HBM (one grid):
//   state A, B : [Q][n1 + 2h][ld] in the storage type, ld = n2 + 2 GC rounded
//                up to 32 elements; rows 0..h-1 and n1+h..n1+2h-1 are the
//                ghost rows the boundary kernel fills, columns 0..GC-1 and
//                n2+GC.. hold periodic copies (interior column j sits at
//                j + GC), written by whichever kernel writes the row.  A population is stored as
//                its deviation from the rest equilibrium of its own row,
//                sigma_alpha(i) = N'_alpha(i) - ref_alpha(i), zero at rest
//                (ghost rows use the mirrored row's reference).
//   tab        : [n1][Tab<Q>::S] per-row coefficients in the compute type.
//   geo        : [n1][Geo::stride(Q)] per-row FP64 geometry + references.
//   wall       : [2 walls][h][n2] x {rho, Ut^2} of the last collision (the
//                boundary kernel's input when ghost rows must be rebuilt).
// Each update writes the interior, the ghost rows and the periodic ghost
// columns of the buffer it fills; the boundary kernel rebuilds them only
// after the state or the case was set from outside.
//   ghost      : [2 walls][h][Q] x {offset, correction coefficient}.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "clbm_lattice.cuh"

namespace clbm {

// Storage conversions.  FP16 keeps deviations scaled by SCALE = 2^12 (out of
// the subnormal range; scaling by a power of two is exact).  ld reads global
// memory through the read-only path, lds any address, rt rounds a value the
// way a store and a load would; ldr (global, read-only path) and ldsr (any
// address) read the stored value as it is (SCALE times the deviation), for
// an update that carries the scale through its arithmetic instead.
constexpr float F16_SCALE = 4096.0f;
template <typename S> struct Store;
template <> struct Store<double> {
    using C = double;
    static constexpr int SCALE = 1;
    __device__ static __forceinline__ double ld(const double* p) { return __ldg(p); }
    __device__ static __forceinline__ double lds(const double* p) { return *p; }
    __device__ static __forceinline__ double ldsr(const double* p) { return *p; }
    __device__ static __forceinline__ double ldr(const double* p) { return __ldg(p); }
    __device__ static __forceinline__ void st(double* p, double v) { *p = v; }
    __device__ static __forceinline__ double rt(double v) { return v; }
};
template <> struct Store<float> {
    using C = float;
    static constexpr int SCALE = 1;
    __device__ static __forceinline__ float ld(const float* p) { return __ldg(p); }
    __device__ static __forceinline__ float lds(const float* p) { return *p; }
    __device__ static __forceinline__ float ldsr(const float* p) { return *p; }
    __device__ static __forceinline__ float ldr(const float* p) { return __ldg(p); }
    __device__ static __forceinline__ void st(float* p, float v) { *p = v; }
    __device__ static __forceinline__ float rt(float v) { return v; }
};
template <> struct Store<__half> {
    using C = float;
    static constexpr int SCALE = 4096;   // F16_SCALE
    __device__ static __forceinline__ float ldsr(const __half* p) { return __half2float(*p); }
    __device__ static __forceinline__ float ldr(const __half* p) { return __half2float(__ldg(p)); }
    __device__ static __forceinline__ float ld(const __half* p) {
        return __half2float(__ldg(p)) * (1.0f / F16_SCALE);
    }
    __device__ static __forceinline__ float lds(const __half* p) {
        return __half2float(*p) * (1.0f / F16_SCALE);
    }
    __device__ static __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v * F16_SCALE); }
    __device__ static __forceinline__ float rt(float v) {
        return __half2float(__float2half_rn(v * F16_SCALE)) * (1.0f / F16_SCALE);
    }
};
template <> struct Store<__nv_bfloat16> {
    using C = float;
    static constexpr int SCALE = 1;
    __device__ static __forceinline__ float ldsr(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static __forceinline__ float ldr(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    __device__ static __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    __device__ static __forceinline__ float lds(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
    __device__ static __forceinline__ float rt(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
};

// Stores of the update's output with the streaming cache hint (st.global.cs:
// evict-first): what a launch writes is read only by the next launch, so it
// gives way first to the rows this launch reads again (the halo rows of the
// next bands).  str stores a value already in the storage scale
// (Store<S>::SCALE times the deviation), st a deviation.
template <typename S>
struct StStream {
    using C = typename Store<S>::C;
    __device__ static __forceinline__ void str(S* p, C v) { __stcs(p, S(v)); }
    __device__ static __forceinline__ void st(S* p, C v) { str(p, v * C(Store<S>::SCALE)); }
};

constexpr int GC = 8;  // ghost columns on each side (>= widest |c^2| = 3; 16-byte TMA origins)

// Scalars of the case, in both compute types (converted once on the host).
struct StepScalars {
    double rho0, g1, g2, tau_inv, omt, pref;
    float frho0, fg1, fg2, ftau_inv, fomt, fpref;
};

// Everything one launch of the fused update or of the boundary fill needs.
struct StepArgs {
    StepScalars k;
    const void* src;        // state A (read)
    void* dst;              // state B (written)
    const void* tab;        // per-row coefficients, compute type
    void* wall_rho;         // [2][h][n2] compute type
    void* wall_ut2;
    const void* ghost;      // [2][h][Q][2], compute type
    int n1, n2, ld, h;
    long long plane;        // elements per population plane = (n1+2h)*ld
    double tau, rho0, g1, g2, U0_lo, U0_hi;
    int bc_lo, bc_hi;
    int ncol;               // geometry / ghost-table columns: 1 (planar, polar) or n2 (general)
    int iters;              // extra passes of the implicit force
    int* err;               // device error word (bounded waits that gave up)
};

// Diagnostics launch arguments.
struct MomArgs {
    StepScalars k;
    const void* src;
    const void* tab;
    const double* geo;
    int n1, n2, ld, h;
    long long plane;
    double tau, rho0, g1, g2;
    int ncol;               // 1 (planar, polar) or n2 (general grids: per-cell tables)
    // outputs (device, [n1][n2] FP64, may be null)
    double *rho, *U1, *U2, *Ut1, *Ut2, *F1, *F2;
    // residual mode
    double* ut_prev;        // [2][n1][n2] FP64 snapshot of Ut^k
    double* partial;        // [blocks][NRED]
    int have_prev;
    int* err;               // device error word of bounded waits (pipelined residual)
};

constexpr int NRED = 10;  // reduced quantities per block

// Launchers (defined in the .cu files); all asynchronous on `stream`.
// Geometry of n1 rows x ncol columns (ncol = 1: one column serves the row;
// ncol = n2: general grids), reference states of `count` geometry entries,
// and the coefficient + ghost tables (row tables, or per-cell tables when
// ncol > 1).
void launch_geometry(int Q, const double* pos, int n1, int ncol, double dx, int moments,
                     double* geo, cudaStream_t stream);
void launch_reference(int Q, double* geo, int count, double rho0, cudaStream_t stream);
void launch_tables(int Q, int prec, const double* geo, void* tab, void* ghost, int n1, int n2,
                   int ncol, int bc_lo, int bc_hi, cudaStream_t stream);
void launch_boundary(int Q, int prec, const StepArgs& a, void* state, cudaStream_t stream);
void launch_step(int Q, int prec, const StepArgs& a, cudaStream_t stream);
void launch_moments(int Q, int prec, const MomArgs& a, int iters, int reduce,
                    cudaStream_t stream);
int moments_blocks(int n1, int n2);
void launch_reduce_final(const double* partial, int nblocks, double* out, cudaStream_t stream);
// ncol: geometry columns, 1 (planar, polar) or n2 (general grids).
void launch_state_from_fp64(int Q, int prec, const double* Np, const double* geo, void* state,
                            int n1, int n2, int ld, int h, int ncol, cudaStream_t stream);
void launch_state_to_fp64(int Q, int prec, const void* state, const double* geo, double* Np,
                          int n1, int n2, int ld, int h, int ncol, cudaStream_t stream);
// rho_nf: no-flow density per row (ncol = 1) or per cell (ncol = n2).
void launch_wall_copy(int prec, void* wall_rho, void* wall_ut2, const double* src_rho,
                      const double* src_ut2, const double* rho_nf, int n1, int n2, int h,
                      double rho0, int ncol, cudaStream_t stream);
void launch_equilibrium(int Q, const double* rho, const double* U1, const double* U2,
                        const double* geo, double* Np, int n1, int n2, int ncol, double rho0,
                        cudaStream_t s);
void launch_wall_init(int prec, void* wall_rho, void* wall_ut2, const double* rho,
                      const double* ut2, int n1, int n2, int h, double rho0, cudaStream_t stream);
// rho0 times the total volume of `count` geometry entries of `mult` cells
// each, written to *out (device).
void launch_rest_mass(int Q, const double* geo, int count, int mult, double rho0, double* out,
                      cudaStream_t stream);
// Eq. 23 on `count` geometry entries (rows, or cells of a general grid).
void launch_scale_volume(int Q, double* geo, const double* rho_nf, int count, double rho0,
                         cudaStream_t stream);
void launch_row_mean(const double* field, int n1, int n2, double* out, cudaStream_t stream);
// Halo strips of slabs along q^2 (k_halo.cu): entries per side (D2Q21 12,
// D2Q9 3) and the pack (unpack = 0) / unpack of one side's strips.
int halo_entries(int Q);
void launch_halo(int Q, int prec, void* state, void* buf, long long plane, int ld, int rows, int n2,
                 int side, int unpack, cudaStream_t stream);

// TMA-staged fused update (k_step_tma.cu): tensor maps of the two state
// buffers, their construction, and the launch (src = physical source buffer).
struct TmaMaps;
int make_tma_maps(int Q, int prec, TmaMaps** out, void* bufA, void* bufB, int n1, int n2, int ld);
void free_tma_maps(TmaMaps* m);
// Copy the 2 x 8 load maps of both buffers to out (host); returns their bytes
// (out may be NULL to ask the size).
size_t tma_load_maps(const TmaMaps* m, void* out);
// Residual sums of the pipelined (TMA-staged) pass over the current buffer
// src of the maps: one partial per CTA; returns the number of partials, or
// -1 when it cannot run (FP64 storage, launch failure).
int launch_residual_tma(int Q, int prec, const TmaMaps& maps, const MomArgs& m, int src, int nsm,
                        cudaStream_t s);
// The pipelined update of a general grid (per-cell tables read by the
// consumers, state staged by TMA); the maps as for launch_step_tma.
int launch_step_tma_general(int Q, int prec, const TmaMaps& maps, const StepArgs& a, int src, int nsm,
                            cudaStream_t s);
int launch_step_tma(int Q, int prec, const TmaMaps& maps, const StepArgs& a, int src, int nsm,
                    int pipelined, cudaStream_t s);
// nsteps time steps of the pipelined update (mode 1: one cell per consumer
// thread, 2: two) in one cooperative launch whose CTAs order the steps among
// themselves: prog holds one progress word per CTA and the run's tile
// counter (nsm + 1 words, zero when allocated), epoch a value no earlier
// launch on prog used.  Returns the launch's CUDA error (cudaSuccess when it
// was launched).
int run_tiles(int Q, int mode, int n1, int n2);
cudaError_t launch_step_tma_run(int Q, int prec, const TmaMaps& maps, const StepArgs& a, int src, int nsm,
                                int mode, int nsteps, unsigned long long* prog, unsigned epoch,
                                cudaStream_t s);

// Set the thread-local message returned by clbm_last_error (clbm_api.cu).
void set_last_error(const char* msg);

// Size in bytes of one stored population.
inline int storage_bytes(int prec) { return prec == 0 ? 8 : (prec == 1 ? 4 : 2); }
inline int compute_bytes(int prec) { return prec == 0 ? 8 : 4; }

}  // namespace clbm
