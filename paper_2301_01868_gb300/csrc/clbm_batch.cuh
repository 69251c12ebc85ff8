// clbm_batch.cuh -- device descriptor of one lattice inside a batch and the
// batched launchers (k_batch.cu).
#pragma once

#include "clbm_internal.cuh"

namespace clbm {

struct BatchGrid {
    void* phys[2];          // the lattice's two state buffers
    const void* tab;        // per-row coefficients (compute type)
    void* wall_rho;
    void* wall_ut2;
    const void* ghost;      // compute type
    const double* geo;
    double* prev;           // Ut snapshot of the residual
    StepScalars k;
    double U0_lo, U0_hi;
    long long plane;
    int n1, n2, ld;
    int parity;             // physical buffer that is the source at batch phase 0
    int bc_lo, bc_hi, have_prev;
    int iters;              // extra passes of the implicit force (0: lagged, Sec. 2)
};

constexpr int BATCH_VARIANTS = 4;

// what: 0 boundary items, 1 update tiles (variant) of lagged-force lattices,
// 2 diagnostics tiles of lagged-force lattices, 3 update tiles (variant 0
// shape) and 4 diagnostics tiles of lattices that iterate the force.  Work
// item e writes partial[e] (diagnostics).
void launch_batch(int Q, int prec, int what, int variant, const BatchGrid* grids, const int4* work,
                  int nwork, int parity, int nblk, double* partial, cudaStream_t s);
void launch_batch_reduce(const double* partial, const int2* range, int ngrids, double* out,
                         cudaStream_t s);
// Update tile (columns x rows) of a variant.
void batch_tile_shape(int variant, int* tj, int* tr);

// Variant BATCH_WS: the pipelined TMA update over 8 x 64 tiles of every
// lattice (k_step_tma.cu).  maps: per lattice the 2 x 8 load maps of its two
// state buffers (device memory, tma_load_maps layout); err: device error word
// of bounded waits.  Returns nonzero if it could not be launched.
constexpr int BATCH_WS = BATCH_VARIANTS;
constexpr int BATCH_ALL = BATCH_VARIANTS + 1;
int launch_batch_ws(int Q, int prec, const BatchGrid* grids, const void* maps, const int4* work, int nwork,
                    int parity, int nsm, int* err, cudaStream_t s);

}  // namespace clbm
