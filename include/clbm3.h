/*
 * clbm3.h -- C ABI of the three-dimensional form of the volumetric
 * curvilinear lattice Boltzmann update (arXiv:2301.01868, Sec. 2, whose
 * equations are written for three coordinates; its tests are 2-D).
 *
 * Lattice D3Q39: shells (0,0,0), (1,0,0), (1,1,1), (2,0,0), (2,2,0), (3,0,0),
 * weights 1/12, 1/12, 1/27, 2/135, 1/432, 1/1620, T0 = 2/3 -- isotropic
 * through the sixth order, the order the paper requires of the lattice
 * (Sec. 4: D2Q21 in 2-D); the paper prints no 3-D set.  Population order:
 * shell by shell, each shell in lexicographic order of (c1, c2, c3).
 *
 * Grids: q^1 = i is wall-normal (walls at i = 1/2 and n1 + 1/2, App. B),
 * q^2 = j and q^3 = k are periodic.  CLBM3_CHANNEL: nodes at (x_i, (j-1/2)
 * step2, (k-1/2) step3) with x_i the midpoints of the wall-normal edges
 * (App. C); CLBM3_ANNULUS: nodes at (r_i cos th_j, r_i sin th_j, (k-1/2)
 * step3), th_j = (j-1/2) 2 pi / n2, r_i the midpoints of the radial edges.
 * Both are invariant along q^2 and q^3, so the geometry (metric, volume,
 * Christoffel contractions, Eqs. 1-5) is evaluated per row on the device in
 * FP64.  The walls move along q^2 (moving-wall correction of App. B with the
 * tangential components 2 and 3).
 *
 * Every entry point returns a clbm_status (clbm.h); clbm_last_error() gives
 * the message.  Populations cross the ABI as FP64 [39][n1][n2][n3] N'(q,t-1),
 * cell fields as [n1][n2][n3], vector fields as [3][n1][n2][n3]; host or
 * device per the *_is_device flag, caller-owned, used during the call only.
 * Handles are not thread-safe.
 */
#ifndef CLBM3_H
#define CLBM3_H

#include <stddef.h>

#include "clbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct clbm3_grid* clbm3_handle;

typedef enum { CLBM3_CHANNEL = 0, CLBM3_ANNULUS = 1 } clbm3_kind;

typedef struct {
    int precision;          /* clbm_precision: FP64, FP32, or FP32 compute with FP16 /
                               BF16 storage of the deviations (as in clbm.h) */
    int n1, n2, n3;         /* n1 >= 4; n2, n3 >= 1 */
    int kind;               /* clbm3_kind */
    const double* edges;    /* n1 + 1 increasing wall-normal / radial edges (host) */
    double step2;           /* CLBM3_CHANNEL: node spacing along q^2 */
    double step3;           /* node spacing along q^3 */
    double dx;              /* Delta x of the tangent vectors; <= 0: average wall-normal step */
    int bc_lo, bc_hi;       /* clbm_wall_bc of the walls at i = 1/2 and n1 + 1/2 */
    int device;             /* CUDA device ordinal */
    void* stream;           /* cudaStream_t the grid works on (NULL: default stream) */
} clbm3_grid_desc;

typedef struct {
    double tau;             /* BGK relaxation time > 1/2 (Eq. 11) */
    double rho0;            /* reference density */
    double u_wall_lo;       /* contravariant wall velocity U0^2 of the low wall */
    double u_wall_hi;       /* ... of the high wall (CLBM_BC_MOVING walls) */
    double g_ext[3];        /* contravariant body acceleration, F^k += rho g^k */
} clbm3_case;

/* Allocate device state and run the FP64 geometry precompute (Eqs. 1-5).
 * CLBM_EINVAL on a bad description, CLBM_ENOMEM / CLBM_ECUDA on device
 * failures.  The state is undefined until clbm3_set_case. */
clbm_status clbm3_create_grid(const clbm3_grid_desc* desc, clbm3_handle* out);

/* Set the case and start from rest: N'(q,-1) = J f^eq(rho0, 0; g^{ij}(q)),
 * last-collision wall moments (rho0, 0, 0), t = 0. */
clbm_status clbm3_set_case(clbm3_handle h, const clbm3_case* cs);

/* Replace N'(q,t-1) and, optionally, the last-collision moments rho, Ut^2,
 * Ut^3 the moving walls read (NULL: rho0, 0, 0).  Synchronises. */
clbm_status clbm3_set_state(clbm3_handle h, const double* Np, const double* rho_prev,
                            const double* ut2_prev, const double* ut3_prev, int src_is_device);
clbm_status clbm3_get_state(clbm3_handle h, double* Np, int dst_is_device);

/* Start from the local equilibrium of given fields: N'(q,-1) = J f^eq(rho,
 * U, Ut = U; g^{ij}(q)) (Eq. 19, formed in FP64 on the device), the walls'
 * last-collision moments (rho, U^2, U^3), t = 0.  rho [n1][n2][n3] and U
 * [3][n1][n2][n3] (contravariant) FP64, host or device; NULL: rho0 / 0.
 * Requires clbm3_set_case.  Synchronises. */
clbm_status clbm3_set_equilibrium(clbm3_handle h, const double* rho, const double* U, int src_is_device);

/* Checkpoint / resume: clbm3_checkpoint copies the case, the time, the raw
 * current state buffer (storage type, ghost rows included) and the wall
 * moments into buf (host memory of clbm3_checkpoint_bytes bytes,
 * caller-owned); clbm3_restore loads it into a grid with the same
 * description (no case needed first) and stepping then continues bit for
 * bit.  CLBM_EINVAL if precision, sizes or kind differ.  The paper has no
 * counterpart.  Both synchronise. */
clbm_status clbm3_checkpoint_bytes(clbm3_handle h, size_t* bytes);
clbm_status clbm3_checkpoint(clbm3_handle h, void* buf);
clbm_status clbm3_restore(clbm3_handle h, const void* buf);

/* Advance n >= 0 time steps (Sec. 2: advection Eq. 12, moments Eqs. 7-10,
 * lagged force Eq. 15, Ut Eq. 18, f^eq Eq. 19, dPi Eq. 16, dN Eq. 17, BGK
 * Eqs. 6, 11; App. B walls): one launch per step, which also fills the
 * ghost rows the next step reads (a second launch fills the current ones
 * after a new state or case), asynchronous on the grid's stream.  Runs of more than 21 steps replay a
 * CUDA graph of 10 steps (rebuilt when the case changes; bitwise the plain
 * launches; plain launches on a stream that cannot be captured). */
clbm_status clbm3_step(clbm3_handle h, long long n);

/* rho and Ut^k of the collision the next step makes (Ut: [3][n1][n2][n3]);
 * either pointer may be NULL.  Synchronises. */
clbm_status clbm3_moments(clbm3_handle h, double* rho, double* Ut, int dst_is_device);

/* out[0] = sum N' (mass), out[1..3] = sum c N' (momentum) of the current
 * state, reduced on the device in a fixed order.  Synchronises. */
clbm_status clbm3_totals(clbm3_handle h, double out[4]);

/* Update kernel: 0 the automatic choice, 1 the pulled populations held in
 * registers until the collision (six blocks per SM for FP32 compute; the
 * only form of FP64 grids), 2 held in shared memory (seven blocks per SM; the
 * automatic choice of FP32, FP16 and BF16 storage).  The same arithmetic in
 * the same order (Eqs. 6-19, App. B): both give the same bits.  FP64 grids
 * accept 0 and 1; CLBM_EINVAL otherwise.  Synchronises the grid's stream and
 * drops its captured graph. */
clbm_status clbm3_set_kernel(clbm3_handle h, int kernel);

clbm_status clbm3_time(clbm3_handle h, long long* t);
clbm_status clbm3_destroy(clbm3_handle h);

#ifdef __cplusplus
}
#endif
#endif
