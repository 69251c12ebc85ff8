/*
 * clbm.h -- C ABI of the GB300 library for the volumetric lattice Boltzmann
 * method in general curvilinear coordinates (Chekhlov, Staroselsky, Zhang,
 * Chen, arXiv:2301.01868).
 *
 * The library advances the populations N_alpha(q, t) of a 2-D coordinate-space
 * lattice by the paper's update, Eq. 6 of Sec. 2:
 *     N_alpha(q + c_alpha, t + 1) = N_alpha(q, t) + Omega_alpha + dN_alpha,
 * with exact one-to-one advection (Eq. 12), BGK collision (Eq. 11) towards the
 * curvilinear third-order equilibrium (Eq. 19), the lagged inertial force of
 * Eq. 15 with the momentum-flux correction of Eq. 16 and the source of Eq. 17,
 * and the periodic, no-slip and moving-wall boundaries of App. B.  Lattices
 * are D2Q9 (T0 = 1/3) and D2Q21 (T0 = 2/3) of App. A.
 *
 * Index conventions.  q^1 = i is the wall-normal direction (1 <= i <= n1,
 * walls at i = 1/2 and n1 + 1/2, App. B); q^2 = j is periodic (1 <= j <= n2).
 * Every array crossing this interface is row-major and 0-based:
 * populations are double [Q][n1][n2], cell fields double [n1][n2].
 *
 * Ownership.  The library owns the device state of a grid unless the caller
 * passes a workspace; the caller owns every host pointer, which is read or
 * written only during the call.  Device pointers passed in (workspace,
 * outputs with dst_is_device) stay owned by the caller.
 *
 * Errors.  Every entry point returns a clbm_status; clbm_last_error() gives a
 * thread-local message.  Asynchronous CUDA errors and device-side flags
 * surface at the next synchronising call (moments, residual, get_state).
 * Handles are not thread-safe; distinct handles are independent.
 */
#ifndef CLBM_H
#define CLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct clbm_grid* clbm_handle;

typedef enum {
    CLBM_OK = 0,
    CLBM_EINVAL = 1,     /* invalid argument or unsupported combination */
    CLBM_ENOMEM = 2,     /* device or host allocation failed / workspace too small */
    CLBM_ECUDA = 3,      /* a CUDA call failed */
    CLBM_EUNSTABLE = 4,  /* a non-finite or non-positive density was found */
    CLBM_ETIMEOUT = 5,   /* a bounded device wait gave up */
    CLBM_EBUSY = 6       /* the handle is in use (e.g. captured in a graph) */
} clbm_status;

typedef enum { CLBM_D2Q9 = 9, CLBM_D2Q21 = 21 } clbm_lattice;

/* Arithmetic of the bulk update and storage of the populations. */
typedef enum {
    CLBM_FP64 = 0,            /* FP64 compute, FP64 storage */
    CLBM_FP32 = 1,            /* FP32 compute, FP32 storage */
    CLBM_FP32_F16STORE = 2,   /* FP32 compute, FP16 storage (scaled) */
    CLBM_FP32_BF16STORE = 3   /* FP32 compute, BF16 storage */
} clbm_precision;

/* Geometry of the coordinate map x(q) (Sec. 2, App. C, App. D). */
typedef enum {
    CLBM_GEOM_PLANAR = 0,  /* x = (x^1_i, (j - 1/2) step2), x^1_i edge midpoints */
    CLBM_GEOM_POLAR = 1,   /* x = r_i (cos th_j, sin th_j), th_j = (j - 1/2) 2 pi / n2
                              (n2_period in place of n2 when set) */
    CLBM_GEOM_GENERAL = 2  /* node positions given (nodes); Sec. 2 in full generality:
                              metric, volume and Theta of every cell, per-cell tables */
} clbm_geom_kind;

/* Wall conditions of App. B (direction q^2 is always periodic). */
typedef enum {
    CLBM_BC_NOSLIP = 0,  /* bounce-back of N through the mirrored node */
    CLBM_BC_MOVING = 1   /* specular reflection plus the moving-wall correction */
} clbm_wall_bc;

typedef struct {
    int lattice;            /* clbm_lattice */
    int precision;          /* clbm_precision */
    int n1, n2;             /* interior size: wall-normal x periodic; n1 >= 4, n2 >= 1 */
    int kind;               /* clbm_geom_kind */
    const double* edges1;   /* host, n1+1 increasing wall-normal edges x'_0..x'_n1
                               (radii for POLAR, all > 0); nodes sit at midpoints,
                               walls at edges1[0] and edges1[n1]; unused by GENERAL */
    double step2;           /* PLANAR: physical step along q^2 (> 0) */
    double dx;              /* Delta x of the tangent vectors (Sec. 2); <= 0 picks
                               the average wall-normal step (edges1[n1]-edges1[0])/n1;
                               GENERAL needs dx > 0 */
    int bc_lo, bc_hi;       /* clbm_wall_bc of the walls at edges1[0] / edges1[n1] */
    int device;             /* CUDA device ordinal */
    void* stream;           /* cudaStream_t for all work of this grid (NULL: legacy default) */
    void* workspace;        /* optional caller-owned device memory (NULL: library allocates) */
    size_t workspace_bytes; /* size of workspace */
    const double* nodes;    /* GENERAL only, host: positions (x, y) of the nodes
                               i = -3..n1+4 (wall-normal) by j = -3..n2+4 (periodic),
                               row-major [(n1+8)][(n2+8)][2], node (i, j) at
                               q = (i - 1/2, j - 1/2); the rows beyond the walls
                               are the ghost nodes of App. B (e.g. mirror images
                               through straight walls), the columns beyond the ends
                               the periodic images.  Read during create only. */
    int n2_period;          /* POLAR: columns of the whole ring, th_j = (j - 1/2) 2 pi /
                               n2_period (a slab of a ring split along q^2); <= 0
                               means n2.  Ignored by the other kinds. */
} clbm_grid_desc;

typedef struct {
    double tau;             /* BGK relaxation time, > 1/2 (Eq. 11) */
    double rho0;            /* reference density of the rest state (> 0) */
    double u_wall_lo;       /* contravariant tangential velocity U0^2 of the low wall */
    double u_wall_hi;       /* ... of the high wall (used by CLBM_BC_MOVING walls) */
    double g_ext[2];        /* contravariant body acceleration g^k, added to F^k as rho g^k */
    int force_iterations;   /* 0: the paper's lag, F from N'(q,t-1) (Sec. 2);
                               n > 0: n extra passes of the implicit force relation */
} clbm_case;

/* Bytes of device workspace a grid with this description needs. */
clbm_status clbm_workspace_bytes(const clbm_grid_desc* desc, size_t* bytes);

/* Validate desc, allocate (or carve) device state, run the geometry / metric /
 * Christoffel precompute (Sec. 2, Eqs. 1-5) on the device in FP64, and return
 * a handle.  The state is undefined until clbm_set_case. */
clbm_status clbm_create_grid(const clbm_grid_desc* desc, clbm_handle* out);

/* Set the case and start from rest: N'(q,-1) = J f^eq(rho0, U = 0; g^{ij}(q)),
 * previous-step wall moments (rho0, 0), t = 0.  Asynchronous. */
clbm_status clbm_set_case(clbm_handle h, const clbm_case* cs);

/* Replace the state N'(q, t-1) ([Q][n1][n2] FP64, host or device) and,
 * optionally, the previous-step moments used by moving walls (rho, Ut^2 as
 * [n1][n2]; NULL: rho0 and 0).  Synchronises. */
clbm_status clbm_set_state(clbm_handle h, const double* Np, const double* rho_prev,
                           const double* Ut2_prev, int src_is_device);

/* Start from the local equilibrium of given macroscopic fields:
 * N'(q,-1) = J f^eq(rho, U, Ut = U; g^{ij}(q)) with f^eq the third-order
 * Hermite equilibrium of Eq. 19 (with no force known at the start Ut = U),
 * formed on the device in FP64 and stored in the grid's precision; the
 * moving-wall moments of the last collision are (rho, U^2) on the wall rows;
 * t = 0.  rho, U1, U2: [n1][n2] FP64 (contravariant U^1, U^2, lattice units),
 * host or device per src_is_device, caller-owned, read during the call; NULL
 * gives rho0 / 0.  Starting a steady solve from the equilibrium of the exact
 * or a coarser solution shortens the transient (the steady state does not
 * depend on the start).  Requires clbm_set_case.  Synchronises. */
clbm_status clbm_set_equilibrium(clbm_handle h, const double* rho, const double* U1,
                                 const double* U2, int src_is_device);

/* Read the state N'(q, t-1) as [Q][n1][n2] FP64 into host or device memory.
 * Synchronises. */
clbm_status clbm_get_state(clbm_handle h, double* Np, int dst_is_device);

/* Advance n time steps: one launch of the fused stream-collide-force update
 * per step, which also writes the ghost rows (App. B) and periodic ghost
 * columns of the buffer it fills; the ghosts are rebuilt once first when the
 * state or case was set since.  Asynchronous on the grid's stream.  Runs of
 * more than 21 steps replay a CUDA graph of 10 launches (captured on first
 * use and again whenever the case, kernel or buffers it was captured with
 * change; the same launches, so the results are identical bit for bit);
 * if a capture fails the grid keeps to plain launches. */
clbm_status clbm_step(clbm_handle h, long long n);

/* Moments of the current state, i.e. of the post-advection populations
 * N(q, t) with the lagged force (what the next collision uses): rho, U^k
 * (Eq. 10), Ut^k (Eq. 18), F^k (Eq. 15).  Each output is [n1][n2] FP64; any
 * may be NULL.  Synchronises. */
clbm_status clbm_moments(clbm_handle h, double* rho, double* U1, double* U2,
                         double* Ut1, double* Ut2, double* F1, double* F2,
                         int dst_is_device);

/* Asynchronous host copies, for a caller that streams starts in and results
 * out while the grid computes (the copies run on a copy stream the grid
 * creates on first use, with two FP64 upload slots of Q n1 n2 values and two
 * moment slots of 3 n1 n2 values that it allocates then and keeps).  Host
 * buffers should be page-locked: from pageable memory a copy does not
 * overlap.  Every host buffer must stay valid, and an upload's unchanged,
 * until clbm_wait_copies returns (or, for an upload, until the grid's stream
 * has run the clbm_set_uploaded_state that consumes it).
 *   clbm_upload_state_async: start copying N'(q, t-1) (host, FP64
 *     [Q][n1][n2]) into the next upload slot; returns at once.  CLBM_EBUSY
 *     when two uploads wait to be set already.
 *   clbm_set_uploaded_state: make the oldest waiting upload the grid's state,
 *     as clbm_set_state does, ordered on the grid's stream after its copy
 *     (no host wait); CLBM_EINVAL if none waits.
 *   clbm_download_moments_async: the moments rho, Ut^1, Ut^2 (as
 *     clbm_moments gives them) of the current state, computed on the grid's
 *     stream into the next moment slot and copied into the host buffers
 *     ([n1][n2] FP64 each, any may be NULL) on the copy stream; returns at
 *     once.
 *   clbm_wait_copies: block until every copy issued so far has landed;
 *     reports errors of the grid's earlier work as a synchronising call.
 * The paper has no counterpart: these keep host transfers off the update's
 * critical path when every step's input comes from, and its result goes
 * to, host memory. */
clbm_status clbm_upload_state_async(clbm_handle h, const double* Np);
clbm_status clbm_set_uploaded_state(clbm_handle h);
clbm_status clbm_download_moments_async(clbm_handle h, double* rho, double* Ut1, double* Ut2);
clbm_status clbm_wait_copies(clbm_handle h);

/* Convergence and conservation diagnostics (Sec. 3.1: mass, kinetic energy,
 * angular momentum).  res = ||u(t) - u(t')||_J / ((t - t') ||u(t)||_J) with
 * physical u = Ut^k g_k and t' the time of the previous call (+inf on the
 * first call).  cons = {sum N', sum c^1 N', sum c^2 N', kinetic energy
 * 1/2 sum J rho |u|^2, angular momentum sum J rho (x cross u) about the
 * origin (POLAR and GENERAL, else 0), max |u|}.  Per-cell terms are formed in
 * the compute type and summed in FP64 (FP32 compute: a thread's cells with
 * Kahan compensation in FP32 first).  Returns CLBM_EUNSTABLE if a density is
 * not finite and positive, CLBM_ETIMEOUT if a bounded device wait of an
 * earlier update gave up.  Synchronises. */
clbm_status clbm_residual(clbm_handle h, double* res, double cons[6]);

/* The sums behind clbm_residual, for callers that combine several grids (the
 * slabs of one lattice split along q^2 over several GPUs): parts = {sum J
 * |u(t) - u(t')|^2, sum J |u|^2, sum N', sum c^1 N', sum c^2 N', kinetic
 * energy, angular momentum, max |u|, cells with a non-finite or non-positive
 * density}, *dt = t - t' (0 on the first call).  Over several grids the
 * parts add (max |u| takes the maximum) and the residual is
 * sqrt(sum parts[0]) / (dt sqrt(sum parts[1])).  Moves the snapshot like
 * clbm_residual; same errors.  Synchronises. */
clbm_status clbm_residual_parts(clbm_handle h, double parts[9], long long* dt);

/* Slabs along q^2 (one lattice split over several GPUs, each holding a run of
 * columns as a grid of its own; POLAR slabs give the ring's size in
 * n2_period).  The update (Eq. 12) pulls population a from the cell c_a
 * behind, so a slab's first |c2| columns read the lower neighbour's last
 * columns for every population with c2 > 0, and its last columns the upper
 * neighbour's first columns for c2 < 0: one strip per (population, depth),
 * 12 per side for D2Q21 (7 at depth 1, 4 at depth 2, 1 at depth 3), 3 for
 * D2Q9, each covering the n1 + 2h stored rows (App. B's ghost rows
 * included: they are filled per column).  Protocol: after clbm_set_case /
 * clbm_set_state (and the like) call clbm_fill_ghosts, then exchange; after
 * every clbm_step(1) exchange; an exchange packs both sides, sends side 0 to
 * the lower and side 1 to the upper neighbour, and unpacks what the lower
 * neighbour sent as side 0 and what the upper one sent as side 1.  Every
 * call that reads the state (step, moments, residual) then sees the
 * neighbours' columns; without exchanges the grid is periodic on its own.
 *   clbm_fill_ghosts: rebuild the current state's ghost rows and columns now
 *     if it was set from outside (what clbm_step would do first).  Async.
 *   clbm_halo_values: values of one side's strips, in the storage type
 *     (8 / 4 / 2 bytes per value for FP64 / FP32 / FP16 and BF16).
 *   clbm_halo_pack / clbm_halo_unpack: side 0 or 1, buf device memory of
 *     clbm_halo_values values, caller-owned; values move as stored, bit for
 *     bit.  Async on the grid's stream.  CLBM_EINVAL for general grids and
 *     slabs narrower than the stencil (n2 < 3 for D2Q21). */
clbm_status clbm_fill_ghosts(clbm_handle h);
clbm_status clbm_halo_values(clbm_handle h, size_t* values);
clbm_status clbm_halo_pack(clbm_handle h, int side, void* buf);
clbm_status clbm_halo_unpack(clbm_handle h, int side, const void* buf);

/* "No flow" adjustment (Sec. 3.1, Eq. 23): in FP64, run the grid from rest
 * with U0 = 0 and no body force for nsteps, then J <- J rho_nf / rho0 (per
 * row on planar and polar grids, where the no-flow state does not depend on
 * j; per cell on general grids), and leave the state at that no-flow
 * solution (a fixed point of the adjusted update).  rho_nf (host, may be
 * NULL) receives the no-flow density [n1][n2].  Requires a prior
 * clbm_set_case.  Synchronises. */
clbm_status clbm_no_flow_adjust(clbm_handle h, long long nsteps, double* rho_nf);

/* Time step counter t. */
clbm_status clbm_time(clbm_handle h, long long* t);

/* Change the stream the grid's work is issued on. */
clbm_status clbm_set_stream(clbm_handle h, void* stream);

/* period > 0: clbm_step records a CUDA event pair around every period-th
 * launch of the fused update (1: every launch; a larger period keeps the
 * events' own cost out of the timed stream); a graph replay is recorded as a
 * whole, one pair around its 10 back-to-back launches, and so is a
 * multi-step launch (kernels 5 and 6), counted as its number of time steps,
 * whatever the period; period 0 switches it off.
 * clbm_kernel_time returns the recorded launches' summed duration (ms) and
 * their count since the last reset, and resets.  Synchronises. */
clbm_status clbm_set_profiling(clbm_handle h, int period);
clbm_status clbm_kernel_time(clbm_handle h, double* ms, long long* launches);

/* Kernel of the bulk update: 0 automatic (general grids: 1; planar and polar
 * grids with TMA maps: 4 for FP16 / BF16 storage, run as 6 when the grid
 * has at least 8 tiles per SM and the GPU can hold every CTA of the
 * cooperative launch, 3 for FP32; else 1), 1 one thread per cell
 * with direct loads, 2 TMA-staged tiles with a shared output tile (planar
 * and polar grids), 3 TMA-staged tiles in a warp-specialised pipeline
 * (general grids: the state staged, the per-cell tables read by the
 * consumers), 4 the same pipeline with two neighbouring cells per thread in
 * packed FP32 arithmetic (planar and polar grids), 5 / 6 kernels 3 / 4 with up
 * to 1000 time steps per launch (planar and polar grids): the CTAs of one
 * cooperative launch order the steps among themselves -- a tile of step
 * s waits until step s - 1 has finished the row bands its pull reaches
 * (Eq. 12: |c^1| <= 3 rows) -- so the ramp-up, tail and gap of a launch come
 * once per run; a wait that gives up is reported as the pipeline's bounded
 * waits are, CLBM_ETIMEOUT from clbm_moments (2-6: FP32 / FP16 / BF16 storage and rows of at least
 * 16 bytes; the implicit-force passes always use variant 1).  All run the
 * same update; 5 and 6 give the bits of 3 and 4; the packed form rounds each
 * lane as the scalar form but may contract a different multiply-add
 * pairing, so FP32 results agree to rounding, not bit for bit.  CLBM_EINVAL
 * for a variant the grid cannot use. */
clbm_status clbm_set_kernel(clbm_handle h, int variant);

/* Number of kernel launches this grid has issued since creation. */
clbm_status clbm_launch_count(clbm_handle h, long long* launches);

/* Totals of a population array without allocating device memory: out[0] =
 * sum N', out[1] = sum c^1 N', out[2] = sum c^2 N' over Np, a device array of
 * FP64 populations [Q][n1][n2] (the layout clbm_get_state writes).  out is 3
 * doubles in device memory (out_is_device = 1, asynchronous) or host memory
 * (synchronises).  Work goes on `stream` of the current device.
 * The paper has no counterpart: this is for callers that must not allocate,
 * such as code running while a stream is captured into a CUDA graph
 * (cudaMalloc cannot be captured) or a process confined to a fixed memory
 * budget.  It calls no cudaMalloc or cudaFree; its scratch is a static device
 * array of 8192 * 3 + 3 doubles (196 632 bytes) that every GPU which loads
 * the library keeps until exit, so n1 * n2 may not exceed 2 097 152 (larger
 * grids get CLBM_EINVAL).  The first call on each device looks up that
 * array's device address, and so does the first call after the device's
 * context changed (a cudaDeviceReset loads the module again); make such a
 * call before any stream capture.  A CUDA error already pending when the
 * call starts is reported (CLBM_ECUDA) and left in place.
 * All calls share the scratch: calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller. */
clbm_status clbm_totals_noalloc(int lattice, const double* Np, int n1, int n2, double* out,
                                int out_is_device, void* stream);

/* ---- Batches: many lattices advanced together (one persistent launch per
 * phase over a work-list of tiles, two steps per CUDA graph).  The grids
 * share lattice, precision, device and stream and are not owned by the
 * batch; step them only through the batch while it exists (a grid stepped on
 * its own is picked up again on the next batch step).  Grids whose case sets
 * force_iterations > 0 (the implicit force of Sec. 2) are updated by a second
 * persistent launch per step with a fixed 128 x 1 tile; the variant and the
 * autotuner apply to the lagged-force grids.  Each grid gives the same
 * result as its own clbm_step.  Work goes on the first grid's stream
 * (graphs need a non-default stream). */
typedef struct clbm_batch* clbm_batch_handle;
clbm_status clbm_batch_create(const clbm_handle* grids, int n, clbm_batch_handle* out);
/* Advance every grid of the batch n time steps.  Asynchronous. */
clbm_status clbm_batch_step(clbm_batch_handle b, long long n);
/* clbm_residual for every grid in one pass: res[n], cons[n][6].  Synchronises.
 * Every entry is filled; res[k] is NaN for a grid with a non-finite or
 * non-positive density, and the call then returns CLBM_EUNSTABLE. */
clbm_status clbm_batch_residual(clbm_batch_handle b, double* res, double* cons);
/* Update tile of the batched kernel: 0 = 128 x 1 cells, 1 = 256 x 1 cells
 * (2 per thread), 2 = 32 x 4 cells, 3 = 64 x 1 cells, one thread per cell;
 * 4 = 64 x 8 tiles staged by TMA in a warp-specialised pipeline (needs
 * FP32 / FP16 / BF16 storage and TMA maps on every grid, else CLBM_EINVAL). */
clbm_status clbm_batch_set_variant(clbm_batch_handle b, int variant);
/* Autotuner: times every usable variant for `steps` steps on this batch
 * (advancing every grid by steps + 1 steps per variant), keeps the fastest and
 * caches the choice for batches of the same lattice, precision and shape
 * class in this process.  best (may be NULL) receives the variant,
 * ms_per_step[5] (may be NULL) the timings (-1 for a variant the batch
 * cannot use).  Synchronises. */
clbm_status clbm_batch_tune(clbm_batch_handle b, int steps, int* best, double* ms_per_step);
/* Each batched time step runs as one launch per wave: consecutive lattices
 * whose workspaces add up to at most `bytes` (4 GiB by default; a lattice
 * larger than that forms a wave alone).  The update slows as the state one
 * launch sweeps grows into tens of GB (512 lattices, 39.5 GB: 72 % of the
 * copy rate in one launch, 77 % in waves of 4 GiB).  Host only. */
clbm_status clbm_batch_set_wave_bytes(clbm_batch_handle b, size_t bytes);

/* The batch's update variant (0-4, as clbm_batch_set_variant) and whether it
 * came from the tuner's cache when the batch was created (1) or is the
 * default / a later choice (0): a caller that rebuilds batches as lattices
 * come and go re-tunes only classes it has not timed.  variant and cached
 * may be NULL.  Host only. */
clbm_status clbm_batch_get_variant(clbm_batch_handle b, int* variant, int* cached);
clbm_status clbm_batch_launch_count(clbm_batch_handle b, long long* launches);
clbm_status clbm_batch_destroy(clbm_batch_handle b);

/* Free everything the grid owns.  NULL is accepted. */
/* Checkpoint / resume.  clbm_checkpoint copies the grid's case and dynamic
 * state -- the current population buffer as stored (deviations in the
 * storage type, ghost rows and columns included), the wall moments of the
 * last collision, the residual snapshot, the geometry (which holds a no-flow
 * adjustment of J) and the time counters -- into buf (host memory of
 * clbm_checkpoint_bytes bytes, caller-owned; a set case is required).
 * clbm_restore loads it into a grid created with the same description (no
 * clbm_set_case needed; the saved case replaces the grid's); stepping then
 * continues bit for bit as the saved grid would have, with the same kernel
 * choice.  CLBM_EINVAL if lattice, precision or size differ.  The buffer is
 * machine-native (no byte-order conversion).  The paper has no counterpart:
 * runs to steady state are long, and a step cap or a failure need not lose
 * them.  Both synchronise. */
clbm_status clbm_checkpoint_bytes(clbm_handle h, size_t* bytes);
clbm_status clbm_checkpoint(clbm_handle h, void* buf);
clbm_status clbm_restore(clbm_handle h, const void* buf);

clbm_status clbm_destroy(clbm_handle h);

/* Self-test of failure detection.  One CTA waits, with at most `polls` polls
 * (1..2^22), on an mbarrier that nothing completes, through the same bounded
 * wait that every spin of the pipelined kernels uses (the update's waits
 * take 2^18 polls, about one second).  The wait must give up and the kernel
 * return: CLBM_ETIMEOUT is the expected result, *ms the kernel's duration,
 * and the context stays usable; CLBM_OK would mean the barrier completed.
 * The paper has no counterpart. */
clbm_status clbm_selftest_bounded_wait(int device, int polls, double* ms);

/* Thread-local message of the last failing call ("" if none). */
const char* clbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CLBM_H */
