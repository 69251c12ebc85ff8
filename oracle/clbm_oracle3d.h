/*
 * clbm_oracle3d.h -- plain FP64 CPU oracle of the volumetric curvilinear
 * lattice Boltzmann method in three dimensions (Sec. 2 of arXiv:2301.01868 is
 * written for three-dimensional coordinates; its tests are two-dimensional).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load it.  It shares no code, header, table or helper with the CUDA path.
 *
 * Lattice: D3Q39 (the 39-velocity set with isotropy through the sixth order
 * at T0 = 2/3: shells (0,0,0), (1,0,0), (1,1,1), (2,0,0), (2,2,0), (3,0,0)),
 * the three-dimensional counterpart of the paper's D2Q21 requirement of
 * sixth-order isotropy (Sec. 4); the paper gives no 3-D set, so this one is
 * taken from the lattice Boltzmann literature and pinned by its moments.
 *
 * Index conventions: q^1 = i wall-normal, 1 <= i <= n1, walls at i = 1/2 and
 * n1 + 1/2; q^2 = j and q^3 = k periodic.  Arrays are 0-based, row-major:
 * a population array is [alpha][i-1][j-1][k-1], a cell field [i-1][j-1][k-1].
 */
#ifndef CLBM_ORACLE3D_H
#define CLBM_ORACLE3D_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct o3_grid o3_grid;

enum { O3_CHANNEL = 0, O3_ANNULUS = 1 };

/* c is [39][3], w [39], star (reversal) / hat (c^1 flipped) [39]. */
int o3_lattice(int* c, double* w, int* star, int* hat, double* T0);

/*
 * O3_CHANNEL: nodes at (x(i), (j-1/2) step2, (k-1/2) step3), x(i) the midpoint
 *             of wall-normal edges[i-1], edges[i] (App. C), mirrored beyond
 *             the walls (App. B);
 * O3_ANNULUS: nodes at (r(i) cos th, r(i) sin th, (k-1/2) step3) with
 *             th = (j-1/2) 2 pi / n2 and r(i) the midpoint of radial edges.
 * dx is the Delta x of the tangent vectors; dx <= 0 takes the average
 * wall-normal step.  Returns NULL on invalid input.
 */
o3_grid* o3_create(int n1, int n2, int n3, int kind, const double* edges, double step2,
                   double step3, double dx, int bc_lo, int bc_hi);
void o3_destroy(o3_grid* g);

/* BGK time, reference density, contravariant wall velocities U0^2 of the
 * low / high wall (the walls move along q^2), contravariant body force. */
void o3_set_case(o3_grid* g, double tau, double rho0, double U0_lo, double U0_hi,
                 double g1, double g2, double g3);
/* N'(q,-1) = J f^eq(rho0, 0; g^{ij}(q)); last-collision moments (rho0, 0). */
void o3_init_rest(o3_grid* g);
/* State [39][n1][n2][n3]; last-collision moments rho, Ut^2, Ut^3 [n1][n2][n3]
 * (NULL: rho0, 0, 0). */
void o3_set_state(o3_grid* g, const double* Np, const double* rho_prev, const double* ut2_prev,
                  const double* ut3_prev);
void o3_get_state(const o3_grid* g, double* Np);
void o3_step(o3_grid* g, long long nsteps);
long long o3_time(const o3_grid* g);

/* Moments of the collision the next step would make: rho, U^k, Ut^k, F^k
 * (each of the vector fields [3][n1][n2][n3]). */
void o3_moments(const o3_grid* g, double* rho, double* U, double* Ut, double* F);
/* sum N' and sum c N' (4 values) of the current state. */
void o3_totals(const o3_grid* g, double* out);
/* Row geometry of 1-based row i: J, g^{ij} (9), g_ij (9).  -1 if out of range. */
int o3_row_geometry(const o3_grid* g, int i, double* out);
/* Theta^k_m(q + s c_alpha, q) at row i as [k][m] (9). */
void o3_theta(const o3_grid* g, int i, int alpha, int s, double* out);
/* f^eq of Eq. 19 for one direction, ginv [3][3]. */
double o3_feq(const o3_grid* g, int alpha, double rho, const double* U, const double* Ut,
              const double* ginv);
/* One cell's collision from the current state (1-based i, j, k): outgoing
 * and incoming populations and the force. */
void o3_collide_one(const o3_grid* g, int i, int j, int k, double* Npost, double* Nin, double* F,
                    double* rho);

#ifdef __cplusplus
}
#endif
#endif
