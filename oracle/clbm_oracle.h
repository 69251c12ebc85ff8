/*
 * clbm_oracle.h -- plain FP64 CPU oracle of the volumetric curvilinear lattice
 * Boltzmann method (Chekhlov, Staroselsky, Zhang, Chen, arXiv:2301.01868).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library.
 * Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference leg
 * of bench.py may load it.  It shares no code, header, table or helper with
 * the CUDA path, and the CUDA path never calls it.
 *
 * Index conventions (App. B of the paper): q^1 = i is the wall-normal
 * direction, 1 <= i <= n1, walls at i = 1/2 and i = n1 + 1/2; q^2 = j is the
 * periodic direction, 1 <= j <= n2.  Arrays passed through this interface are
 * 0-based and row-major: a population array is [alpha][i-1][j-1].
 */
#ifndef CLBM_ORACLE_H
#define CLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_grid orc_grid;

enum { ORC_PLANAR = 0, ORC_POLAR = 1, ORC_GENERAL = 2 };
enum { ORC_NOSLIP = 0, ORC_MOVING = 1 };

/* Lattice tables as the oracle holds them (App. A, App. B index maps).
 * c is [Q][2] ints, w is [Q], star/hat are [Q] (bounce-back / specular). */
int orc_lattice(int Q, int* c, double* w, int* star, int* hat, double* T0);

/*
 * Build a grid.
 *  kind ORC_PLANAR : edges[0..n1] are the wall-normal cell edges x'_i (App. C);
 *                    nodes sit at edge midpoints; q^2 nodes at (j-1/2)*step2.
 *  kind ORC_POLAR  : edges[0..n1] are radial edges r'_i; theta_j=(j-1/2)*2pi/n2.
 *  kind ORC_GENERAL: nodes holds (n1+8)*(n2+8)*2 doubles: positions of nodes
 *                    i=-3..n1+4, j=-3..n2+4 (1-based), ghosts included.
 *  dx is the Delta x of the tangent-vector definition (Sec. 2); dx<=0 picks the
 *  average wall-normal step (edges[n1]-edges[0])/n1.
 * Returns NULL on invalid input.
 */
orc_grid* orc_create(int Q, int n1, int n2, int kind, const double* edges,
                     double step2, const double* nodes, double dx,
                     int bc_lo, int bc_hi);
void orc_destroy(orc_grid* g);

/* Case: BGK time tau, reference density rho0, contravariant tangential wall
 * velocities U0^2 of the low/high walls, contravariant body acceleration. */
void orc_set_case(orc_grid* g, double tau, double rho0, double U0_lo,
                  double U0_hi, double gext1, double gext2);

/* Initial post-collision state N'(q,-1) = J f^eq(rho0, U=0; g^{ij}(q)); the
 * previous-step moments used by a moving wall are set to (rho0, 0). */
void orc_init_rest(orc_grid* g);

/* State N'(q,t-1), [Q][n1][n2].  set_state also takes the previous-step
 * moments of every cell as rho/Ut2 arrays [n1][n2] (NULL -> rho0 and 0). */
void orc_set_state(orc_grid* g, const double* Np, const double* rho_prev,
                   const double* Ut2_prev);
void orc_get_state(const orc_grid* g, double* Np);
void orc_get_prev_moments(const orc_grid* g, double* rho_prev, double* Ut2_prev);

/* Advance nsteps time steps (Eq. 6 with Eq. 12 advection and App. B BCs). */
void orc_step(orc_grid* g, long long nsteps);
long long orc_time(const orc_grid* g);

/* Moments of the current state: the post-advection populations N(q,t)
 * (pulled from N'(t-1) with the boundary conditions) and the lagged force.
 * Each output is [n1][n2]; any pointer may be NULL. */
void orc_moments(const orc_grid* g, double* rho, double* U1, double* U2,
                 double* Ut1, double* Ut2, double* F1, double* F2);

/* One cell's collision from the current state, without advancing time.
 * i, j are 1-based.  Outputs (any may be NULL): Npost[Q], Nin[Q], feq[Q],
 * dN[Q], F[2], Ut[2], dPi[4] (row-major [i][j]), rho. */
void orc_collide_one(const orc_grid* g, int i, int j, double* Npost,
                     double* Nin, double* feq, double* dN, double* F,
                     double* Ut, double* dPi, double* rho);

/* Geometry at node (i,j), 1-based, including ghosts (i in [-2, n1+3]); for
 * planar and polar grids only columns j in [-2, 4] are held (column 1 serves
 * every column by symmetry).
 * out: g_1(2), g_2(2), g^1(2), g^2(2), J, g^{11}, g^{12}, g^{22}  (12 doubles).
 * Returns 0 on success. */
int orc_node_geometry(const orc_grid* g, int i, int j, double* out);

/* Discrete Christoffel symbol Theta^k_m(q + s*c_alpha, q), s = +1 or -1,
 * at cell (i,j) (1-based): out[k*2+m]. */
void orc_theta(const orc_grid* g, int i, int j, int alpha, int s, double* out);

/* The equilibrium of Eq. (19) for one direction, given rho, U, Ut, g^{ij}. */
double orc_feq(const orc_grid* g, int alpha, double rho, const double* U,
               const double* Ut, const double* ginv /* [2][2] */);

/* Totals of the state N'(t-1): out[0]=sum N', out[1..2]=sum c^k N'. */
void orc_totals(const orc_grid* g, double* out);

/* Flow diagnostics of Sec. 3.1, where a steady state is judged by the total
 * kinetic energy (and, for the circular flows, the angular momentum) no
 * longer changing while the mass stays fixed.  Inputs are cell fields
 * [n1][n2]: the density rho and the contravariant velocity Ut^k (Eq. 18) of
 * every cell, as orc_moments gives them; Ut1_prev / Ut2_prev (both may be
 * NULL) hold the velocity dt steps earlier.  The physical velocity of a cell
 * is u = Ut^1 g_1 + Ut^2 g_2 with the tangent vectors of its node (Sec. 2),
 * J is the cell volume of N = J f (after a no-flow adjustment, the adjusted
 * one), x the node position.
 *   out[0]  residual ||u - u_prev||_J / (dt ||u||_J), ||v||_J^2 = sum J v.v
 *           (+inf without a previous velocity or with dt <= 0; 0 when u and
 *           u_prev both vanish);
 *   out[1]  kinetic energy 1/2 sum J rho |u|^2;
 *   out[2]  angular momentum about the origin, sum J rho (x cross u).z, on
 *           polar and general grids (planar grids have no natural origin:
 *           0 there);
 *   out[3]  max |u|;
 *   out[4]  sum J |u|^2. */
void orc_flow_diagnostics(const orc_grid* g, const double* rho, const double* Ut1,
                          const double* Ut2, const double* Ut1_prev,
                          const double* Ut2_prev, long long dt, double* out);

/* Volume J used by N = J f; set_volume overwrites it ([n1][n2]). */
void orc_get_volume(const orc_grid* g, double* J);
void orc_set_volume(orc_grid* g, const double* J);

/* "No flow" adjustment (Sec. 3.1, Eq. 23): run the same grid with U0 = 0 and
 * no body force for nsteps from rest, then J <- J rho_nf / rho0 per cell.
 * The state is left at that no-flow solution, which is a fixed point of the
 * adjusted problem; the case (walls, force) is restored afterwards.
 * rho_nf (may be NULL) receives the no-flow density [n1][n2]. */
void orc_no_flow_adjust(orc_grid* g, long long nsteps, double* rho_nf);

/* Extra fixed-point passes of the implicit force relation (Sec. 2): 0 (the
 * default) is the paper's lag, F from N'(q,t-1); n > 0 re-evaluates Eq. 15
 * n times with the newest N'(q,t). */
void orc_set_force_iterations(orc_grid* g, int iters);

/* Number of OpenMP threads the step uses (1 without OpenMP). */
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
