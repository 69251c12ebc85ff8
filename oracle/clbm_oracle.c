/*
 * clbm_oracle.c -- plain FP64 CPU oracle of the volumetric curvilinear lattice
 * Boltzmann method of Chekhlov, Staroselsky, Zhang and Chen (arXiv:2301.01868),
 * which implements the formulation it cites as [HChen].
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file;
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline/reference
 * leg load it.  It shares no code with the CUDA library.
 *
 * Everything is written the plain way: one loop over cells per time step, the
 * geometry recomputed from node positions, every tensor sum written out over
 * its indices.  No precontraction, no deviation storage, no per-row tables.
 * Compile with -ffp-contract=off so that the C source is the arithmetic.
 *
 * Readings taken where the paper is silent, garbled or ambiguous (the same
 * readings the CUDA library implements):
 *   R1  D2Q21 weights of the |c|=(2,2) and (3,0) shells are 1/432 and 1/1620
 *       (the printed 7/432 and 7/1620 break sum w = 1; App. A isotropy holds
 *       exactly with the corrected values).
 *   R2  velocity order taken from the App. B index maps (first component is
 *       wall-normal).
 *   R4  Delta x of the tangent vectors is the average wall-normal step (App. D).
 *   R5  an external body force enters as F^k += rho g^k, g^k contravariant.
 *   R6  the lagged state at t=0 is N'(q,-1) = J f^eq(rho0, 0; g^{ij}(q)).
 *   R7  moving-wall correction is (2/T0) w J rho c^2 (U0^2 - Ut^2) at the
 *       mirrored source node, the j=1 term dropped as App. B states.
 *   R8  the source node "x - c_alpha extended through the boundary by
 *       symmetry" is the mirror image of the ghost node through the wall.
 *   R9  the "no flow" run uses the same grid and boundaries with U0 = 0 and no
 *       body force; J is then rescaled per cell, g_i, g^i and Theta unchanged.
 */
#include "clbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define QMAX 21
#define PG 4 /* ghost layers of node positions */
#define GG 3 /* ghost layers of geometry (widest stencil, D2Q21) */

typedef struct { double x, y; } vec2;

struct orc_grid {
    int Q, n1, n2, kind, bc_lo, bc_hi;
    int ncol;             /* columns held by the geometry arrays: n2, or 1 */
    double T0, w[QMAX];
    int c[QMAX][2], star[QMAX], hat[QMAX];
    double dx;
    vec2* pos;            /* (n1+2PG) x (ncol+2PG), i=1-PG..n1+PG, j likewise */
    vec2 *g1, *g2;        /* tangent basis, (n1+2GG) x (ncol+2GG) */
    vec2 *G1, *G2;        /* co-tangent basis */
    double* Jgeo;         /* geometric J = (g_1 x g_2).z */
    double* Jvol;         /* volume used in N = J f (no-flow adjustable), n1 x n2 */
    double tau, rho0, U0_lo, U0_hi, gext[2];
    int iters;            /* extra fixed-point passes of the implicit force */
    double *Np, *Nn;      /* N'(t-1) and the next N', Q x n1 x n2 */
    double *rho_p, *Ut1_p, *Ut2_p; /* moments of the last collision, n1 x n2 */
    double *rho_n, *Ut1_n, *Ut2_n;
    long long t;
};

/* ---------------------------------------------------------------- lattices */

/* App. A tables.  Velocity order from the App. B index maps (reading R2). */
static const int C9[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                             {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
static const int C21[21][2] = {{0, 0},  {1, 0},   {0, 1},  {-1, 0}, {0, -1},
                               {1, 1},  {-1, 1},  {-1, -1}, {1, -1}, {2, 0},
                               {0, 2},  {-2, 0},  {0, -2}, {2, 2},  {-2, 2},
                               {-2, -2}, {2, -2}, {3, 0},  {0, 3},  {-3, 0},
                               {0, -3}};
/* Bounce-back alpha* and specular alpha-hat exactly as App. B tabulates them
 * for the wall-crossing directions; the c^1 = 0 directions never cross a wall
 * and map to their reverse (alpha*) and to themselves (alpha-hat). */
static const int STAR21[21] = {0, 3, 4, 1, 2, 7, 8, 5, 6, 11, 12,
                               9, 10, 15, 16, 13, 14, 19, 20, 17, 18};
static const int HAT21[21] = {0, 3, 2, 1, 4, 6, 5, 8, 7, 11, 10,
                              9, 12, 14, 13, 16, 15, 19, 18, 17, 20};

int orc_lattice(int Q, int* c, double* w, int* star, int* hat, double* T0) {
    if (Q != 9 && Q != 21) return -1;
    for (int a = 0; a < Q; ++a) {
        c[2 * a] = (Q == 9) ? C9[a][0] : C21[a][0];
        c[2 * a + 1] = (Q == 9) ? C9[a][1] : C21[a][1];
        star[a] = STAR21[a];
        hat[a] = HAT21[a];
    }
    if (Q == 9) {
        *T0 = 1.0 / 3.0;
        w[0] = 4.0 / 9.0;
        for (int a = 1; a <= 4; ++a) w[a] = 1.0 / 9.0;
        for (int a = 5; a <= 8; ++a) w[a] = 1.0 / 36.0;
    } else {
        *T0 = 2.0 / 3.0;
        w[0] = 91.0 / 324.0;
        for (int a = 1; a <= 4; ++a) w[a] = 1.0 / 12.0;
        for (int a = 5; a <= 8; ++a) w[a] = 2.0 / 27.0;
        for (int a = 9; a <= 12; ++a) w[a] = 7.0 / 360.0;
        for (int a = 13; a <= 16; ++a) w[a] = 1.0 / 432.0;   /* reading R1 */
        for (int a = 17; a <= 20; ++a) w[a] = 1.0 / 1620.0;  /* reading R1 */
    }
    return 0;
}

/* ------------------------------------------------------------- indexing */

static inline int wrapj(const orc_grid* g, int j) { /* 1-based periodic */
    int m = (j - 1) % g->n2;
    if (m < 0) m += g->n2;
    return m + 1;
}
static inline size_t pidx(const orc_grid* g, int i, int j) {
    return (size_t)(i - 1 + PG) * (size_t)(g->ncol + 2 * PG) + (size_t)(j - 1 + PG);
}
static inline size_t gidx(const orc_grid* g, int i, int j) {
    return (size_t)(i - 1 + GG) * (size_t)(g->ncol + 2 * GG) + (size_t)(j - 1 + GG);
}
/* Column whose geometry serves cell column j.  Planar and polar grids are
 * invariant under a shift along q^2 (a translation, a rotation), so their
 * metric, volume and Theta are evaluated once, at column 1, and reused along
 * the row: a state that does not depend on j then stays exactly independent
 * of j, as in the paper's runs (App. B: only the radial index matters). */
static inline int geo_col(const orc_grid* g, int j) {
    return g->kind == ORC_GENERAL ? j : 1;
}
static inline size_t cidx(const orc_grid* g, int i, int j) { /* interior cell */
    return (size_t)(i - 1) * (size_t)g->n2 + (size_t)(j - 1);
}
static inline size_t nidx(const orc_grid* g, int a, int i, int j) {
    return (size_t)a * (size_t)g->n1 * (size_t)g->n2 + cidx(g, i, j);
}

/* ------------------------------------------------------------- geometry */

/* Wall-normal node coordinate of row i (1-based), ghosts mirrored through the
 * walls at edges[0] and edges[n1] (App. B "extended ... using symmetry"). */
static double node_coord(const double* e, int n1, int i) {
    if (i >= 1 && i <= n1) return 0.5 * (e[i - 1] + e[i]); /* App. C, Eq. 58 */
    if (i < 1) {
        int k = 1 - i;
        return 2.0 * e[0] - 0.5 * (e[k - 1] + e[k]);
    }
    int k = i - n1;
    int m = n1 + 1 - k;
    return 2.0 * e[n1] - 0.5 * (e[m - 1] + e[m]);
}

static int build_positions(orc_grid* g, const double* edges, double step2,
                           const double* nodes) {
    int n1 = g->n1, n2 = g->n2;
    if (g->kind == ORC_GENERAL) {
        size_t cnt = (size_t)(n1 + 2 * PG) * (size_t)(n2 + 2 * PG);
        for (size_t p = 0; p < cnt; ++p) {
            g->pos[p].x = nodes[2 * p];
            g->pos[p].y = nodes[2 * p + 1];
        }
        return 0;
    }
    const double pi = 3.14159265358979323846;
    for (int i = 1 - PG; i <= n1 + PG; ++i) {
        double s = node_coord(edges, n1, i);
        if (g->kind == ORC_POLAR && s <= 0.0) return -1;
        for (int j = 1 - PG; j <= g->ncol + PG; ++j) {
            vec2 p;
            if (g->kind == ORC_PLANAR) {
                p.x = s;
                p.y = ((double)j - 0.5) * step2;
            } else { /* polar, App. D: theta_j = (j - 1/2) Delta theta */
                double th = ((double)j - 0.5) * (2.0 * pi / (double)n2);
                p.x = s * cos(th);
                p.y = s * sin(th);
            }
            g->pos[pidx(g, i, j)] = p;
        }
    }
    return 0;
}

/* Sec. 2: distance vectors (Eq. 1), tangent vectors g_i = [D_i - D_-i]/2dx,
 * metric and volume (Eq. 2), co-tangent vectors (Eq. 3).  In 2-D g_3 = z. */
static void build_geometry(orc_grid* g) {
    int n1 = g->n1;
    for (int i = 1 - GG; i <= n1 + GG; ++i)
        for (int j = 1 - GG; j <= g->ncol + GG; ++j) {
            vec2 xq = g->pos[pidx(g, i, j)];
            vec2 xp1 = g->pos[pidx(g, i + 1, j)], xm1 = g->pos[pidx(g, i - 1, j)];
            vec2 xp2 = g->pos[pidx(g, i, j + 1)], xm2 = g->pos[pidx(g, i, j - 1)];
            vec2 Dp1 = {xp1.x - xq.x, xp1.y - xq.y}, Dm1 = {xm1.x - xq.x, xm1.y - xq.y};
            vec2 Dp2 = {xp2.x - xq.x, xp2.y - xq.y}, Dm2 = {xm2.x - xq.x, xm2.y - xq.y};
            vec2 t1 = {(Dp1.x - Dm1.x) / (2.0 * g->dx), (Dp1.y - Dm1.y) / (2.0 * g->dx)};
            vec2 t2 = {(Dp2.x - Dm2.x) / (2.0 * g->dx), (Dp2.y - Dm2.y) / (2.0 * g->dx)};
            double J = t1.x * t2.y - t1.y * t2.x; /* (g_1 x g_2) . g_3 */
            /* g^1 = (g_2 x g_3)/J, g^2 = (g_3 x g_1)/J */
            vec2 c1 = {t2.y / J, -t2.x / J};
            vec2 c2 = {-t1.y / J, t1.x / J};
            size_t k = gidx(g, i, j);
            g->g1[k] = t1;
            g->g2[k] = t2;
            g->G1[k] = c1;
            g->G2[k] = c2;
            g->Jgeo[k] = J;
        }
}

static inline vec2 tangent(const orc_grid* g, int m, int i, int j) {
    size_t k = gidx(g, i, j);
    return m == 0 ? g->g1[k] : g->g2[k];
}
static inline vec2 cotangent(const orc_grid* g, int m, int i, int j) {
    size_t k = gidx(g, i, j);
    return m == 0 ? g->G1[k] : g->G2[k];
}

/* Eq. 5: Theta^k_m(q + s c_a, q) = [g_m(q + s c_a) - g_m(q)] . g^k(q). */
static double theta(const orc_grid* g, int k, int m, int i, int j, int a, int s) {
    j = geo_col(g, j);
    int ii = i + s * g->c[a][0], jj = j + s * g->c[a][1];
    vec2 gn = tangent(g, m, ii, jj), gq = tangent(g, m, i, j);
    vec2 gk = cotangent(g, k, i, j);
    return (gn.x - gq.x) * gk.x + (gn.y - gq.y) * gk.y;
}

static void inverse_metric(const orc_grid* g, int i, int j, double ginv[2][2]) {
    j = geo_col(g, j);
    for (int k = 0; k < 2; ++k)
        for (int m = 0; m < 2; ++m) {
            vec2 a = cotangent(g, k, i, j), b = cotangent(g, m, i, j);
            ginv[k][m] = a.x * b.x + a.y * b.y; /* Eq. 3 */
        }
}

/* ------------------------------------------------------------ equilibrium */

/* Eq. 19: third-order curvilinear Hermite equilibrium, every sum written out. */
static double feq_one(const orc_grid* g, int a, double rho, const double U[2],
                      const double Ut[2], const double gi[2][2]) {
    const double T0 = g->T0;
    double c[2] = {(double)g->c[a][0], (double)g->c[a][1]};
    double t1 = 0.0;
    for (int i = 0; i < 2; ++i) t1 += c[i] * U[i] / T0;
    double t2 = 0.0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double dij = (i == j) ? 1.0 : 0.0;
            t2 += (c[i] * c[j] / T0 - dij) * ((gi[i][j] - dij) * T0 + Ut[i] * Ut[j]);
        }
    t2 /= 2.0 * T0;
    double t3 = 0.0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k) {
                double dij = (i == j), djk = (j == k), dki = (k == i);
                double H3 = c[i] * c[j] * c[k] - T0 * (c[i] * djk + c[j] * dki + c[k] * dij);
                double A3 = T0 * ((gi[i][j] * Ut[k] - dij * U[k]) +
                                  (gi[j][k] * Ut[i] - djk * U[i]) +
                                  (gi[k][i] * Ut[j] - dki * U[j])) +
                            Ut[i] * Ut[j] * Ut[k];
                t3 += H3 * A3;
            }
    t3 /= 6.0 * T0 * T0 * T0;
    return rho * g->w[a] * (1.0 + t1 + t2 + t3);
}

double orc_feq(const orc_grid* g, int alpha, double rho, const double* U,
               const double* Ut, const double* ginv) {
    double gi[2][2] = {{ginv[0], ginv[1]}, {ginv[2], ginv[3]}};
    return feq_one(g, alpha, rho, U, Ut, gi);
}

/* -------------------------------------------------------------- advection */

/* N_a(q,t) = N'_a(q - c_a, t-1) (Eq. 12), with App. B at the walls:
 * periodic in q^2; a source row beyond a wall is mirrored through that wall
 * (reading R8) and supplies N'_{a*} (no-slip) or N'_{a-hat} plus the moving
 * wall correction (reading R7).  rho_p/Ut2_p hold the source's moments of the
 * previous collision. */
static double incoming(const orc_grid* g, int a, int i, int j) {
    int si = i - g->c[a][0];
    int sj = wrapj(g, j - g->c[a][1]);
    if (si >= 1 && si <= g->n1) return g->Np[nidx(g, a, si, sj)];
    int lo = si < 1;
    int k = lo ? 1 - si : si - g->n1;          /* ghost depth */
    int mi = lo ? k : g->n1 + 1 - k;           /* mirrored fluid row */
    int bc = lo ? g->bc_lo : g->bc_hi;
    if (bc == ORC_NOSLIP) return g->Np[nidx(g, g->star[a], mi, sj)];
    int b = g->hat[a];
    double U0 = lo ? g->U0_lo : g->U0_hi;
    size_t m = cidx(g, mi, sj);
    double corr = (2.0 / g->T0) * g->w[b] * g->Jvol[m] * g->rho_p[m] *
                  (double)g->c[b][1] * (U0 - g->Ut2_p[m]);
    return g->Np[nidx(g, b, mi, sj)] + corr;
}

/* ---------------------------------------------------------------- collide */

typedef struct {
    double Npost[QMAX], Nin[QMAX], feq[QMAX], dN[QMAX];
    double F[2], U[2], Ut[2], dPi[2][2], rho;
} cell_out;

/* Everything of one cell's collision that follows advection: f = N/J
 * (Eq. 7), moments (Eqs. 8, 10), the inertial force of Eq. 15 evaluated with
 * the outgoing populations Nout, Ut (Eq. 18), f^eq (Eq. 19), dPi (Eq. 16),
 * dN (Eq. 17) and the BGK update of Eq. 6 with Eq. 11. */
static void collide_from(const orc_grid* g, int i, int j, const double* N,
                         const double* Nout, cell_out* o) {
    const int Q = g->Q;
    const double T0 = g->T0, tau = g->tau;
    double f[QMAX];
    double J = g->Jvol[cidx(g, i, j)];
    for (int a = 0; a < Q; ++a) f[a] = N[a] / J;
    double rho = 0.0, mU[2] = {0.0, 0.0};
    for (int a = 0; a < Q; ++a) {
        rho += f[a];
        for (int k = 0; k < 2; ++k) mU[k] += (double)g->c[a][k] * f[a];
    }
    double U[2] = {mU[0] / rho, mU[1] / rho};

    double F[2];
    for (int k = 0; k < 2; ++k) {
        double s = 0.0;
        for (int a = 0; a < Q; ++a)
            for (int m = 0; m < 2; ++m)
                s += (double)g->c[a][m] * (theta(g, k, m, i, j, a, +1) * Nout[a] -
                                           theta(g, k, m, i, j, a, -1) * N[a]);
        F[k] = -s / (2.0 * J) + rho * g->gext[k]; /* reading R5 */
    }
    double Ut[2] = {U[0] + F[0] / (2.0 * rho), U[1] + F[1] / (2.0 * rho)};

    double gi[2][2];
    inverse_metric(g, i, j, gi);
    double feq[QMAX];
    for (int a = 0; a < Q; ++a) feq[a] = feq_one(g, a, rho, U, Ut, gi);

    double dPi[2][2];
    double pref = -0.5 * (1.0 - 1.0 / (2.0 * tau));
    for (int p = 0; p < 2; ++p)
        for (int r = 0; r < 2; ++r) {
            double s = 0.0;
            for (int a = 0; a < Q; ++a)
                for (int k = 0; k < 2; ++k)
                    s += (double)g->c[a][p] * (double)g->c[a][k] *
                         (theta(g, r, k, i, j, a, +1) - theta(g, r, k, i, j, a, -1)) * feq[a];
            dPi[p][r] = pref * s;
        }

    for (int a = 0; a < Q; ++a) {
        double s1 = 0.0, s2 = 0.0;
        for (int p = 0; p < 2; ++p) s1 += (double)g->c[a][p] * F[p] / T0;
        for (int p = 0; p < 2; ++p)
            for (int r = 0; r < 2; ++r) {
                double dpr = (p == r) ? 1.0 : 0.0;
                s2 += ((double)g->c[a][p] * (double)g->c[a][r] / T0 - dpr) * dPi[p][r] / T0;
            }
        double dN = g->w[a] * J * (s1 + s2);
        double Om = -J * (f[a] - feq[a]) / tau;
        o->Npost[a] = N[a] + Om + dN;
        o->Nin[a] = N[a];
        o->feq[a] = feq[a];
        o->dN[a] = dN;
    }
    o->F[0] = F[0];
    o->F[1] = F[1];
    o->U[0] = U[0];
    o->U[1] = U[1];
    o->Ut[0] = Ut[0];
    o->Ut[1] = Ut[1];
    o->rho = rho;
    for (int p = 0; p < 2; ++p)
        for (int r = 0; r < 2; ++r) o->dPi[p][r] = dPi[p][r];
}

/* One cell of Eq. 6 in the order of Sec. 2.  The outgoing populations in the
 * force of Eq. 15 are those of the previous step, N'(q, t-1), as the paper
 * does; with iters > 0 the implicit relation is then iterated, each pass
 * putting the last N'(q, t) back into Eq. 15 (the iterative procedure the
 * paper mentions as an alternative to the lag). */
static void collide_cell(const orc_grid* g, int i, int j, cell_out* o) {
    const int Q = g->Q;
    double N[QMAX], Nout[QMAX];
    for (int a = 0; a < Q; ++a) {
        N[a] = incoming(g, a, i, j);
        Nout[a] = g->Np[nidx(g, a, i, j)]; /* lag: N'(q, t-1) */
    }
    collide_from(g, i, j, N, Nout, o);
    for (int it = 0; it < g->iters; ++it) {
        for (int a = 0; a < Q; ++a) Nout[a] = o->Npost[a];
        collide_from(g, i, j, N, Nout, o);
    }
}

/* ------------------------------------------------------------------ API */

orc_grid* orc_create(int Q, int n1, int n2, int kind, const double* edges,
                     double step2, const double* nodes, double dx, int bc_lo,
                     int bc_hi) {
    if ((Q != 9 && Q != 21) || n1 < PG || n2 < 1) return NULL;
    if (kind == ORC_GENERAL ? nodes == NULL : edges == NULL) return NULL;
    if (kind < 0 || kind > 2) return NULL;
    orc_grid* g = (orc_grid*)calloc(1, sizeof(orc_grid));
    if (!g) return NULL;
    g->Q = Q;
    g->n1 = n1;
    g->n2 = n2;
    g->kind = kind;
    g->bc_lo = bc_lo;
    g->bc_hi = bc_hi;
    int c[2 * QMAX];
    orc_lattice(Q, c, g->w, g->star, g->hat, &g->T0);
    for (int a = 0; a < Q; ++a) {
        g->c[a][0] = c[2 * a];
        g->c[a][1] = c[2 * a + 1];
    }
    if (dx <= 0.0) {
        if (kind == ORC_GENERAL) { free(g); return NULL; }
        dx = (edges[n1] - edges[0]) / (double)n1;
    }
    g->dx = dx;
    g->ncol = (kind == ORC_GENERAL) ? n2 : 1;
    size_t np = (size_t)(n1 + 2 * PG) * (size_t)(g->ncol + 2 * PG);
    size_t ng = (size_t)(n1 + 2 * GG) * (size_t)(g->ncol + 2 * GG);
    size_t nc = (size_t)n1 * (size_t)n2;
    g->pos = (vec2*)malloc(np * sizeof(vec2));
    g->g1 = (vec2*)malloc(ng * sizeof(vec2));
    g->g2 = (vec2*)malloc(ng * sizeof(vec2));
    g->G1 = (vec2*)malloc(ng * sizeof(vec2));
    g->G2 = (vec2*)malloc(ng * sizeof(vec2));
    g->Jgeo = (double*)malloc(ng * sizeof(double));
    g->Jvol = (double*)malloc(nc * sizeof(double));
    g->Np = (double*)calloc((size_t)Q * nc, sizeof(double));
    g->Nn = (double*)calloc((size_t)Q * nc, sizeof(double));
    g->rho_p = (double*)calloc(nc, sizeof(double));
    g->Ut1_p = (double*)calloc(nc, sizeof(double));
    g->Ut2_p = (double*)calloc(nc, sizeof(double));
    g->rho_n = (double*)calloc(nc, sizeof(double));
    g->Ut1_n = (double*)calloc(nc, sizeof(double));
    g->Ut2_n = (double*)calloc(nc, sizeof(double));
    if (!g->pos || !g->g1 || !g->g2 || !g->G1 || !g->G2 || !g->Jgeo || !g->Jvol ||
        !g->Np || !g->Nn || !g->rho_p || !g->Ut1_p || !g->Ut2_p || !g->rho_n ||
        !g->Ut1_n || !g->Ut2_n || build_positions(g, edges, step2, nodes) != 0) {
        orc_destroy(g);
        return NULL;
    }
    build_geometry(g);
    for (int i = 1; i <= n1; ++i)
        for (int j = 1; j <= n2; ++j) {
            double J = g->Jgeo[gidx(g, i, geo_col(g, j))];
            if (!(J > 0.0)) { orc_destroy(g); return NULL; }
            g->Jvol[cidx(g, i, j)] = J;
        }
    g->tau = 1.0;
    g->rho0 = 1.0;
    return g;
}

void orc_destroy(orc_grid* g) {
    if (!g) return;
    free(g->pos); free(g->g1); free(g->g2); free(g->G1); free(g->G2);
    free(g->Jgeo); free(g->Jvol); free(g->Np); free(g->Nn);
    free(g->rho_p); free(g->Ut1_p); free(g->Ut2_p);
    free(g->rho_n); free(g->Ut1_n); free(g->Ut2_n);
    free(g);
}

void orc_set_case(orc_grid* g, double tau, double rho0, double U0_lo,
                  double U0_hi, double gext1, double gext2) {
    g->tau = tau;
    g->rho0 = rho0;
    g->U0_lo = U0_lo;
    g->U0_hi = U0_hi;
    g->gext[0] = gext1;
    g->gext[1] = gext2;
}

void orc_init_rest(orc_grid* g) { /* reading R6 */
    const double zero[2] = {0.0, 0.0};
    for (int i = 1; i <= g->n1; ++i)
        for (int j = 1; j <= g->n2; ++j) {
            double gi[2][2];
            inverse_metric(g, i, j, gi);
            double J = g->Jvol[cidx(g, i, j)];
            for (int a = 0; a < g->Q; ++a)
                g->Np[nidx(g, a, i, j)] = J * feq_one(g, a, g->rho0, zero, zero, gi);
            size_t m = cidx(g, i, j);
            g->rho_p[m] = g->rho0;
            g->Ut1_p[m] = 0.0;
            g->Ut2_p[m] = 0.0;
        }
    g->t = 0;
}

void orc_set_state(orc_grid* g, const double* Np, const double* rho_prev,
                   const double* Ut2_prev) {
    size_t nc = (size_t)g->n1 * (size_t)g->n2;
    memcpy(g->Np, Np, (size_t)g->Q * nc * sizeof(double));
    for (size_t m = 0; m < nc; ++m) {
        g->rho_p[m] = rho_prev ? rho_prev[m] : g->rho0;
        g->Ut2_p[m] = Ut2_prev ? Ut2_prev[m] : 0.0;
        g->Ut1_p[m] = 0.0;
    }
}

void orc_get_state(const orc_grid* g, double* Np) {
    memcpy(Np, g->Np, (size_t)g->Q * (size_t)g->n1 * (size_t)g->n2 * sizeof(double));
}

void orc_get_prev_moments(const orc_grid* g, double* rho_prev, double* Ut2_prev) {
    size_t nc = (size_t)g->n1 * (size_t)g->n2;
    if (rho_prev) memcpy(rho_prev, g->rho_p, nc * sizeof(double));
    if (Ut2_prev) memcpy(Ut2_prev, g->Ut2_p, nc * sizeof(double));
}

void orc_step(orc_grid* g, long long nsteps) {
    const int n1 = g->n1, n2 = g->n2, Q = g->Q;
    for (long long s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int i = 1; i <= n1; ++i)
            for (int j = 1; j <= n2; ++j) {
                cell_out o;
                collide_cell(g, i, j, &o);
                for (int a = 0; a < Q; ++a) g->Nn[nidx(g, a, i, j)] = o.Npost[a];
                size_t m = cidx(g, i, j);
                g->rho_n[m] = o.rho;
                g->Ut1_n[m] = o.Ut[0];
                g->Ut2_n[m] = o.Ut[1];
            }
        double* t;
        t = g->Np; g->Np = g->Nn; g->Nn = t;
        t = g->rho_p; g->rho_p = g->rho_n; g->rho_n = t;
        t = g->Ut1_p; g->Ut1_p = g->Ut1_n; g->Ut1_n = t;
        t = g->Ut2_p; g->Ut2_p = g->Ut2_n; g->Ut2_n = t;
        g->t++;
    }
}

long long orc_time(const orc_grid* g) { return g->t; }

void orc_moments(const orc_grid* g, double* rho, double* U1, double* U2,
                 double* Ut1, double* Ut2, double* F1, double* F2) {
#pragma omp parallel for schedule(static)
    for (int i = 1; i <= g->n1; ++i)
        for (int j = 1; j <= g->n2; ++j) {
            cell_out o;
            collide_cell(g, i, j, &o);
            size_t m = cidx(g, i, j);
            if (rho) rho[m] = o.rho;
            if (U1) U1[m] = o.U[0];
            if (U2) U2[m] = o.U[1];
            if (Ut1) Ut1[m] = o.Ut[0];
            if (Ut2) Ut2[m] = o.Ut[1];
            if (F1) F1[m] = o.F[0];
            if (F2) F2[m] = o.F[1];
        }
}

void orc_collide_one(const orc_grid* g, int i, int j, double* Npost,
                     double* Nin, double* feq, double* dN, double* F,
                     double* Ut, double* dPi, double* rho) {
    cell_out o;
    collide_cell(g, i, j, &o);
    for (int a = 0; a < g->Q; ++a) {
        if (Npost) Npost[a] = o.Npost[a];
        if (Nin) Nin[a] = o.Nin[a];
        if (feq) feq[a] = o.feq[a];
        if (dN) dN[a] = o.dN[a];
    }
    if (F) { F[0] = o.F[0]; F[1] = o.F[1]; }
    if (Ut) { Ut[0] = o.Ut[0]; Ut[1] = o.Ut[1]; }
    if (dPi) { dPi[0] = o.dPi[0][0]; dPi[1] = o.dPi[0][1]; dPi[2] = o.dPi[1][0]; dPi[3] = o.dPi[1][1]; }
    if (rho) *rho = o.rho;
}

int orc_node_geometry(const orc_grid* g, int i, int j, double* out) {
    if (i < 1 - GG || i > g->n1 + GG || j < 1 - GG || j > g->ncol + GG) return -1;
    size_t k = gidx(g, i, j);
    out[0] = g->g1[k].x; out[1] = g->g1[k].y;
    out[2] = g->g2[k].x; out[3] = g->g2[k].y;
    out[4] = g->G1[k].x; out[5] = g->G1[k].y;
    out[6] = g->G2[k].x; out[7] = g->G2[k].y;
    out[8] = g->Jgeo[k];
    double gi[2][2];
    inverse_metric(g, i, j, gi);
    out[9] = gi[0][0]; out[10] = gi[0][1]; out[11] = gi[1][1];
    return 0;
}

void orc_theta(const orc_grid* g, int i, int j, int alpha, int s, double* out) {
    for (int k = 0; k < 2; ++k)
        for (int m = 0; m < 2; ++m) out[k * 2 + m] = theta(g, k, m, i, j, alpha, s);
}

void orc_totals(const orc_grid* g, double* out) {
    double m = 0.0, p1 = 0.0, p2 = 0.0;
    for (int a = 0; a < g->Q; ++a)
        for (int i = 1; i <= g->n1; ++i)
            for (int j = 1; j <= g->n2; ++j) {
                double v = g->Np[nidx(g, a, i, j)];
                m += v;
                p1 += (double)g->c[a][0] * v;
                p2 += (double)g->c[a][1] * v;
            }
    out[0] = m;
    out[1] = p1;
    out[2] = p2;
}

/* Sec. 3.1 diagnostics from given moment fields.  The tangent vectors and the
 * position of a planar or polar cell are those of column 1 (R22): a polar
 * cell at column j is the column-1 cell turned about the origin, and |u| and
 * (x cross u).z do not change under a rotation of both x and u. */
void orc_flow_diagnostics(const orc_grid* g, const double* rho, const double* Ut1,
                          const double* Ut2, const double* Ut1_prev,
                          const double* Ut2_prev, long long dt, double* out) {
    const int have_prev = Ut1_prev != NULL && Ut2_prev != NULL;
    double sum_dd = 0.0, sum_uu = 0.0, ke = 0.0, am = 0.0, umax = 0.0;
    for (int i = 1; i <= g->n1; ++i)
        for (int j = 1; j <= g->n2; ++j) {
            size_t m = cidx(g, i, j);
            int jc = geo_col(g, j);
            vec2 t1 = tangent(g, 0, i, jc), t2 = tangent(g, 1, i, jc);
            vec2 x = g->pos[pidx(g, i, jc)];
            double J = g->Jvol[m];
            vec2 u = {Ut1[m] * t1.x + Ut2[m] * t2.x, Ut1[m] * t1.y + Ut2[m] * t2.y};
            double uu = u.x * u.x + u.y * u.y;
            sum_uu += J * uu;
            ke += 0.5 * J * rho[m] * uu;
            if (g->kind != ORC_PLANAR) am += J * rho[m] * (x.x * u.y - x.y * u.x);
            if (sqrt(uu) > umax) umax = sqrt(uu);
            if (have_prev) {
                vec2 up = {Ut1_prev[m] * t1.x + Ut2_prev[m] * t2.x,
                           Ut1_prev[m] * t1.y + Ut2_prev[m] * t2.y};
                double ex = u.x - up.x, ey = u.y - up.y;
                sum_dd += J * (ex * ex + ey * ey);
            }
        }
    double res = INFINITY;
    if (have_prev && dt > 0) {
        if (sum_uu > 0.0) res = sqrt(sum_dd) / ((double)dt * sqrt(sum_uu));
        else res = sum_dd > 0.0 ? INFINITY : 0.0;
    }
    out[0] = res;
    out[1] = ke;
    out[2] = am;
    out[3] = umax;
    out[4] = sum_uu;
}

void orc_get_volume(const orc_grid* g, double* J) {
    memcpy(J, g->Jvol, (size_t)g->n1 * (size_t)g->n2 * sizeof(double));
}
void orc_set_volume(orc_grid* g, const double* J) {
    memcpy(g->Jvol, J, (size_t)g->n1 * (size_t)g->n2 * sizeof(double));
}

void orc_no_flow_adjust(orc_grid* g, long long nsteps, double* rho_nf) {
    double U0l = g->U0_lo, U0h = g->U0_hi, g1 = g->gext[0], g2 = g->gext[1];
    g->U0_lo = g->U0_hi = 0.0;
    g->gext[0] = g->gext[1] = 0.0;
    orc_init_rest(g);
    orc_step(g, nsteps);
    size_t nc = (size_t)g->n1 * (size_t)g->n2;
    double* r = (double*)malloc(nc * sizeof(double));
    orc_moments(g, r, NULL, NULL, NULL, NULL, NULL, NULL);
    /* Eq. 23.  Under J -> J rho_nf/rho0 every density of the kept state
     * scales by rho0/rho_nf while U, Ut are unchanged, so the stored moments
     * of the last collision are rescaled the same way. */
    for (size_t m = 0; m < nc; ++m) {
        g->Jvol[m] *= r[m] / g->rho0;
        g->rho_p[m] *= g->rho0 / r[m];
    }
    if (rho_nf) memcpy(rho_nf, r, nc * sizeof(double));
    free(r);
    g->U0_lo = U0l;
    g->U0_hi = U0h;
    g->gext[0] = g1;
    g->gext[1] = g2;
    g->t = 0;
}

void orc_set_force_iterations(orc_grid* g, int iters) { g->iters = iters < 0 ? 0 : iters; }

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
