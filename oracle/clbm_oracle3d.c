/*
 * clbm_oracle3d.c -- plain FP64 CPU oracle of the volumetric curvilinear
 * lattice Boltzmann method in three dimensions (arXiv:2301.01868, Sec. 2,
 * whose equations are written for three coordinates), D3Q39 lattice.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file;
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg load
 * it.  It shares no code with the CUDA library.
 *
 * Written the plain way: one loop over cells per time step, every tensor sum
 * written out over its indices, Theta formed from tangent vectors at the
 * neighbour nodes (Eq. 5), f^eq from Eq. 19 directly.  The grids here are
 * invariant under shifts along q^2 and q^3 (a channel: translations; an
 * annulus extruded along z: rotations and translations), so the geometry is
 * evaluated around column (1, 1) and serves every column, as the 2-D oracle
 * does for its planar and polar grids.  Compile with -ffp-contract=off.
 *
 * Readings (the 2-D oracle's, carried to three coordinates):
 *   R4  Delta x of the tangent vectors is the average wall-normal step.
 *   R5  a body force enters as F^k += rho g^k, g^k contravariant.
 *   R6  N'(q,-1) = J f^eq(rho0, 0; g^{ij}(q)).
 *   R7  the moving wall adds (2/T0) w J rho sum_t c^t (U0^t - Ut^t) over the
 *       tangential components t = 2, 3 at the mirrored source node (the
 *       wall moves along q^2, so U0^3 = 0); the normal term is dropped as
 *       App. B drops it.
 *   R8  the source of a population crossing a wall is the mirror image of
 *       the ghost node through that wall: N'_{a*} there (no-slip, a* = -a)
 *       or N'_{a-hat} (moving wall, a-hat = a with c^1 flipped).
 *   R26 the lattice is D3Q39 (no 3-D set is printed in the paper).
 */
#include "clbm_oracle3d.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NQ 39
#define PG 4 /* ghost layers of node positions */
#define GG 3 /* ghost layers of tangent vectors (widest stencil |c| = 3) */
#define NB (2 * PG + 1)  /* position block width along q^2, q^3 */
#define NT (2 * GG + 1)  /* tangent block width */

typedef struct { double v[3]; } vec3;

struct o3_grid {
    int n1, n2, n3, kind, bc_lo, bc_hi;
    double T0, w[NQ];
    int c[NQ][3], star[NQ], hat[NQ];
    double dx, step2, step3;
    double* edges;
    vec3* pos;        /* [i][jb][kb], i = 1-PG..n1+PG, jb, kb = 1-PG..1+PG */
    vec3* tg;         /* tangent vectors g_m: [i][jb][kb][m], i = 1-GG..n1+GG, jb, kb in 1-GG..1+GG */
    vec3* ct;         /* co-tangent g^m at (i, 1, 1): [i][m], interior rows */
    double* J;        /* volume per interior row */
    double tau, rho0, U0_lo, U0_hi, gext[3];
    double *Np, *Nn;  /* N'(t-1), next N' */
    double *rho_p, *ut2_p, *ut3_p, *rho_n, *ut2_n, *ut3_n;
    long long t;
};

/* ---------------------------------------------------------------- lattice */

/* Shells in order, sign and permutation variants in lexicographic order. */
int o3_lattice(int* c, double* w, int* star, int* hat, double* T0) {
    static const int shell[6][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 1}, {2, 0, 0}, {2, 2, 0}, {3, 0, 0}};
    static const double ws[6] = {1.0 / 12.0, 1.0 / 12.0, 1.0 / 27.0, 2.0 / 135.0, 1.0 / 432.0,
                                 1.0 / 1620.0};
    int n = 0;
    for (int s = 0; s < 6; ++s) {
        /* every vector whose sorted absolute values equal the shell's */
        for (int x = -3; x <= 3; ++x)
            for (int y = -3; y <= 3; ++y)
                for (int z = -3; z <= 3; ++z) {
                    int a[3] = {abs(x), abs(y), abs(z)};
                    /* sort descending */
                    for (int p = 0; p < 3; ++p)
                        for (int q = p + 1; q < 3; ++q)
                            if (a[q] > a[p]) { int t = a[p]; a[p] = a[q]; a[q] = t; }
                    if (a[0] != shell[s][0] || a[1] != shell[s][1] || a[2] != shell[s][2]) continue;
                    c[3 * n] = x;
                    c[3 * n + 1] = y;
                    c[3 * n + 2] = z;
                    w[n] = ws[s];
                    ++n;
                }
    }
    if (n != NQ) return -1;
    for (int a = 0; a < NQ; ++a) {
        star[a] = hat[a] = -1;
        for (int b = 0; b < NQ; ++b) {
            if (c[3 * b] == -c[3 * a] && c[3 * b + 1] == -c[3 * a + 1] && c[3 * b + 2] == -c[3 * a + 2])
                star[a] = b;
            if (c[3 * b] == -c[3 * a] && c[3 * b + 1] == c[3 * a + 1] && c[3 * b + 2] == c[3 * a + 2])
                hat[a] = b;
        }
    }
    *T0 = 2.0 / 3.0;
    return 0;
}

/* ------------------------------------------------------------- indexing */

static inline int wrap(int j, int n) { /* 1-based periodic */
    int m = (j - 1) % n;
    if (m < 0) m += n;
    return m + 1;
}
static inline size_t cidx(const o3_grid* g, int i, int j, int k) {
    return ((size_t)(i - 1) * g->n2 + (size_t)(j - 1)) * g->n3 + (size_t)(k - 1);
}
static inline size_t ncells(const o3_grid* g) { return (size_t)g->n1 * g->n2 * g->n3; }
static inline size_t nidx(const o3_grid* g, int a, int i, int j, int k) {
    return (size_t)a * ncells(g) + cidx(g, i, j, k);
}
static inline size_t pidx(const o3_grid* g, int i, int jb, int kb) {
    (void)g;
    return ((size_t)(i - 1 + PG) * NB + (size_t)(jb - 1 + PG)) * NB + (size_t)(kb - 1 + PG);
}
static inline size_t tidx(const o3_grid* g, int i, int jb, int kb, int m) {
    (void)g;
    return (((size_t)(i - 1 + GG) * NT + (size_t)(jb - 1 + GG)) * NT + (size_t)(kb - 1 + GG)) * 3 + m;
}

/* ------------------------------------------------------------- geometry */

/* Wall-normal node coordinate of row i (App. C midpoints, App. B mirror). */
static double node_coord(const double* e, int n1, int i) {
    if (i >= 1 && i <= n1) return 0.5 * (e[i - 1] + e[i]);
    if (i < 1) {
        int k = 1 - i;
        return 2.0 * e[0] - 0.5 * (e[k - 1] + e[k]);
    }
    int k = i - n1, m = n1 + 1 - k;
    return 2.0 * e[n1] - 0.5 * (e[m - 1] + e[m]);
}

static vec3 node(const o3_grid* g, int i, int j, int k) {
    const double pi = 3.14159265358979323846;
    double s = node_coord(g->edges, g->n1, i);
    vec3 p;
    if (g->kind == O3_CHANNEL) {
        p.v[0] = s;
        p.v[1] = ((double)j - 0.5) * g->step2;
    } else {
        double th = ((double)j - 0.5) * (2.0 * pi / (double)g->n2);
        p.v[0] = s * cos(th);
        p.v[1] = s * sin(th);
    }
    p.v[2] = ((double)k - 0.5) * g->step3;
    return p;
}

static vec3 cross(vec3 a, vec3 b) {
    vec3 r = {{a.v[1] * b.v[2] - a.v[2] * b.v[1], a.v[2] * b.v[0] - a.v[0] * b.v[2],
               a.v[0] * b.v[1] - a.v[1] * b.v[0]}};
    return r;
}
static double dot(vec3 a, vec3 b) { return a.v[0] * b.v[0] + a.v[1] * b.v[1] + a.v[2] * b.v[2]; }

/* Sec. 2: D_{+-m} = x(q +- e_m) - x(q) (Eq. 1), g_m = [D_m - D_-m] / (2 dx),
 * J = g_1 . (g_2 x g_3), g^1 = g_2 x g_3 / J and cyclic (Eq. 3). */
static void build_geometry(o3_grid* g) {
    int n1 = g->n1;
    for (int i = 1 - PG; i <= n1 + PG; ++i)
        for (int jb = 1 - PG; jb <= 1 + PG; ++jb)
            for (int kb = 1 - PG; kb <= 1 + PG; ++kb) g->pos[pidx(g, i, jb, kb)] = node(g, i, jb, kb);
    for (int i = 1 - GG; i <= n1 + GG; ++i)
        for (int jb = 1 - GG; jb <= 1 + GG; ++jb)
            for (int kb = 1 - GG; kb <= 1 + GG; ++kb) {
                vec3 xq = g->pos[pidx(g, i, jb, kb)];
                for (int m = 0; m < 3; ++m) {
                    int di = m == 0, dj = m == 1, dk = m == 2;
                    vec3 xp = g->pos[pidx(g, i + di, jb + dj, kb + dk)];
                    vec3 xm = g->pos[pidx(g, i - di, jb - dj, kb - dk)];
                    vec3 t;
                    for (int r = 0; r < 3; ++r)
                        t.v[r] = ((xp.v[r] - xq.v[r]) - (xm.v[r] - xq.v[r])) / (2.0 * g->dx);
                    g->tg[tidx(g, i, jb, kb, m)] = t;
                }
            }
    for (int i = 1; i <= n1; ++i) {
        vec3 t1 = g->tg[tidx(g, i, 1, 1, 0)], t2 = g->tg[tidx(g, i, 1, 1, 1)], t3 = g->tg[tidx(g, i, 1, 1, 2)];
        double J = dot(t1, cross(t2, t3));
        vec3 c1 = cross(t2, t3), c2 = cross(t3, t1), c3 = cross(t1, t2);
        for (int r = 0; r < 3; ++r) {
            c1.v[r] /= J;
            c2.v[r] /= J;
            c3.v[r] /= J;
        }
        g->ct[(size_t)(i - 1) * 3 + 0] = c1;
        g->ct[(size_t)(i - 1) * 3 + 1] = c2;
        g->ct[(size_t)(i - 1) * 3 + 2] = c3;
        g->J[i - 1] = J;
    }
}

/* Eq. 5: Theta^k_m(q + s c_a, q) = [g_m(q + s c_a) - g_m(q)] . g^k(q). */
static double theta(const o3_grid* g, int k, int m, int i, int a, int s) {
    vec3 gn = g->tg[tidx(g, i + s * g->c[a][0], 1 + s * g->c[a][1], 1 + s * g->c[a][2], m)];
    vec3 gq = g->tg[tidx(g, i, 1, 1, m)];
    vec3 d = {{gn.v[0] - gq.v[0], gn.v[1] - gq.v[1], gn.v[2] - gq.v[2]}};
    return dot(d, g->ct[(size_t)(i - 1) * 3 + k]);
}

static void inverse_metric(const o3_grid* g, int i, double gi[3][3]) {
    for (int k = 0; k < 3; ++k)
        for (int m = 0; m < 3; ++m)
            gi[k][m] = dot(g->ct[(size_t)(i - 1) * 3 + k], g->ct[(size_t)(i - 1) * 3 + m]);
}

/* ------------------------------------------------------------ equilibrium */

/* Eq. 19 in three coordinates, every sum written out. */
static double feq_one(const o3_grid* g, int a, double rho, const double U[3], const double Ut[3],
                      const double gi[3][3]) {
    const double T0 = g->T0;
    double c[3] = {(double)g->c[a][0], (double)g->c[a][1], (double)g->c[a][2]};
    double t1 = 0.0;
    for (int i = 0; i < 3; ++i) t1 += c[i] * U[i] / T0;
    double t2 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double dij = (i == j) ? 1.0 : 0.0;
            t2 += (c[i] * c[j] / T0 - dij) * ((gi[i][j] - dij) * T0 + Ut[i] * Ut[j]);
        }
    t2 /= 2.0 * T0;
    double t3 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                double dij = (i == j), djk = (j == k), dki = (k == i);
                double H3 = c[i] * c[j] * c[k] - T0 * (c[i] * djk + c[j] * dki + c[k] * dij);
                double A3 = T0 * ((gi[i][j] * Ut[k] - dij * U[k]) + (gi[j][k] * Ut[i] - djk * U[i]) +
                                  (gi[k][i] * Ut[j] - dki * U[j])) +
                            Ut[i] * Ut[j] * Ut[k];
                t3 += H3 * A3;
            }
    t3 /= 6.0 * T0 * T0 * T0;
    return rho * g->w[a] * (1.0 + t1 + t2 + t3);
}

double o3_feq(const o3_grid* g, int alpha, double rho, const double* U, const double* Ut,
              const double* ginv) {
    double gi[3][3];
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) gi[p][q] = ginv[3 * p + q];
    return feq_one(g, alpha, rho, U, Ut, gi);
}

/* -------------------------------------------------------------- advection */

/* N_a(q,t) = N'_a(q - c_a, t-1) (Eq. 12): periodic in q^2 and q^3; a source
 * beyond a wall is mirrored through it (R8) and supplies N'_{a*} (no-slip)
 * or N'_{a-hat} plus the moving-wall term (R7). */
static double incoming(const o3_grid* g, int a, int i, int j, int k) {
    int si = i - g->c[a][0];
    int sj = wrap(j - g->c[a][1], g->n2), sk = wrap(k - g->c[a][2], g->n3);
    if (si >= 1 && si <= g->n1) return g->Np[nidx(g, a, si, sj, sk)];
    int lo = si < 1;
    int d = lo ? 1 - si : si - g->n1;
    int mi = lo ? d : g->n1 + 1 - d;
    int bc = lo ? g->bc_lo : g->bc_hi;
    if (bc == 0) return g->Np[nidx(g, g->star[a], mi, sj, sk)];
    int b = g->hat[a];
    double U0 = lo ? g->U0_lo : g->U0_hi;
    size_t m = cidx(g, mi, sj, sk);
    double corr = (2.0 / g->T0) * g->w[b] * g->J[mi - 1] * g->rho_p[m] *
                  ((double)g->c[b][1] * (U0 - g->ut2_p[m]) + (double)g->c[b][2] * (0.0 - g->ut3_p[m]));
    return g->Np[nidx(g, b, mi, sj, sk)] + corr;
}

/* ---------------------------------------------------------------- collide */

typedef struct {
    double Npost[NQ], Nin[NQ];
    double F[3], U[3], Ut[3], rho;
} cell_out;

/* f = N/J (Eq. 7), moments (Eqs. 8, 10), the lagged force of Eq. 15 with
 * N'(q, t-1), Ut (Eq. 18), f^eq (Eq. 19), dPi (Eq. 16), dN (Eq. 17), BGK
 * (Eqs. 6, 11). */
static void collide_cell(const o3_grid* g, int i, int j, int k, cell_out* o) {
    const double T0 = g->T0, tau = g->tau;
    double N[NQ], Nout[NQ], f[NQ];
    for (int a = 0; a < NQ; ++a) {
        N[a] = incoming(g, a, i, j, k);
        Nout[a] = g->Np[nidx(g, a, i, j, k)];
    }
    double J = g->J[i - 1];
    for (int a = 0; a < NQ; ++a) f[a] = N[a] / J;
    double rho = 0.0, mU[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < NQ; ++a) {
        rho += f[a];
        for (int p = 0; p < 3; ++p) mU[p] += (double)g->c[a][p] * f[a];
    }
    double U[3] = {mU[0] / rho, mU[1] / rho, mU[2] / rho};
    double F[3];
    for (int p = 0; p < 3; ++p) {
        double s = 0.0;
        for (int a = 0; a < NQ; ++a)
            for (int m = 0; m < 3; ++m)
                s += (double)g->c[a][m] * (theta(g, p, m, i, a, +1) * Nout[a] - theta(g, p, m, i, a, -1) * N[a]);
        F[p] = -s / (2.0 * J) + rho * g->gext[p];
    }
    double Ut[3];
    for (int p = 0; p < 3; ++p) Ut[p] = U[p] + F[p] / (2.0 * rho);
    double gi[3][3];
    inverse_metric(g, i, gi);
    double feq[NQ];
    for (int a = 0; a < NQ; ++a) feq[a] = feq_one(g, a, rho, U, Ut, gi);
    double dPi[3][3];
    double pref = -0.5 * (1.0 - 1.0 / (2.0 * tau));
    for (int p = 0; p < 3; ++p)
        for (int r = 0; r < 3; ++r) {
            double s = 0.0;
            for (int a = 0; a < NQ; ++a)
                for (int m = 0; m < 3; ++m)
                    s += (double)g->c[a][p] * (double)g->c[a][m] *
                         (theta(g, r, m, i, a, +1) - theta(g, r, m, i, a, -1)) * feq[a];
            dPi[p][r] = pref * s;
        }
    for (int a = 0; a < NQ; ++a) {
        double s1 = 0.0, s2 = 0.0;
        for (int p = 0; p < 3; ++p) s1 += (double)g->c[a][p] * F[p] / T0;
        for (int p = 0; p < 3; ++p)
            for (int r = 0; r < 3; ++r) {
                double dpr = (p == r) ? 1.0 : 0.0;
                s2 += ((double)g->c[a][p] * (double)g->c[a][r] / T0 - dpr) * dPi[p][r] / T0;
            }
        double dN = g->w[a] * J * (s1 + s2);
        double Om = -J * (f[a] - feq[a]) / tau;
        o->Npost[a] = N[a] + Om + dN;
        o->Nin[a] = N[a];
    }
    for (int p = 0; p < 3; ++p) {
        o->F[p] = F[p];
        o->U[p] = U[p];
        o->Ut[p] = Ut[p];
    }
    o->rho = rho;
}

/* ------------------------------------------------------------------ API */

o3_grid* o3_create(int n1, int n2, int n3, int kind, const double* edges, double step2,
                   double step3, double dx, int bc_lo, int bc_hi) {
    if (n1 < 4 || n2 < 1 || n3 < 1 || !edges) return NULL;
    if (kind != O3_CHANNEL && kind != O3_ANNULUS) return NULL;
    for (int i = 0; i < n1; ++i)
        if (!(edges[i + 1] > edges[i])) return NULL;
    if (kind == O3_ANNULUS && !(edges[0] > 0.0)) return NULL;
    o3_grid* g = (o3_grid*)calloc(1, sizeof(o3_grid));
    if (!g) return NULL;
    g->n1 = n1;
    g->n2 = n2;
    g->n3 = n3;
    g->kind = kind;
    g->bc_lo = bc_lo;
    g->bc_hi = bc_hi;
    int cc[3 * NQ];
    o3_lattice(cc, g->w, g->star, g->hat, &g->T0);
    for (int a = 0; a < NQ; ++a)
        for (int p = 0; p < 3; ++p) g->c[a][p] = cc[3 * a + p];
    g->dx = dx > 0.0 ? dx : (edges[n1] - edges[0]) / (double)n1;
    g->step2 = step2;
    g->step3 = step3;
    g->edges = (double*)malloc((size_t)(n1 + 1) * sizeof(double));
    memcpy(g->edges, edges, (size_t)(n1 + 1) * sizeof(double));
    g->pos = (vec3*)calloc((size_t)(n1 + 2 * PG) * NB * NB, sizeof(vec3));
    g->tg = (vec3*)calloc((size_t)(n1 + 2 * GG) * NT * NT * 3, sizeof(vec3));
    g->ct = (vec3*)calloc((size_t)n1 * 3, sizeof(vec3));
    g->J = (double*)calloc((size_t)n1, sizeof(double));
    size_t nc = ncells(g);
    g->Np = (double*)calloc(nc * NQ, sizeof(double));
    g->Nn = (double*)calloc(nc * NQ, sizeof(double));
    g->rho_p = (double*)calloc(nc, sizeof(double));
    g->ut2_p = (double*)calloc(nc, sizeof(double));
    g->ut3_p = (double*)calloc(nc, sizeof(double));
    g->rho_n = (double*)calloc(nc, sizeof(double));
    g->ut2_n = (double*)calloc(nc, sizeof(double));
    g->ut3_n = (double*)calloc(nc, sizeof(double));
    build_geometry(g);
    g->tau = 1.0;
    g->rho0 = 1.0;
    return g;
}

void o3_destroy(o3_grid* g) {
    if (!g) return;
    free(g->edges);
    free(g->pos);
    free(g->tg);
    free(g->ct);
    free(g->J);
    free(g->Np);
    free(g->Nn);
    free(g->rho_p);
    free(g->ut2_p);
    free(g->ut3_p);
    free(g->rho_n);
    free(g->ut2_n);
    free(g->ut3_n);
    free(g);
}

void o3_set_case(o3_grid* g, double tau, double rho0, double U0_lo, double U0_hi, double g1,
                 double g2, double g3) {
    g->tau = tau;
    g->rho0 = rho0;
    g->U0_lo = U0_lo;
    g->U0_hi = U0_hi;
    g->gext[0] = g1;
    g->gext[1] = g2;
    g->gext[2] = g3;
}

void o3_init_rest(o3_grid* g) {
    double zero[3] = {0.0, 0.0, 0.0};
    for (int i = 1; i <= g->n1; ++i) {
        double gi[3][3];
        inverse_metric(g, i, gi);
        for (int a = 0; a < NQ; ++a) {
            double v = g->J[i - 1] * feq_one(g, a, g->rho0, zero, zero, gi);
            for (int j = 1; j <= g->n2; ++j)
                for (int k = 1; k <= g->n3; ++k) g->Np[nidx(g, a, i, j, k)] = v;
        }
    }
    for (size_t m = 0; m < ncells(g); ++m) {
        g->rho_p[m] = g->rho0;
        g->ut2_p[m] = 0.0;
        g->ut3_p[m] = 0.0;
    }
    g->t = 0;
}

void o3_set_state(o3_grid* g, const double* Np, const double* rho_prev, const double* ut2_prev,
                  const double* ut3_prev) {
    size_t nc = ncells(g);
    memcpy(g->Np, Np, nc * NQ * sizeof(double));
    for (size_t m = 0; m < nc; ++m) {
        g->rho_p[m] = rho_prev ? rho_prev[m] : g->rho0;
        g->ut2_p[m] = ut2_prev ? ut2_prev[m] : 0.0;
        g->ut3_p[m] = ut3_prev ? ut3_prev[m] : 0.0;
    }
}

void o3_get_state(const o3_grid* g, double* Np) { memcpy(Np, g->Np, ncells(g) * NQ * sizeof(double)); }

void o3_step(o3_grid* g, long long nsteps) {
    for (long long s = 0; s < nsteps; ++s) {
        for (int i = 1; i <= g->n1; ++i)
            for (int j = 1; j <= g->n2; ++j)
                for (int k = 1; k <= g->n3; ++k) {
                    cell_out o;
                    collide_cell(g, i, j, k, &o);
                    for (int a = 0; a < NQ; ++a) g->Nn[nidx(g, a, i, j, k)] = o.Npost[a];
                    size_t m = cidx(g, i, j, k);
                    g->rho_n[m] = o.rho;
                    g->ut2_n[m] = o.Ut[1];
                    g->ut3_n[m] = o.Ut[2];
                }
        double* t;
        t = g->Np; g->Np = g->Nn; g->Nn = t;
        t = g->rho_p; g->rho_p = g->rho_n; g->rho_n = t;
        t = g->ut2_p; g->ut2_p = g->ut2_n; g->ut2_n = t;
        t = g->ut3_p; g->ut3_p = g->ut3_n; g->ut3_n = t;
        g->t++;
    }
}

long long o3_time(const o3_grid* g) { return g->t; }

void o3_moments(const o3_grid* g, double* rho, double* U, double* Ut, double* F) {
    size_t nc = ncells(g);
    for (int i = 1; i <= g->n1; ++i)
        for (int j = 1; j <= g->n2; ++j)
            for (int k = 1; k <= g->n3; ++k) {
                cell_out o;
                collide_cell(g, i, j, k, &o);
                size_t m = cidx(g, i, j, k);
                if (rho) rho[m] = o.rho;
                for (int p = 0; p < 3; ++p) {
                    if (U) U[p * nc + m] = o.U[p];
                    if (Ut) Ut[p * nc + m] = o.Ut[p];
                    if (F) F[p * nc + m] = o.F[p];
                }
            }
}

void o3_totals(const o3_grid* g, double* out) {
    for (int p = 0; p < 4; ++p) out[p] = 0.0;
    for (int a = 0; a < NQ; ++a)
        for (int i = 1; i <= g->n1; ++i)
            for (int j = 1; j <= g->n2; ++j)
                for (int k = 1; k <= g->n3; ++k) {
                    double v = g->Np[nidx(g, a, i, j, k)];
                    out[0] += v;
                    for (int p = 0; p < 3; ++p) out[1 + p] += (double)g->c[a][p] * v;
                }
}

int o3_row_geometry(const o3_grid* g, int i, double* out) {
    if (i < 1 || i > g->n1) return -1;
    double gi[3][3];
    inverse_metric(g, i, gi);
    out[0] = g->J[i - 1];
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
            out[1 + 3 * p + q] = gi[p][q];
            out[10 + 3 * p + q] = dot(g->tg[tidx(g, i, 1, 1, p)], g->tg[tidx(g, i, 1, 1, q)]);
        }
    return 0;
}

void o3_theta(const o3_grid* g, int i, int alpha, int s, double* out) {
    for (int k = 0; k < 3; ++k)
        for (int m = 0; m < 3; ++m) out[3 * k + m] = theta(g, k, m, i, alpha, s);
}

void o3_collide_one(const o3_grid* g, int i, int j, int k, double* Npost, double* Nin, double* F,
                    double* rho) {
    cell_out o;
    collide_cell(g, i, j, k, &o);
    for (int a = 0; a < NQ; ++a) {
        Npost[a] = o.Npost[a];
        Nin[a] = o.Nin[a];
    }
    for (int p = 0; p < 3; ++p) F[p] = o.F[p];
    *rho = o.rho;
}
