/*
 * lbref.c -- plain FP64 CPU reference ("the oracle") for the linear
 * lattice-Boltzmann (LB) acoustic scheme of Dhuri, Hanasoge, Perlekar and
 * Robertsson, "Numerical analysis of the lattice Boltzmann method for
 * simulation of linear acoustic waves" (arXiv:1704.03172).
 *
 * TEST INFRASTRUCTURE.  This file exists so that the tests, the smoke check
 * and the CPU-baseline leg of the benchmark can compare the CUDA path with a
 * slow, obviously correct restatement of the paper.  The product path never
 * calls, links or loads it, and it shares no code, header, table or helper
 * with the CUDA path.
 *
 * Everything is FP64, plain loops, no blocking or fusion beyond the order in
 * which the paper states the scheme.  The only parallelism is an OpenMP loop
 * over rows, which does not change any arithmetic.
 *
 * Discrete scheme (one time step n -> n+1, for every lattice site x):
 *   1. moments      rho = sum_i g_i                      (Eq. macroscopic density)
 *                   j   = sum_i c_i g_i  (= rho_0 v)     (Eq. macroscopic velocity)
 *   2. equilibrium  g_i^eq = (w_i / c_s^2) [p + c_i . j],  p = c_s^2 rho
 *                                                        (Eq. linear eqm dist, Eq. state)
 *   3. collision    BGK: g* = g - (g - g^eq)/tau         (Eq. BGK-LB)
 *                   MRT: m = M g, m^eq = M g^eq,
 *                        g* = M^-1 [m - S (m - m^eq)]    (Eq. MRT-LB basic, App. A)
 *   4. source       g*_i += w_i S^n at the source site   (Eq. MRT-LB linear acoustic)
 *   5. sponge       g*_i *= (1 - sigma(x))               (Sec. 4, overlap/sponge layers)
 *   6. streaming    g_i(x + c_i, n+1) = g*_i(x)          (push; periodic wrap, or the
 *                   population is dropped when it leaves the domain and 0 enters)
 * Receivers record p = c_s^2 rho of the state entering step n (row n of the
 * trace holds the pressure at time n).
 *
 * Weights (Sec. 2.3, Eq. LB lattice moments and Eq. 0th lattice weight):
 *   eta = c / c_ref.  D2Q5: w_0 = 1 - eta^2, w_1..4 = (1 - w_0)/4.
 *   D2Q9 (the paper leaves the split open): w_1..4 = eta^2 w1_ref,
 *   w_5..8 = eta^2 w5_ref, w_0 = 1 - sum of the others.
 *   In both cases c_s^2 = sum_i w_i c_ix^2 (the second-moment constraint).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#include "lbref.h"

#ifdef _OPENMP
#include <omp.h>
#endif

/* Lattice velocities (Table I; numbering fixed by the rows of M, App. A). */
static const int C5[5][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}};
static const int C9[9][2] = {{0, 0},  {1, 0},  {0, 1},   {-1, 0}, {0, -1},
                             {1, 1},  {-1, 1}, {-1, -1}, {1, -1}};

/* Moment matrices printed in App. A. */
static const double M5[5][5] = {
    {1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0},
    {0, 0, 1, 0, -1},
    {-4, 1, 1, 1, 1},
    {0, 1, -1, 1, -1},
};
static const double M9[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, 1, -1, 1, -1},
};

static const int (*velocities(int Q))[2] { return Q == 9 ? C9 : C5; }

int orc_velocities(int Q, int *c) {
    if (Q != 5 && Q != 9) return -1;
    const int(*cv)[2] = velocities(Q);
    for (int i = 0; i < Q; i++) {
        c[2 * i] = cv[i][0];
        c[2 * i + 1] = cv[i][1];
    }
    return 0;
}

int orc_moment_matrix(int Q, double *M) {
    if (Q != 5 && Q != 9) return -1;
    for (int r = 0; r < Q; r++)
        for (int c = 0; c < Q; c++) M[r * Q + c] = (Q == 5) ? M5[r][c] : M9[r][c];
    return 0;
}

/* M^-1 by Gauss-Jordan elimination with partial pivoting (App. A gives M;
 * App. B prints the D2Q5 inverse, which the tests compare against). */
int orc_moment_inverse(int Q, double *Minv) {
    double a[9][18];
    if (Q != 5 && Q != 9) return -1;
    for (int r = 0; r < Q; r++)
        for (int c = 0; c < 2 * Q; c++)
            a[r][c] = (c < Q) ? ((Q == 5) ? M5[r][c] : M9[r][c]) : (c - Q == r ? 1.0 : 0.0);
    for (int col = 0; col < Q; col++) {
        int piv = col;
        for (int r = col + 1; r < Q; r++)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (fabs(a[piv][col]) < 1e-300) return -2;
        if (piv != col)
            for (int c = 0; c < 2 * Q; c++) {
                double t = a[col][c];
                a[col][c] = a[piv][c];
                a[piv][c] = t;
            }
        double d = a[col][col];
        for (int c = 0; c < 2 * Q; c++) a[col][c] /= d;
        for (int r = 0; r < Q; r++) {
            if (r == col) continue;
            double f = a[r][col];
            if (f == 0.0) continue;
            for (int c = 0; c < 2 * Q; c++) a[r][c] -= f * a[col][c];
        }
    }
    for (int r = 0; r < Q; r++)
        for (int c = 0; c < Q; c++) Minv[r * Q + c] = a[r][Q + c];
    return 0;
}

/* Weights and lattice sound speed from eta (Sec. 2.3). */
int orc_weights(int Q, double eta, const double *w_ref, double *w, double *cs2) {
    const int(*cv)[2] = velocities(Q);
    if (Q == 5) {
        double w0 = 1.0 - eta * eta; /* Eq. 0th lattice weight */
        w[0] = w0;
        for (int i = 1; i < 5; i++) w[i] = (1.0 - w0) / 4.0; /* sum_i w_i = 1, symmetry */
    } else if (Q == 9) {
        double e2 = eta * eta, moving = 0.0;
        for (int i = 1; i < 5; i++) w[i] = e2 * w_ref[1];
        for (int i = 5; i < 9; i++) w[i] = e2 * w_ref[2];
        for (int i = 1; i < 9; i++) moving += w[i];
        w[0] = 1.0 - moving; /* sum_i w_i = 1 */
    } else {
        return -1;
    }
    double s = 0.0;
    for (int i = 0; i < Q; i++) s += w[i] * cv[i][0] * cv[i][0]; /* sum w c_x c_x = c_s^2 */
    *cs2 = s;
    return 0;
}

/* Eq. linear eqm dist with p = c_s^2 rho and rho_0 v = j. */
void orc_equilibrium(int Q, const double *w, double cs2, double rho, double jx, double jy,
                     double *geq) {
    const int(*cv)[2] = velocities(Q);
    double p = cs2 * rho;
    for (int i = 0; i < Q; i++) geq[i] = (w[i] / cs2) * (p + cv[i][0] * jx + cv[i][1] * jy);
}

static void moments(int Q, const double *g, double *rho, double *jx, double *jy) {
    const int(*cv)[2] = velocities(Q);
    double r = 0.0, x = 0.0, y = 0.0;
    for (int i = 0; i < Q; i++) {
        r += g[i];
        x += cv[i][0] * g[i];
        y += cv[i][1] * g[i];
    }
    *rho = r;
    *jx = x;
    *jy = y;
}

/* One-site collision: BGK (Eq. BGK-LB) or MRT (Eq. MRT-LB basic). */
static void collide_with(int Q, int mrt, double tau, const double *s, const double *Minv,
                         const double *w, double cs2, const double *g, double *gs) {
    double rho, jx, jy, geq[9];
    moments(Q, g, &rho, &jx, &jy);
    orc_equilibrium(Q, w, cs2, rho, jx, jy, geq);
    if (!mrt) {
        for (int i = 0; i < Q; i++) gs[i] = g[i] - (g[i] - geq[i]) / tau;
        return;
    }
    double m[9], meq[9], ms[9];
    for (int k = 0; k < Q; k++) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < Q; i++) {
            double Mki = (Q == 5) ? M5[k][i] : M9[k][i];
            a += Mki * g[i];
            b += Mki * geq[i];
        }
        m[k] = a;
        meq[k] = b;
    }
    for (int k = 0; k < Q; k++) ms[k] = m[k] - s[k] * (m[k] - meq[k]);
    for (int i = 0; i < Q; i++) {
        double a = 0.0;
        for (int k = 0; k < Q; k++) a += Minv[i * Q + k] * ms[k];
        gs[i] = a;
    }
}

int orc_collide(int Q, int mrt, double tau, const double *s, const double *w, double cs2,
                const double *g, double *gs) {
    double Minv[81];
    if (orc_moment_inverse(Q, Minv)) return -1;
    collide_with(Q, mrt, tau, s, Minv, w, cs2, g, gs);
    return 0;
}

/* Sponge profile (Sec. 4 "sponge layers"; the paper gives no profile):
 * sigma = sigma_max ((W - d)/W)^2 for d < W, d = distance to the nearest edge. */
double orc_sponge_sigma(int x, int y, int nx, int ny, int W, double smax) {
    if (W <= 0) return 0.0;
    int d = x;
    if (y < d) d = y;
    if (nx - 1 - x < d) d = nx - 1 - x;
    if (ny - 1 - y < d) d = ny - 1 - y;
    if (d >= W) return 0.0;
    double r = (double)(W - d) / (double)W;
    return smax * r * r;
}

static void site_weights(const orc_problem *P, size_t idx, double *w, double *cs2) {
    double eta = (double)P->c_map[idx] / P->c_ref;
    orc_weights(P->Q, eta, P->w_ref, w, cs2);
}

int orc_init_pressure(const orc_problem *P, const double *p0, double *g) {
    const size_t N = (size_t)P->nx * P->ny;
    for (size_t idx = 0; idx < N; idx++) {
        double w[9], cs2, geq[9];
        site_weights(P, idx, w, &cs2);
        double p = p0 ? p0[idx] : 0.0;
        orc_equilibrium(P->Q, w, cs2, p / cs2, 0.0, 0.0, geq); /* rho = p/c_s^2, j = 0 */
        for (int i = 0; i < P->Q; i++) g[(size_t)i * N + idx] = geq[i];
    }
    return 0;
}

int orc_pressure(const orc_problem *P, const double *g, double *p) {
    const size_t N = (size_t)P->nx * P->ny;
    for (size_t idx = 0; idx < N; idx++) {
        double w[9], cs2, rho = 0.0;
        site_weights(P, idx, w, &cs2);
        for (int i = 0; i < P->Q; i++) rho += g[(size_t)i * N + idx];
        p[idx] = cs2 * rho; /* Eq. state */
    }
    return 0;
}

static void record(const orc_problem *P, const double *g, double *row) {
    const size_t N = (size_t)P->nx * P->ny;
    for (int r = 0; r < P->nrec; r++) {
        int x = P->rec_xy[2 * r], y = P->rec_xy[2 * r + 1];
        size_t idx = (size_t)y * P->nx + x;
        double w[9], cs2, rho = 0.0;
        site_weights(P, idx, w, &cs2);
        for (int i = 0; i < P->Q; i++) rho += g[(size_t)i * N + idx];
        row[r] = cs2 * rho;
    }
}

/* One full time step t: g (time t) -> gn (time t+1). */
static void step(const orc_problem *P, const double *Minv, int t, const double *g, double *gn) {
    const int Q = P->Q, nx = P->nx, ny = P->ny;
    const size_t N = (size_t)nx * ny;
    const int(*cv)[2] = velocities(Q);
    memset(gn, 0, sizeof(double) * Q * N);
    const double S = (P->src && t >= 0 && t < P->nt_src) ? P->src[t] : 0.0;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++) {
        for (int x = 0; x < nx; x++) {
            size_t idx = (size_t)y * nx + x;
            double gl[9], gs[9], w[9], cs2;
            for (int i = 0; i < Q; i++) gl[i] = g[(size_t)i * N + idx];
            site_weights(P, idx, w, &cs2);
            collide_with(Q, P->mrt, P->tau, P->s, Minv, w, cs2, gl, gs);
            if (P->src && x == P->src_x && y == P->src_y)
                for (int i = 0; i < Q; i++) gs[i] += w[i] * S;
            double sig = orc_sponge_sigma(x, y, nx, ny, P->sponge_width, P->sponge_sigma_max);
            for (int i = 0; i < Q; i++) gs[i] *= (1.0 - sig);
            for (int i = 0; i < Q; i++) {
                int xd = x + cv[i][0], yd = y + cv[i][1];
                if (P->periodic) {
                    xd = (xd + nx) % nx;
                    yd = (yd + ny) % ny;
                } else if (xd < 0 || xd >= nx || yd < 0 || yd >= ny) {
                    continue; /* leaves the domain */
                }
                gn[(size_t)i * N + (size_t)yd * nx + xd] = gs[i];
            }
        }
    }
}

int orc_run(const orc_problem *P, double *g, int t0, int nsteps, double *trace) {
    double Minv[81];
    if (P->Q != 5 && P->Q != 9) return -1;
    if (orc_moment_inverse(P->Q, Minv)) return -2;
#ifdef _OPENMP
    if (P->nthreads > 0) omp_set_num_threads(P->nthreads);
#endif
    const size_t len = (size_t)P->Q * P->nx * P->ny;
    double *gn = (double *)malloc(sizeof(double) * len);
    if (!gn) return -3;
    for (int k = 0; k < nsteps; k++) {
        if (trace && P->nrec > 0) record(P, g, trace + (size_t)k * P->nrec);
        step(P, Minv, t0 + k, g, gn);
        memcpy(g, gn, sizeof(double) * len);
    }
    free(gn);
    return 0;
}

/* orc_run with the stored state rounded to FP32 (round to nearest even) after every step:
 * the arithmetic stays FP64, so the result differs from orc_run's by what storing the
 * populations in FP32 alone costs -- the floor below which no FP32-storage implementation
 * of the scheme can agree with orc_run after nsteps steps. */
int orc_run_f32_stored(const orc_problem *P, double *g, int t0, int nsteps, double *trace) {
    double Minv[81];
    if (P->Q != 5 && P->Q != 9) return -1;
    if (orc_moment_inverse(P->Q, Minv)) return -2;
#ifdef _OPENMP
    if (P->nthreads > 0) omp_set_num_threads(P->nthreads);
#endif
    const size_t len = (size_t)P->Q * P->nx * P->ny;
    double *gn = (double *)malloc(sizeof(double) * len);
    if (!gn) return -3;
    for (size_t i = 0; i < len; i++) g[i] = (double)(float)g[i];
    for (int k = 0; k < nsteps; k++) {
        if (trace && P->nrec > 0) record(P, g, trace + (size_t)k * P->nrec);
        step(P, Minv, t0 + k, g, gn);
        for (size_t i = 0; i < len; i++) g[i] = (double)(float)gn[i];
    }
    free(gn);
    return 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Exported for the refinement and adjoint oracles (same library). */
void orc_collide_site(int Q, int mrt, double tau, const double *s, const double *Minv,
                      const double *w, double cs2, const double *g, double *gs) {
    collide_with(Q, mrt, tau, s, Minv, w, cs2, g, gs);
}

void orc_step_grid(const orc_problem *P, const double *Minv, int t, const double *g, double *gn) {
    step(P, Minv, t, g, gn);
}

void orc_record(const orc_problem *P, const double *g, double *row) { record(P, g, row); }

void orc_site_weights(const orc_problem *P, size_t idx, double *w, double *cs2) {
    site_weights(P, idx, w, cs2);
}
