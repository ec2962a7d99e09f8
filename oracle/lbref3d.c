/*
 * lbref3d.c -- FP64 oracle of the three-dimensional linear LB acoustic scheme
 * on the D3Q7 lattice.  TEST INFRASTRUCTURE: used only by the tests, the smoke
 * check and the CPU-baseline leg of the benchmark.
 *
 * The paper works in 2-D and states that the method carries over to 3-D
 * (DnQm lattices, Sec. 2; conclusions).  Reading: D3Q7 is the 3-D counterpart
 * of D2Q5 -- velocities 0, +-e_x, +-e_y, +-e_z -- with the weight rule of
 * Eq. 0th lattice weight carried over, w_0 = 1 - eta^2 and w_1..6 = eta^2 / 6,
 * which makes sum_i w_i c_i c_i = c_s^2 I with c_s^2 = eta^2 / 3.  The linear
 * equilibrium is Eq. linear eqm dist, g^eq_i = w_i rho + (w_i / c_s^2) c_i . j,
 * and the collision is BGK (Eq. BGK-LB).  Source (post-collision w_i S[t] at the
 * source node), sponge ((1 - sigma) after collision, sigma = sigma_max
 * ((W - d) / W)^2 with d the distance to the nearest face) and receivers
 * (p = c_s^2 rho of the state entering step t) follow the 2-D oracle.
 * Push streaming: populations leaving a zero-ghost domain are dropped.
 */
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "lbref.h"

static const int V7[7][3] = {{0, 0, 0},  {1, 0, 0}, {0, 1, 0}, {-1, 0, 0},
                             {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

static void weights3(const orc3_problem *P, size_t idx, double w[7], double *cs2) {
    const double eta = (double)P->c_map[idx] / P->c_ref, e2 = eta * eta;
    w[0] = 1.0 - e2;
    for (int i = 1; i < 7; i++) w[i] = e2 / 6.0;
    *cs2 = e2 / 3.0;
}

static double sponge3(const orc3_problem *P, int x, int y, int z) {
    const int W = P->sponge_width;
    if (W <= 0) return 0.0;
    int d = x;
    if (P->nx - 1 - x < d) d = P->nx - 1 - x;
    if (y < d) d = y;
    if (P->ny - 1 - y < d) d = P->ny - 1 - y;
    if (z < d) d = z;
    if (P->nz - 1 - z < d) d = P->nz - 1 - z;
    if (d >= W) return 0.0;
    const double r = (double)(W - d) / (double)W;
    return P->sponge_sigma_max * r * r;
}

static size_t sites(const orc3_problem *P) { return (size_t)P->nx * P->ny * P->nz; }

int orc3_init_pressure(const orc3_problem *P, const double *p0, double *g) {
    const size_t N = sites(P);
    for (size_t idx = 0; idx < N; idx++) {
        double w[7], cs2;
        weights3(P, idx, w, &cs2);
        const double rho = (p0 ? p0[idx] : 0.0) / cs2;  /* j = 0 */
        for (int i = 0; i < 7; i++) g[(size_t)i * N + idx] = w[i] * rho;
    }
    return 0;
}

int orc3_pressure(const orc3_problem *P, const double *g, double *p) {
    const size_t N = sites(P);
    for (size_t idx = 0; idx < N; idx++) {
        double w[7], cs2, rho = 0.0;
        weights3(P, idx, w, &cs2);
        for (int i = 0; i < 7; i++) rho += g[(size_t)i * N + idx];
        p[idx] = cs2 * rho;
    }
    return 0;
}

static void record3(const orc3_problem *P, const double *g, double *row) {
    const size_t N = sites(P);
    for (int r = 0; r < P->nrec; r++) {
        const int x = P->rec_xyz[3 * r], y = P->rec_xyz[3 * r + 1], z = P->rec_xyz[3 * r + 2];
        const size_t idx = ((size_t)z * P->ny + y) * P->nx + x;
        double w[7], cs2, rho = 0.0;
        weights3(P, idx, w, &cs2);
        for (int i = 0; i < 7; i++) rho += g[(size_t)i * N + idx];
        row[r] = cs2 * rho;
    }
}

/* one step t: g (time t) -> gn (time t + 1) */
static void step3(const orc3_problem *P, int t, const double *g, double *gn) {
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const size_t N = sites(P);
    memset(gn, 0, sizeof(double) * 7 * N);
    const double S = (P->src && t >= 0 && t < P->nt_src) ? P->src[t] : 0.0;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; z++) {
        for (int y = 0; y < ny; y++) {
            for (int x = 0; x < nx; x++) {
                const size_t idx = ((size_t)z * ny + y) * nx + x;
                double gl[7], w[7], cs2, rho = 0.0, j[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < 7; i++) {
                    gl[i] = g[(size_t)i * N + idx];
                    rho += gl[i];
                    for (int d = 0; d < 3; d++) j[d] += V7[i][d] * gl[i];
                }
                weights3(P, idx, w, &cs2);
                const double sig = sponge3(P, x, y, z);
                for (int i = 0; i < 7; i++) {
                    const double cj = V7[i][0] * j[0] + V7[i][1] * j[1] + V7[i][2] * j[2];
                    const double geq = w[i] * rho + w[i] / cs2 * cj;
                    double v = gl[i] - (gl[i] - geq) / P->tau;
                    if (P->src && x == P->src_x && y == P->src_y && z == P->src_z) v += w[i] * S;
                    v *= 1.0 - sig;
                    int xd = x + V7[i][0], yd = y + V7[i][1], zd = z + V7[i][2];
                    if (P->periodic) {
                        xd = (xd + nx) % nx;
                        yd = (yd + ny) % ny;
                        zd = (zd + nz) % nz;
                    } else if (xd < 0 || xd >= nx || yd < 0 || yd >= ny || zd < 0 || zd >= nz) {
                        continue;
                    }
                    gn[(size_t)i * N + ((size_t)zd * ny + yd) * nx + xd] = v;
                }
            }
        }
    }
}

int orc3_run(const orc3_problem *P, double *g, int t0, int nsteps, double *trace) {
#ifdef _OPENMP
    if (P->nthreads > 0) omp_set_num_threads(P->nthreads);
#endif
    const size_t len = 7 * sites(P);
    double *gn = (double *)malloc(sizeof(double) * len);
    if (!gn) return -3;
    for (int k = 0; k < nsteps; k++) {
        if (trace && P->nrec > 0) record3(P, g, trace + (size_t)k * P->nrec);
        step3(P, t0 + k, g, gn);
        memcpy(g, gn, sizeof(double) * len);
    }
    free(gn);
    return 0;
}
