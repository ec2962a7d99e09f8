/*
 * lbrefine.c -- FP64 oracle of the two-level grid refinement of Sec. 4 of
 * arXiv:1704.03172 (after Dupuis and Chopard).  TEST INFRASTRUCTURE: used only
 * by the tests, the smoke check and the CPU-baseline leg of the benchmark.
 *
 * Geometry.  The coarse grid covers the whole domain.  A patch of coarse cells
 * [x0, x0 + nxp] x [y0, y0 + nyp] (closed rectangle of coarse nodes) is covered
 * by a fine grid with spacing and time step halved (n = 2): fine node (a, b),
 * 0 <= a <= 2 nxp, 0 <= b <= 2 nyp, sits at coarse position
 * (x0 + a/2, y0 + b/2).  The fine sound speed is the coarse c_map interpolated
 * bilinearly to the fine nodes (rounded to float), so both grids share eta and
 * hence the lattice sound speed; the physical speed is continuous.
 * The interface I is the rectangle's boundary, a line of nodes of both grids.
 *
 * Coupling (Eq. grid refinement eqm dist, Eq. coarse-fine dist connect): the
 * equilibrium part is shared and the non-equilibrium part is scaled,
 *   fine   <- coarse:  g^f = g^eq + (g^c - g^eq) / n,
 *   coarse <- fine:    g^c = g^eq + (g^f - g^eq) * n,
 * with g^eq formed from the moments of the transferred vector and the
 * receiving grid's weights.  Sec. 4 lets the direction in which waves cross the
 * interface decide which grid supplies a value; that choice is read here per
 * population (reading R3): at a fine node of I the populations whose upstream
 * node x - c_i lies outside the fine grid come from the coarse grid; at a
 * coarse node of I the populations whose upstream node lies strictly inside
 * the patch come from the fine grid.  The coarse grid keeps evolving under the
 * patch (its overlap with the fine domain), which supplies the full coarse
 * vector at I for the coarse -> fine transfer.
 *
 * Time sequence per coarse step T -> T+1 (Sec. 4, itemised procedure):
 *   record the pressure at time T;
 *   coarse collide + stream -> coarse state at T+1 (provisional on I); keep its
 *     values on I, U(T+1);
 *   fine step 2T -> 2T+1, then set the coarse-side populations on I from the
 *     spatial (linear along I) and temporal (midpoint) interpolation of U(T),
 *     U(T+1);
 *   fine step 2T+1 -> 2T+2, then the same from U(T+1);
 *   correct the coarse populations on I from the fine state at 2T+2.
 * The same coupling is applied once to the initial state (time 0).
 *
 * Nested patches ("multiples of 2", Sec. 4): orc_ref_nest places a further patch inside the
 * innermost fine grid, in that grid's node coordinates, refined by 2 again (ratio 4, 8, ...
 * to the coarse grid).  Each pair of adjacent levels is coupled exactly as above; a "fine
 * step" of a level that holds a patch is the whole procedure for that level and its patch
 * (two steps of the next level per step, recursively).  The fine rates follow reading R6 level
 * by level: tau_{l+1} - 1/2 = 2 (tau_l - 1/2).  Receivers and pressures come from the deepest
 * level whose closed patch holds the node.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "lbref.h"

typedef struct ref_s {
    orc_problem C, F;
    struct ref_s *sub; /* nested patch inside F, or NULL */
    int rule;
    /* direction of the coupling (Sec. 4, the switch on which way waves cross the interface):
     * 0 both ways, population by population (reading R3); 1 coarse -> fine only (the
     * coarse grid is never corrected from the fine one); 2 fine -> coarse only (no coarse
     * population enters the fine grid: what enters it across I is zero, the zero ghost) */
    int dir;
    int x0, y0, nxp, nyp, nxf, nyf, nI;
    float *cf;
    double *gc, *gf, *tc, *tf, *Uprev, *Unext;
    int *Ix, *Iy, *idxI;
    double M[81], Minv[81];
    /* non-equilibrium factors per moment (MRT) or for all populations (BGK, entry 0):
     * coarse -> fine and fine -> coarse */
    double fc2f[9], ff2c[9];
    long t;
} ref_t;

/* Relaxation time of a rate and its fine-grid counterpart.  With dx and dt halved, the
 * physical viscosity c_s^2 (tau - 1/2) dx^2 / dt is the same on both grids when
 * tau_f - 1/2 = n (tau_c - 1/2) (reading R6); the non-equilibrium parts then scale
 * as g_neq_f = tau_f / (n tau_c) g_neq_c (Chapman-Enskog: g_neq ~ tau dt times
 * gradients that are n times smaller per fine cell).  At tau = 1/2 (s = 2, the
 * paper's lossless setting) this is the paper's factor 1/n, and tau_f = tau_c. */
static double fine_tau(double tau_c) { return 0.5 + 2.0 * (tau_c - 0.5); }

/* n_k(g - geq): the non-equilibrium part rescaled by fac (per moment for MRT) */
static void rescale_neq(const ref_t *R, const double *fac, const double *g, const double *geq,
                        double *out) {
    const int Q = R->C.Q;
    if (!R->C.mrt) {
        for (int i = 0; i < Q; i++) out[i] = geq[i] + fac[0] * (g[i] - geq[i]);
        return;
    }
    double m[9];
    for (int k = 0; k < Q; k++) {
        double v = 0;
        for (int i = 0; i < Q; i++) v += R->M[k * Q + i] * (g[i] - geq[i]);
        m[k] = fac[k] * v;
    }
    for (int i = 0; i < Q; i++) {
        double v = 0;
        for (int k = 0; k < Q; k++) v += R->Minv[i * Q + k] * m[k];
        out[i] = geq[i] + v;
    }
}

static const int V5[5][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}};
static const int V9[9][2] = {{0, 0},  {1, 0},  {0, 1},   {-1, 0}, {0, -1},
                             {1, 1},  {-1, 1}, {-1, -1}, {1, -1}};

static const int (*vel(int Q))[2] { return Q == 9 ? V9 : V5; }

static int on_I(const ref_t *R, int X, int Y) {
    if (X < R->x0 || X > R->x0 + R->nxp || Y < R->y0 || Y > R->y0 + R->nyp) return 0;
    return X == R->x0 || X == R->x0 + R->nxp || Y == R->y0 || Y == R->y0 + R->nyp;
}

static int strictly_inside(const ref_t *R, int X, int Y) {
    return X > R->x0 && X < R->x0 + R->nxp && Y > R->y0 && Y < R->y0 + R->nyp;
}

static int in_closed_patch(const ref_t *R, int X, int Y) {
    return X >= R->x0 && X <= R->x0 + R->nxp && Y >= R->y0 && Y <= R->y0 + R->nyp;
}

/* Eq. coarse-fine dist connect for one vector g that arrives at node idx of the receiving
 * grid (the fine grid when to_fine, else the coarse one): g^eq is formed from g's own
 * moments with the receiving grid's weights (Eq. grid refinement eqm dist), and the
 * non-equilibrium part g - g^eq is scaled by that direction's factors (1/n and n at
 * tau = 1/2; reading R6 otherwise). */
static void transfer(const ref_t *R, int to_fine, size_t idx, const double *g, double *out) {
    const int Q = R->C.Q;
    const int(*cv)[2] = vel(Q);
    double rho = 0, jx = 0, jy = 0;
    for (int i = 0; i < Q; i++) {
        rho += g[i];
        jx += cv[i][0] * g[i];
        jy += cv[i][1] * g[i];
    }
    double w[9], cs2, geq[9];
    orc_site_weights(to_fine ? &R->F : &R->C, idx, w, &cs2);
    orc_equilibrium(Q, w, cs2, rho, jx, jy, geq);
    rescale_neq(R, to_fine ? R->fc2f : R->ff2c, g, geq, out);
}

static const double *U_at(const ref_t *R, const double *U, int X, int Y) {
    int k = R->idxI[(Y - R->y0) * (R->nxp + 1) + (X - R->x0)];
    return U + (size_t)k * R->C.Q;
}

static void snapshot(const ref_t *R, const double *gc, double *U) {
    const int Q = R->C.Q;
    const size_t N = (size_t)R->C.nx * R->C.ny;
    for (int k = 0; k < R->nI; k++)
        for (int i = 0; i < Q; i++)
            U[(size_t)k * Q + i] = gc[(size_t)i * N + (size_t)R->Iy[k] * R->C.nx + R->Ix[k]];
}

/* coarse -> fine on I: ghat = (1 - alpha) Ua + alpha Ub, interpolated along I */
static void c2f(const ref_t *R, double *gf, const double *Ua, const double *Ub, double alpha) {
    const int Q = R->C.Q;
    const int(*cv)[2] = vel(Q);
    const size_t Nf = (size_t)R->nxf * R->nyf;
    for (int b = 0; b < R->nyf; b++) {
        for (int a = 0; a < R->nxf; a++) {
            if (!(a == 0 || a == R->nxf - 1 || b == 0 || b == R->nyf - 1)) continue;
            int X = R->x0 + a / 2, Y = R->y0 + b / 2;
            const double *pa[2], *pb[2];
            int np = 1;
            pa[0] = U_at(R, Ua, X, Y);
            pb[0] = U_at(R, Ub, X, Y);
            if (a % 2 == 1) {
                pa[1] = U_at(R, Ua, X + 1, Y);
                pb[1] = U_at(R, Ub, X + 1, Y);
                np = 2;
            } else if (b % 2 == 1) {
                pa[1] = U_at(R, Ua, X, Y + 1);
                pb[1] = U_at(R, Ub, X, Y + 1);
                np = 2;
            }
            double gh[9], gr[9];
            for (int i = 0; i < Q; i++) {
                double s = 0;
                for (int k = 0; k < np; k++) s += (1.0 - alpha) * pa[k][i] + alpha * pb[k][i];
                gh[i] = s / np;
            }
            transfer(R, 1, (size_t)b * R->nxf + a, gh, gr);
            for (int i = 0; i < Q; i++) {
                int ua = a - cv[i][0], ub = b - cv[i][1];
                if (ua >= 0 && ua < R->nxf && ub >= 0 && ub < R->nyf) continue;  /* from fine */
                gf[(size_t)i * Nf + (size_t)b * R->nxf + a] = gr[i];
            }
        }
    }
}

/* fine -> coarse on I */
static void f2c(const ref_t *R, double *gc, const double *gf) {
    const int Q = R->C.Q;
    const int(*cv)[2] = vel(Q);
    const size_t N = (size_t)R->C.nx * R->C.ny, Nf = (size_t)R->nxf * R->nyf;
    for (int k = 0; k < R->nI; k++) {
        int X = R->Ix[k], Y = R->Iy[k];
        size_t fidx = (size_t)(2 * (Y - R->y0)) * R->nxf + 2 * (X - R->x0);
        double G[9], gr[9];
        for (int i = 0; i < Q; i++) G[i] = gf[(size_t)i * Nf + fidx];
        size_t cidx = (size_t)Y * R->C.nx + X;
        transfer(R, 0, cidx, G, gr);
        for (int i = 0; i < Q; i++)
            if (strictly_inside(R, X - cv[i][0], Y - cv[i][1])) gc[(size_t)i * N + cidx] = gr[i];
    }
}

void *orc_ref_create(const orc_problem *coarse, int x0, int y0, int nxp, int nyp, int rule) {
    if (!coarse || nxp < 1 || nyp < 1 || x0 < 1 || y0 < 1 || x0 + nxp > coarse->nx - 2 ||
        y0 + nyp > coarse->ny - 2)
        return NULL;
    ref_t *R = (ref_t *)calloc(1, sizeof(ref_t));
    R->C = *coarse;
    R->x0 = x0;
    R->y0 = y0;
    R->nxp = nxp;
    R->nyp = nyp;
    R->nxf = 2 * nxp + 1;
    R->nyf = 2 * nyp + 1;
    R->rule = rule;
    const int Q = coarse->Q, nx = coarse->nx;
    const size_t N = (size_t)nx * coarse->ny, Nf = (size_t)R->nxf * R->nyf;
    /* fine medium: bilinear interpolation of the coarse sound speed */
    R->cf = (float *)malloc(sizeof(float) * Nf);
    for (int b = 0; b < R->nyf; b++)
        for (int a = 0; a < R->nxf; a++) {
            int X = x0 + a / 2, Y = y0 + b / 2, ox = a % 2, oy = b % 2;
            double s = 0;
            int cnt = 0;
            for (int dy = 0; dy <= oy; dy++)
                for (int dx = 0; dx <= ox; dx++) {
                    s += (double)coarse->c_map[(size_t)(Y + dy) * nx + X + dx];
                    cnt++;
                }
            R->cf[(size_t)b * R->nxf + a] = (float)(s / cnt);
        }
    memset(&R->F, 0, sizeof(R->F));
    R->F.Q = Q;
    R->F.nx = R->nxf;
    R->F.ny = R->nyf;
    R->F.periodic = 0;
    R->F.mrt = coarse->mrt;
    R->F.tau = coarse->tau;
    memcpy(R->F.s, coarse->s, sizeof(R->F.s));
    memcpy(R->F.w_ref, coarse->w_ref, sizeof(R->F.w_ref));
    R->F.c_map = R->cf;
    R->F.c_ref = coarse->c_ref;
    R->F.nthreads = coarse->nthreads;
    /* interface nodes */
    R->idxI = (int *)malloc(sizeof(int) * (nxp + 1) * (nyp + 1));
    R->Ix = (int *)malloc(sizeof(int) * 2 * (nxp + nyp + 2));
    R->Iy = (int *)malloc(sizeof(int) * 2 * (nxp + nyp + 2));
    for (int Y = y0; Y <= y0 + nyp; Y++)
        for (int X = x0; X <= x0 + nxp; X++) {
            int *slot = &R->idxI[(Y - y0) * (nxp + 1) + (X - x0)];
            *slot = -1;
            if (on_I(R, X, Y)) {
                *slot = R->nI;
                R->Ix[R->nI] = X;
                R->Iy[R->nI] = Y;
                R->nI++;
            }
        }
    R->gc = (double *)calloc((size_t)Q * N, sizeof(double));
    R->tc = (double *)calloc((size_t)Q * N, sizeof(double));
    R->gf = (double *)calloc((size_t)Q * Nf, sizeof(double));
    R->tf = (double *)calloc((size_t)Q * Nf, sizeof(double));
    R->Uprev = (double *)calloc((size_t)Q * R->nI, sizeof(double));
    R->Unext = (double *)calloc((size_t)Q * R->nI, sizeof(double));
    orc_moment_matrix(Q, R->M);
    orc_moment_inverse(Q, R->Minv);
    /* rule 0 (R6): viscosity-continuous fine rates and per-moment factors; rule 1: the
     * paper's printed factors 1/2 and 2 with the coarse rates on both grids (exact for
     * tau = 1/2 / s = 2, where both rules coincide) */
    if (rule == 0) {
        R->F.tau = fine_tau(coarse->tau);
        for (int k = 0; k < Q; k++) R->F.s[k] = 1.0 / fine_tau(1.0 / coarse->s[k]);
    }
    for (int k = 0; k < 9; k++) {
        double tc = coarse->mrt ? (k < Q ? 1.0 / coarse->s[k] : 1.0) : coarse->tau;
        double tf = rule == 0 ? fine_tau(tc) : tc;
        R->fc2f[k] = rule == 0 ? tf / (2.0 * tc) : 0.5;
        R->ff2c[k] = rule == 0 ? 2.0 * tc / tf : 2.0;
    }
    return R;
}

void orc_ref_destroy(void *h) {
    ref_t *R = (ref_t *)h;
    if (!R) return;
    orc_ref_destroy(R->sub);
    free(R->cf);
    free(R->idxI);
    free(R->Ix);
    free(R->Iy);
    free(R->gc);
    free(R->tc);
    free(R->gf);
    free(R->tf);
    free(R->Uprev);
    free(R->Unext);
    free(R);
}

int orc_ref_dims(void *h, int *nxf, int *nyf) {
    ref_t *R = (ref_t *)h;
    *nxf = R->nxf;
    *nyf = R->nyf;
    return R->nI;
}

int orc_ref_fine_cmap(void *h, float *cf) {
    ref_t *R = (ref_t *)h;
    memcpy(cf, R->cf, sizeof(float) * R->nxf * R->nyf);
    return 0;
}

/* The start of a run from states already set on every level: for each pair of adjacent
 * levels, innermost first, the snapshot U(0) of the coarser side on I and the coupling at
 * time 0 (when `couple`; the couplings of different pairs touch different nodes when every
 * patch keeps a margin of at least one node, so their order is immaterial). */
static void start_level(ref_t *R, double *gcs, int couple) {
    if (R->sub) start_level(R->sub, R->gf, couple);
    snapshot(R, gcs, R->Uprev);
    if (!couple) return;
    if (R->dir != 2) c2f(R, R->gf, R->Uprev, R->Uprev, 1.0);
    if (R->dir != 1) f2c(R, gcs, R->gf);
}

/* Fine grid of R from the pressure pc on R's coarse grid (NULL: zero): g = g^eq(p / c_s^2, 0)
 * with p interpolated bilinearly, the same for every nested level. */
static void init_level(ref_t *R, const double *pc) {
    const int nx = R->C.nx;
    const size_t Nf = (size_t)R->nxf * R->nyf;
    double *pf = NULL;
    if (pc) {
        pf = (double *)malloc(sizeof(double) * Nf);
        for (int b = 0; b < R->nyf; b++)
            for (int a = 0; a < R->nxf; a++) {
                int X = R->x0 + a / 2, Y = R->y0 + b / 2, ox = a % 2, oy = b % 2, cnt = 0;
                double s = 0;
                for (int dy = 0; dy <= oy; dy++)
                    for (int dx = 0; dx <= ox; dx++) {
                        s += pc[(size_t)(Y + dy) * nx + X + dx];
                        cnt++;
                    }
                pf[(size_t)b * R->nxf + a] = s / cnt;
            }
    }
    orc_init_pressure(&R->F, pf, R->gf);
    if (R->sub) init_level(R->sub, pf);
    free(pf);
}

/* g = g^eq(p0 / c_s^2, 0) on every grid (p0 interpolated bilinearly to the fine
 * nodes, level by level), then the coupling at time 0. */
int orc_ref_init_pressure(void *h, const double *p0) {
    ref_t *R = (ref_t *)h;
    orc_init_pressure(&R->C, p0, R->gc);
    init_level(R, p0);
    start_level(R, R->gc, 1);
    R->t = 0;
    return 0;
}

/* pressure at node (a, b) of R's fine grid, from the deepest level holding it */
static double fine_p(const ref_t *R, int a, int b) {
    if (R->sub && in_closed_patch(R->sub, a, b))
        return fine_p(R->sub, 2 * (a - R->sub->x0), 2 * (b - R->sub->y0));
    const size_t Nf = (size_t)R->nxf * R->nyf, fidx = (size_t)b * R->nxf + a;
    double w[9], cs2, rho = 0;
    orc_site_weights(&R->F, fidx, w, &cs2);
    for (int i = 0; i < R->C.Q; i++) rho += R->gf[(size_t)i * Nf + fidx];
    return cs2 * rho;
}

static void record_all(const ref_t *R, double *row) {
    const orc_problem *C = &R->C;
    const size_t N = (size_t)C->nx * C->ny;
    for (int r = 0; r < C->nrec; r++) {
        int X = C->rec_xy[2 * r], Y = C->rec_xy[2 * r + 1];
        if (in_closed_patch(R, X, Y)) {
            row[r] = fine_p(R, 2 * (X - R->x0), 2 * (Y - R->y0));
        } else {
            double w[9], cs2, rho = 0;
            size_t idx = (size_t)Y * C->nx + X;
            orc_site_weights(C, idx, w, &cs2);
            for (int i = 0; i < C->Q; i++) rho += R->gc[(size_t)i * N + idx];
            row[r] = cs2 * rho;
        }
    }
}

static void pair_advance(ref_t *R, double *gin, double *gout, long T);

/* one step of R's fine grid from fin to fout, with every level nested in it */
static void fine_advance(ref_t *R, double *fin, double *fout, long t) {
    if (R->sub)
        pair_advance(R->sub, fin, fout, t);
    else
        orc_step_grid(&R->F, R->Minv, 0, fin, fout);
}

/* R's coarse grid from time T (gin) to T+1 (gout), its fine grid from 2T to 2T+2 */
static void pair_advance(ref_t *R, double *gin, double *gout, long T) {
    orc_step_grid(&R->C, R->Minv, (int)T, gin, gout); /* provisional coarse T+1 */
    snapshot(R, gout, R->Unext);
    fine_advance(R, R->gf, R->tf, 2 * T); /* fine 2T -> 2T+1 */
    if (R->dir != 2) c2f(R, R->tf, R->Uprev, R->Unext, 0.5);
    fine_advance(R, R->tf, R->gf, 2 * T + 1); /* fine 2T+1 -> 2T+2 */
    if (R->dir != 2) c2f(R, R->gf, R->Uprev, R->Unext, 1.0);
    if (R->dir != 1) f2c(R, gout, R->gf);
    double *s = R->Uprev;
    R->Uprev = R->Unext;
    R->Unext = s;
}

int orc_ref_run(void *h, int nsteps, double *trace) {
    ref_t *R = (ref_t *)h;
    for (int k = 0; k < nsteps; k++) {
        if (trace && R->C.nrec > 0) record_all(R, trace + (size_t)k * R->C.nrec);
        pair_advance(R, R->gc, R->tc, R->t);
        double *s = R->gc;
        R->gc = R->tc;
        R->tc = s;
        R->t++;
    }
    return 0;
}

/* pressure on the coarse grid; nodes of the closed patch from the finest level holding them */
int orc_ref_pressure(void *h, double *p) {
    ref_t *R = (ref_t *)h;
    orc_pressure(&R->C, R->gc, p);
    for (int Y = R->y0; Y <= R->y0 + R->nyp; Y++)
        for (int X = R->x0; X <= R->x0 + R->nxp; X++)
            p[(size_t)Y * R->C.nx + X] = fine_p(R, 2 * (X - R->x0), 2 * (Y - R->y0));
    return 0;
}

int orc_ref_fine_pressure(void *h, double *pf) {
    ref_t *R = (ref_t *)h;
    return orc_pressure(&R->F, R->gf, pf);
}

int orc_ref_states(void *h, double *gc, double *gf) {
    ref_t *R = (ref_t *)h;
    if (gc) memcpy(gc, R->gc, sizeof(double) * R->C.Q * R->C.nx * R->C.ny);
    if (gf) memcpy(gf, R->gf, sizeof(double) * R->C.Q * R->nxf * R->nyf);
    return 0;
}

/* A patch of nodes [x0, x0 + nxp] x [y0, y0 + nyp] of the innermost fine grid, refined by 2
 * again (same rule).  Call before orc_ref_init_pressure.  Returns the new level's index
 * (2 for the first nested patch), or -1 for a patch without a one-node margin. */
int orc_ref_nest(void *h, int x0, int y0, int nxp, int nyp) {
    ref_t *R = (ref_t *)h;
    int level = 1;
    while (R->sub) {
        R = R->sub;
        level++;
    }
    ref_t *S = (ref_t *)orc_ref_create(&R->F, x0, y0, nxp, nyp, R->rule);
    if (!S) return -1;
    R->sub = S;
    return level + 1;
}

/* Direction of the coupling between level `level` - 1 and `level` (1: the first patch):
 * 0 both ways, 1 coarse -> fine only, 2 fine -> coarse only.  Before init_pressure. */
int orc_ref_direction(void *h, int level, int dir) {
    ref_t *R = (ref_t *)h;
    if (dir < 0 || dir > 2 || level < 1) return -1;
    for (int l = 1; l < level && R; l++) R = R->sub;
    if (!R) return -1;
    R->dir = dir;
    return 0;
}

static const ref_t *level_of(const ref_t *R, int level) {
    for (int l = 1; l < level && R; l++) R = R->sub;
    return R;
}

/* node counts of level >= 1 (level 1 is the first patch's fine grid) */
int orc_ref_level_dims(void *h, int level, int *nx, int *ny) {
    const ref_t *R = level_of((const ref_t *)h, level);
    if (!R || level < 1) return -1;
    *nx = R->nxf;
    *ny = R->nyf;
    return 0;
}

/* pressure of level >= 1 on its own nodes [ny][nx] */
int orc_ref_level_pressure(void *h, int level, double *p) {
    const ref_t *R = level_of((const ref_t *)h, level);
    if (!R || level < 1) return -1;
    return orc_pressure(&R->F, R->gf, p);
}

int orc_ref_level_cmap(void *h, int level, float *c) {
    const ref_t *R = level_of((const ref_t *)h, level);
    if (!R || level < 1) return -1;
    memcpy(c, R->cf, sizeof(float) * R->nxf * R->nyf);
    return 0;
}

/* ---- Access to the individual transfer functions, for the tests that pin them ---- */

/* the state array of level `level` (0: the coarse grid, l >= 1: the fine grid of patch l) and
 * its node counts */
static double *level_state(ref_t *R, int level, int *nx, int *ny) {
    if (level == 0) {
        *nx = R->C.nx;
        *ny = R->C.ny;
        return R->gc;
    }
    ref_t *L = (ref_t *)level_of(R, level);
    if (!L) return NULL;
    *nx = L->nxf;
    *ny = L->nyf;
    return L->gf;
}

/* Copy a state [Q][ny][nx] into (set != 0) or out of level `level` (0: coarse). */
int orc_ref_level_state(void *h, int level, int set, double *g) {
    ref_t *R = (ref_t *)h;
    int nx = 0, ny = 0;
    double *st = level < 0 ? NULL : level_state(R, level, &nx, &ny);
    if (!st || !g) return -1;
    const size_t n = sizeof(double) * (size_t)R->C.Q * nx * ny;
    if (set)
        memcpy(st, g, n);
    else
        memcpy(g, st, n);
    return 0;
}

/* Start a run (time 0) from the states set with orc_ref_level_state: the snapshots U(0) and,
 * when couple != 0, the coupling at time 0, exactly as orc_ref_init_pressure does. */
int orc_ref_start(void *h, int couple) {
    ref_t *R = (ref_t *)h;
    start_level(R, R->gc, couple);
    R->t = 0;
    return 0;
}

/* The transfer of one vector g[Q] into node (ax, ay) of the receiving grid of the pair
 * coupling level `level` to the level above it: the fine grid of patch `level` when
 * to_fine, else the grid above (its node coordinates). */
int orc_ref_transfer(void *h, int level, int to_fine, int ax, int ay, const double *g,
                     double *out) {
    const ref_t *R = level_of((const ref_t *)h, level);
    if (!R || level < 1) return -1;
    const orc_problem *P = to_fine ? &R->F : &R->C;
    if (ax < 0 || ax >= P->nx || ay < 0 || ay >= P->ny) return -1;
    transfer(R, to_fine, (size_t)ay * P->nx + ax, g, out);
    return 0;
}

/* The interface nodes I of patch `level` in the coordinates of the grid above, in the
 * order of the rows of the snapshots U; returns their number (Ix, Iy may be NULL). */
int orc_ref_interface(void *h, int level, int *Ix, int *Iy) {
    const ref_t *R = level_of((const ref_t *)h, level);
    if (!R || level < 1) return -1;
    for (int k = 0; k < R->nI; k++) {
        if (Ix) Ix[k] = R->Ix[k];
        if (Iy) Iy[k] = R->Iy[k];
    }
    return R->nI;
}

/* One coarse -> fine transfer into the fine grid of patch `level` from snapshots
 * Ua, Ub [nI][Q] at weight alpha (the values (1 - alpha) Ua + alpha Ub), as the run applies
 * it; or one fine -> coarse correction of the grid above from that fine grid. */
int orc_ref_apply_c2f(void *h, int level, const double *Ua, const double *Ub, double alpha) {
    ref_t *R = (ref_t *)level_of((const ref_t *)h, level);
    if (!R || level < 1 || !Ua || !Ub) return -1;
    c2f(R, R->gf, Ua, Ub, alpha);
    return 0;
}

int orc_ref_apply_f2c(void *h, int level) {
    ref_t *top = (ref_t *)h;
    ref_t *R = (ref_t *)level_of(top, level);
    if (!R || level < 1) return -1;
    int nx, ny;
    f2c(R, level_state(top, level - 1, &nx, &ny), R->gf);
    return 0;
}
