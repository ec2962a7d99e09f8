/*
 * lbref.h -- interface of the FP64 CPU oracle for the linear LB acoustic
 * scheme (arXiv:1704.03172).  TEST INFRASTRUCTURE: only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark use it.  It is independent
 * of the CUDA library and of include/lbac.h.
 *
 * Arrays: populations g[Q][ny][nx] (x fastest), FP64, pre-collision state at
 * the current time.  c_map[ny][nx] FP32 sound speeds (the same values the CUDA
 * path receives).  rec_xy[nrec][2] = (x, y).  trace[nsteps][nrec].
 */
#ifndef LBREF_H
#define LBREF_H
#include <stddef.h>

typedef struct {
    int Q;                 /* 5 (D2Q5) or 9 (D2Q9) */
    int nx, ny;
    int periodic;          /* 1: periodic; 0: zero ghost outside the domain */
    int mrt;               /* 0: BGK, 1: MRT */
    double tau;            /* BGK relaxation time */
    double s[9];           /* MRT rates: diagonal of S in moment order (App. A) */
    double w_ref[3];       /* D2Q9 weights (w0, w1, w5) at eta = 1 */
    const float *c_map;    /* [ny][nx] sound speed */
    double c_ref;          /* eta = c / c_ref */
    int sponge_width;      /* W; 0 = no sponge */
    double sponge_sigma_max;
    int src_x, src_y;
    const double *src;     /* S^n for n < nt_src; NULL: no source */
    int nt_src;
    const int *rec_xy;     /* [nrec][2] */
    int nrec;
    int nthreads;          /* OpenMP threads, <= 0: runtime default */
} orc_problem;

int orc_velocities(int Q, int *c);
int orc_moment_matrix(int Q, double *M);
int orc_moment_inverse(int Q, double *Minv);
int orc_weights(int Q, double eta, const double *w_ref, double *w, double *cs2);
void orc_equilibrium(int Q, const double *w, double cs2, double rho, double jx, double jy,
                     double *geq);
int orc_collide(int Q, int mrt, double tau, const double *s, const double *w, double cs2,
                const double *g, double *gs);
double orc_sponge_sigma(int x, int y, int nx, int ny, int W, double smax);
int orc_init_pressure(const orc_problem *P, const double *p0, double *g);
int orc_pressure(const orc_problem *P, const double *g, double *p);
int orc_run(const orc_problem *P, double *g, int t0, int nsteps, double *trace);
/* orc_run with the state rounded to FP32 after every step (FP32-storage floor) */
int orc_run_f32_stored(const orc_problem *P, double *g, int t0, int nsteps, double *trace);
int orc_max_threads(void);

/* building blocks shared by the oracle's own files (refinement, adjoint) */
void orc_collide_site(int Q, int mrt, double tau, const double *s, const double *Minv,
                      const double *w, double cs2, const double *g, double *gs);
void orc_step_grid(const orc_problem *P, const double *Minv, int t, const double *g, double *gn);
void orc_record(const orc_problem *P, const double *g, double *row);
void orc_site_weights(const orc_problem *P, size_t idx, double *w, double *cs2);

/* Grid refinement (Sec. 4), lbrefine.c: two levels, or more with nested patches.  Opaque
 * handle. */
/* rule 0: viscosity-continuous fine rates and non-equilibrium factors (reading R6);
 * rule 1: the paper's printed factors 1/2 and 2 with the coarse rates on both grids.
 * Both coincide at tau = 1/2 (MRT: s = 2 for every relaxed moment). */
void *orc_ref_create(const orc_problem *coarse, int x0, int y0, int nxp, int nyp, int rule);
void orc_ref_destroy(void *h);
int orc_ref_dims(void *h, int *nxf, int *nyf);
int orc_ref_fine_cmap(void *h, float *cf);
int orc_ref_init_pressure(void *h, const double *p0);
int orc_ref_run(void *h, int nsteps, double *trace);
int orc_ref_pressure(void *h, double *p);
int orc_ref_fine_pressure(void *h, double *pf);
int orc_ref_states(void *h, double *gc, double *gf);
/* nested patches: a patch of the innermost fine grid (its node coordinates), refined by 2 */
int orc_ref_nest(void *h, int x0, int y0, int nxp, int nyp);
/* coupling direction of level `level` (1: the first patch): 0 both ways (population by
 * population), 1 coarse -> fine only, 2 fine -> coarse only (Sec. 4) */
int orc_ref_direction(void *h, int level, int dir);
int orc_ref_level_dims(void *h, int level, int *nx, int *ny);
int orc_ref_level_pressure(void *h, int level, double *p);
int orc_ref_level_cmap(void *h, int level, float *c);
/* access to the individual transfer functions (for the tests that pin them) */
int orc_ref_level_state(void *h, int level, int set, double *g);
int orc_ref_start(void *h, int couple);
int orc_ref_transfer(void *h, int level, int to_fine, int ax, int ay, const double *g,
                     double *out);
int orc_ref_interface(void *h, int level, int *Ix, int *Iy);
int orc_ref_apply_c2f(void *h, int level, const double *Ua, const double *Ub, double alpha);
int orc_ref_apply_f2c(void *h, int level);

/* Discrete adjoint (lbadjoint.c): gradients of J with dJ/dp^t_r = resid[t][r]
 * for nt steps from g0.  grad_c [ny][nx]; grad_src [nt] and grad_g0 [Q][ny][nx]
 * may be NULL. */
int orc_adjoint(const orc_problem *P, const double *g0, int nt, const double *resid,
                double *grad_c, double *grad_src, double *grad_g0);

/* Three-dimensional D3Q7 BGK (lbref3d.c): arrays [nz][ny][nx], populations [7][nz][ny][nx]. */
typedef struct {
    int nx, ny, nz;
    int periodic;
    double tau;
    const float *c_map;    /* [nz][ny][nx] */
    double c_ref;
    int sponge_width;
    double sponge_sigma_max;
    int src_x, src_y, src_z;
    const double *src;
    int nt_src;
    const int *rec_xyz;    /* [nrec][3] */
    int nrec;
    int nthreads;
} orc3_problem;

int orc3_init_pressure(const orc3_problem *P, const double *p0, double *g);
int orc3_pressure(const orc3_problem *P, const double *g, double *p);
int orc3_run(const orc3_problem *P, double *g, int t0, int nsteps, double *trace);

#endif
