/*
 * lbadjoint.c -- FP64 discrete adjoint of the linear LB scheme (oracle).
 * TEST INFRASTRUCTURE: used only by the tests and the CPU-baseline leg.
 *
 * The paper has no adjoint; this is the exact transpose of the forward map of
 * lbref.c, written as its own loop (no automatic differentiation):
 *   forward   h^t = D_sigma (K(x) g^t + b S^t),  g^{t+1} = P h^t,
 *             p^t_r = c_s^2(x_r) sum_i g^t_i(x_r)        (trace row t)
 *   with K = I - C (I - E), C = M^-1 S M (MRT) or I / tau (BGK),
 *   E_kj = d g^eq_k / d g_j = w_k (1 + c_k . c_j / c_s^2)  (Eq. linear eqm dist),
 *   b = w(x_s) at the source node, D_sigma = diag(1 - sigma(x)), P = push streaming.
 * For a functional J whose gradient with respect to the traces is R^t_r,
 *   mu^t   = D_sigma P^T lambda^{t+1}      (P^T: pull from x + c_i; lambda^{nt} = 0)
 *   lambda^t = K^T mu^t + sum_r R^t_r c_s^2(x_r) [x = x_r]  (every population)
 *   dJ/dS^t  = b . mu^t(x_s)
 *   dJ/deta(x) = sum_t rho^t(x) mu^t(x) . (C dw/deta)
 *              + [x = x_s] S^t mu^t(x_s) . dw/deta
 *              + sum_r [x = x_r] R^t_r d(c_s^2)/deta rho^t(x_r)
 * (the velocity part of g^eq has weights w_k / c_s^2 that do not depend on eta
 * under the weight rule of Sec. 2.3, so dE/deta g = dw/deta rho), and
 * dJ/dc = dJ/deta / c_ref, dJ/dg^0 = lambda^0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "lbref.h"

static const int A5[5][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}};
static const int A9[9][2] = {{0, 0},  {1, 0},  {0, 1},   {-1, 0}, {0, -1},
                             {1, 1},  {-1, 1}, {-1, -1}, {1, -1}};

/* d w_i / d eta for the weight rule of Sec. 2.3 (D2Q5) and its D2Q9 reading */
static void dweights(int Q, double eta, const double *w_ref, double *dw, double *dcs2) {
    if (Q == 5) {
        dw[0] = -2.0 * eta;                          /* w_0 = 1 - eta^2 */
        for (int i = 1; i < 5; i++) dw[i] = 0.5 * eta; /* w_i = eta^2 / 4 */
        *dcs2 = eta;                                 /* c_s^2 = eta^2 / 2 */
    } else {
        double s = 0.0;
        for (int i = 1; i < 5; i++) dw[i] = 2.0 * eta * w_ref[1];
        for (int i = 5; i < 9; i++) dw[i] = 2.0 * eta * w_ref[2];
        for (int i = 1; i < 9; i++) s += dw[i];
        dw[0] = -s;
        *dcs2 = 2.0 * eta * (2.0 * w_ref[1] + 4.0 * w_ref[2]);
    }
}

static void collision_matrix(const orc_problem *P, double *C) {
    const int Q = P->Q;
    memset(C, 0, sizeof(double) * Q * Q);
    if (!P->mrt) {
        for (int i = 0; i < Q; i++) C[i * Q + i] = 1.0 / P->tau;
        return;
    }
    double M[81], Minv[81];
    orc_moment_matrix(Q, M);
    orc_moment_inverse(Q, Minv);
    for (int i = 0; i < Q; i++)
        for (int j = 0; j < Q; j++) {
            double a = 0.0;
            for (int k = 0; k < Q; k++) a += Minv[i * Q + k] * P->s[k] * M[k * Q + j];
            C[i * Q + j] = a;
        }
}

int orc_adjoint(const orc_problem *P, const double *g0, int nt, const double *resid,
                double *grad_c, double *grad_src, double *grad_g0) {
    const int Q = P->Q, nx = P->nx, ny = P->ny;
    const size_t N = (size_t)nx * ny, len = (size_t)Q * N;
    const int(*cv)[2] = Q == 9 ? A9 : A5;
    double Minv[81], C[81];
    orc_moment_inverse(Q, Minv);
    collision_matrix(P, C);
    /* forward: keep every state */
    double *G = (double *)malloc(sizeof(double) * len * (size_t)(nt > 0 ? nt : 1));
    double *lam = (double *)calloc(len, sizeof(double));
    double *lnew = (double *)calloc(len, sizeof(double));
    double *geta = (double *)calloc(N, sizeof(double));
    if (!G || !lam || !lnew || !geta) return -3;
    if (nt > 0) memcpy(G, g0, sizeof(double) * len);
    for (int t = 0; t + 1 < nt; t++) orc_step_grid(P, Minv, t, G + (size_t)t * len, G + (size_t)(t + 1) * len);
    if (grad_src)
        for (int t = 0; t < nt; t++) grad_src[t] = 0.0;
    for (int t = nt - 1; t >= 0; t--) {
        const double *g = G + (size_t)t * len;
        const double S = (P->src && t < P->nt_src) ? P->src[t] : 0.0;
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                size_t idx = (size_t)y * nx + x;
                double w[9], cs2, dw[9], dcs2, mu[9], gl[9], rho = 0.0;
                orc_site_weights(P, idx, w, &cs2);
                double eta = (double)P->c_map[idx] / P->c_ref;
                dweights(Q, eta, P->w_ref, dw, &dcs2);
                double sig = orc_sponge_sigma(x, y, nx, ny, P->sponge_width, P->sponge_sigma_max);
                for (int i = 0; i < Q; i++) {
                    int xd = x + cv[i][0], yd = y + cv[i][1];
                    double v = 0.0;
                    if (P->periodic) {
                        xd = (xd + nx) % nx;
                        yd = (yd + ny) % ny;
                        v = lam[(size_t)i * N + (size_t)yd * nx + xd];
                    } else if (xd >= 0 && xd < nx && yd >= 0 && yd < ny) {
                        v = lam[(size_t)i * N + (size_t)yd * nx + xd];
                    }
                    mu[i] = (1.0 - sig) * v;
                    gl[i] = g[(size_t)i * N + idx];
                    rho += gl[i];
                }
                /* K = I - C (I - E) built entry by entry; lambda^t = K^T mu */
                double K[81];
                for (int k = 0; k < Q; k++)
                    for (int j = 0; j < Q; j++) {
                        double a = 0.0;
                        for (int m = 0; m < Q; m++) {
                            double E = w[m] * (1.0 + (cv[m][0] * cv[j][0] + cv[m][1] * cv[j][1]) / cs2);
                            a += C[k * Q + m] * ((m == j ? 1.0 : 0.0) - E);
                        }
                        K[k * Q + j] = (k == j ? 1.0 : 0.0) - a;
                    }
                for (int j = 0; j < Q; j++) {
                    double a = 0.0;
                    for (int k = 0; k < Q; k++) a += K[k * Q + j] * mu[k];
                    lnew[(size_t)j * N + idx] = a;
                }
                /* dK/deta = C dE/deta with dE_kj/deta = dw_k/deta (velocity part eta-free) */
                double gsum = 0.0;
                for (int k = 0; k < Q; k++) {
                    double Cdw = 0.0;
                    for (int m = 0; m < Q; m++) Cdw += C[k * Q + m] * dw[m];
                    gsum += mu[k] * Cdw;
                }
                geta[idx] += rho * gsum;
                if (P->src && x == P->src_x && y == P->src_y) {
                    double a = 0.0, b = 0.0;
                    for (int i = 0; i < Q; i++) {
                        a += mu[i] * dw[i];
                        b += mu[i] * w[i];
                    }
                    geta[idx] += S * a;
                    if (grad_src) grad_src[t] = b;
                }
            }
        /* receivers: p^t_r = c_s^2 rho^t(x_r) */
        for (int r = 0; r < P->nrec; r++) {
            int x = P->rec_xy[2 * r], y = P->rec_xy[2 * r + 1];
            size_t idx = (size_t)y * nx + x;
            double w[9], cs2, dw[9], dcs2, rho = 0.0;
            orc_site_weights(P, idx, w, &cs2);
            dweights(Q, (double)P->c_map[idx] / P->c_ref, P->w_ref, dw, &dcs2);
            for (int i = 0; i < Q; i++) rho += g[(size_t)i * N + idx];
            double R = resid[(size_t)t * P->nrec + r];
            for (int i = 0; i < Q; i++) lnew[(size_t)i * N + idx] += R * cs2;
            geta[idx] += R * dcs2 * rho;
        }
        double *s = lam;
        lam = lnew;
        lnew = s;
    }
    for (size_t k = 0; k < N; k++) grad_c[k] = geta[k] / P->c_ref;
    if (grad_g0) memcpy(grad_g0, lam, sizeof(double) * len);
    free(G);
    free(lam);
    free(lnew);
    free(geta);
    return 0;
}
