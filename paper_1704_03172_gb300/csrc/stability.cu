// stability.cu -- linear (von Neumann) stability of a configuration, on the host.
//
// One LB step maps a Fourier mode g(x) = g_k exp(i k.x) of a homogeneous medium to
// T(k) g_k with T(k) = D(k) (I - C A) (Eq. MRT-LB dispersion, collide then stream):
//   A_ij = delta_ij - w_i (1 + c_i.c_j / c_s^2)  (g^eq = (I - A) g, Eq. linear eqm dist),
//   C    = I / tau (BGK) or M^-1 S M (MRT, M of App. A, S = diag of the rates),
//   D(k) = diag(exp(-i k.c_i)).
// The scheme is stable at a wave vector when every eigenvalue of T(k) has modulus <= 1
// (Sec. 3's single-mode analysis; Sec. 2.3 on choices of rates and weights that are not).
// lb_create evaluates max |lambda| over a grid of wave vectors at the medium's values of
// eta = c / c_ref and refuses a configuration above 1 + 1e-12.
//
// Eigenvalues: Householder reduction to upper Hessenberg form, then the complex QR
// algorithm with Wilkinson shifts and deflation (Golub & Van Loan, Matrix Computations,
// Sec. 7.4-7.5), in complex double precision on at most 9 x 9 matrices.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lbac.h"
#include "lb_runtime.h"

namespace {

using cd = std::complex<double>;

// lattice velocities in the order of the rows of M (App. A)
const int kC5[5][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}};
const int kC9[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};

// moment matrices of App. A (rows are mutually orthogonal)
const double kM5[5][5] = {{1, 1, 1, 1, 1},
                          {0, 1, 0, -1, 0},
                          {0, 0, 1, 0, -1},
                          {-4, 1, 1, 1, 1},
                          {0, 1, -1, 1, -1}};
const double kM9[9][9] = {{1, 1, 1, 1, 1, 1, 1, 1, 1},
                          {0, 1, 0, -1, 0, 1, -1, -1, 1},
                          {0, 0, 1, 0, -1, 1, 1, -1, -1},
                          {-4, -1, -1, -1, -1, 2, 2, 2, 2},
                          {0, 1, -1, 1, -1, 0, 0, 0, 0},
                          {4, -2, -2, -2, -2, 1, 1, 1, 1},
                          {0, -2, 0, 2, 0, 1, -1, -1, 1},
                          {0, 0, -2, 0, 2, 1, 1, -1, -1},
                          {0, 0, 0, 0, 0, 1, -1, 1, -1}};

double mrow(int Q, int k, int i) { return Q == 5 ? kM5[k][i] : kM9[k][i]; }
int cvel(int Q, int i, int d) { return Q == 5 ? kC5[i][d] : kC9[i][d]; }

// Eigenvalues of the n x n complex matrix a (row-major, overwritten).  False if the QR
// iteration did not converge.
bool eigenvalues(int n, cd *a, cd *ev) {
    auto A = [&](int i, int j) -> cd & { return a[i * n + j]; };
    // 1. Householder reduction to upper Hessenberg form
    for (int k = 0; k + 2 < n; k++) {
        double xn = 0;
        for (int i = k + 1; i < n; i++) xn += std::norm(A(i, k));
        xn = std::sqrt(xn);
        if (xn == 0) continue;
        const cd x0 = A(k + 1, k);
        const cd ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1);
        cd v[9];
        for (int i = 0; i < n; i++) v[i] = 0;
        v[k + 1] = x0 + ph * xn;
        for (int i = k + 2; i < n; i++) v[i] = A(i, k);
        double vn = 0;
        for (int i = k + 1; i < n; i++) vn += std::norm(v[i]);
        if (vn == 0) continue;
        // A <- H A H with H = I - 2 v v^H / (v^H v)
        for (int j = 0; j < n; j++) {
            cd s = 0;
            for (int i = k + 1; i < n; i++) s += std::conj(v[i]) * A(i, j);
            s *= 2.0 / vn;
            for (int i = k + 1; i < n; i++) A(i, j) -= v[i] * s;
        }
        for (int i = 0; i < n; i++) {
            cd s = 0;
            for (int j = k + 1; j < n; j++) s += A(i, j) * v[j];
            s *= 2.0 / vn;
            for (int j = k + 1; j < n; j++) A(i, j) -= s * std::conj(v[j]);
        }
        for (int i = k + 2; i < n; i++) A(i, k) = 0;
    }
    // 2. shifted QR on the active block [lo, hi]
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, iter = 0;
    while (hi >= 0) {
        if (hi == 0) {
            ev[0] = A(0, 0);
            break;
        }
        int lo = hi;
        while (lo > 0) {
            const double scale = std::abs(A(lo, lo)) + std::abs(A(lo - 1, lo - 1));
            if (std::abs(A(lo, lo - 1)) <= eps * (scale > 0 ? scale : 1.0)) {
                A(lo, lo - 1) = 0;
                break;
            }
            lo--;
        }
        if (lo == hi) {  // a 1 x 1 block has split off
            ev[hi] = A(hi, hi);
            hi--;
            iter = 0;
            continue;
        }
        if (++iter > 60 * n) return false;
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer to A(hi, hi)
        const cd p = A(hi - 1, hi - 1), q = A(hi - 1, hi), r = A(hi, hi - 1), d = A(hi, hi);
        const cd half = 0.5 * (p + d), disc = std::sqrt(0.25 * (p - d) * (p - d) + q * r);
        cd mu = std::abs(half + disc - d) < std::abs(half - disc - d) ? half + disc : half - disc;
        if (iter % 10 == 0) mu += std::abs(A(hi, hi - 1));  // exceptional shift
        for (int i = lo; i <= hi; i++) A(i, i) -= mu;
        cd cs[9], sn[9];
        for (int k = lo; k < hi; k++) {  // Givens rotations zero the subdiagonal: A = Q R
            const cd x = A(k, k), y = A(k + 1, k);
            const double rr = std::sqrt(std::norm(x) + std::norm(y));
            cs[k] = rr > 0 ? x / rr : cd(1);
            sn[k] = rr > 0 ? y / rr : cd(0);
            for (int j = k; j < n; j++) {
                const cd u = A(k, j), w = A(k + 1, j);
                A(k, j) = std::conj(cs[k]) * u + std::conj(sn[k]) * w;
                A(k + 1, j) = -sn[k] * u + cs[k] * w;
            }
        }
        for (int k = lo; k < hi; k++) {  // R Q
            const int top = std::min(k + 2, hi);
            for (int i = 0; i <= top; i++) {
                const cd u = A(i, k), w = A(i, k + 1);
                A(i, k) = u * cs[k] + w * sn[k];
                A(i, k + 1) = -u * std::conj(sn[k]) + w * std::conj(cs[k]);
            }
        }
        for (int i = lo; i <= hi; i++) A(i, i) += mu;
    }
    return true;
}

// weights and c_s^2 at eta: D2Q5 w_0 = 1 - eta^2, w_1..4 = eta^2 / 4 (Eq. 0th lattice
// weight); D2Q9 w_1..4 = eta^2 w1_ref, w_5..8 = eta^2 w5_ref, w_0 = 1 - sum of the others
void weights(int Q, double eta, const double *w_ref, double *w, double *cs2) {
    const double e2 = eta * eta;
    if (Q == 5) {
        w[0] = 1 - e2;
        for (int i = 1; i < 5; i++) w[i] = 0.25 * e2;
        *cs2 = 0.5 * e2;
        return;
    }
    const double w1 = e2 * w_ref[1], w5 = e2 * w_ref[2];
    w[0] = 1 - 4 * (w1 + w5);
    for (int i = 1; i < 5; i++) w[i] = w1;
    for (int i = 5; i < 9; i++) w[i] = w5;
    *cs2 = e2 * (2 * w_ref[1] + 4 * w_ref[2]);
}

struct Rates {
    int Q, mrt;
    double tau, s[9], w_ref[3];
};

// K = I - C A for the rates r at eta (real Q x Q, row-major)
void collision_map(const Rates &r, double eta, double *K) {
    const int Q = r.Q;
    double w[9], cs2;
    weights(Q, eta, r.w_ref, w, &cs2);
    double A[81];
    for (int i = 0; i < Q; i++)
        for (int j = 0; j < Q; j++) {
            const double cc = cvel(Q, i, 0) * cvel(Q, j, 0) + cvel(Q, i, 1) * cvel(Q, j, 1);
            A[i * Q + j] = (i == j ? 1.0 : 0.0) - w[i] * (1.0 + cc / cs2);
        }
    double C[81];
    if (!r.mrt) {
        for (int i = 0; i < Q * Q; i++) C[i] = 0;
        for (int i = 0; i < Q; i++) C[i * Q + i] = 1.0 / r.tau;
    } else {  // M^-1 S M with M^-1 = M^T diag(1 / |row_k|^2) (orthogonal rows)
        for (int i = 0; i < Q; i++)
            for (int j = 0; j < Q; j++) {
                double v = 0;
                for (int k = 0; k < Q; k++) {
                    double nk = 0;
                    for (int m = 0; m < Q; m++) nk += mrow(Q, k, m) * mrow(Q, k, m);
                    v += mrow(Q, k, i) * (r.s[k] / nk) * mrow(Q, k, j);
                }
                C[i * Q + j] = v;
            }
    }
    for (int i = 0; i < Q; i++)
        for (int j = 0; j < Q; j++) {
            double v = i == j ? 1.0 : 0.0;
            for (int k = 0; k < Q; k++) v -= C[i * Q + k] * A[k * Q + j];
            K[i * Q + j] = v;
        }
}

// max over k = 2 pi (m, n) / nk of max |lambda(T(k))|; -1 if the QR did not converge.
// T(-k) is the complex conjugate of T(k), so n = 0 .. nk / 2 covers every modulus.
double radius(const Rates &r, double eta, int nk) {
    const int Q = r.Q;
    double K[81];
    collision_map(r, eta, K);
    double best = 0;
    for (int m = 0; m < nk; m++)
        for (int n = 0; n <= nk / 2; n++) {
            const double kx = 2 * M_PI * m / nk, ky = 2 * M_PI * n / nk;
            cd T[81], ev[9];
            for (int i = 0; i < Q; i++) {
                const cd d = std::exp(cd(0, -(kx * cvel(Q, i, 0) + ky * cvel(Q, i, 1))));
                for (int j = 0; j < Q; j++) T[i * Q + j] = d * K[i * Q + j];
            }
            if (!eigenvalues(Q, T, ev)) return -1;
            for (int i = 0; i < Q; i++) best = std::max(best, std::abs(ev[i]));
        }
    return best;
}

// rates of refinement level `level` (reading R6: tau_l - 1/2 = 2^l (tau - 1/2), moment by
// moment for MRT)
Rates level_rates(const lb_config *cfg, int level) {
    Rates r;
    memset(&r, 0, sizeof(r));
    r.Q = cfg->lattice;
    r.mrt = cfg->collision == LB_MRT;
    const double f = std::ldexp(1.0, level);
    r.tau = 0.5 + f * (cfg->tau - 0.5);
    for (int k = 0; k < 9; k++) {
        const double s = k < r.Q ? cfg->s[k] : 1.0;
        r.s[k] = 1.0 / (0.5 + f * (1.0 / s - 0.5));
    }
    for (int k = 0; k < 3; k++) r.w_ref[k] = cfg->w_ref[k];
    return r;
}

std::mutex g_mu;
std::map<std::string, double> g_cache;  // radius by (rates, eta, nk)

double radius_cached(const Rates &r, double eta, int nk) {
    std::string key(reinterpret_cast<const char *>(&r), sizeof(r));
    key.append(reinterpret_cast<const char *>(&eta), sizeof(eta));
    key.append(reinterpret_cast<const char *>(&nk), sizeof(nk));
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) return it->second;
    }
    const double v = radius(r, eta, nk);
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_cache.size() > 4096) g_cache.clear();
    g_cache[key] = v;
    return v;
}

}  // namespace

namespace lbrt {

// Whether a configuration needs the check: the D2Q5 BGK step is stable for every tau >=
// 1/2 and eta <= 1 (its tau = 1/2 form is the leapfrog scheme at Courant number
// c_s <= 1/sqrt(2), App. C), and D3Q7 is its BGK extension; MRT rates and D2Q9 weight
// choices can be unstable.
bool stability_needed(const lb_config *cfg) {
    return cfg->lattice == LB_D2Q9 || (cfg->lattice == LB_D2Q5 && cfg->collision == LB_MRT);
}

// The values of eta at which lb_create checks: the distinct values of the medium when there
// are at most 8, else 8 values spread over [eta_min, eta_max] (both ends included).
std::vector<double> stability_etas(double eta_min, double eta_max, const std::vector<double> &distinct) {
    if (!distinct.empty() && distinct.size() <= 8) return distinct;
    std::vector<double> e;
    for (int k = 0; k < 8; k++) e.push_back(eta_min + (eta_max - eta_min) * k / 7.0);
    return e;
}

// max |lambda| over the checked etas and every refinement level; the eta that attains it
double stability_worst(const lb_config *cfg, const std::vector<double> &etas, double *eta_at,
                       int *level_at) {
    double worst = 0;
    const int levels = 1 + std::max(0, cfg->n_patches);
    for (int l = 0; l < levels; l++) {
        const Rates r = level_rates(cfg, l);
        for (double eta : etas) {
            const double v = radius_cached(r, eta, 64);
            if (v < 0 || v > worst) {
                worst = v < 0 ? 1e300 : v;
                if (eta_at) *eta_at = eta;
                if (level_at) *level_at = l;
            }
        }
    }
    return worst;
}

}  // namespace lbrt

extern "C" lb_status lb_stability_radius(const lb_config *cfg, double eta, int level, int nk,
                                         double *radius_out) {
    if (!cfg || !radius_out) return LB_EINVAL;
    if ((cfg->lattice != LB_D2Q5 && cfg->lattice != LB_D2Q9) || !(eta > 0.0 && eta <= 1.0) ||
        level < 0 || level > LB_MAX_PATCHES || nk < 2 || nk > 4096)
        return LB_EINVAL;
    if (cfg->collision == LB_BGK && !(cfg->tau >= 0.5)) return LB_EINVAL;
    if (cfg->collision == LB_MRT)
        for (int k = 0; k < cfg->lattice; k++)
            if (!(cfg->s[k] > 0.0 && cfg->s[k] <= 2.0)) return LB_EINVAL;
    const double v = radius_cached(level_rates(cfg, level), eta, nk);
    if (v < 0) return lbrt::fail(nullptr, LB_EINVAL, "eigenvalue iteration did not converge");
    *radius_out = v;
    return LB_OK;
}
