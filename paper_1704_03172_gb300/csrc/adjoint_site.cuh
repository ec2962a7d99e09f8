// adjoint_site.cuh -- the per-site arithmetic of the discrete adjoint (adjoint.cu: the
// one-step and tile-blocked reverse sweeps; adjoint5.cu: the D2Q5 wavefront sweep) and the
// arguments the sweeps share.  The derivation is at the top of adjoint.cu.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "lb_kernels.cuh"
#include "lb_runtime.h"

namespace lbadj {

using namespace lbk;

// d w_i / d(eta^2) and d c_s^2 / d(eta^2) under the weight rule of Sec. 2.3
template <int Q>
__device__ __forceinline__ float dweight(int i, const StepArgs &a) {
    if (Q == 5) return i == 0 ? -1.f : 0.25f;
    if (i == 0) return -4.f * (a.w1r + a.w5r);
    return i < 5 ? a.w1r : a.w5r;
}

template <int Q>
__device__ __forceinline__ float dcs2(const StepArgs &a) {
    return Q == 5 ? 0.5f : a.c2r;
}

// Source terms of one site's adjoint, from m = sigma(x) mu(x) before adj_site: src_w = w . m
// (dJ/dS^t at the source) and src_dw = dw/d(eta^2) . m (times S^t: the source's medium
// gradient).
template <int Q>
__device__ __forceinline__ void adj_src(const float (&m)[Q], float e2, const StepArgs &a,
                                        float &src_w, float &src_dw) {
    src_w = 0.f;
    src_dw = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        src_w += weight_i<Q>(i, e2, a) * m[i];
        src_dw += dweight<Q>(i, a) * m[i];
    }
}

// Adjoint of one site's collision.  In: m = sigma(x) mu(x), the pulled adjoint populations
// times the sponge factor.  Out: m = K^T m = m - (I - E^T) v with v = C^T m, the site's
// lambda^t before receiver terms; returns gsum = v . dw/d(eta^2) (times rho^t: the medium
// gradient).  (E^T v)_i = A + c_i . B with A = sum_j w_j v_j, B = sum_j (w_j / c_s^2) c_j v_j.
template <int Q, bool MRT>
__device__ __forceinline__ float adj_site(float (&m)[Q], float e2, const StepArgs &a) {
    if constexpr (Q == 5) {
        // D2Q5: w_0 = 1 - eta^2, w_i = eta^2 / 4, w_i / c_s^2 = 1/2, dw = (-1, 1/4, 1/4, 1/4, 1/4)
        const float w0 = 1.f - e2, w1 = 0.25f * e2;
        const float s14 = m[1] + m[2] + m[3] + m[4];
        if (!MRT) {
            // v = omega m: A = omega (w . m), B = omega / 2 (m1 - m3, m2 - m4), and
            // m - v + E^T v = (1 - omega) m + A + c . B
            const float om = a.omega, A = om * (w0 * m[0] + w1 * s14);
            const float hb = 0.5f * om, Bx = hb * (m[1] - m[3]), By = hb * (m[2] - m[4]);
            const float keep = 1.f - om;
            const float gsum = om * (0.25f * s14 - m[0]);
            m[0] = keep * m[0] + A;
            m[1] = keep * m[1] + (A + Bx);
            m[2] = keep * m[2] + (A + By);
            m[3] = keep * m[3] + (A - Bx);
            m[4] = keep * m[4] + (A - By);
            return gsum;
        }
        // MRT: only e (row 3 of M, norm 20) and p_xx (row 4, norm 4) relax; both are even
        // in c, so B = 0, and v = (-4 e', e' + p', e' - p', e' + p', e' - p')
        const float me = (-4.f * m[0] + s14) * a.s[3];  // rates arrive as s_e / 20, s_p / 4
        const float mp = (m[1] - m[2] + m[3] - m[4]) * a.s[4];
        const float v13 = me + mp, v24 = me - mp;
        const float A = 4.f * me * (w1 - w0);  // w0 v0 + w1 (2 v13 + 2 v24)
        m[0] = m[0] + 4.f * me + A;
        m[1] = m[1] - v13 + A;
        m[2] = m[2] - v24 + A;
        m[3] = m[3] - v13 + A;
        m[4] = m[4] - v24 + A;
        return 5.f * me;  // v . dw = 4 e' + e'
    } else {
        // D2Q9: w_j and w_j / c_s^2 (eta-independent for j > 0)
        float w[Q], wc[Q];
#pragma unroll
        for (int i = 0; i < Q; i++) {
            w[i] = weight_i<Q>(i, e2, a);
            wc[i] = i == 0 ? 0.f : (i < 5 ? a.a1 : a.a5);
        }
        float v[Q];
        if (!MRT) {
#pragma unroll
            for (int i = 0; i < Q; i++) v[i] = a.omega * m[i];
        } else {
            const float s14 = m[1] + m[2] + m[3] + m[4], s58 = m[5] + m[6] + m[7] + m[8];
            // rates arrive divided by the squared row norms (36, 4, 36, 12, 12, 4)
            const float d3 = a.s[3] * (-4.f * m[0] - s14 + 2.f * s58);
            const float d4 = a.s[4] * (m[1] - m[2] + m[3] - m[4]);
            const float d5 = a.s[5] * (4.f * m[0] - 2.f * s14 + s58);
            const float d6 = a.s[6] * (-2.f * m[1] + 2.f * m[3] + m[5] - m[6] - m[7] + m[8]);
            const float d7 = a.s[7] * (-2.f * m[2] + 2.f * m[4] + m[5] + m[6] - m[7] - m[8]);
            const float d8 = a.s[8] * (m[5] - m[6] + m[7] - m[8]);
            v[0] = -4.f * d3 + 4.f * d5;
            v[1] = -d3 + d4 - 2.f * d5 - 2.f * d6;
            v[2] = -d3 - d4 - 2.f * d5 - 2.f * d7;
            v[3] = -d3 + d4 - 2.f * d5 + 2.f * d6;
            v[4] = -d3 - d4 - 2.f * d5 + 2.f * d7;
            const float c5 = 2.f * d3 + d5;
            v[5] = c5 + d6 + d7 + d8;
            v[6] = c5 - d6 + d7 - d8;
            v[7] = c5 - d6 - d7 + d8;
            v[8] = c5 + d6 - d7 - d8;
        }
        float A = 0.f, Bx = 0.f, By = 0.f;
#pragma unroll
        for (int j = 0; j < Q; j++) {
            A += w[j] * v[j];
            Bx += wc[j] * Lat<Q>::cx(j) * v[j];
            By += wc[j] * Lat<Q>::cy(j) * v[j];
        }
        float gsum = 0.f;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            gsum += v[i] * dweight<Q>(i, a);
            m[i] = m[i] - v[i] + (A + Lat<Q>::cx(i) * Bx + Lat<Q>::cy(i) * By);
        }
        return gsum;
    }
}

struct AdjArgs {
    const float *lam_in;   // lambda^{t+1} [Q][ny][pitch]
    float *lam_out;        // lambda^t
    const float *rho;      // rho(x, t) of the forward state g^t, [ny][pitch] (replay tape)
    double *grad;          // dJ/d(eta^2), [ny][pitch]
    double *grad_src;      // [nt] (indexed by t - t0) or nullptr
    long long t0;
    const float *resid;    // dJ/dp, [nt][nrec] (row t - t0)
    int nrec;
    int segs;              // warps per row: ceil(nx / 128)
};

}  // namespace lbadj

// The D2Q5 wavefront reverse sweep (adjoint5.cu): levels per launch, the receivers' row lists
// ([ny + 1] offsets, x ascending, receiver ids) and the launch of kAdj5Levels levels
// t_hi .. t_hi - kAdj5Levels + 1 (rho^t at rho_hi - (t_hi - t) plane) on ctx's stream.
constexpr int kAdj5Levels = 4;
void adj5_row_lists(const lb_ctx *ctx, std::vector<int> &off, std::vector<int> &xs,
                    std::vector<int> &ids);
cudaError_t adj5_launch(lb_ctx *ctx, const lbk::StepArgs &a, const lbadj::AdjArgs &d,
                        const float *rho_hi, long long t_hi, const int *row_off, const int *rec_x,
                        const int *rec_id);
