// adjoint.cu -- discrete adjoint of the fused LB step, with two-level
// checkpointing, for gradients of a receiver-trace functional with respect to
// the sound-speed map, the source samples and the initial state.
//
// The paper has no adjoint.  Because the scheme is linear in the populations,
// the adjoint of one step is its exact transpose:
//   forward   h^t = D_sigma (K g^t + b S^t),  g^{t+1} = P h^t,  p^t_r = c_s^2 rho^t(x_r)
//   adjoint   mu^t = D_sigma P^T lambda^{t+1}          (pull from x + c_i: reverse streaming)
//             lambda^t = K^T mu^t + R^t_r c_s^2(x_r) at the receivers
//             dJ/dS^t = w(x_s) . mu^t(x_s)
//             dJ/d(eta^2)(x) += rho^t(x) (C^T mu^t) . dw/d(eta^2) (+ source, receiver terms)
// with K = I - C (I - E), E_kj = w_k (1 + c_k . c_j / c_s^2) (Eq. linear eqm dist),
// C = M^-1 S M (Eq. MRT-LB) or I / tau (Eq. BGK-LB).  Only the non-conserved
// moments of C^T mu contribute (the conserved ones are annihilated by I - E^T,
// and dw sums to zero with zero first moment), so s_rho and s_v drop out as in
// the forward step.  dJ/dc = dJ/d(eta^2) * 2 eta / c_ref.
//
// Checkpoints: lb_step copies the state every C steps (C = lb_checkpoint_every).
// The backward sweep walks the segments newest first; each segment is replayed
// once to place sub-checkpoints every ceil(sqrt(C)) steps, and each
// sub-segment is replayed again keeping all its states, then swept backwards.
// Device memory: the checkpoints, ~2 sqrt(C) + 3 states, the adjoint pair and
// an FP64 gradient.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lb_kernels.cuh"
#include "lb_runtime.h"

using namespace lbk;
using namespace lbrt;

namespace {

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

struct AdjArgs {
    const float *lam_in;   // lambda^{t+1} [Q][ny][pitch]
    float *lam_out;        // lambda^t
    const float *fwd;      // forward buffer whose pull gives g^t (raw: g^t itself)
    int fwd_raw;
    double *grad;          // dJ/d(eta^2), [ny][pitch]
    double *grad_src;      // [nt] (indexed by t - t0) or nullptr
    long long t0;
    const float *resid;    // dJ/dp, [nt][nrec] (row t - t0)
    int nrec;
};

template <int Q, bool MRT, bool PERIODIC>
__global__ void __launch_bounds__(256) adjoint_kernel(const StepArgs a, const AdjArgs d) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)a.ny * a.pitch) return;
    const int y = (int)(idx / a.pitch), x = (int)(idx - (long long)y * a.pitch);
    if (x >= a.nx) return;
    const float e2 = a.eta2[idx];
    const float f = a.sponge_w > 0 ? sponge_factor(x, y, a) : 1.f;
    float mu[Q], rho = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        int xd = x + Lat<Q>::cx(i), yd = y + Lat<Q>::cy(i);
        float v = 0.f;
        bool ok = true;
        if (PERIODIC) {
            xd = (xd + a.nx) % a.nx;
            yd = (yd + a.ny) % a.ny;
        } else {
            ok = xd >= 0 && xd < a.nx && yd >= 0 && yd < a.ny;
        }
        if (ok) v = d.lam_in[i * a.plane + (long long)yd * a.pitch + xd];
        mu[i] = f * v;
        // forward population g^t_i(x)
        int xs = x, ys = y;
        if (!d.fwd_raw) {
            xs -= Lat<Q>::cx(i);
            ys -= Lat<Q>::cy(i);
        }
        bool okf = true;
        if (PERIODIC) {
            xs = (xs + a.nx) % a.nx;
            ys = (ys + a.ny) % a.ny;
        } else {
            okf = xs >= 0 && xs < a.nx && ys >= 0 && ys < a.ny;
        }
        if (okf) rho += d.fwd[i * a.plane + (long long)ys * a.pitch + xs];
    }
    // w_j and w_j / c_s^2 (eta-independent for j > 0)
    float w[Q], wc[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        w[i] = weight_i<Q>(i, e2, a);
        wc[i] = i == 0 ? 0.f : (Q == 5 ? 0.5f : (i < 5 ? a.a1 : a.a5));
    }
    // v = C^T mu (non-conserved part for MRT; all of it for BGK)
    float v[Q];
    if (!MRT) {
#pragma unroll
        for (int i = 0; i < Q; i++) v[i] = a.omega * mu[i];
    } else if (Q == 5) {
        // rows 3 (e) and 4 (p_xx) of M, norms 20 and 4
        const float me = (-4.f * mu[0] + mu[1] + mu[2] + mu[3] + mu[4]) * a.s[3] * (1.f / 20.f);
        const float mp = (mu[1] - mu[2] + mu[3] - mu[4]) * a.s[4] * 0.25f;
        v[0] = -4.f * me;
        v[1] = me + mp;
        v[2] = me - mp;
        v[3] = me + mp;
        v[4] = me - mp;
    } else {
        const float s14 = mu[1] + mu[2] + mu[3] + mu[4], s58 = mu[5] + mu[6] + mu[7] + mu[8];
        const float d3 = a.s[3] * (-4.f * mu[0] - s14 + 2.f * s58) * (1.f / 36.f);
        const float d4 = a.s[4] * (mu[1] - mu[2] + mu[3] - mu[4]) * 0.25f;
        const float d5 = a.s[5] * (4.f * mu[0] - 2.f * s14 + s58) * (1.f / 36.f);
        const float d6 = a.s[6] * (-2.f * mu[1] + 2.f * mu[3] + mu[5] - mu[6] - mu[7] + mu[8]) *
                         (1.f / 12.f);
        const float d7 = a.s[7] * (-2.f * mu[2] + 2.f * mu[4] + mu[5] + mu[6] - mu[7] - mu[8]) *
                         (1.f / 12.f);
        const float d8 = a.s[8] * (mu[5] - mu[6] + mu[7] - mu[8]) * 0.25f;
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
    // K^T mu = mu - (I - E^T) v, (E^T v)_i = sum_j w_j v_j + c_i . sum_j (w_j / c_s^2) c_j v_j
    float A = 0.f, Bx = 0.f, By = 0.f;
#pragma unroll
    for (int j = 0; j < Q; j++) {
        A += w[j] * v[j];
        Bx += wc[j] * Lat<Q>::cx(j) * v[j];
        By += wc[j] * Lat<Q>::cy(j) * v[j];
    }
    float gsum = 0.f, src_w = 0.f, src_dw = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const float et = A + Lat<Q>::cx(i) * Bx + Lat<Q>::cy(i) * By;
        d.lam_out[i * a.plane + idx] = mu[i] - v[i] + et;
        const float dw = dweight<Q>(i, a);
        gsum += v[i] * dw;
        src_w += w[i] * mu[i];
        src_dw += dw * mu[i];
    }
    double gadd = (double)rho * (double)gsum;
    if (x == a.src_x && y == a.src_y && a.src_tab) {
        if (d.grad_src) d.grad_src[a.t - d.t0] = (double)src_w;
        if (a.t < a.src_nt) gadd += (double)a.src_tab[a.t] * (double)src_dw;
    }
    d.grad[idx] += gadd;
}

// receivers: lambda^t += R^t_r c_s^2(x_r) (every population), dJ/d(eta^2) += R dc_s^2 rho^t
template <int Q, bool PERIODIC>
__global__ void adjoint_receivers(const StepArgs a, const AdjArgs d) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.nrec) return;
    const int2 xy = a.rec[r];
    const long long idx = (long long)xy.y * a.pitch + xy.x;
    const float R = d.resid[(a.t - d.t0) * d.nrec + r];
    float rho = 0.f;
    for (int i = 0; i < Q; i++) {
        int xs = xy.x, ys = xy.y;
        if (!d.fwd_raw) {
            xs -= Lat<Q>::cx(i);
            ys -= Lat<Q>::cy(i);
        }
        if (PERIODIC) {
            xs = (xs + a.nx) % a.nx;
            ys = (ys + a.ny) % a.ny;
        } else if (xs < 0 || xs >= a.nx || ys < 0 || ys >= a.ny) {
            continue;
        }
        rho += d.fwd[i * a.plane + (long long)ys * a.pitch + xs];
    }
    const float c2 = cs2_of<Q>(a.eta2[idx], a);
    for (int i = 0; i < Q; i++) atomicAdd(d.lam_out + i * a.plane + idx, R * c2);
    atomicAdd(d.grad + idx, (double)R * (double)dcs2<Q>(a) * (double)rho);
}

// dJ/dc = dJ/d(eta^2) * 2 eta / c_ref, and lambda^0 unpadded
__global__ void adjoint_finish(const StepArgs a, const double *grad, float *grad_c, double inv_cref,
                               const float *lam, float *grad_g0, int Q) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = (long long)a.nx * a.ny;
    if (k >= total) return;
    int y = (int)(k / a.nx), x = (int)(k - (long long)y * a.nx);
    long long idx = (long long)y * a.pitch + x;
    if (grad_c) grad_c[k] = (float)(grad[idx] * 2.0 * sqrt((double)a.eta2[idx]) * inv_cref);
    if (grad_g0)
        for (int i = 0; i < Q; i++) grad_g0[i * total + k] = lam[i * a.plane + idx];
}

using AdjFn = void (*)(const StepArgs, const AdjArgs);

template <int Q, bool MRT> AdjFn adj_fn(bool per) {
    return per ? adjoint_kernel<Q, MRT, true> : adjoint_kernel<Q, MRT, false>;
}

AdjFn pick_adj(int Q, bool mrt, bool per) {
    if (Q == 9) return mrt ? adj_fn<9, true>(per) : adj_fn<9, false>(per);
    return mrt ? adj_fn<5, true>(per) : adj_fn<5, false>(per);
}

AdjFn pick_adj_rec(int Q, bool per) {
    if (Q == 9) return per ? adjoint_receivers<9, true> : adjoint_receivers<9, false>;
    return per ? adjoint_receivers<5, true> : adjoint_receivers<5, false>;
}

}  // namespace

void ckpt_reset(lb_ctx *ctx) {
    ctx->ckpt_count = 0;
    ctx->ckpt_t0 = ctx->t;
}

lb_status ckpt_maybe_save(lb_ctx *ctx) {
    const long long rel = ctx->t - ctx->ckpt_t0;
    if (rel < 0 || rel % ctx->ckpt_every != 0) return LB_OK;
    const long long k = rel / ctx->ckpt_every;
    if (k != ctx->ckpt_count) return LB_OK;  // only extend a contiguous run
    const size_t bytes = (size_t)ctx->Q * ctx->ny * ctx->pitch * ctx->ebytes;
    if ((size_t)k >= ctx->ckpt.size()) {
        void *p = dev_alloc(ctx, bytes);
        if (!p) return fail(ctx, LB_ENOMEM, "checkpoint %lld", k);
        ctx->ckpt.push_back(p);
    }
    cudaError_t e = cudaMemcpyAsync(ctx->ckpt[k], ctx->pop[ctx->cur], bytes,
                                    cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "checkpoint copy");
    if (k == 0) ctx->ckpt_raw0 = ctx->raw;
    ctx->ckpt_count = (int)k + 1;
    return LB_OK;
}

bool ckpt_reserve(lb_ctx *ctx, void **dst, const void **src, size_t *bytes) {
    const long long rel = ctx->t - ctx->ckpt_t0;
    if (rel < 0 || rel % ctx->ckpt_every != 0) return false;
    const long long k = rel / ctx->ckpt_every;
    if (k != ctx->ckpt_count) return false;
    const size_t b = (size_t)ctx->Q * ctx->ny * ctx->pitch * ctx->ebytes;
    if ((size_t)k >= ctx->ckpt.size()) {
        void *p = dev_alloc(ctx, b);
        if (!p) return false;
        ctx->ckpt.push_back(p);
    }
    *dst = ctx->ckpt[k];
    *src = ctx->pop[ctx->cur];
    *bytes = b;
    if (k == 0) ctx->ckpt_raw0 = ctx->raw;
    ctx->ckpt_count = (int)k + 1;
    return true;
}

extern "C" lb_status lb_checkpoint_every(lb_ctx *ctx, int every) {
    if (!ctx) return LB_EINVAL;
    if (every < 0) return fail(ctx, LB_EINVAL, "every < 0");
    if (every > 0 && (ctx->refined || ctx->cfg.storage != LB_F32))
        return fail(ctx, LB_ESTATE, "the adjoint needs an FP32 context without a patch");
    ctx->ckpt_every = every;
    ckpt_reset(ctx);
    return LB_OK;
}

extern "C" lb_status lb_adjoint(lb_ctx *ctx, const float *dJdp, int nt, float *grad_c,
                                double *grad_src, float *grad_g0, int on_device) {
    if (!ctx) return LB_EINVAL;
    const int C = ctx->ckpt_every;
    if (C <= 0) return fail(ctx, LB_ESTATE, "call lb_checkpoint_every before stepping");
    if (nt < 1) return fail(ctx, LB_EINVAL, "nt < 1");
    if (ctx->nrec > 0 && !dJdp) return fail(ctx, LB_EINVAL, "dJdp is NULL");
    if (ctx->t - ctx->ckpt_t0 < nt || (long long)ctx->ckpt_count * C < nt)
        return fail(ctx, LB_ESTATE, "checkpoints cover %lld steps, %d requested",
                    std::min<long long>(ctx->t - ctx->ckpt_t0, (long long)ctx->ckpt_count * C), nt);
    if (ctx->nrec > 0 && ctx->ckpt_t0 != ctx->t_rec0)
        return fail(ctx, LB_ESTATE, "receivers must be set at the checkpointed start time");
    const int Q = ctx->Q;
    const size_t plane = (size_t)ctx->ny * ctx->pitch, sbytes = (size_t)Q * plane * 4;
    const int C2 = std::max(1, (int)std::ceil(std::sqrt((double)C)));
    const int nsub = (C + C2 - 1) / C2;
    std::vector<void *> mine;
    auto grab = [&](size_t b) {
        void *p = dev_alloc(ctx, b);
        if (p) mine.push_back(p);
        return p;
    };
    auto release = [&](lb_status st) {
        cudaStreamSynchronize(ctx->stream);
        for (void *p : mine) dev_free(ctx, p);
        return st;
    };
    std::vector<float *> X(C2 + 1), SC(nsub);
    for (auto &p : X)
        if (!(p = static_cast<float *>(grab(sbytes)))) return release(fail(ctx, LB_ENOMEM, "replay states"));
    for (auto &p : SC)
        if (!(p = static_cast<float *>(grab(sbytes)))) return release(fail(ctx, LB_ENOMEM, "sub-checkpoints"));
    float *L[2];
    for (auto &p : L)
        if (!(p = static_cast<float *>(grab(sbytes)))) return release(fail(ctx, LB_ENOMEM, "adjoint state"));
    double *grad = static_cast<double *>(grab(plane * 8));
    double *gsrc = static_cast<double *>(grab((size_t)nt * 8));
    float *resid = nullptr;
    if (!grad || !gsrc) return release(fail(ctx, LB_ENOMEM, "gradient"));
    if (ctx->nrec > 0) {
        if (on_device) {
            resid = const_cast<float *>(dJdp);
        } else {
            resid = static_cast<float *>(grab((size_t)nt * ctx->nrec * 4));
            if (!resid) return release(fail(ctx, LB_ENOMEM, "residual"));
            cudaMemcpyAsync(resid, dJdp, (size_t)nt * ctx->nrec * 4, cudaMemcpyHostToDevice,
                            ctx->stream);
        }
    }
    cudaMemsetAsync(L[0], 0, sbytes, ctx->stream);
    cudaMemsetAsync(L[1], 0, sbytes, ctx->stream);
    cudaMemsetAsync(grad, 0, plane * 8, ctx->stream);
    cudaMemsetAsync(gsrc, 0, (size_t)nt * 8, ctx->stream);

    const bool mrt = ctx->cfg.collision == LB_MRT, per = ctx->cfg.boundary == LB_PERIODIC;
    StepFn fwd = pick_step(ctx);
    AdjFn adj = pick_adj(Q, mrt, per), adj_rec = pick_adj_rec(Q, per);
    StepArgs base = base_args(ctx);
    base.trace_row = nullptr;  // replays record nothing
    const long long t0 = ctx->ckpt_t0;
    const int grid_sites = (int)((plane + 255) / 256);
    // one forward step of the replay: in -> out at absolute time t
    auto replay = [&](const float *in, bool raw, float *out, long long t) {
        StepArgs a = base;
        a.in = in;
        a.out = out;
        a.raw = raw ? 1 : 0;
        a.t = t;
        fwd<<<a.main_blocks, kThreads, 0, ctx->stream>>>(a);
    };
    int li = 0;  // L[li] holds lambda^{t+1}
    const int nseg = (nt + C - 1) / C;
    for (int k = nseg - 1; k >= 0; k--) {
        const long long ta = t0 + (long long)k * C, tb = std::min<long long>(ta + C, t0 + nt);
        const bool raw_a = (k == 0) && ctx->ckpt_raw0;
        // place sub-checkpoints
        cudaMemcpyAsync(SC[0], ctx->ckpt[k], sbytes, cudaMemcpyDeviceToDevice, ctx->stream);
        const int nsc = (int)((tb - ta + C2 - 1) / C2);
        for (int j = 1; j < nsc; j++) {
            const float *cur = SC[j - 1];
            bool raw = raw_a && j == 1;
            for (int m = 0; m < C2; m++) {
                long long t = ta + (long long)(j - 1) * C2 + m;
                float *out = (m == C2 - 1) ? SC[j] : X[m & 1];
                replay(cur, raw, out, t);
                cur = out;
                raw = false;
            }
        }
        // sweep the sub-segments backwards
        for (int j = nsc - 1; j >= 0; j--) {
            const long long sa = ta + (long long)j * C2, sb = std::min<long long>(sa + C2, tb);
            const int len = (int)(sb - sa);
            const bool raw0 = raw_a && j == 0;
            cudaMemcpyAsync(X[0], SC[j], sbytes, cudaMemcpyDeviceToDevice, ctx->stream);
            for (int m = 0; m + 1 < len; m++) replay(X[m], raw0 && m == 0, X[m + 1], sa + m);
            for (int m = len - 1; m >= 0; m--) {
                StepArgs a = base;
                a.t = sa + m;
                AdjArgs d;
                d.lam_in = L[li];
                d.lam_out = L[li ^ 1];
                d.fwd = X[m];
                d.fwd_raw = (raw0 && m == 0) ? 1 : 0;
                d.grad = grad;
                d.grad_src = gsrc;
                d.t0 = t0;
                d.resid = resid;
                d.nrec = ctx->nrec;
                adj<<<grid_sites, 256, 0, ctx->stream>>>(a, d);
                if (ctx->nrec > 0)
                    adj_rec<<<(ctx->nrec + 255) / 256, 256, 0, ctx->stream>>>(a, d);
                li ^= 1;
            }
        }
    }
    lb_status st = check_launch(ctx, "adjoint");
    if (st != LB_OK) return release(st);
    // outputs
    const size_t N = (size_t)ctx->nx * ctx->ny;
    float *gc_dev = grad_c, *gg_dev = grad_g0;
    if (!on_device) {
        gc_dev = grad_c ? static_cast<float *>(grab(N * 4)) : nullptr;
        gg_dev = grad_g0 ? static_cast<float *>(grab(N * Q * 4)) : nullptr;
        if ((grad_c && !gc_dev) || (grad_g0 && !gg_dev))
            return release(fail(ctx, LB_ENOMEM, "output staging"));
    }
    StepArgs a = base;
    adjoint_finish<<<(int)((N + 255) / 256), 256, 0, ctx->stream>>>(a, grad, gc_dev,
                                                                   1.0 / ctx->cfg.c_ref, L[li],
                                                                   gg_dev, Q);
    cudaError_t e = cudaSuccess;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (!on_device) {
        if (grad_c) e = cudaMemcpyAsync(grad_c, gc_dev, N * 4, kind, ctx->stream);
        if (e == cudaSuccess && grad_g0)
            e = cudaMemcpyAsync(grad_g0, gg_dev, N * Q * 4, kind, ctx->stream);
    }
    if (e == cudaSuccess && grad_src)
        e = cudaMemcpyAsync(grad_src, gsrc, (size_t)nt * 8, kind, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return release(cuda_fail(ctx, e, "adjoint output"));
    return release(check_launch(ctx, "adjoint output"));
}
