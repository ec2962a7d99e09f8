// refine.cu -- two-level grid refinement of Sec. 4 (ratio n = 2 in space and
// time) on the GPU.
//
// The coarse grid is the context's grid; a patch of coarse cells
// [x0, x0 + nxp] x [y0, y0 + nyp] is covered by a fine grid of
// (2 nxp + 1) x (2 nyp + 1) nodes, fine node (a, b) at coarse position
// (x0 + a/2, y0 + b/2), whose sound speed is the coarse c_map interpolated
// bilinearly.  The fine grid is stored with a one-node ghost ring: the
// populations that enter the fine grid across the interface I (the patch
// boundary) are written into the ghost ring, so the ordinary fused step kernel
// pulls them in.
//
// Coupling (Eq. grid refinement eqm dist, Eq. coarse-fine dist connect), read
// per population: a fine node of I takes from the coarse grid exactly the
// populations whose upstream node lies outside the fine grid,
//   g^f_i = g^eq_i + (g^c_i - g^eq_i) / 2,
// from coarse vectors interpolated linearly along I and in time (midpoint at
// odd fine times); a coarse node of I takes from the fine grid the populations
// whose upstream node lies strictly inside the patch,
//   g^c_i = g^eq_i + 2 (g^f_i - g^eq_i),
// g^eq being formed from the transferred vector's moments with the receiving
// grid's weights.  The factors 1/2 and 2 are those of the paper's lossless
// setting (tau = 1/2, s = 2).  For other rates the fine grid relaxes with
// tau_f - 1/2 = 2 (tau_c - 1/2) per relaxed moment, which keeps the physical
// viscosity continuous, and the non-equilibrium parts scale by tau_f / (2 tau_c)
// (coarse -> fine) and 2 tau_c / tau_f (fine -> coarse), moment by moment;
// at tau = 1/2 these are the paper's factors.  The coarse grid keeps running under the patch, which gives
// the full coarse vector on I (U, kept for two coarse times).
//
// One coarse step T (fused kernels, all on the context stream):
//   coarse step T (pull, collide, store; receivers outside the patch)
//   snapshot U(T) = coarse populations on I at time T (before correction)
//   [T >= 1] c2f into the fine ghost ring from (U(T-1) + U(T)) / 2, fine step 2T-1
//   c2f from U(T), fine step 2T (receivers inside the closed patch)
//   f2c: coarse nodes of I re-pulled, corrected from the fine state at 2T,
//        re-collided and stored over the coarse step's output.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "lb_kernels.cuh"
#include "lb_runtime.h"

using namespace lbk;
using namespace lbrt;

struct lb_refine {
    int x0, y0, nxp, nyp, nxf, nyf;  // patch (coarse cells) and fine node counts
    int gx, gy, pitch;               // fine grid with its ghost ring
    void *pop[2] = {nullptr, nullptr};
    int cur = 0;
    bool raw = false;
    float *eta2 = nullptr;
    int nI = 0;
    int2 *Ic = nullptr;              // coarse nodes of I
    float *U[3] = {nullptr, nullptr, nullptr};  // [nI][Q]: slots T % 2, plus one for peeks
    int nIf = 0;
    int4 *If = nullptr;              // fine nodes of I: (a, b, k1, k2), k2 < 0 when single
    int2 *rec_c = nullptr, *rec_f = nullptr;
    int *col_c = nullptr, *col_f = nullptr;
    int nrec_c = 0, nrec_f = 0;
    // relaxation on the fine grid, and the non-equilibrium rescales written as collisions:
    // g' = geq + F (g - geq) per non-conserved moment is a collision with rates 1 - F
    float omega_f = 2.f, s_f[9] = {};
    float c2f_omega = 0.5f, c2f_s[9] = {}, f2c_omega = -1.f, f2c_s[9] = {};
};

namespace {

__global__ void ref_medium_kernel(const float *c_map, int nx, int x0, int y0, int nxf, int nyf,
                                  int gx, int gy, int pitch, double inv_cref, float *eta2) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)gy * pitch) return;
    int pb = (int)(idx / pitch), pa = (int)(idx - (long long)pb * pitch);
    if (pa >= gx) {
        eta2[idx] = 0.f;
        return;
    }
    int a = min(max(pa - 1, 0), nxf - 1), b = min(max(pb - 1, 0), nyf - 1);
    int X = x0 + a / 2, Y = y0 + b / 2, ox = a & 1, oy = b & 1, cnt = 0;
    double s = 0.0;
    for (int dy = 0; dy <= oy; dy++)
        for (int dx = 0; dx <= ox; dx++) {
            s += (double)c_map[(long long)(Y + dy) * nx + X + dx];
            cnt++;
        }
    float cf = (float)(s / cnt);
    double eta = (double)cf * inv_cref;
    if (eta > 1.0) eta = 1.0;
    eta2[idx] = (float)(eta * eta);
}

// raw fine state g = g^eq(p / c_s^2, 0), p = bilinear interpolation of the coarse p0
template <int Q>
__global__ void ref_init_fine_kernel(StepArgs af, const float *p0, int nx, int x0, int y0,
                                     int nxf, int nyf) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= af.plane) return;
    int pb = (int)(idx / af.pitch), pa = (int)(idx - (long long)pb * af.pitch);
    int a = pa - 1, b = pb - 1;
    float p = 0.f;
    bool inside = a >= 0 && a < nxf && b >= 0 && b < nyf;
    if (inside && p0) {
        int X = x0 + a / 2, Y = y0 + b / 2, ox = a & 1, oy = b & 1, cnt = 0;
        double s = 0.0;
        for (int dy = 0; dy <= oy; dy++)
            for (int dx = 0; dx <= ox; dx++) {
                s += (double)p0[(long long)(Y + dy) * nx + X + dx];
                cnt++;
            }
        p = (float)(s / cnt);
    }
    float *o = static_cast<float *>(af.out);
    const float e2 = af.eta2[idx];
    for (int i = 0; i < Q; i++)
        o[i * af.plane + idx] = inside ? weight_i<Q>(i, e2, af) / cs2_of<Q>(e2, af) * p : 0.f;
}

template <int Q>
__device__ __forceinline__ float pull1(const float *in, int raw, int periodic, int x, int y,
                                       int i, int nx, int ny, int pitch, long long plane) {
    int xs = x, ys = y;
    if (!raw) {
        xs -= Lat<Q>::cx(i);
        ys -= Lat<Q>::cy(i);
    }
    if (periodic) {
        xs = (xs + nx) % nx;
        ys = (ys + ny) % ny;
    } else if (xs < 0 || xs >= nx || ys < 0 || ys >= ny) {
        return 0.f;
    }
    return in[i * plane + (long long)ys * pitch + xs];
}

template <int Q>
__global__ void ref_snapshot_kernel(StepArgs ac, const int2 *Ic, int nI, float *U) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nI) return;
    const float *in = static_cast<const float *>(ac.in);
    int2 X = Ic[k];  // at least one node from the coarse edges: no wrap needed
    for (int i = 0; i < Q; i++)
        U[(long long)k * Q + i] = pull1<Q>(in, ac.raw, 0, X.x, X.y, i, ac.nx, ac.ny, ac.pitch,
                                           ac.plane);
}

// coarse -> fine: write the entering populations of the fine nodes of I into
// the fine input buffer (at the upstream ghost node, or in place when raw).
template <int Q, bool MRT>
__global__ void ref_c2f_kernel(StepArgs af, StepArgs rs, const int4 *If, int nIf, const float *Ua,
                               const float *Ub, float alpha, int nxf, int nyf) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nIf) return;
    const int4 e = If[j];
    const int a = e.x, b = e.y;
    float gh[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        float v = (1.f - alpha) * Ua[(long long)e.z * Q + i] + alpha * Ub[(long long)e.z * Q + i];
        if (e.w >= 0) {
            v += (1.f - alpha) * Ua[(long long)e.w * Q + i] + alpha * Ub[(long long)e.w * Q + i];
            v *= 0.5f;
        }
        gh[i] = v;
    }
    const long long node = (long long)(b + 1) * af.pitch + (a + 1);
    // g^eq (fine weights) + factor (g - g^eq): a collision with the rescale rates rs
    if (Q == 5)
        collide5<MRT>(gh, af.eta2[node], rs);
    else
        collide9<MRT>(gh, af.eta2[node], rs);
    float *in = static_cast<float *>(const_cast<void *>(af.in));
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int ua = a - Lat<Q>::cx(i), ub = b - Lat<Q>::cy(i);
        if (ua >= 0 && ua < nxf && ub >= 0 && ub < nyf) continue;  // comes from the fine grid
        const long long pos =
            af.raw ? node : (long long)(ub + 1) * af.pitch + (ua + 1);
        in[i * af.plane + pos] = gh[i];
    }
}

// fine -> coarse on I, then collide (+ sponge) and overwrite the coarse output
template <int Q, bool MRT, bool PERIODIC>
__global__ void ref_f2c_kernel(StepArgs ac, StepArgs rs, const float *fin, int fraw, int fpitch,
                               long long fplane, const int2 *Ic, int nI, int x0, int y0, int nxp,
                               int nyp) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nI) return;
    const int2 X = Ic[k];
    const float *cin = static_cast<const float *>(ac.in);
    float g[Q], G[Q];
    const int fa = 1 + 2 * (X.x - x0), fb = 1 + 2 * (X.y - y0);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        g[i] = pull1<Q>(cin, ac.raw, PERIODIC, X.x, X.y, i, ac.nx, ac.ny, ac.pitch, ac.plane);
        G[i] = pull1<Q>(fin, fraw, 0, fa, fb, i, 1 << 30, 1 << 30, fpitch, fplane);
    }
    const float e2 = ac.eta2[(long long)X.y * ac.pitch + X.x];
    // g^eq (coarse weights) + factor (G - g^eq): a collision with the rescale rates rs
    if (Q == 5)
        collide5<MRT>(G, e2, rs);
    else
        collide9<MRT>(G, e2, rs);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int ux = X.x - Lat<Q>::cx(i), uy = X.y - Lat<Q>::cy(i);
        if (ux > x0 && ux < x0 + nxp && uy > y0 && uy < y0 + nyp) g[i] = G[i];
    }
    if (Q == 5)
        collide5<MRT>(g, e2, ac);
    else
        collide9<MRT>(g, e2, ac);
    float f = ac.sponge_w > 0 ? sponge_factor(X.x, X.y, ac) : 1.f;
    float *out = static_cast<float *>(ac.out);
#pragma unroll
    for (int i = 0; i < Q; i++) out[i * ac.plane + (long long)X.y * ac.pitch + X.x] = g[i] * f;
}

// pressure at the nodes of the closed patch from the coincident fine nodes
template <int Q>
__global__ void ref_overlay_kernel(StepArgs af, float *p, int nx, int x0, int y0, int nxp,
                                   int nyp) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int w = nxp + 1;
    if (k >= w * (nyp + 1)) return;
    int ca = k % w, cb = k / w;
    int fa = 1 + 2 * ca, fb = 1 + 2 * cb;
    const float *in = static_cast<const float *>(af.in);
    float rho = 0.f;
    for (int i = 0; i < Q; i++)
        rho += pull1<Q>(in, af.raw, 0, fa, fb, i, 1 << 30, 1 << 30, af.pitch, af.plane);
    p[(long long)(y0 + cb) * nx + (x0 + ca)] =
        cs2_of<Q>(af.eta2[(long long)fb * af.pitch + fa], af) * rho;
}

int blocks_for(long long n) { return (int)((n + 255) / 256); }

StepArgs fine_args(const lb_ctx *ctx) {
    const lb_refine *R = ctx->ref;
    StepArgs a = base_args(ctx);
    a.eta2 = R->eta2;
    a.mid = nullptr;  // the fine grid reads its own eta^2 plane
    a.mid_tab = nullptr;
    a.omega = R->omega_f;  // viscosity-continuous fine relaxation
    for (int k = 0; k < 9; k++) a.s[k] = R->s_f[k];
    a.nx = R->gx;
    a.ny = R->gy;
    a.pitch = R->pitch;
    a.plane = (long long)R->gy * R->pitch;
    a.segs = (R->gx + kSitesPerWarp - 1) / kSitesPerWarp;
    a.main_blocks = (int)(((long long)a.segs * R->gy + kWarps - 1) / kWarps);
    a.sponge_w = 0;
    a.src_tab = nullptr;
    a.src_nt = 0;
    a.rec = nullptr;
    a.nrec = 0;
    a.trace_row = nullptr;
    a.rec_col = nullptr;
    a.scale_in = nullptr;
    return a;
}

// rates whose collision is the non-equilibrium rescale g^eq + F (g - g^eq)
StepArgs rescale_args(StepArgs a, float omega, const float *s) {
    a.omega = omega;
    for (int k = 0; k < 9; k++) a.s[k] = s[k];
    return a;
}

template <int Q, bool MRT>
void c2f_q(lb_ctx *ctx, const StepArgs &af, const float *Ua, const float *Ub, float alpha) {
    lb_refine *R = ctx->ref;
    ref_c2f_kernel<Q, MRT><<<blocks_for(R->nIf), 256, 0, ctx->stream>>>(
        af, rescale_args(af, R->c2f_omega, R->c2f_s), R->If, R->nIf, Ua, Ub, alpha, R->nxf, R->nyf);
}

void launch_c2f(lb_ctx *ctx, const float *Ua, const float *Ub, float alpha) {
    lb_refine *R = ctx->ref;
    StepArgs af = fine_args(ctx);
    af.in = R->pop[R->cur];
    af.raw = R->raw ? 1 : 0;
    const bool mrt = ctx->cfg.collision == LB_MRT;
    if (ctx->Q == 9) {
        if (mrt) c2f_q<9, true>(ctx, af, Ua, Ub, alpha); else c2f_q<9, false>(ctx, af, Ua, Ub, alpha);
    } else {
        if (mrt) c2f_q<5, true>(ctx, af, Ua, Ub, alpha); else c2f_q<5, false>(ctx, af, Ua, Ub, alpha);
    }
}

// one fine step (pull from pop[cur], store into pop[cur ^ 1]); receivers at trace row `row`
void launch_fine_step(lb_ctx *ctx, float *trace_row) {
    lb_refine *R = ctx->ref;
    StepArgs af = fine_args(ctx);
    af.in = R->pop[R->cur];
    af.out = R->pop[R->cur ^ 1];
    af.raw = R->raw ? 1 : 0;
    int rec_blocks = 0;
    if (trace_row && R->nrec_f > 0) {
        af.rec = R->rec_f;
        af.nrec = R->nrec_f;
        af.rec_col = R->col_f;
        af.trace_row = trace_row;
        rec_blocks = (R->nrec_f + kThreads - 1) / kThreads;
    }
    StepFn fn = pick_step_for(ctx->Q, ctx->cfg.collision == LB_MRT, false, LB_F32);
    fn<<<af.main_blocks + rec_blocks, kThreads, 0, ctx->stream>>>(af);
    R->cur ^= 1;
    R->raw = false;
}

void launch_snapshot(lb_ctx *ctx, const void *coarse_in, bool raw, float *U) {
    lb_refine *R = ctx->ref;
    StepArgs ac = base_args(ctx);
    ac.in = coarse_in;
    ac.raw = raw ? 1 : 0;
    if (ctx->Q == 9)
        ref_snapshot_kernel<9><<<blocks_for(R->nI), 256, 0, ctx->stream>>>(ac, R->Ic, R->nI, U);
    else
        ref_snapshot_kernel<5><<<blocks_for(R->nI), 256, 0, ctx->stream>>>(ac, R->Ic, R->nI, U);
}

template <int Q, bool MRT>
void f2c_q(lb_ctx *ctx, const StepArgs &ac, const float *fin, int fraw) {
    lb_refine *R = ctx->ref;
    long long fplane = (long long)R->gy * R->pitch;
    if (ctx->cfg.boundary == LB_PERIODIC)
        ref_f2c_kernel<Q, MRT, true><<<blocks_for(R->nI), 256, 0, ctx->stream>>>(
            ac, rescale_args(ac, R->f2c_omega, R->f2c_s), fin, fraw, R->pitch, fplane, R->Ic,
            R->nI, R->x0, R->y0, R->nxp, R->nyp);
    else
        ref_f2c_kernel<Q, MRT, false><<<blocks_for(R->nI), 256, 0, ctx->stream>>>(
            ac, rescale_args(ac, R->f2c_omega, R->f2c_s), fin, fraw, R->pitch, fplane, R->Ic,
            R->nI, R->x0, R->y0, R->nxp, R->nyp);
}

void launch_f2c(lb_ctx *ctx, const StepArgs &ac, const float *fin, int fraw) {
    bool mrt = ctx->cfg.collision == LB_MRT;
    if (ctx->Q == 9) {
        if (mrt) f2c_q<9, true>(ctx, ac, fin, fraw); else f2c_q<9, false>(ctx, ac, fin, fraw);
    } else {
        if (mrt) f2c_q<5, true>(ctx, ac, fin, fraw); else f2c_q<5, false>(ctx, ac, fin, fraw);
    }
}

}  // namespace

lb_status refine_setup(lb_ctx *ctx, const lb_config *cfg, const float *c_map_dev) {
    const lb_patch P = cfg->patches[0];
    if (P.ratio != 2) return fail(ctx, LB_EINVAL, "patch ratio must be 2");
    if (cfg->storage != LB_F32) return fail(ctx, LB_EINVAL, "refinement needs FP32 storage");
    if (P.nx_c < 1 || P.ny_c < 1 || P.x0 < 1 || P.y0 < 1 || P.x0 + P.nx_c > ctx->nx - 2 ||
        P.y0 + P.ny_c > ctx->ny - 2)
        return fail(ctx, LB_EINVAL, "patch must lie inside the grid with a 1-node margin");
    lb_refine *R = new lb_refine();
    ctx->ref = R;
    {  // fine rates and rescale factors (tau_f - 1/2 = 2 (tau_c - 1/2), per relaxed moment)
        auto fine_tau = [](double tc) { return 0.5 + 2.0 * (tc - 0.5); };
        const double tc = cfg->tau, tf = fine_tau(tc);
        R->omega_f = (float)(1.0 / tf);
        R->c2f_omega = (float)(1.0 - tf / (2.0 * tc));
        R->f2c_omega = (float)(1.0 - 2.0 * tc / tf);
        for (int k = 0; k < 9; k++) {
            const double tck = 1.0 / cfg->s[k], tfk = fine_tau(tck);
            R->s_f[k] = (float)(1.0 / tfk);
            R->c2f_s[k] = (float)(1.0 - tfk / (2.0 * tck));
            R->f2c_s[k] = (float)(1.0 - 2.0 * tck / tfk);
        }
    }
    R->x0 = P.x0;
    R->y0 = P.y0;
    R->nxp = P.nx_c;
    R->nyp = P.ny_c;
    R->nxf = 2 * P.nx_c + 1;
    R->nyf = 2 * P.ny_c + 1;
    R->gx = R->nxf + 2;
    R->gy = R->nyf + 2;
    R->pitch = round_up(R->gx, 32);
    const size_t plane = (size_t)R->gy * R->pitch;
    const int Q = ctx->Q;
    for (int b = 0; b < 2; b++) {
        R->pop[b] = dev_alloc(ctx, (size_t)Q * plane * 4);
        if (!R->pop[b]) return fail(ctx, LB_ENOMEM, "fine population buffer");
        cudaMemsetAsync(R->pop[b], 0, (size_t)Q * plane * 4, ctx->stream);
    }
    R->eta2 = static_cast<float *>(dev_alloc(ctx, plane * 4));
    if (!R->eta2) return fail(ctx, LB_ENOMEM, "fine medium");
    ref_medium_kernel<<<blocks_for((long long)plane), 256, 0, ctx->stream>>>(
        c_map_dev, ctx->nx, R->x0, R->y0, R->nxf, R->nyf, R->gx, R->gy, R->pitch,
        1.0 / ctx->cfg.c_ref, R->eta2);
    // interface node lists
    std::vector<int2> Ic;
    std::vector<int> idx((size_t)(R->nxp + 1) * (R->nyp + 1), -1);
    for (int Y = R->y0; Y <= R->y0 + R->nyp; Y++)
        for (int X = R->x0; X <= R->x0 + R->nxp; X++)
            if (X == R->x0 || X == R->x0 + R->nxp || Y == R->y0 || Y == R->y0 + R->nyp) {
                idx[(size_t)(Y - R->y0) * (R->nxp + 1) + (X - R->x0)] = (int)Ic.size();
                Ic.push_back(make_int2(X, Y));
            }
    auto kidx = [&](int X, int Y) { return idx[(size_t)(Y - R->y0) * (R->nxp + 1) + (X - R->x0)]; };
    std::vector<int4> If;
    for (int b = 0; b < R->nyf; b++)
        for (int a = 0; a < R->nxf; a++) {
            if (!(a == 0 || a == R->nxf - 1 || b == 0 || b == R->nyf - 1)) continue;
            int X = R->x0 + a / 2, Y = R->y0 + b / 2;
            int k1 = kidx(X, Y), k2 = -1;
            if (a & 1)
                k2 = kidx(X + 1, Y);
            else if (b & 1)
                k2 = kidx(X, Y + 1);
            If.push_back(make_int4(a, b, k1, k2));
        }
    R->nI = (int)Ic.size();
    R->nIf = (int)If.size();
    R->Ic = static_cast<int2 *>(dev_alloc(ctx, Ic.size() * sizeof(int2)));
    R->If = static_cast<int4 *>(dev_alloc(ctx, If.size() * sizeof(int4)));
    for (int s = 0; s < 3; s++) R->U[s] = static_cast<float *>(dev_alloc(ctx, (size_t)R->nI * Q * 4));
    if (!R->Ic || !R->If || !R->U[0] || !R->U[1] || !R->U[2])
        return fail(ctx, LB_ENOMEM, "interface buffers");
    cudaMemcpyAsync(R->Ic, Ic.data(), Ic.size() * sizeof(int2), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(R->If, If.data(), If.size() * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "refinement setup");
    ctx->refined = true;
    return check_launch(ctx, "refinement setup");
}

void refine_destroy(lb_ctx *ctx) {
    delete ctx->ref;  // device buffers are owned by the context's allocation list
    ctx->ref = nullptr;
}

bool refine_contains(const lb_ctx *ctx, int x, int y) {
    const lb_refine *R = ctx->ref;
    return R && x >= R->x0 && x <= R->x0 + R->nxp && y >= R->y0 && y <= R->y0 + R->nyp;
}

lb_status refine_set_receivers(lb_ctx *ctx, const int *xy, int nrec) {
    lb_refine *R = ctx->ref;
    std::vector<int2> rc, rf;
    std::vector<int> cc, cf;
    for (int r = 0; r < nrec; r++) {
        int x = xy[2 * r], y = xy[2 * r + 1];
        if (refine_contains(ctx, x, y)) {
            rf.push_back(make_int2(1 + 2 * (x - R->x0), 1 + 2 * (y - R->y0)));
            cf.push_back(r);
        } else {
            rc.push_back(make_int2(x, y));
            cc.push_back(r);
        }
    }
    R->nrec_c = (int)rc.size();
    R->nrec_f = (int)rf.size();
    R->rec_c = static_cast<int2 *>(dev_alloc(ctx, std::max<size_t>(1, rc.size()) * sizeof(int2)));
    R->rec_f = static_cast<int2 *>(dev_alloc(ctx, std::max<size_t>(1, rf.size()) * sizeof(int2)));
    R->col_c = static_cast<int *>(dev_alloc(ctx, std::max<size_t>(1, cc.size()) * sizeof(int)));
    R->col_f = static_cast<int *>(dev_alloc(ctx, std::max<size_t>(1, cf.size()) * sizeof(int)));
    if (!R->rec_c || !R->rec_f || !R->col_c || !R->col_f)
        return fail(ctx, LB_ENOMEM, "receiver lists");
    if (!rc.empty()) {
        cudaMemcpyAsync(R->rec_c, rc.data(), rc.size() * sizeof(int2), cudaMemcpyHostToDevice,
                        ctx->stream);
        cudaMemcpyAsync(R->col_c, cc.data(), cc.size() * sizeof(int), cudaMemcpyHostToDevice,
                        ctx->stream);
    }
    if (!rf.empty()) {
        cudaMemcpyAsync(R->rec_f, rf.data(), rf.size() * sizeof(int2), cudaMemcpyHostToDevice,
                        ctx->stream);
        cudaMemcpyAsync(R->col_f, cf.data(), cf.size() * sizeof(int), cudaMemcpyHostToDevice,
                        ctx->stream);
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "receiver upload");
    return LB_OK;
}

lb_status refine_after_set_state(lb_ctx *ctx, const float *p0_dev) {
    lb_refine *R = ctx->ref;
    StepArgs af = fine_args(ctx);
    R->cur = 0;
    af.out = R->pop[0];
    if (ctx->Q == 9)
        ref_init_fine_kernel<9><<<blocks_for(af.plane), 256, 0, ctx->stream>>>(
            af, p0_dev, ctx->nx, R->x0, R->y0, R->nxf, R->nyf);
    else
        ref_init_fine_kernel<5><<<blocks_for(af.plane), 256, 0, ctx->stream>>>(
            af, p0_dev, ctx->nx, R->x0, R->y0, R->nxf, R->nyf);
    R->raw = true;
    return check_launch(ctx, "refined initial state");
}

lb_status refine_step(lb_ctx *ctx, int n) {
    lb_refine *R = ctx->ref;
    StepFn coarse_fn = pick_step(ctx);
    for (int k = 0; k < n; k++) {
        const long long T = ctx->t;
        float *Ucur = R->U[T & 1], *Uprev = R->U[(T + 1) & 1];
        long long row = T - ctx->t_rec0;
        float *trace_row = (ctx->trace && row >= 0 && row < ctx->trace_cap)
                               ? ctx->trace + row * ctx->nrec : nullptr;
        // coarse step T
        StepArgs ac = base_args(ctx);
        ac.in = ctx->pop[ctx->cur];
        ac.out = ctx->pop[ctx->cur ^ 1];
        ac.t = T;
        ac.raw = ctx->raw ? 1 : 0;
        ac.rec = R->rec_c;
        ac.nrec = R->nrec_c;
        ac.rec_col = R->col_c;
        ac.trace_row = R->nrec_c > 0 ? trace_row : nullptr;
        int rec_blocks = ac.trace_row ? (R->nrec_c + kThreads - 1) / kThreads : 0;
        coarse_fn<<<ac.main_blocks + rec_blocks, kThreads, 0, ctx->stream>>>(ac);
        launch_snapshot(ctx, ac.in, ctx->raw, Ucur);
        if (T >= 1) {
            launch_c2f(ctx, Uprev, Ucur, 0.5f);
            launch_fine_step(ctx, nullptr);
        }
        launch_c2f(ctx, Ucur, Ucur, 1.0f);
        const float *fin_last = static_cast<const float *>(R->pop[R->cur]);
        const int fraw = R->raw ? 1 : 0;
        launch_fine_step(ctx, trace_row);
        launch_f2c(ctx, ac, fin_last, fraw);
        ctx->cur ^= 1;
        ctx->raw = false;
        ctx->t += 1;
    }
    return check_launch(ctx, "refined step");
}

// Pressure at the current time inside the closed patch.  The fine state at
// fine time 2t does not exist yet between steps, so the coupling and the fine
// sub-steps of step t are replayed into the buffers they will overwrite
// anyway (the spare fine buffer, its ghost ring, and the third U slot).
lb_status refine_overlay_pressure(lb_ctx *ctx, float *p_dev) {
    lb_refine *R = ctx->ref;
    const long long T = ctx->t;
    float *Ucur = R->U[2], *Uprev = R->U[(T + 1) & 1];
    launch_snapshot(ctx, ctx->pop[ctx->cur], ctx->raw, Ucur);
    const int cur0 = R->cur;
    const bool raw0 = R->raw;
    if (T >= 1) {
        launch_c2f(ctx, Uprev, Ucur, 0.5f);
        launch_fine_step(ctx, nullptr);
    }
    launch_c2f(ctx, Ucur, Ucur, 1.0f);
    StepArgs af = fine_args(ctx);
    af.in = R->pop[R->cur];
    af.raw = R->raw ? 1 : 0;
    int cnt = (R->nxp + 1) * (R->nyp + 1);
    if (ctx->Q == 9)
        ref_overlay_kernel<9><<<blocks_for(cnt), 256, 0, ctx->stream>>>(af, p_dev, ctx->nx, R->x0,
                                                                      R->y0, R->nxp, R->nyp);
    else
        ref_overlay_kernel<5><<<blocks_for(cnt), 256, 0, ctx->stream>>>(af, p_dev, ctx->nx, R->x0,
                                                                      R->y0, R->nxp, R->nyp);
    R->cur = cur0;  // the replay committed nothing
    R->raw = raw0;
    return check_launch(ctx, "refined pressure");
}
