// f64.cu -- the test-only FP64 storage (LB_F64): populations, eta^2, the source table
// and the collision coefficients in FP64, so that a GPU run can be held to the FP64
// oracle at rounding level (about 1e-12) instead of FP32's 1e-5.
//
// The per-site arithmetic is the production code itself: collide5 / collide9 / collide7,
// weight_i, cs2_of, the source and the sponge of lb_kernels.cuh, instantiated with
// R = double.  Only the data movement is plain here: one thread per site, a direct
// indexed pull of g_i(x - c_i, t - 1) (Eq. streaming), no vector loads and no shuffles.
// Speed is not a goal of this path; the FP32 and 16-bit kernels are the product.
//
// Available: lb_step, lb_init_pressure, lb_set_state / lb_get_state / lb_get_pressure
// (FP32 arrays) and their FP64 forms below, receivers and the source.  Not available:
// refinement patches, time blocking, the adjoint, invariants, mode projections, serving.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "lbac.h"
#include "lb_kernels.cuh"
#include "lb_runtime.h"

using namespace lbk;

namespace {

constexpr int kT = 256;

// eta^2 = (c / c_ref)^2 in FP64 (pads 0), clamped at 1 as the FP32 medium is
__global__ void medium64_kernel(const float *c_map, double *eta2, int nx, int ny, int pitch,
                                double inv_cref) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)ny * pitch) return;
    const int y = (int)(idx / pitch), x = (int)(idx - (long long)y * pitch);
    double v = 0.0;
    if (x < nx) {
        double eta = (double)c_map[(long long)y * nx + x] * inv_cref;
        if (eta > 1.0) eta = 1.0;
        v = eta * eta;
    }
    eta2[idx] = v;
}

// g_i(x, t) for the site (x, row r): the pulled value g*_i(x - c_i, t - 1), or the stored
// value itself when the buffer holds g(t) (raw); zero outside a zero-ghost domain
template <int Q, bool PERIODIC>
__device__ __forceinline__ double pulled64(const StepArgs &a, const double *in, int x, int r,
                                           int i) {
    int xs = x, ys = r;
    if (!a.raw) {
        xs = x - Lat<Q>::cx(i);
        ys = pull_row<Q, PERIODIC>(a, r, i);
    }
    if (PERIODIC)
        xs = (xs + a.nx) % a.nx;
    else if (xs < 0 || xs >= a.nx || ys < 0)
        return 0.0;
    return in[i * a.plane + (long long)ys * a.pitch + xs];
}

// One step t-1 -> t at every site: pull, collision, source, sponge, store (pads stay 0)
template <int Q, bool MRT, bool PERIODIC>
__global__ void step64_kernel(StepArgs a) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)a.ny * a.pitch) return;
    const int r = (int)(idx / a.pitch), x = (int)(idx - (long long)r * a.pitch);
    const double *in = static_cast<const double *>(a.in);
    double *out = static_cast<double *>(a.out);
    if (x >= a.nx) {
        for (int i = 0; i < Q; i++) out[i * a.plane + idx] = 0.0;
        return;
    }
    double g[Q][1];
#pragma unroll
    for (int i = 0; i < Q; i++) g[i][0] = pulled64<Q, PERIODIC>(a, in, x, r, i);
    const double e2[1] = {a.eta2_64[idx]};
    const bool has_src =
        r == a.src_y && x == a.src_x && a.src64 != nullptr && a.t < a.src_nt;
    collide_sites<Q, MRT, 1, true, double>(g, e2, a, x, row_face_dist<Q>(r, a), has_src);
#pragma unroll
    for (int i = 0; i < Q; i++) out[i * a.plane + idx] = g[i][0];
}

// p_r(t) = c_s^2(x_r) sum_i g_i(x_r, t) of the pulled state, rounded once to the FP32 trace
template <int Q, bool PERIODIC>
__global__ void rec64_kernel(StepArgs a) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.nrec) return;
    const int2 xy = a.rec[k];
    const double *in = static_cast<const double *>(a.in);
    double rho = 0.0;
    for (int i = 0; i < Q; i++) rho += pulled64<Q, PERIODIC>(a, in, xy.x, xy.y, i);
    a.trace_row[k] = (float)(cs2_of<Q>(a.eta2_64[(long long)xy.y * a.pitch + xy.x], a) * rho);
}

// Write g(t) in place (raw).  mode 0: from pressure, g_i = (w_i / c_s^2) p (linear
// equilibrium at rest); mode 1: populations [Q][ny][nx].  Source in FP32 (f) or FP64 (d);
// both null: zero.
template <int Q>
__global__ void set64_kernel(StepArgs a, const float *f, const double *d, int mode) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)a.ny * a.pitch) return;
    const int y = (int)(idx / a.pitch), x = (int)(idx - (long long)y * a.pitch);
    double *o = static_cast<double *>(a.out);
    const long long n = (long long)a.ny * a.nx, s = (long long)y * a.nx + x;
    for (int i = 0; i < Q; i++) {
        double v = 0.0;
        if (x < a.nx && (f || d)) {
            if (mode == 0) {
                const double e2 = a.eta2_64[idx], p = f ? (double)f[s] : d[s];
                v = weight_i<Q>(i, e2, a) / cs2_of<Q>(e2, a) * p;
            } else {
                v = f ? (double)f[i * n + s] : d[i * n + s];
            }
        }
        o[i * a.plane + idx] = v;
    }
}

// mode 0: pressure [ny][nx]; mode 1: populations g(t) [Q][ny][nx]; into f (FP32) or d (FP64)
template <int Q, bool PERIODIC>
__global__ void get64_kernel(StepArgs a, float *f, double *d, int mode) {
    const long long n = (long long)a.ny * a.nx;
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int y = (int)(idx / a.nx), x = (int)(idx - (long long)y * a.nx);
    const double *in = static_cast<const double *>(a.in);
    double rho = 0.0;
    for (int i = 0; i < Q; i++) {
        const double v = pulled64<Q, PERIODIC>(a, in, x, y, i);
        if (mode == 1) {
            if (f) f[i * n + idx] = (float)v;
            else d[i * n + idx] = v;
        }
        rho += v;
    }
    if (mode == 0) {
        const double p = cs2_of<Q>(a.eta2_64[(long long)y * a.pitch + x], a) * rho;
        if (f) f[idx] = (float)p;
        else d[idx] = p;
    }
}

using Step64 = void (*)(StepArgs);
using Rec64 = void (*)(StepArgs);
using Get64 = void (*)(StepArgs, float *, double *, int);
using Set64 = void (*)(StepArgs, const float *, const double *, int);

template <int Q, bool MRT> Step64 step64_b(bool per) {
    return per ? step64_kernel<Q, MRT, true> : step64_kernel<Q, MRT, false>;
}
Step64 pick_step64(int Q, bool mrt, bool per) {
    if (Q == 7) return step64_b<7, false>(per);
    if (Q == 9) return mrt ? step64_b<9, true>(per) : step64_b<9, false>(per);
    return mrt ? step64_b<5, true>(per) : step64_b<5, false>(per);
}
template <int Q> Rec64 rec64_q(bool per) {
    return per ? rec64_kernel<Q, true> : rec64_kernel<Q, false>;
}
Rec64 pick_rec64(int Q, bool per) {
    return Q == 7 ? rec64_q<7>(per) : Q == 9 ? rec64_q<9>(per) : rec64_q<5>(per);
}
template <int Q> Get64 get64_q(bool per) {
    return per ? get64_kernel<Q, true> : get64_kernel<Q, false>;
}
Get64 pick_get64(int Q, bool per) {
    return Q == 7 ? get64_q<7>(per) : Q == 9 ? get64_q<9>(per) : get64_q<5>(per);
}
Set64 pick_set64(int Q) {
    return Q == 7 ? set64_kernel<7> : Q == 9 ? set64_kernel<9> : set64_kernel<5>;
}

unsigned blocks_for(long long n) { return (unsigned)((n + kT - 1) / kT); }

}  // namespace

using namespace lbrt;

lb_status f64_setup(lb_ctx *c, const float *cmap_dev, double cref) {
    const size_t plane = (size_t)c->ny * c->pitch;
    c->eta2_64 = static_cast<double *>(dev_alloc(c, plane * 8));
    c->coef64 = static_cast<double *>(dev_alloc(c, kNCo64 * 8));
    if (!c->eta2_64 || !c->coef64) return fail(c, LB_ENOMEM, "FP64 medium");
    medium64_kernel<<<blocks_for((long long)plane), kT, 0, c->stream>>>(
        cmap_dev, c->eta2_64, c->nx, c->ny, c->pitch, 1.0 / cref);
    // the FP64 counterparts of base_args' FP32 coefficients
    std::vector<double> co(kNCo64, 0.0);
    const lb_config &g = c->cfg;
    co[kCoOmega] = 1.0 / g.tau;
    for (int k = 0; k < 9; k++) co[kCoS + k] = g.s[k] / mrt_norm(c->Q, k);
    const double c2r = 2.0 * g.w_ref[1] + 4.0 * g.w_ref[2];
    co[kCoW1r] = g.w_ref[1];
    co[kCoW5r] = g.w_ref[2];
    co[kCoC2r] = c2r;
    co[kCoA1] = c2r > 0 ? g.w_ref[1] / c2r : 0.0;
    co[kCoA5] = c2r > 0 ? g.w_ref[2] / c2r : 0.0;
    co[kCoSmax] = g.sponge_sigma_max;
    co[kCoInvW] = g.sponge_width > 0 ? 1.0 / g.sponge_width : 0.0;
    cudaError_t e = cudaMemcpyAsync(c->coef64, co.data(), kNCo64 * 8, cudaMemcpyHostToDevice,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // co goes out of scope
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "FP64 medium");
    return LB_OK;
}

lb_status f64_set_source(lb_ctx *c, const double *wavelet, int nt) {
    if (c->src64) dev_free(c, c->src64);
    c->src64 = nullptr;
    if (nt == 0) return LB_OK;
    c->src64 = static_cast<double *>(dev_alloc(c, (size_t)nt * 8));
    if (!c->src64) return fail(c, LB_ENOMEM, "FP64 source table");
    cudaError_t e =
        cudaMemcpyAsync(c->src64, wavelet, (size_t)nt * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "FP64 source upload");
    return LB_OK;
}

lb_status f64_step(lb_ctx *c, int n) {
    const Step64 fn = pick_step64(c->Q, c->cfg.collision == LB_MRT, c->cfg.boundary == LB_PERIODIC);
    const Rec64 rec = pick_rec64(c->Q, c->cfg.boundary == LB_PERIODIC);
    const long long total = (long long)c->ny * c->pitch;
    for (int k = 0; k < n; k++) {
        StepArgs a = base_args(c);
        a.in = c->pop[c->cur];
        a.out = c->pop[c->cur ^ 1];
        a.t = c->t;
        a.raw = c->raw ? 1 : 0;
        const long long row = c->t - c->t_rec0;
        a.trace_row =
            (c->trace && row >= 0 && row < c->trace_cap) ? c->trace + row * c->nrec : nullptr;
        if (a.trace_row) rec<<<blocks_for(c->nrec), kT, 0, c->stream>>>(a);
        fn<<<blocks_for(total), kT, 0, c->stream>>>(a);
        c->raw = false;
        c->cur ^= 1;
        c->t += 1;
    }
    return check_launch(c, "step64_kernel");
}

// mode 0: pressure (nx ny values), 1: populations (Q nx ny); f (FP32) or d (FP64)
lb_status f64_set(lb_ctx *c, const float *f, const double *d, int on_device, int mode) {
    const size_t n = (size_t)c->nx * c->ny * (mode == 0 ? 1 : c->Q), eb = f ? 4 : 8;
    const void *src = f ? static_cast<const void *>(f) : static_cast<const void *>(d);
    void *tmp = nullptr;
    if (src && !on_device) {
        tmp = dev_alloc(c, n * eb);
        if (!tmp) return fail(c, LB_ENOMEM, "staging buffer");
        cudaError_t e = cudaMemcpyAsync(tmp, src, n * eb, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(c->stream);
            dev_free(c, tmp);
            return cuda_fail(c, e, "upload");
        }
        src = tmp;
    }
    StepArgs a = base_args(c);
    a.out = c->pop[c->cur];
    c->raw = true;
    pick_set64(c->Q)<<<blocks_for((long long)c->ny * c->pitch), kT, 0, c->stream>>>(
        a, f ? static_cast<const float *>(src) : nullptr,
        f ? nullptr : static_cast<const double *>(src), mode);
    lb_status st = check_launch(c, "set64_kernel");
    if (tmp) {
        cudaStreamSynchronize(c->stream);
        dev_free(c, tmp);
    }
    return st;
}

lb_status f64_get(lb_ctx *c, float *f, double *d, int on_device, int mode) {
    if (!f && !d) return fail(c, LB_EINVAL, "out is NULL");
    const size_t n = (size_t)c->nx * c->ny * (mode == 0 ? 1 : c->Q), eb = f ? 4 : 8;
    void *dst = f ? static_cast<void *>(f) : static_cast<void *>(d);
    if (!on_device) {
        dst = dev_alloc(c, n * eb);
        if (!dst) return fail(c, LB_ENOMEM, "staging buffer");
    }
    StepArgs a = base_args(c);
    a.in = c->pop[c->cur];
    a.raw = c->raw ? 1 : 0;
    pick_get64(c->Q, c->cfg.boundary == LB_PERIODIC)<<<blocks_for((long long)c->nx * c->ny), kT,
                                                       0, c->stream>>>(
        a, f ? static_cast<float *>(dst) : nullptr, f ? nullptr : static_cast<double *>(dst), mode);
    lb_status st = check_launch(c, "get64_kernel");
    cudaError_t e = cudaSuccess;
    if (st == LB_OK && !on_device)
        e = cudaMemcpyAsync(f ? static_cast<void *>(f) : static_cast<void *>(d), dst, n * eb,
                            cudaMemcpyDeviceToHost, c->stream);
    const cudaError_t e2 = cudaStreamSynchronize(c->stream);
    if (!on_device) dev_free(c, dst);
    if (st != LB_OK) return st;
    if (e != cudaSuccess) return cuda_fail(c, e, "download");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "stream");
    return LB_OK;
}

extern "C" {

lb_status lb_get_state_f64(lb_ctx *ctx, double *out, int on_device) {
    if (!ctx) return LB_EINVAL;
    if (ctx->cfg.storage != LB_F64) return fail(ctx, LB_EINVAL, "lb_get_state_f64 needs LB_F64 storage");
    if (!out) return fail(ctx, LB_EINVAL, "out is NULL");
    return f64_get(ctx, nullptr, out, on_device, 1);
}

lb_status lb_get_pressure_f64(lb_ctx *ctx, double *out, int on_device) {
    if (!ctx) return LB_EINVAL;
    if (ctx->cfg.storage != LB_F64)
        return fail(ctx, LB_EINVAL, "lb_get_pressure_f64 needs LB_F64 storage");
    if (!out) return fail(ctx, LB_EINVAL, "out is NULL");
    return f64_get(ctx, nullptr, out, on_device, 0);
}

lb_status lb_set_state_f64(lb_ctx *ctx, const double *in, int on_device) {
    if (!ctx) return LB_EINVAL;
    if (ctx->cfg.storage != LB_F64) return fail(ctx, LB_EINVAL, "lb_set_state_f64 needs LB_F64 storage");
    if (!in) return fail(ctx, LB_EINVAL, "state is NULL");
    return f64_set(ctx, nullptr, in, on_device, 1);
}

}  // extern "C"
