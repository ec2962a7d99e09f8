// modes.cu -- Fourier projections of the pressure field, in FP64, for the
// dispersion diagnostics (the single-mode runs behind the paper's dispersion
// analysis, Sec. 3 and Fig. 3 / Fig. 4): for integer wave numbers (mx, my) on
// the nx x ny grid, k = 2 pi (mx / nx, my / ny) and
//     P(k, t) = sum_x p(x, t) exp(-i k . x),   p = c_s^2 rho (Eq. state).
// On a periodic homogeneous grid each Fourier mode evolves on its own under
// the one-step amplification matrix (Eq. MRT-LB dispersion), so the time
// series P(k, t) of a run started from a superposition of modes carries the
// eigenvalues of every excited mode; the host fits them (dispersion.py).
//
// rho is summed in FP64 from the stored populations; the phase is reduced
// exactly with integer arithmetic before sincospi.  Block partials are
// summed on the host in a fixed order, so results are reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "lb_kernels.cuh"
#include "lb_runtime.h"

using namespace lbk;
using namespace lbrt;

namespace {

constexpr int kModeChunk = 8;       // modes per launch (2 FP64 accumulators each)
constexpr int kModeThreads = 256;
constexpr int kModeBlocks = 304;    // 2 per SM on GB300, grid-stride over the sites

struct ModeArgs {
    const void *pop;        // current buffer
    int raw;                // 1: g(t) unshifted; 0: post-collision h(t-1), pulled
    int swap;               // in-place streaming: h(t-1)'s population i in slot opp(i)
    int periodic;
    const float *eta2;
    const float *scale;     // per-population scale (FP16 storage) or nullptr
    float c2r;              // D2Q9: c_s^2 / eta^2
    int nx, ny, pitch;
    long long plane;
    const int *modes;       // [m][2] integer wave numbers of this chunk
    int m;                  // modes in this chunk (<= kModeChunk)
    double *partial;        // [gridDim.x][kModeChunk][2]
};

template <int Q, typename ST>
__global__ void __launch_bounds__(kModeThreads) mode_partial_kernel(const ModeArgs a) {
    double acc[2 * kModeChunk];
#pragma unroll
    for (int j = 0; j < 2 * kModeChunk; j++) acc[j] = 0.0;
    const ST *pop = static_cast<const ST *>(a.pop);
    const long long n = (long long)a.nx * a.ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(s / a.nx), x = (int)(s - (long long)y * a.nx);
        double rho = 0.0;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            int xs = x - (a.raw ? 0 : Lat<Q>::cx(i)), ys = y - (a.raw ? 0 : Lat<Q>::cy(i));
            if (a.periodic) {
                xs = (xs + a.nx) % a.nx;
                ys = (ys + a.ny) % a.ny;
            } else if (xs < 0 || xs >= a.nx || ys < 0 || ys >= a.ny) {
                continue;
            }
            const int slot = a.swap ? Lat<Q>::opp(i) : i;
            rho += (double)Store<ST>::load1(pop + slot * a.plane + (long long)ys * a.pitch + xs) *
                   (double)(a.scale ? a.scale[i] : 1.f);
        }
        const double e2 = (double)a.eta2[(long long)y * a.pitch + x];
        const double p = (Q == 5 ? 0.5 * e2 : e2 * (double)a.c2r) * rho;
#pragma unroll
        for (int j = 0; j < kModeChunk; j++) {  // unrolled: the accumulators stay in registers
            if (j >= a.m) break;
            const long long mx = a.modes[2 * j], my = a.modes[2 * j + 1];
            // k . x / (2 pi) = mx x / nx + my y / ny, each term reduced mod 1 exactly
            const long long rx = ((mx * x) % a.nx + a.nx) % a.nx;
            const long long ry = ((my * y) % a.ny + a.ny) % a.ny;
            const double ph = (double)rx / a.nx + (double)ry / a.ny;
            double sn, cs;
            sincospi(2.0 * ph, &sn, &cs);
            acc[2 * j] += p * cs;
            acc[2 * j + 1] -= p * sn;
        }
    }
    // block reduction in a fixed order: warp tree, then warp 0 over the warp sums
    __shared__ double sm[2 * kModeChunk][kModeThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 2 * kModeChunk; j++) {
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sm[j][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * kModeChunk) {
        double v = 0.0;
        for (int k = 0; k < kModeThreads / 32; k++) v += sm[threadIdx.x][k];
        a.partial[(long long)blockIdx.x * 2 * kModeChunk + threadIdx.x] = v;
    }
}

using ModeFn = void (*)(const ModeArgs);

template <typename ST> ModeFn mode_fn(int Q) {
    return Q == 9 ? mode_partial_kernel<9, ST> : mode_partial_kernel<5, ST>;
}

}  // namespace

extern "C" lb_status lb_mode_projection(lb_ctx *ctx, const int *modes, int n_modes, double *out) {
    if (!ctx) return LB_EINVAL;
    if (!modes || !out || n_modes < 1) return fail(ctx, LB_EINVAL, "modes, out and n_modes >= 1");
    if (ctx->refined) return fail(ctx, LB_ESTATE, "mode projection of a refined context");
    if (ctx->Q == 7) return fail(ctx, LB_ESTATE, "mode projection is 2-D (D2Q5 / D2Q9)");
    if (ctx->cfg.storage == LB_F64)
        return fail(ctx, LB_ESTATE, "mode projection reads FP32 / 16-bit storage, not LB_F64");
    const int blocks = (int)std::min<long long>(
        kModeBlocks, ((long long)ctx->nx * ctx->ny + kModeThreads - 1) / kModeThreads);
    int *d_modes = static_cast<int *>(dev_alloc(ctx, (size_t)n_modes * 2 * sizeof(int)));
    double *d_part = static_cast<double *>(dev_alloc(ctx, (size_t)blocks * 2 * kModeChunk * 8));
    auto release = [&](lb_status st) {
        cudaStreamSynchronize(ctx->stream);
        if (d_modes) dev_free(ctx, d_modes);
        if (d_part) dev_free(ctx, d_part);
        return st;
    };
    if (!d_modes || !d_part) return release(fail(ctx, LB_ENOMEM, "mode projection buffers"));
    cudaError_t e = cudaMemcpyAsync(d_modes, modes, (size_t)n_modes * 2 * sizeof(int),
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return release(cuda_fail(ctx, e, "modes upload"));
    ModeArgs a;
    a.pop = ctx->pop[ctx->cur];
    a.raw = ctx->raw ? 1 : 0;
    a.swap = ctx->swap ? 1 : 0;
    a.periodic = ctx->cfg.boundary == LB_PERIODIC;
    a.eta2 = ctx->eta2;
    a.scale = current_scale(ctx);
    a.c2r = (float)(2.0 * ctx->cfg.w_ref[1] + 4.0 * ctx->cfg.w_ref[2]);
    a.nx = ctx->nx;
    a.ny = ctx->ny;
    a.pitch = ctx->pitch;
    a.plane = (long long)ctx->ny * ctx->pitch;
    a.partial = d_part;
    const ModeFn fn = ctx->cfg.storage == LB_BF16  ? mode_fn<__nv_bfloat16>(ctx->Q)
                      : ctx->cfg.storage == LB_F16 ? mode_fn<__half>(ctx->Q)
                                                   : mode_fn<float>(ctx->Q);
    std::vector<double> part((size_t)blocks * 2 * kModeChunk);
    for (int m0 = 0; m0 < n_modes; m0 += kModeChunk) {
        a.modes = d_modes + 2 * m0;
        a.m = std::min(kModeChunk, n_modes - m0);
        fn<<<blocks, kModeThreads, 0, ctx->stream>>>(a);
        e = cudaMemcpyAsync(part.data(), d_part, part.size() * 8, cudaMemcpyDeviceToHost,
                            ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return release(cuda_fail(ctx, e, "mode projection"));
        for (int j = 0; j < a.m; j++) {  // fixed order over the blocks
            double re = 0.0, im = 0.0;
            for (int b = 0; b < blocks; b++) {
                re += part[(size_t)b * 2 * kModeChunk + 2 * j];
                im += part[(size_t)b * 2 * kModeChunk + 2 * j + 1];
            }
            out[2 * (m0 + j)] = re;
            out[2 * (m0 + j) + 1] = im;
        }
    }
    return release(check_launch(ctx, "mode projection"));
}
