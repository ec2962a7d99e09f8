// tblock.cu -- temporal blocking: K fused LB steps per launch with the tile
// resident in shared memory (overlapped tiling).  D2Q9 contexts use this kernel; D2Q5
// contexts use the row wavefront of tblock5.cu (the dispatch below).
//
// Each CTA owns an OUT x OUT tile of output sites, OUT = 48 - 2K, and loads
// the stored post-collision populations h^{t-1} of the 48 x 48 region made of
// the tile and a halo of K sites on every side.  It then performs K steps in
// shared memory, ping-ponging between two copies of the region: in step j
// every site whose distance to the region edge exceeds j (its neighbourhood is
// still valid) pulls g_i(x) = h_i(x - c_i) from one copy, collides (BGK or
// MRT), adds the source, applies the sponge and writes h into the other copy;
// one barrier per step.  After K steps the tile holds h^{t+K-1} and is stored.
// HBM traffic per output site falls from (2Q + 1) * 4 bytes per step to
// ((48 / OUT)^2 (Q + 1) + Q) * 4 bytes per K steps, for K * (48 - j)^2-type
// recomputation of the halo.  Receivers are gathered at each of the K time
// levels by the tile that owns them, from a per-tile receiver list.
//
// Thread layout: 384 threads, each owning the same 6 sites of the region for
// all K steps (site s = thread + 384 m, row-major, so a warp touches 32
// consecutive shared-memory words: no bank conflicts, including the +-1 and
// +-48 shifted pulls).  Per-site medium, sponge factor and ring distance are
// computed once and kept in registers.
//
// The arithmetic per site is the same as in step_kernel (lb_kernels.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "lb_kernels.cuh"
#include "lb_runtime.h"

using namespace lbk;
using namespace lbrt;

namespace {

constexpr int kW = kTbW;      // region width (tile + 2K halo)
constexpr int kNS = kTbNS;    // sites in the region
constexpr int kPer = kTbPer;  // 6 sites per thread

struct TbArgs {
    const int *tile_off;  // [ntiles + 1] receiver list offsets per tile
    const int *tile_rec;  // receiver indices grouped by tile
    int tiles_x;
};


// REC: also record rho of every level of the own tile (adjoint replays only)
template <int Q, bool MRT, bool PERIODIC, int K, bool REC>
__global__ void __launch_bounds__(kTbThreads) tb_kernel(const StepArgs a, const TbArgs tb) {
    pdl_trigger_and_wait();
    constexpr int W = kW, NS = kNS, OUT = W - 2 * K;
    extern __shared__ float smem[];  // two copies of [Q][NS]
    float *bufA = smem, *bufB = smem + Q * NS;
    const int X0 = blockIdx.x * OUT - K, Y0 = blockIdx.y * OUT - K;
    const int tid = threadIdx.x;
    const float *in = static_cast<const float *>(a.in);

    // ---- load the region into copy A (zero outside a zero-ghost domain)
    const bool interior = (K % 4 == 0) && (OUT % 4 == 0) && X0 >= 0 && Y0 >= 0 &&
                          X0 + W <= a.nx && Y0 + W <= a.ny;
    if (interior) {  // 16-byte loads: X0 = OUT bx - K is a multiple of 4
        constexpr int CH = W / 4;
        for (int e = tid; e < Q * W * CH; e += kTbThreads) {
            const int i = e / (W * CH), rem = e - i * (W * CH), r = rem / CH, c = rem - r * CH;
            const float4 v = *reinterpret_cast<const float4 *>(
                in + i * a.plane + (long long)(Y0 + r) * a.pitch + X0 + 4 * c);
            *reinterpret_cast<float4 *>(bufA + i * NS + r * W + 4 * c) = v;
        }
    } else {
        for (int e = tid; e < Q * NS; e += kTbThreads) {
            const int i = e / NS, s = e - i * NS, r = s / W, c = s - r * W;
            int gx = X0 + c, gy = Y0 + r;
            float v = 0.f;
            if (PERIODIC) {
                v = in[i * a.plane + (long long)wrap_mod(gy, a.ny) * a.pitch + wrap_mod(gx, a.nx)];
            } else if (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny) {
                v = in[i * a.plane + (long long)gy * a.pitch + gx];
            }
            bufA[i * NS + s] = v;
        }
    }
    // ---- per-thread sites: ring distance (-1: outside the domain), medium, sponge, source
    int ring[kPer];
    float e2[kPer], sf[kPer];
    unsigned srcmask = 0u, ownmask = 0u;  // ownmask: sites of this block's output tile
#pragma unroll
    for (int m = 0; m < kPer; m++) {
        const int s = tid + m * kTbThreads, r = s / W, c = s - r * W;
        int gx = X0 + c, gy = Y0 + r;
        bool live = true;
        if (PERIODIC) {
            gx = wrap_mod(gx, a.nx);
            gy = wrap_mod(gy, a.ny);
        } else {
            live = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny;
        }
        ring[m] = live ? min(min(r, c), min(W - 1 - r, W - 1 - c)) : -1;
        e2[m] = live ? a.eta2[(long long)gy * a.pitch + gx] : 0.f;
        sf[m] = (live && a.sponge_w > 0) ? sponge_factor(gx, gy, a) : 1.f;
        if (live && gx == a.src_x && gy == a.src_y) srcmask |= 1u << m;
        // own output sites, unwrapped coordinates inside the grid (the last tile row / column
        // may extend past nx / ny)
        if (live && r >= K && r < K + OUT && c >= K && c < K + OUT && X0 + c < a.nx &&
            Y0 + r < a.ny)
            ownmask |= 1u << m;
        if (!live)
#pragma unroll
            for (int i = 0; i < Q; i++) bufB[i * NS + s] = 0.f;  // copy A is already 0 there
    }
    __syncthreads();

    const int tile = blockIdx.y * tb.tiles_x + blockIdx.x;
    const int r0 = tb.tile_off ? tb.tile_off[tile] : 0;
    const int r1 = tb.tile_off ? tb.tile_off[tile + 1] : 0;
#pragma unroll 1
    for (int j = 0; j < K; j++) {
        const float *src = (j & 1) ? bufB : bufA;
        float *dst = (j & 1) ? bufA : bufB;
        const long long t = a.t + j;
        // receivers owned by this tile, at time t (level j, before its collision)
        if (a.trace_row) {
            for (int q = r0 + tid; q < r1; q += kTbThreads) {
                const int r = tb.tile_rec[q];
                const int2 xy = a.rec[r];
                const int ls = (xy.y - Y0) * W + (xy.x - X0);
                float rho = 0.f;
#pragma unroll
                for (int i = 0; i < Q; i++)
                    rho += src[i * NS + ls - Lat<Q>::cy(i) * W - Lat<Q>::cx(i)];
                a.trace_row[(long long)j * a.nrec + (a.rec_col ? a.rec_col[r] : r)] =
                    cs2_of<Q>(a.eta2[(long long)xy.y * a.pitch + xy.x], a) * rho;
            }
        }
        const float S = (srcmask && a.src_tab != nullptr && t < a.src_nt) ? a.src_tab[t] : 0.f;
#pragma unroll
        for (int m = 0; m < kPer; m++) {
            if (ring[m] <= j) continue;
            const int s = tid + m * kTbThreads;
            float g[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) g[i] = src[i * NS + s - Lat<Q>::cy(i) * W - Lat<Q>::cx(i)];
            if (REC && (ownmask & (1u << m))) {  // adjoint replay: rho of level j
                const int r = s / W, c = s - r * W;
                float rho = 0.f;
#pragma unroll
                for (int i = 0; i < Q; i++) rho += g[i];
                a.rho_out[j * a.rho_stride + (long long)(Y0 + r) * a.pitch + X0 + c] = rho;
            }
            if (Q == 5)
                collide5<MRT>(g, e2[m], a);
            else
                collide9<MRT>(g, e2[m], a);
            if (srcmask & (1u << m)) {
#pragma unroll
                for (int i = 0; i < Q; i++) g[i] += weight_i<Q>(i, e2[m], a) * S;
            }
#pragma unroll
            for (int i = 0; i < Q; i++) dst[i * NS + s] = g[i] * sf[m];
        }
        __syncthreads();
    }
    // ---- store the tile from the copy the last step wrote
    const float *fin = (K % 2 == 0) ? bufA : bufB;
    float *out = static_cast<float *>(a.out);
    const int OX = blockIdx.x * OUT, OY = blockIdx.y * OUT;
    const bool full = (K % 4 == 0) && (OUT % 4 == 0) && OX + OUT <= a.nx && OY + OUT <= a.ny;
    if (full) {
        constexpr int CH = OUT / 4;
        for (int e = tid; e < Q * OUT * CH; e += kTbThreads) {
            const int i = e / (OUT * CH), rem = e - i * (OUT * CH), r = rem / CH, c = rem - r * CH;
            const float4 v = *reinterpret_cast<const float4 *>(fin + i * NS + (r + K) * W + K + 4 * c);
            *reinterpret_cast<float4 *>(out + i * a.plane + (long long)(OY + r) * a.pitch + OX + 4 * c) = v;
        }
    } else {
        for (int e = tid; e < Q * OUT * OUT; e += kTbThreads) {
            const int i = e / (OUT * OUT), s = e - i * (OUT * OUT), r = s / OUT, c = s - r * OUT;
            const int gx = OX + c, gy = OY + r;
            if (gy < a.ny && gx < a.pitch)
                out[i * a.plane + (long long)gy * a.pitch + gx] =
                    gx < a.nx ? fin[i * NS + (r + K) * W + c + K] : 0.f;
        }
    }
}

using TbFn = void (*)(const StepArgs, const TbArgs);

template <int Q, bool MRT, int K> TbFn tb_fn_p(bool per, bool rec) {
    if (rec) return per ? tb_kernel<Q, MRT, true, K, true> : tb_kernel<Q, MRT, false, K, true>;
    return per ? tb_kernel<Q, MRT, true, K, false> : tb_kernel<Q, MRT, false, K, false>;
}
template <int K> TbFn tb_fn(int Q, bool mrt, bool per, bool rec) {
    if constexpr (K <= 4) {
        if (Q == 9) return mrt ? tb_fn_p<9, true, K>(per, rec) : tb_fn_p<9, false, K>(per, rec);
    }
    return nullptr;  // D2Q5 runs the wavefront kernel (tblock5.cu); see tb_supported
}

int tile_out(int K) { return kW - 2 * K; }

}  // namespace

// supported fused-step counts (D2Q9: shared memory holds two copies of 9 x 48^2 floats)
bool tb_supported(int Q, int K) { return Q == 5 ? tb5_supported(K) : (K == 2 || K == 4); }

lb_status tb_set_receivers(lb_ctx *ctx, const int *xy, int nrec) {
    if (ctx->Q == 5) return tb5_set_receivers(ctx, xy, nrec);
    const int T = tile_out(ctx->cfg.time_block);
    const int tx = (ctx->nx + T - 1) / T, ty = (ctx->ny + T - 1) / T;
    std::vector<int> cnt((size_t)tx * ty + 1, 0), order(std::max(nrec, 1));
    for (int r = 0; r < nrec; r++) cnt[(size_t)(xy[2 * r + 1] / T) * tx + xy[2 * r] / T + 1]++;
    for (size_t k = 1; k < cnt.size(); k++) cnt[k] += cnt[k - 1];
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    for (int r = 0; r < nrec; r++) order[pos[(size_t)(xy[2 * r + 1] / T) * tx + xy[2 * r] / T]++] = r;
    ctx->tb_off = static_cast<int *>(dev_alloc(ctx, cnt.size() * sizeof(int)));
    ctx->tb_rec = static_cast<int *>(dev_alloc(ctx, order.size() * sizeof(int)));
    if (!ctx->tb_off || !ctx->tb_rec) return fail(ctx, LB_ENOMEM, "tile receiver lists");
    cudaMemcpyAsync(ctx->tb_off, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice,
                    ctx->stream);
    cudaMemcpyAsync(ctx->tb_rec, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice,
                    ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tile receiver lists");
    return LB_OK;
}

// Launch K fused steps with the caller's arguments (a.in / a.out / a.t / a.trace_row /
// a.rho_out; a.in must not be raw).  Receivers only when a.trace_row is set and the
// tile lists exist.
lb_status tb_launch_args(lb_ctx *ctx, const StepArgs &a, int K) {
    if (!tb_supported(ctx->Q, K)) return fail(ctx, LB_EINVAL, "time_block %d not supported", K);
    if (ctx->Q == 5) return tb5_launch_args(ctx, a, K);
    const bool mrt = ctx->cfg.collision == LB_MRT, per = ctx->cfg.boundary == LB_PERIODIC;
    const bool rec = a.rho_out != nullptr;
    TbFn fn = nullptr;
    switch (K) {
        case 2: fn = tb_fn<2>(ctx->Q, mrt, per, rec); break;
        case 4: fn = tb_fn<4>(ctx->Q, mrt, per, rec); break;
        default: break;
    }
    if (!fn) return fail(ctx, LB_EINVAL, "time_block %d not supported", K);
    const int T = tile_out(K);
    TbArgs tb;
    tb.tile_off = a.trace_row ? ctx->tb_off : nullptr;
    tb.tile_rec = a.trace_row ? ctx->tb_rec : nullptr;
    tb.tiles_x = (ctx->nx + T - 1) / T;
    dim3 grid(tb.tiles_x, (ctx->ny + T - 1) / T);
    const size_t smem = 2 * (size_t)ctx->Q * kNS * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "temporal-blocking shared memory");
    e = launch_pdl(fn, grid, dim3(kTbThreads), smem, ctx->stream, a, tb);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "temporal-blocking launch");
    return LB_OK;
}

// K fused steps of the context from a non-raw FP32 state; traces for times t .. t+K-1 go
// to consecutive rows, so the caller only uses this while all K rows fit.
lb_status tb_launch(lb_ctx *ctx, int K) {
    StepArgs a = base_args(ctx);
    a.in = ctx->pop[ctx->cur];
    a.out = ctx->pop[ctx->cur ^ 1];
    a.t = ctx->t;
    a.raw = 0;
    long long row = ctx->t - ctx->t_rec0;
    const int *lists = ctx->Q == 5 ? ctx->tb5_off : ctx->tb_off;
    a.trace_row = (ctx->trace && lists && row >= 0 && row + K <= ctx->trace_cap)
                      ? ctx->trace + row * ctx->nrec : nullptr;
    // forward rho tape (the caller keeps K steps inside it): level j at rho_out + j plane
    a.rho_out = tape_row(ctx, ctx->t);
    a.rho_stride = (long long)ctx->ny * ctx->pitch;
    lb_status st = tb_launch_args(ctx, a, K);
    if (st != LB_OK) return st;
    ctx->cur ^= 1;
    ctx->t += K;
    return LB_OK;
}
