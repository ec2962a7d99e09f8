// tblock.cu -- temporal blocking: K fused LB steps per launch with the tile
// resident in shared memory (overlapped tiling).
//
// Each CTA owns a 32 x 32 tile of output sites.  It loads the stored
// post-collision populations h^{t-1} of the tile plus a halo of K sites on
// every side (a (32 + 2K)^2 region) and the per-site eta^2 once, then performs
// K steps in shared memory: in step j every site of the region whose
// neighbourhood is still valid (the valid region shrinks by one site per side
// per step) pulls g_i(x) = h_i(x - c_i) from shared memory, collides (BGK or
// MRT), adds the source, applies the sponge, and writes h back in place after a
// barrier.  After K steps the 32 x 32 interior holds h^{t+K-1} and is stored.
// HBM traffic per output site falls from (2 Q + 1) * 4 bytes per step to
// ((1 + 2K/32)^2 (Q + 1) + Q) * 4 bytes per K steps, at the price of the
// recomputed halo.  Receivers are gathered by the tile that owns them, at
// every one of the K time levels, from a per-tile receiver list.
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

constexpr int kTile = 32;
constexpr int kTbThreads = 256;

struct TbArgs {
    const int *tile_off;  // [ntiles + 1] receiver list offsets per tile
    const int *tile_rec;  // receiver indices grouped by tile
    int tiles_x;
};

template <int Q, bool MRT, bool PERIODIC, int K>
__global__ void __launch_bounds__(kTbThreads) tb_kernel(const StepArgs a, const TbArgs tb) {
    constexpr int W = kTile + 2 * K;       // region width
    constexpr int NS = W * W;              // sites in the region
    constexpr int PER = (NS + kTbThreads - 1) / kTbThreads;
    extern __shared__ float smem[];  // [Q][NS], dynamic (Q W^2 floats can exceed 48 KB)
    float(*sm)[NS] = reinterpret_cast<float(*)[NS]>(smem);
    const int X0 = blockIdx.x * kTile - K, Y0 = blockIdx.y * kTile - K;
    const float *in = static_cast<const float *>(a.in);

    // ---- load the region (zero outside a zero-ghost domain, wrapped when periodic)
    const bool interior = (K % 4 == 0) && X0 >= 0 && Y0 >= 0 && X0 + W <= a.nx && Y0 + W <= a.ny;
    if (interior) {  // 16-byte loads: X0 = 32 bx - K is a multiple of 4 when K is
        constexpr int CH = W / 4;
        for (int e = threadIdx.x; e < Q * W * CH; e += kTbThreads) {
            const int i = e / (W * CH), rem = e - i * (W * CH), r = rem / CH, c = rem - r * CH;
            const float4 v = *reinterpret_cast<const float4 *>(
                in + i * a.plane + (long long)(Y0 + r) * a.pitch + X0 + 4 * c);
            float *d = &sm[i][r * W + 4 * c];
            d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
        }
    } else {
        for (int e = threadIdx.x; e < Q * NS; e += kTbThreads) {
            const int i = e / NS, s = e - i * NS, r = s / W, c = s - r * W;
            int gx = X0 + c, gy = Y0 + r;
            float v = 0.f;
            if (PERIODIC) {
                gx = ((gx % a.nx) + a.nx) % a.nx;
                gy = ((gy % a.ny) + a.ny) % a.ny;
                v = in[i * a.plane + (long long)gy * a.pitch + gx];
            } else if (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny) {
                v = in[i * a.plane + (long long)gy * a.pitch + gx];
            }
            sm[i][s] = v;
        }
    }
    // per-thread sites: medium, sponge factor, domain membership
    float e2[PER], sf[PER];
    bool live[PER];
#pragma unroll
    for (int m = 0; m < PER; m++) {
        const int s = threadIdx.x + m * kTbThreads;
        const int r = s / W, c = s - r * W;
        int gx = X0 + c, gy = Y0 + r;
        bool inside = s < NS;
        if (PERIODIC) {
            gx = ((gx % a.nx) + a.nx) % a.nx;
            gy = ((gy % a.ny) + a.ny) % a.ny;
        } else {
            inside = inside && gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny;
        }
        live[m] = inside;
        e2[m] = inside ? a.eta2[(long long)gy * a.pitch + gx] : 0.f;
        sf[m] = (inside && a.sponge_w > 0) ? sponge_factor(gx, gy, a) : 1.f;
    }
    __syncthreads();

    const int tile = blockIdx.y * tb.tiles_x + blockIdx.x;
    const int r0 = tb.tile_off ? tb.tile_off[tile] : 0, r1 = tb.tile_off ? tb.tile_off[tile + 1] : 0;
#pragma unroll 1
    for (int j = 0; j < K; j++) {
        const long long t = a.t + j;
        // receivers owned by this tile, at time t (level j, before its collision)
        if (a.trace_row) {
            for (int q = r0 + (int)threadIdx.x; q < r1; q += kTbThreads) {
                const int r = tb.tile_rec[q];
                const int2 xy = a.rec[r];
                const int lx = xy.x - X0, ly = xy.y - Y0;
                float rho = 0.f;
#pragma unroll
                for (int i = 0; i < Q; i++)
                    rho += sm[i][(ly - Lat<Q>::cy(i)) * W + lx - Lat<Q>::cx(i)];
                a.trace_row[(long long)j * a.nrec + (a.rec_col ? a.rec_col[r] : r)] =
                    cs2_of<Q>(a.eta2[(long long)xy.y * a.pitch + xy.x], a) * rho;
            }
        }
        const bool src_on = a.src_tab != nullptr && t < a.src_nt;
        const float S = src_on ? a.src_tab[t] : 0.f;
        float nh[PER][Q];
#pragma unroll
        for (int m = 0; m < PER; m++) {
            const int s = threadIdx.x + m * kTbThreads;
            const int r = s / W, c = s - r * W;
            const bool upd = live[m] && r > j && r < W - 1 - j && c > j && c < W - 1 - j;
            if (!upd) continue;
            float g[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) g[i] = sm[i][s - Lat<Q>::cy(i) * W - Lat<Q>::cx(i)];
            if (Q == 5)
                collide5<MRT>(g, e2[m], a);
            else
                collide9<MRT>(g, e2[m], a);
            if (src_on && X0 + c == a.src_x && Y0 + r == a.src_y) {
#pragma unroll
                for (int i = 0; i < Q; i++) g[i] += weight_i<Q>(i, e2[m], a) * S;
            }
#pragma unroll
            for (int i = 0; i < Q; i++) nh[m][i] = g[i] * sf[m];
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < PER; m++) {
            const int s = threadIdx.x + m * kTbThreads;
            const int r = s / W, c = s - r * W;
            const bool upd = live[m] && r > j && r < W - 1 - j && c > j && c < W - 1 - j;
            if (!upd) continue;
#pragma unroll
            for (int i = 0; i < Q; i++) sm[i][s] = nh[m][i];
        }
        __syncthreads();
    }
    // ---- store the interior
    float *out = static_cast<float *>(a.out);
    const int OX = blockIdx.x * kTile, OY = blockIdx.y * kTile;
    for (int e = threadIdx.x; e < Q * kTile * kTile; e += kTbThreads) {
        const int i = e / (kTile * kTile), s = e - i * (kTile * kTile);
        const int r = s / kTile, c = s - r * kTile;
        const int gx = OX + c, gy = OY + r;
        if (gy < a.ny && gx < a.pitch) {
            float v = (gx < a.nx) ? sm[i][(r + K) * W + c + K] : 0.f;
            out[i * a.plane + (long long)gy * a.pitch + gx] = v;
        }
    }
}

using TbFn = void (*)(const StepArgs, const TbArgs);

template <int Q, bool MRT, int K> TbFn tb_fn_p(bool per) {
    return per ? tb_kernel<Q, MRT, true, K> : tb_kernel<Q, MRT, false, K>;
}
template <int K> TbFn tb_fn(int Q, bool mrt, bool per) {
    if constexpr (K <= 4) {
        if (Q == 9) return mrt ? tb_fn_p<9, true, K>(per) : tb_fn_p<9, false, K>(per);
    }
    if (Q == 9) return nullptr;  // beyond the D2Q9 register / shared-memory budget
    return mrt ? tb_fn_p<5, true, K>(per) : tb_fn_p<5, false, K>(per);
}

}  // namespace

// supported fused-step counts (register and shared-memory budget per lattice)
bool tb_supported(int Q, int K) {
    return Q == 5 ? (K == 2 || K == 4 || K == 6 || K == 8) : (K == 2 || K == 4);
}

static size_t tb_smem_bytes(int Q, int K) {
    const size_t W = kTile + 2 * K;
    return (size_t)Q * W * W * sizeof(float);
}

lb_status tb_set_receivers(lb_ctx *ctx, const int *xy, int nrec) {
    const int tx = (ctx->nx + kTile - 1) / kTile, ty = (ctx->ny + kTile - 1) / kTile;
    std::vector<int> cnt((size_t)tx * ty + 1, 0), order(nrec);
    for (int r = 0; r < nrec; r++) cnt[(size_t)(xy[2 * r + 1] / kTile) * tx + xy[2 * r] / kTile + 1]++;
    for (size_t k = 1; k < cnt.size(); k++) cnt[k] += cnt[k - 1];
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    for (int r = 0; r < nrec; r++) order[pos[(size_t)(xy[2 * r + 1] / kTile) * tx + xy[2 * r] / kTile]++] = r;
    ctx->tb_off = static_cast<int *>(dev_alloc(ctx, cnt.size() * sizeof(int)));
    ctx->tb_rec = static_cast<int *>(dev_alloc(ctx, std::max(1, nrec) * sizeof(int)));
    if (!ctx->tb_off || !ctx->tb_rec) return fail(ctx, LB_ENOMEM, "tile receiver lists");
    cudaMemcpyAsync(ctx->tb_off, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice,
                    ctx->stream);
    if (nrec > 0)
        cudaMemcpyAsync(ctx->tb_rec, order.data(), nrec * sizeof(int), cudaMemcpyHostToDevice,
                        ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tile receiver lists");
    return LB_OK;
}

// K fused steps from a non-raw FP32 state; traces for times t .. t+K-1 go to
// consecutive rows, so the caller only uses this while all K rows fit.
lb_status tb_launch(lb_ctx *ctx, int K) {
    const bool mrt = ctx->cfg.collision == LB_MRT, per = ctx->cfg.boundary == LB_PERIODIC;
    TbFn fn = nullptr;
    if (!tb_supported(ctx->Q, K)) return fail(ctx, LB_EINVAL, "time_block %d not supported", K);
    switch (K) {
        case 2: fn = tb_fn<2>(ctx->Q, mrt, per); break;
        case 4: fn = tb_fn<4>(ctx->Q, mrt, per); break;
        case 6: fn = tb_fn<6>(ctx->Q, mrt, per); break;
        case 8: fn = tb_fn<8>(ctx->Q, mrt, per); break;
        default: return fail(ctx, LB_EINVAL, "time_block %d not supported", K);
    }
    StepArgs a = base_args(ctx);
    a.in = ctx->pop[ctx->cur];
    a.out = ctx->pop[ctx->cur ^ 1];
    a.t = ctx->t;
    a.raw = 0;
    long long row = ctx->t - ctx->t_rec0;
    a.trace_row = (ctx->trace && row >= 0 && row + K <= ctx->trace_cap)
                      ? ctx->trace + row * ctx->nrec : nullptr;
    TbArgs tb;
    tb.tile_off = ctx->tb_off;
    tb.tile_rec = ctx->tb_rec;
    tb.tiles_x = (ctx->nx + kTile - 1) / kTile;
    if (!ctx->tb_off) a.trace_row = nullptr;
    dim3 grid(tb.tiles_x, (ctx->ny + kTile - 1) / kTile);
    const size_t smem = tb_smem_bytes(ctx->Q, K);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "temporal-blocking shared memory");
    fn<<<grid, kTbThreads, smem, ctx->stream>>>(a, tb);
    ctx->cur ^= 1;
    ctx->t += K;
    return LB_OK;
}
