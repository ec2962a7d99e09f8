// tblock5.cu -- host side of the D2Q5 wavefront temporal blocking (kernels: tblock5.cuh):
// FP32 instances, launch sizing, receiver row lists and the served batches.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "lb_kernels.cuh"
#include "lb_runtime.h"
#include "tblock5.cuh"

using namespace lbk;
using namespace lbrt;
using namespace lbtb5;

namespace lbtb5 {
Tb5Fn pick_f32(int K, bool mrt, bool rec) {
    switch (K) {
        case 2: return pick_k<2, float>(mrt, rec);
        case 4: return pick_k<4, float>(mrt, rec);
        case 6: return pick_k<6, float>(mrt, rec);
        case 8: return pick_k<8, float>(mrt, rec);
        case 16: return pick_k<16, float>(mrt, rec);
        default: return nullptr;
    }
}
Tb5BatchFn pick_batch_f32(int K, bool mrt) {
    if (K != kServeTb) return nullptr;
    return mrt ? tb5_batch_kernel<true, kServeTb, float> : tb5_batch_kernel<false, kServeTb, float>;
}
}  // namespace lbtb5

bool tb5_supported(int K) { return K == 2 || K == 4 || K == 6 || K == 8 || K == 16; }

// Per-row receiver lists of the wavefront kernel (rows of the context, x ascending).
lb_status tb5_set_receivers(lb_ctx *ctx, const int *xy, int nrec) {
    std::vector<int> off((size_t)ctx->ny + 2, 0), order(std::max(nrec, 1));
    for (int r = 0; r < nrec; r++) off[(size_t)xy[2 * r + 1] + 1]++;
    for (size_t k = 1; k < off.size(); k++) off[k] += off[k - 1];
    for (int r = 0; r < nrec; r++) order[r] = r;
    std::stable_sort(order.begin(), order.begin() + nrec, [&](int p, int q) {
        return xy[2 * p + 1] != xy[2 * q + 1] ? xy[2 * p + 1] < xy[2 * q + 1] : xy[2 * p] < xy[2 * q];
    });
    std::vector<int> xs(std::max(nrec, 1));
    for (int k = 0; k < nrec; k++) xs[k] = xy[2 * order[k]];
    ctx->tb5_off = static_cast<int *>(dev_alloc(ctx, off.size() * sizeof(int)));
    ctx->tb5_x = static_cast<int *>(dev_alloc(ctx, xs.size() * sizeof(int)));
    ctx->tb5_id = static_cast<int *>(dev_alloc(ctx, order.size() * sizeof(int)));
    if (!ctx->tb5_off || !ctx->tb5_x || !ctx->tb5_id) return fail(ctx, LB_ENOMEM, "row receiver lists");
    cudaMemcpyAsync(ctx->tb5_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice,
                    ctx->stream);
    cudaMemcpyAsync(ctx->tb5_x, xs.data(), xs.size() * sizeof(int), cudaMemcpyHostToDevice,
                    ctx->stream);
    cudaMemcpyAsync(ctx->tb5_id, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice,
                    ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "row receiver lists");
    return LB_OK;
}

// K fused D2Q5 steps with the caller's arguments (a.in must not be raw); receivers when
// a.trace_row is set and the row lists exist; rho of every level when a.rho_out is set
// (FP32 storage).
lb_status tb5_launch_args(lb_ctx *ctx, const StepArgs &a, int K) {
    const bool mrt = ctx->cfg.collision == LB_MRT, per = ctx->cfg.boundary == LB_PERIODIC;
    const bool rec = a.rho_out != nullptr;
    Tb5Fn fn = ctx->cfg.storage == LB_BF16 ? pick_bf16(K, mrt, rec)
             : ctx->cfg.storage == LB_F32  ? pick_f32(K, mrt, rec)
                                           : nullptr;
    if (!fn) return fail(ctx, LB_EINVAL, "time_block %d not supported for this storage", K);
    static int occ[17] = {0};  // resident CTAs per SM by K (the same for every variant)
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (!occ[K]) {
        int nb = 0;
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)4 * K * (kWS + 2) * sizeof(float)));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kWS,
                                                      (size_t)4 * K * (kWS + 2) * sizeof(float));
        occ[K] = std::max(1, nb);
    }
    const int OUT = kWS - 2 * K;
    const int strips = (ctx->nx + OUT - 1) / OUT;
    // rows per CTA: the chunks of one wave of CTAs over the SMs.  A CTA sweeps its H + 2K
    // rows one after another, so a wave of short chunks beats fewer tall ones even though
    // each chunk recomputes 2K warm-up rows (GB300, two-layer 1024^2, K = 8: chunks of at
    // least 8K rows gave 80 CTAs and 60 GLUPS)
    const int slots = std::max(1, occ[K] * std::max(sms, 1));
    const int chunks = std::max(1, slots / strips);
    const int H = std::max(1, (ctx->ny + chunks - 1) / chunks);
    Tb5Args tb;
    tb.row_off = a.trace_row ? ctx->tb5_off : nullptr;
    tb.rec_x = ctx->tb5_x;
    tb.rec_id = ctx->tb5_id;
    tb.H = H;
    tb.per = per ? 1 : 0;
    dim3 grid(strips, (ctx->ny + H - 1) / H);
    const size_t smem = (size_t)2 * K * 2 * (kWS + 2) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "temporal-blocking shared memory");
    e = launch_pdl(fn, grid, dim3(kWS), smem, ctx->stream, a, tb);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "temporal-blocking launch");
    return LB_OK;
}

// ------------------------------------------------------------- served batches --
// One launch of tb5_batch_kernel: the descriptors of its n shots in one staging block,
// [n] StepArgs, [n] Tb5Args, [n] strips, [n + 1] block prefixes.
size_t tb5_batch_bytes(int n) {
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    return up(n * sizeof(StepArgs)) + up(n * sizeof(Tb5Args)) + up(n * sizeof(int)) +
           up((n + 1) * sizeof(int));
}

namespace {
struct BatchLayout {
    StepArgs *a;
    Tb5Args *tb;
    int *strips, *first;
};
BatchLayout batch_layout(void *base, int n) {
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    char *p = static_cast<char *>(base);
    BatchLayout L;
    L.a = reinterpret_cast<StepArgs *>(p);
    p += up(n * sizeof(StepArgs));
    L.tb = reinterpret_cast<Tb5Args *>(p);
    p += up(n * sizeof(Tb5Args));
    L.strips = reinterpret_cast<int *>(p);
    p += up(n * sizeof(int));
    L.first = reinterpret_cast<int *>(p);
    return L;
}
}  // namespace

// Whether a served shot can take K steps in one batched launch now: D2Q5, FP32 or BF16,
// not from a raw state, no checkpoint or rho tape, its receiver rows listed, and K trace
// rows left.
bool tb5_batch_ready(const lb_ctx *ctx, int K) {
    if (ctx->Q != 5 || (ctx->cfg.storage != LB_F32 && ctx->cfg.storage != LB_BF16) || ctx->raw ||
        ctx->ckpt_every > 0 || ctx->rho_tape || ctx->refined || ctx->slab_nyg || !tb5_supported(K))
        return false;
    if (ctx->nrec > 0) {
        const long long row = ctx->t - ctx->t_rec0;
        if (!ctx->tb5_off || row < 0 || row + K > ctx->trace_cap) return false;
    }
    return true;
}

int tb5_strips(const lb_ctx *ctx, int K) {
    const int OUT = kWS - 2 * K;
    return (ctx->nx + OUT - 1) / OUT;
}

int tb5_batch_blocks(const lb_ctx *ctx, int K, int H) {
    H = std::max(1, std::min(ctx->ny, H));
    return tb5_strips(ctx, K) * ((ctx->ny + H - 1) / H);
}

int tb5_batch_wave(int K) {
    int dev = 0, sms = 0, nb = 0;
    Tb5BatchFn fn = pick_batch_f32(K, false);
    const size_t smem = (size_t)2 * K * 2 * (kWS + 2) * sizeof(float);
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && fn)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && fn) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kWS, smem);
    if (e != cudaSuccess) cudaGetLastError();  // this query's own failure: one CTA per SM
    return std::max(1, sms) * std::max(1, nb);
}

// Fill the host staging block `h` for K steps of ctxs[0 .. n), H output rows per CTA
// (advancing their time and buffers as if the launch ran); returns the launch's block count.
int tb5_batch_fill(lb_ctx *const *ctxs, int n, int K, int H, void *h) {
    BatchLayout L = batch_layout(h, n);
    const int OUT = kWS - 2 * K;
    int blocks = 0;
    for (int k = 0; k < n; k++) {
        lb_ctx *ctx = ctxs[k];
        StepArgs a = base_args(ctx);
        a.in = ctx->pop[ctx->cur];
        a.out = ctx->pop[ctx->cur ^ 1];
        a.t = ctx->t;
        a.raw = 0;
        const long long row = ctx->t - ctx->t_rec0;
        a.trace_row = ctx->nrec > 0 ? ctx->trace + row * ctx->nrec : nullptr;
        Tb5Args tb;
        tb.row_off = a.trace_row ? ctx->tb5_off : nullptr;
        tb.rec_x = ctx->tb5_x;
        tb.rec_id = ctx->tb5_id;
        tb.H = std::max(1, std::min(ctx->ny, H));
        tb.per = ctx->cfg.boundary == LB_PERIODIC ? 1 : 0;
        const int strips = (ctx->nx + OUT - 1) / OUT, chunks = (ctx->ny + tb.H - 1) / tb.H;
        L.a[k] = a;
        L.tb[k] = tb;
        L.strips[k] = strips;
        L.first[k] = blocks;
        blocks += strips * chunks;
        ctx->cur ^= 1;
        ctx->t += K;
    }
    L.first[n] = blocks;
    return blocks;
}

// The launch of a block filled by tb5_batch_fill and copied to device memory `d`.
cudaError_t tb5_batch_launch(const void *d, int n, int K, int blocks, bool mrt, bool per,
                             int storage, cudaStream_t stream) {
    (void)per;  // the periodic flag travels in each shot's Tb5Args
    Tb5BatchFn fn = storage == LB_BF16 ? pick_batch_bf16(K, mrt) : pick_batch_f32(K, mrt);
    if (!fn || n < 1 || blocks < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)2 * K * 2 * (kWS + 2) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    BatchLayout L = batch_layout(const_cast<void *>(d), n);
    return launch_pdl(fn, dim3(blocks), dim3(kWS), smem, stream, (const StepArgs *)L.a,
                      (const Tb5Args *)L.tb, (const int *)L.strips, (const int *)L.first, n);
}
