// tblock5.cu -- temporal blocking for D2Q5: K fused steps per launch as a row wavefront.
//
// A CTA of 256 threads owns a vertical strip of 256 columns (its output columns plus K
// on each side, recomputed) and a chunk of output rows, which it sweeps upward.  Thread c
// owns column c of the strip at every time level.  In wavefront iteration r
//   level 0   loads row r of h^{t-1} (the stored post-collision populations),
//   level l   (1 <= l <= K) pulls, collides and writes row r - l from level l-1,
// so each level lags the one below by a row and every level advances one row per
// iteration.  What a site of level l pulls from level l-1 (Eq. BGK-LB lhs, streaming
// g_i(x, t) = h_i(x - c_i, t - 1)):
//   g0 (x, y)      this thread, kept in a register from the previous iteration,
//   g2 (x, y - 1)  this thread, kept from two iterations back,
//   g4 (x, y + 1)  this thread, computed just before in this iteration,
//   g1 (x - 1, y), g3 (x + 1, y)  neighbouring threads, written to shared memory in the
//                  previous iteration.
// One barrier per iteration orders all of it.  Each level keeps three registers (g0 and
// g2 of its newest row, g2 of the row before), so K levels cost about 3K registers, and
// HBM sees one read and one write of the state per K steps (plus the x-halo columns and
// the K warm-up rows at each end of a chunk).  The per-site arithmetic (collision, source,
// sponge, zero ghost) is that of step_kernel (lb_kernels.cuh).  Level K is stored in the
// storage type; the levels in between stay FP32.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "lb_kernels.cuh"
#include "lb_runtime.h"

using namespace lbk;
using namespace lbrt;

namespace {

constexpr int kWS = 256;  // strip width in columns = threads per CTA
static_assert(kWS == 256, "one medium-table entry per thread");

struct Tb5Args {
    const int *row_off;  // [ny + 1]: the receivers of row y are entries row_off[y] .. row_off[y+1]
    const int *rec_x;    // their x, ascending within a row
    const int *rec_id;   // their receiver index
    int H;               // output rows per CTA
};

// One level's site: collision, source and sponge of step_kernel (finish_sites).
template <bool MRT>
__device__ __forceinline__ void level_site(float (&g)[5], float e2, const StepArgs &a, int x, int y,
                                           long long t, bool edge) {
    collide5<MRT>(g, e2, a);
    if (y == a.src_y && x == a.src_x && a.src_tab != nullptr && t < a.src_nt) {
        const float S = a.src_tab[t];
#pragma unroll
        for (int i = 0; i < 5; i++) g[i] += weight_i<5>(i, e2, a) * S;
    }
    if (edge) {
        const float f = sponge_of_dist(min(min(x, a.nx - 1 - x), min(y, a.ny - 1 - y)), a);
#pragma unroll
        for (int i = 0; i < 5; i++) g[i] *= f;
    }
}

// The strip bx and row chunk by of one grid, K levels (the body of both kernels below).
// REC: also record rho of every level of the own output sites (adjoint replays, rho tape).
// xs_mem: [2][K][2][kWS + 2] floats of shared memory; s_tab: [kWS] floats.
template <bool MRT, bool PER, int K, bool REC, typename ST>
__device__ __forceinline__ void tb5_body(const StepArgs &a, const Tb5Args &tb, int bx, int by,
                                         float *xs_mem, float *s_tab) {
    constexpr int OUT = kWS - 2 * K;
    // g1 and g3 of each level's newest row, by iteration parity
    auto xs = reinterpret_cast<float(*)[K][2][kWS + 2]>(xs_mem);
    const int c = threadIdx.x;
    const int OX = bx * OUT, gx = OX - K + c;
    bool col_in = true;
    int gxw = gx;
    if (PER)
        gxw = wrap_mod(gx, a.nx);
    else if (gx < 0 || gx >= a.nx)
        col_in = false, gxw = 0;
    const bool own_col = c >= K && c < K + OUT && gx < a.nx;
    const bool pad_col = c >= K && c < K + OUT && gx >= a.nx && gx < a.pitch;
    const int Y0 = by * tb.H, Y1 = min(Y0 + tb.H, a.ny);
    if (a.mid) s_tab[c] = a.mid_tab[c];
    if (c < 4 * K) {  // the pads either side of every row (the strip's outermost neighbours)
        float *row = &xs[c & 1][(c >> 1) % K][(c >> 1) / K][0];
        row[0] = 0.f;
        row[kWS + 1] = 0.f;
    }
    const int dxs = min(gxw, a.nx - 1 - gxw);  // distance to the nearest x face
    const bool wx_edge = __any_sync(0xffffffffu, a.sponge_w > 0 && col_in && dxs < a.sponge_w);
    const bool has_rec = a.trace_row != nullptr && tb.row_off != nullptr &&
                         tb.row_off[Y1] > tb.row_off[Y0];
    const ST *in = static_cast<const ST *>(a.in);
    __syncthreads();

    // level-0 row r, zero outside a zero-ghost domain
    auto load_row = [&](int r, float (&v)[5], float &e2) {
        int yw = r;
        bool live = col_in;
        if (PER)
            yw = wrap_mod(r, a.ny);
        else
            live = live && r >= 0 && r < a.ny;
        if (!live) {
#pragma unroll
            for (int i = 0; i < 5; i++) v[i] = 0.f;
            e2 = 0.f;
            return;
        }
        const long long o = (long long)yw * a.pitch + gxw;
#pragma unroll
        for (int i = 0; i < 5; i++) v[i] = Store<ST>::load1(in + i * a.plane + o);
        e2 = a.mid ? s_tab[a.mid[o]] : a.eta2[o];
    };

    float P0[K], P2a[K], P2b[K];  // per level: g0, g2 of the newest-but-one row; g2 before it
    float E[K + 1];               // eta^2 of rows r, r - 1, ..., r - K
#pragma unroll
    for (int l = 0; l < K; l++) P0[l] = P2a[l] = P2b[l] = 0.f;
#pragma unroll
    for (int l = 0; l <= K; l++) E[l] = 0.f;
    float pre[5], pre_e2;
    load_row(Y0 - K, pre, pre_e2);
    const int rend = Y1 + K;
#pragma unroll 1
    for (int r = Y0 - K; r < rend; r++) {
        float nw[5];
#pragma unroll
        for (int i = 0; i < 5; i++) nw[i] = pre[i];
#pragma unroll
        for (int l = K; l > 0; l--) E[l] = E[l - 1];
        E[0] = pre_e2;
        if (r + 1 < rend) load_row(r + 1, pre, pre_e2);  // in flight during this iteration
        const int p = r & 1;
#pragma unroll
        for (int l = 0; l < K; l++) {
            // level l's newest row (r - l): publish the populations the neighbours pull
            xs[p][l][0][c + 1] = nw[1];
            xs[p][l][1][c + 1] = nw[3];
            float g[5];
            g[0] = P0[l];
            g[2] = P2b[l];
            g[4] = nw[4];
            g[1] = xs[p ^ 1][l][0][c];      // h_1 (x - 1, y), written last iteration
            g[3] = xs[p ^ 1][l][1][c + 2];  // h_3 (x + 1, y)
            P2b[l] = P2a[l];
            P2a[l] = nw[2];
            P0[l] = nw[0];
            // level l + 1 computes row y = r - l - 1 once its inputs exist (warp-uniform)
            const int y = r - l - 1;
            if (r >= Y0 - K + 2 * (l + 1)) {
                bool live = col_in;
                int yw = y;
                if (PER)
                    yw = wrap_mod(y, a.ny);
                else
                    live = live && y >= 0 && y < a.ny;
                const long long t = a.t + l;
                const bool mine = own_col && y >= Y0 && y < Y1;
                const bool row_rec = has_rec && y >= Y0 && y < Y1 &&
                                     tb.row_off[y + 1] > tb.row_off[y];  // warp-uniform
                if ((REC && mine) || row_rec) {
                    const float rho = g[0] + g[1] + g[2] + g[3] + g[4];
                    if (REC && mine)
                        a.rho_out[l * a.rho_stride + (long long)y * a.pitch + gx] = rho;
                    if (row_rec && mine) {  // receivers of this site: binary search in the row
                        int lo = tb.row_off[y], hi = tb.row_off[y + 1];
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (tb.rec_x[mid] < gx)
                                lo = mid + 1;
                            else
                                hi = mid;
                        }
                        for (; lo < tb.row_off[y + 1] && tb.rec_x[lo] == gx; lo++) {
                            const int q = tb.rec_id[lo];
                            a.trace_row[(long long)l * a.nrec + (a.rec_col ? a.rec_col[q] : q)] =
                                cs2_of<5>(E[l + 1], a) * rho;
                        }
                    }
                }
                if (live) {
                    const int dy = min(yw, a.ny - 1 - yw);
                    const bool edge = a.sponge_w > 0 && (wx_edge || dy < a.sponge_w);
                    level_site<MRT>(g, E[l + 1], a, gxw, yw, t, edge);
                } else {
#pragma unroll
                    for (int i = 0; i < 5; i++) g[i] = 0.f;
                }
            }
#pragma unroll
            for (int i = 0; i < 5; i++) nw[i] = g[i];
        }
        // level K holds row r - K: store it when it is one of this CTA's output rows
        const int yo = r - K;
        if (yo >= Y0 && yo < Y1 && (own_col || pad_col)) {
            ST *o = static_cast<ST *>(a.out) + (long long)yo * a.pitch + gx;
#pragma unroll
            for (int i = 0; i < 5; i++) Store<ST>::store1(o + i * a.plane, own_col ? nw[i] : 0.f);
        }
        __syncthreads();
    }
}

template <bool MRT, bool PER, int K, bool REC, typename ST>
__global__ void __launch_bounds__(kWS, 2) tb5_kernel(const StepArgs a, const Tb5Args tb) {
    pdl_trigger_and_wait();
    extern __shared__ float xs_mem[];
    __shared__ float s_tab[kWS];
    tb5_body<MRT, PER, K, REC, ST>(a, tb, blockIdx.x, blockIdx.y, xs_mem, s_tab);
}

// Several independent grids ("shots") advanced by K steps in one launch: shot k owns
// blocks [first[k], first[k + 1]) of the grid, laid out as its strips x row chunks, and
// reads its own descriptors (the served batches; no rho tape).
template <bool MRT, bool PER, int K, typename ST>
__global__ void __launch_bounds__(kWS, 2)
    tb5_batch_kernel(const StepArgs *__restrict__ args, const Tb5Args *__restrict__ tbs,
                     const int *__restrict__ strips, const int *__restrict__ first, int nshots) {
    pdl_trigger_and_wait();
    extern __shared__ float xs_mem[];
    __shared__ float s_tab[kWS];
    __shared__ StepArgs sa;
    __shared__ Tb5Args stb;
    __shared__ int s_blk, s_strips;
    if (threadIdx.x == 0) {
        int lo = 0, hi = nshots - 1;  // shot with first[k] <= blockIdx.x < first[k + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first[mid] <= (int)blockIdx.x)
                lo = mid;
            else
                hi = mid - 1;
        }
        sa = args[lo];
        stb = tbs[lo];
        s_strips = strips[lo];
        s_blk = (int)blockIdx.x - first[lo];
    }
    __syncthreads();
    const int blk = s_blk, ns = s_strips;
    tb5_body<MRT, PER, K, false, ST>(sa, stb, blk % ns, blk / ns, xs_mem, s_tab);
}

using Tb5Fn = void (*)(const StepArgs, const Tb5Args);

template <int K, typename ST> Tb5Fn pick5(bool mrt, bool per, bool rec) {
    if constexpr (sizeof(ST) == 4) {
        if (rec) {
            if (mrt) return per ? tb5_kernel<true, true, K, true, ST> : tb5_kernel<true, false, K, true, ST>;
            return per ? tb5_kernel<false, true, K, true, ST> : tb5_kernel<false, false, K, true, ST>;
        }
    }
    if (rec) return nullptr;  // the rho tape of 16-bit contexts is recorded by the one-step kernel
    if (mrt) return per ? tb5_kernel<true, true, K, false, ST> : tb5_kernel<true, false, K, false, ST>;
    return per ? tb5_kernel<false, true, K, false, ST> : tb5_kernel<false, false, K, false, ST>;
}

template <typename ST> Tb5Fn pick5_k(int K, bool mrt, bool per, bool rec) {
    switch (K) {
        case 2: return pick5<2, ST>(mrt, per, rec);
        case 4: return pick5<4, ST>(mrt, per, rec);
        case 6: return pick5<6, ST>(mrt, per, rec);
        case 8: return pick5<8, ST>(mrt, per, rec);
        case 16: return pick5<16, ST>(mrt, per, rec);
        default: return nullptr;
    }
}

}  // namespace

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
    Tb5Fn fn = ctx->cfg.storage == LB_BF16 ? pick5_k<__nv_bfloat16>(K, mrt, per, rec)
             : ctx->cfg.storage == LB_F32  ? pick5_k<float>(K, mrt, per, rec)
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
    // rows per CTA: one wave of CTAs over the SMs when the chunks stay tall (>= 8K rows, so
    // the 2K warm-up rows cost little), else chunks of 8K rows
    const int slots = std::max(1, occ[K] * std::max(sms, 1));
    int chunks = std::max(1, slots / strips);
    int H = (ctx->ny + chunks - 1) / chunks;
    H = std::max(H, std::min(ctx->ny, 8 * K));
    Tb5Args tb;
    tb.row_off = a.trace_row ? ctx->tb5_off : nullptr;
    tb.rec_x = ctx->tb5_x;
    tb.rec_id = ctx->tb5_id;
    tb.H = H;
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

// Fill the host staging block `h` for K steps of ctxs[0 .. n) (advancing their time and
// buffers as if the launch ran); returns the launch's block count.
int tb5_batch_fill(lb_ctx *const *ctxs, int n, int K, void *h) {
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
        tb.H = std::min(ctx->ny, 16 * K);  // tall enough that the 2K warm-up rows cost little
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

using Tb5BatchFn = void (*)(const StepArgs *, const Tb5Args *, const int *, const int *, int);

template <int K, typename ST> Tb5BatchFn pick5_batch(bool mrt, bool per) {
    if (mrt) return per ? tb5_batch_kernel<true, true, K, ST> : tb5_batch_kernel<true, false, K, ST>;
    return per ? tb5_batch_kernel<false, true, K, ST> : tb5_batch_kernel<false, false, K, ST>;
}

// The launch of a block filled by tb5_batch_fill and copied to device memory `d`.
cudaError_t tb5_batch_launch(const void *d, int n, int K, int blocks, bool mrt, bool per,
                             int storage, cudaStream_t stream) {
    Tb5BatchFn fn = nullptr;
    const bool bf = storage == LB_BF16;
    if (K == 8) fn = bf ? pick5_batch<8, __nv_bfloat16>(mrt, per) : pick5_batch<8, float>(mrt, per);
    if (!fn || n < 1 || blocks < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)2 * K * 2 * (kWS + 2) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    BatchLayout L = batch_layout(const_cast<void *>(d), n);
    return launch_pdl(fn, dim3(blocks), dim3(kWS), smem, stream, (const StepArgs *)L.a,
                      (const Tb5Args *)L.tb, (const int *)L.strips, (const int *)L.first, n);
}
