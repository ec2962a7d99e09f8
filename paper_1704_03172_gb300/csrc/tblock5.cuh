// tblock5.cuh -- temporal blocking for D2Q5: K fused steps per launch as a row wavefront.
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
#pragma once

#include <cuda_runtime.h>

#include "lb_kernels.cuh"

namespace lbtb5 {

using namespace lbk;

constexpr int kWS = 256;  // strip width in columns = threads per CTA
static_assert(kWS == 256, "one medium-table entry per thread");

struct Tb5Args {
    const int *row_off;  // [ny + 1]: the receivers of row y are entries row_off[y] .. row_off[y+1]
    const int *rec_x;    // their x, ascending within a row
    const int *rec_id;   // their receiver index
    int H;               // output rows per CTA
    int per;             // periodic boundary
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

// Per-thread constants of one strip and row chunk.
struct Tb5Thread {
    int c, gx, gxw, Y0, Y1;
    bool per, col_in, own_col, pad_col, wx_edge, has_rec, edgy_cols, lossless;
    int dxs;             // distance of this column to the nearest x face
    int rec_lo, rec_hi;  // the first and last chunk row that holds a receiver (none: 1, 0)
    float *xs;           // [2][K][2][kWS + 2]: g1, g3 of each level's newest row, by parity
    const float *s_tab;  // medium table (indexed media)
};

// Level state, named by the parity of the iteration that wrote it so that the row loop,
// unrolled by two, renames registers instead of moving them: a value written in
// iteration r and read in r + 1 (g0 and eta^2 of a level's newest row) alternates
// between two names; g2, read two iterations later, reuses its own name.
template <int K> struct Tb5Regs {
    float W0[2][K];   // g0 of level l's newest row, written in an iteration of that parity
    float EE[2][K];   // eta^2 of that row
    float G2[2][K];   // g2 of level l's newest row (read two iterations later)
    float pre[2][5];  // level-0 row prefetched for the next iteration
    float pre_e2[2];  // (unused)
};

// Level-0 row r, zero outside a zero-ghost domain.  v holds the stored bits (tb5_iter
// widens them one iteration later, so the conversion does not wait for the load).
template <typename ST>
__device__ __forceinline__ void tb5_load(const StepArgs &a, const Tb5Thread &T, int r, float (&v)[5],
                                         float &e2) {
    int yw = r;
    bool live = T.col_in;
    if (T.per)
        yw = wrap_mod(r, a.ny);
    else
        live = live && r >= 0 && r < a.ny;
    if (!live) {
#pragma unroll
        for (int i = 0; i < 5; i++) v[i] = 0.f;
        e2 = 0.f;
        return;
    }
    const ST *in = static_cast<const ST *>(a.in);
    const long long o = (long long)yw * a.pitch + T.gxw;
#pragma unroll
    for (int i = 0; i < 5; i++) v[i] = __uint_as_float(Store<ST>::bits1(in + i * a.plane + o));
    // the medium as loaded: eta^2, or the index byte (as a float's bits) that tb5_e2 looks up
    // one iteration later, so that the table read does not wait for the global load
    e2 = a.mid ? __int_as_float((int)a.mid[o]) : a.eta2[o];
}

// eta^2 from what tb5_load left (the index byte of an indexed medium, else eta^2 itself)
__device__ __forceinline__ float tb5_e2(const StepArgs &a, const Tb5Thread &T, bool live, float m) {
    return (a.mid && live) ? T.s_tab[__float_as_int(m)] : m;
}

// One wavefront iteration r (parity P).  FAST: every level's row lies inside the chunk's
// output rows, inside the domain and outside the sponge, holds neither the source nor a
// receiver, and the strip's columns are all live and outside the sponge: no per-site
// checks at all.
// edgy (FAST, CTA-uniform): a column of the strip or a row of the iteration lies outside
// the domain or in the sponge, so the fast path applies a per-site factor.
template <bool MRT, int K, bool REC, typename ST, int P, bool FAST>
__device__ __forceinline__ void tb5_iter(const StepArgs &a, const Tb5Args &tb, const Tb5Thread &T,
                                         float (&W0)[2][K], float (&EE)[2][K], float (&G2)[2][K],
                                         float (&pre)[2][5], float (&pre_e2)[2], int r, int rend,
                                         bool edgy) {
    constexpr int SR = kWS + 2, SL = 2 * SR;  // row and level strides of xs
    float n[5], nE;  // level l's newest row (r - l); level 0: the prefetched row r
#pragma unroll
    for (int i = 0; i < 5; i++) n[i] = Store<ST>::unbits1(__float_as_uint(pre[P][i]));
    nE = tb5_e2(a, T, T.col_in && (T.per || (r >= 0 && r < a.ny)), pre_e2[P]);
    if (r + 1 < rend) tb5_load<ST>(a, T, r + 1, pre[P ^ 1], pre_e2[P ^ 1]);
    float *cur = T.xs + P * K * SL + T.c + 1;        // this iteration's rows, column c
    const float *prv = T.xs + (P ^ 1) * K * SL + T.c;  // last iteration's rows, column c - 1
    // every level's neighbour values at once: they were written last iteration, so none
    // of this iteration's stores (the other parity) has to complete before them
    float h1[K], h3[K];
#pragma unroll
    for (int l = 0; l < K; l++) {
        h1[l] = prv[l * SL];           // h_1 (x - 1, y)
        h3[l] = prv[l * SL + SR + 2];  // h_3 (x + 1, y)
    }
#pragma unroll
    for (int l = 0; l < K; l++) {
        cur[l * SL] = n[1];
        cur[l * SL + SR] = n[3];
        float g[5];
        g[1] = h1[l];
        g[3] = h3[l];
        g[0] = W0[P ^ 1][l];        // h_0 (x, y)
        g[2] = G2[P][l];            // h_2 (x, y - 1), written two iterations back
        g[4] = n[4];                  // h_4 (x, y + 1), computed just before
        const float e2 = EE[P ^ 1][l];
        W0[P][l] = n[0];
        G2[P][l] = n[2];
        EE[P][l] = nE;
        const int y = r - l - 1;  // the row level l + 1 computes
        if (FAST) {
            if (REC && T.own_col)
                a.rho_out[l * a.rho_stride + (long long)y * a.pitch + T.gx] =
                    g[0] + g[1] + g[2] + g[3] + g[4];
            if (!MRT && T.lossless)
                collide5_lossless(g, e2);
            else
                collide5<MRT>(g, e2, a);
            if (edgy) {  // CTA-uniform: sponge columns or rows, or columns outside the domain
                const int yw = T.per ? wrap_mod(y, a.ny) : y;
                const float f = T.col_in ? sponge_of_dist(min(T.dxs, min(yw, a.ny - 1 - yw)), a)
                                         : 0.f;
#pragma unroll
                for (int i = 0; i < 5; i++) g[i] *= f;
            }
        } else if (r >= T.Y0 - K + 2 * (l + 1)) {  // its inputs exist (warp-uniform)
            bool live = T.col_in;
            int yw = y;
            if (T.per)
                yw = wrap_mod(y, a.ny);
            else
                live = live && y >= 0 && y < a.ny;
            const bool mine = T.own_col && y >= T.Y0 && y < T.Y1;
            const bool row_rec = T.has_rec && y >= T.Y0 && y < T.Y1 &&
                                 tb.row_off[y + 1] > tb.row_off[y];  // warp-uniform
            if ((REC && mine) || row_rec) {
                const float rho = g[0] + g[1] + g[2] + g[3] + g[4];
                if (REC && mine) a.rho_out[l * a.rho_stride + (long long)y * a.pitch + T.gx] = rho;
                if (row_rec && mine) {  // receivers of this site: binary search in the row
                    int lo = tb.row_off[y], hi = tb.row_off[y + 1];
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (tb.rec_x[mid] < T.gx)
                            lo = mid + 1;
                        else
                            hi = mid;
                    }
                    for (; lo < tb.row_off[y + 1] && tb.rec_x[lo] == T.gx; lo++) {
                        const int q = tb.rec_id[lo];
                        a.trace_row[(long long)l * a.nrec + (a.rec_col ? a.rec_col[q] : q)] =
                            cs2_of<5>(e2, a) * rho;
                    }
                }
            }
            if (live) {
                const int dy = min(yw, a.ny - 1 - yw);
                const bool edge = a.sponge_w > 0 && (T.wx_edge || dy < a.sponge_w);
                level_site<MRT>(g, e2, a, T.gxw, yw, a.t + l, edge);
            } else {
#pragma unroll
                for (int i = 0; i < 5; i++) g[i] = 0.f;
            }
        }
#pragma unroll
        for (int i = 0; i < 5; i++) n[i] = g[i];
        nE = e2;
    }
    // level K holds row r - K: store it when it is one of this CTA's output rows
    const int yo = r - K;
    if (FAST ? T.own_col : (yo >= T.Y0 && yo < T.Y1 && (T.own_col || T.pad_col))) {
        ST *o = static_cast<ST *>(a.out) + (long long)yo * a.pitch + T.gx;
#pragma unroll
        for (int i = 0; i < 5; i++) Store<ST>::store1(o + i * a.plane, T.own_col ? n[i] : 0.f);
    }
    __syncthreads();
}

// The strip bx and row chunk by of one grid, K levels (the body of both kernels below).
// REC: also record rho of every level of the own output sites (adjoint replays, rho tape).
// xs_mem: [2][K][2][kWS + 2] floats of shared memory; s_tab: [kWS] floats.
template <bool MRT, int K, bool REC, typename ST>
__device__ __forceinline__ void tb5_body(const StepArgs &a, const Tb5Args &tb, int bx, int by,
                                         float *xs_mem, float *s_tab) {
    constexpr int OUT = kWS - 2 * K;
    Tb5Thread T;
    T.c = threadIdx.x;
    const int OX = bx * OUT;
    T.gx = OX - K + T.c;
    T.per = tb.per != 0;
    T.col_in = true;
    T.gxw = T.gx;
    if (T.per)
        T.gxw = wrap_mod(T.gx, a.nx);
    else if (T.gx < 0 || T.gx >= a.nx)
        T.col_in = false, T.gxw = 0;
    T.own_col = T.c >= K && T.c < K + OUT && T.gx < a.nx;
    T.pad_col = T.c >= K && T.c < K + OUT && T.gx >= a.nx && T.gx < a.pitch;
    T.Y0 = by * tb.H;
    T.Y1 = min(T.Y0 + tb.H, a.ny);
    T.xs = xs_mem;
    T.s_tab = s_tab;
    if (a.mid) s_tab[T.c] = a.mid_tab[T.c];
    if (T.c < 4 * K) {  // the pads either side of every row (the strip's outermost neighbours)
        constexpr int SR = kWS + 2;
        float *row = xs_mem + ((T.c & 1) * K + (T.c >> 1) % K) * 2 * SR + ((T.c >> 1) / K) * SR;
        row[0] = 0.f;
        row[kWS + 1] = 0.f;
    }
    T.dxs = min(T.gxw, a.nx - 1 - T.gxw);  // distance to the nearest x face
    const bool x_edge = a.sponge_w > 0 && T.col_in && T.dxs < a.sponge_w;
    T.wx_edge = __any_sync(0xffffffffu, x_edge);
    T.has_rec = a.trace_row != nullptr && tb.row_off != nullptr && tb.row_off[T.Y1] > tb.row_off[T.Y0];
    T.rec_lo = 1;
    T.rec_hi = 0;
    if (T.has_rec) {  // the chunk's first and last receiver rows (row_off is a prefix count)
        int lo = T.Y0, hi = T.Y1 - 1;
        while (lo < hi) {  // first y with receivers: row_off[y + 1] > row_off[Y0]
            const int m = (lo + hi) >> 1;
            if (tb.row_off[m + 1] > tb.row_off[T.Y0]) hi = m; else lo = m + 1;
        }
        T.rec_lo = lo;
        lo = T.Y0;
        hi = T.Y1 - 1;
        while (lo < hi) {  // last y with receivers: row_off[y] < row_off[Y1]
            const int m = (lo + hi + 1) >> 1;
            if (tb.row_off[m] < tb.row_off[T.Y1]) lo = m; else hi = m - 1;
        }
        T.rec_hi = lo;
    }
    T.lossless = a.omega == 2.f;
    // some column of the strip outside the domain or in the sponge, or a sponge in y
    // (CTA-uniform): the fast path then applies a per-site factor
    T.edgy_cols = __syncthreads_or(!T.col_in || x_edge) != 0;

    float W0[2][K], EE[2][K], G2[2][K], pre[2][5], pre_e2[2];
#pragma unroll
    for (int l = 0; l < K; l++)
#pragma unroll
        for (int q = 0; q < 2; q++) W0[q][l] = EE[q][l] = G2[q][l] = 0.f;
    const int rbeg = T.Y0 - K, rend = T.Y1 + K;
    // iterations whose K rows r - K .. r - 1 are all own rows of the chunk
    const int fbeg = T.Y0 + K, fend = T.Y1 + 1;
    // the fast path: every level's row an own row of the chunk, none of them the source
    // row or a receiver row (sponge and edge columns take its per-site factor)
    auto edgy = [&](int r) {  // CTA-uniform: the factor of the fast path is needed
        const int w = a.sponge_w, lo = r - K, hi = r - 1;
        if (T.edgy_cols) return true;
        if (w <= 0) return false;
        if (!T.per) return lo < w || hi > a.ny - 1 - w;
        return true;  // periodic rows wrap: check per site
    };
    auto fast_ok = [&](int r) {  // CTA-uniform
        if (r < fbeg || r >= fend) return false;
        const int lo = r - K, hi = r - 1;  // the rows of levels K .. 1
        if (a.src_tab != nullptr && a.src_y >= lo && a.src_y <= hi && a.t < a.src_nt) return false;
        if (T.rec_lo <= hi && T.rec_hi >= lo) return false;
        return true;
    };
    // iteration parity counts from rbeg: even iterations are parity 0
    tb5_load<ST>(a, T, rbeg, pre[0], pre_e2[0]);
    int r = rbeg;
#pragma unroll 1
    for (; r < rend; r += 2) {
        if (fast_ok(r))
            tb5_iter<MRT, K, REC, ST, 0, true>(a, tb, T, W0, EE, G2, pre, pre_e2, r, rend, edgy(r));
        else
            tb5_iter<MRT, K, REC, ST, 0, false>(a, tb, T, W0, EE, G2, pre, pre_e2, r, rend, edgy(r));
        if (r + 1 >= rend) break;
        if (fast_ok(r + 1))
            tb5_iter<MRT, K, REC, ST, 1, true>(a, tb, T, W0, EE, G2, pre, pre_e2, r + 1, rend, edgy(r + 1));
        else
            tb5_iter<MRT, K, REC, ST, 1, false>(a, tb, T, W0, EE, G2, pre, pre_e2, r + 1, rend, edgy(r + 1));
    }
}

// Resident CTAs per SM the register budget is cut for: three for the shallow blocks
// (<= 80 registers), two for the deep ones.
template <int K> constexpr int tb5_min_blocks() { return K <= 4 ? 3 : 2; }

template <bool MRT, int K, bool REC, typename ST>
__global__ void __launch_bounds__(kWS, tb5_min_blocks<K>()) tb5_kernel(const StepArgs a,
                                                                      const Tb5Args tb) {
    pdl_trigger_and_wait();
    extern __shared__ float xs_mem[];
    __shared__ float s_tab[kWS];
    tb5_body<MRT, K, REC, ST>(a, tb, blockIdx.x, blockIdx.y, xs_mem, s_tab);
}

// Several independent grids ("shots") advanced by K steps in one launch: shot k owns
// blocks [first[k], first[k + 1]) of the grid, laid out as its strips x row chunks, and
// reads its own descriptors (the served batches; no rho tape).
template <bool MRT, int K, typename ST>
__global__ void __launch_bounds__(kWS, tb5_min_blocks<K>())
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
    tb5_body<MRT, K, false, ST>(sa, stb, blk % ns, blk / ns, xs_mem, s_tab);
}


using Tb5Fn = void (*)(const StepArgs, const Tb5Args);
using Tb5BatchFn = void (*)(const StepArgs *, const Tb5Args *, const int *, const int *, int);

// one storage type's kernels (tblock5.cu: FP32, tblock5_bf16.cu: BF16); nullptr where absent
Tb5Fn pick_f32(int K, bool mrt, bool rec);
Tb5Fn pick_bf16(int K, bool mrt, bool rec);
Tb5BatchFn pick_batch_f32(int K, bool mrt);
Tb5BatchFn pick_batch_bf16(int K, bool mrt);

template <int K, typename ST, bool WITH_REC = true> Tb5Fn pick_k(bool mrt, bool rec) {
    if constexpr (WITH_REC) {
        if (rec) return mrt ? tb5_kernel<true, K, true, ST> : tb5_kernel<false, K, true, ST>;
    }
    if (rec) return nullptr;
    return mrt ? tb5_kernel<true, K, false, ST> : tb5_kernel<false, K, false, ST>;
}

}  // namespace lbtb5
