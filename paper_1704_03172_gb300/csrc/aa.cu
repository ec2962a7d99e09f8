// aa.cu -- in-place streaming: one population buffer instead of two (the "AA" pattern).
//
// The pull step streams g_i(x, t) = h_i(x - c_i, t - 1) (Eq. BGK-LB) from one buffer and
// writes the collided h(t) to the other.  Here the steps alternate between two forms that
// both work in one buffer:
//   site-local step   the buffer holds g(t) at its own site, population i in slot i.  The
//                     thread of site x reads slot i at x, collides, and writes h_i(x, t)
//                     to slot opp(i) at x.
//   exchange step     the buffer holds h(t - 1) at its own site, population i in slot
//                     opp(i).  The thread of site x reads g_i(x, t) = h_i(x - c_i, t - 1)
//                     from slot opp(i) at x - c_i, collides, and writes h_i(x, t) to slot i
//                     at x + c_i, which is g_i(x + c_i, t + 1) for the next site-local step.
// In the exchange step slot i at site y is read and written by the thread of site y - c_i
// alone (its population opp(i) in, its population i out); in the site-local step a thread
// touches only its own site.  No slot is shared between threads in either form, so one
// launch per step needs no barrier and no second buffer.  Under the zero ghost no site
// writes slot i at the sites whose x - c_i lies outside the domain: their own threads write
// the zero that the ghost streams in.
//
// The per-site arithmetic is that of step_kernel (collide_sites: collision, source,
// sponge; receivers summed in the same order), so results equal the two-buffer step bit for
// bit.  A thread owns V consecutive sites of a row (4 FP32, 8 16-bit) as step_kernel does.
// The site-local step moves 16-byte vectors only.  The exchange step pulls with the same
// vector-and-shuffle loads as step_kernel; of its pushes, those with no x component are
// 16-byte vectors and the two (D2Q9: six) that move one site in x are element stores.
//
// Loads and stores of one thread's slots never meet another thread's: a vector load of the
// exchange step also covers one element that the neighbouring lane (or, at a warp's edge,
// the neighbouring warp) owns and may be writing; that element is only passed on by the
// shuffle to the lane that owns it, never used, and at a warp's edge the owner loads it
// itself.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "aa_sites.cuh"
#include "lb_kernels.cuh"
#include "lb_runtime.h"

namespace lbaa {

using namespace lbk;

// The medium of a thread's V sites as stored: with a 1-byte medium index its V / 4 words of
// indices (as float bits), else eta^2 itself.  Loaded together with the populations, so that
// a warp waits on memory once.
template <int V>
__device__ __forceinline__ void medium_load(const StepArgs &a, long long off, float (&raw)[V]) {
    if (a.mid) {
        const uint8_t *mp = a.mid + off;
        if (V == 4) {
            raw[0] = __uint_as_float(*reinterpret_cast<const uint32_t *>(mp));
        } else {
            const uint2 u = *reinterpret_cast<const uint2 *>(mp);
            raw[0] = __uint_as_float(u.x);
            raw[1] = __uint_as_float(u.y);
        }
    } else {
#pragma unroll
        for (int k = 0; k < V; k += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(a.eta2 + off + k);
            raw[k] = v.x; raw[k + 1] = v.y; raw[k + 2] = v.z; raw[k + 3] = v.w;
        }
    }
}

// Receivers, medium and collision of one thread's V sites, as step_kernel does them; raw is
// the sites' medium from medium_load.
template <int Q, bool MRT, typename ST>
__device__ __forceinline__ void collide_site_vector(const StepArgs &a, const AaRec &r,
                                                    const float *tab,
                                                    float (&g)[Q][Store<ST>::V], int y, int x0,
                                                    const float (&raw)[Store<ST>::V]) {
    constexpr int V = Store<ST>::V;
    float e2s[V];
    if (a.mid) {  // eta^2 from the shared table
#pragma unroll
        for (int k = 0; k < V; k++)
            e2s[k] = tab[(__float_as_uint(raw[k >> 2]) >> (8 * (k & 3))) & 0xffu];
    } else {
#pragma unroll
        for (int k = 0; k < V; k++) e2s[k] = raw[k];
    }
    aa_receivers<Q, ST>(a, r, g, y, x0);
    aa_collide<Q, MRT, V>(a, g, e2s, y, x0);
}


// The exchange step of a warp whose sites and neighbours are all interior: rows y - 1 and
// y + 1 exist, the warp's first site has a left neighbour and its last a right one, and no
// site is padding.  Nothing is wrapped, absent or a ghost, so the bounds and ghost logic of
// the general form drops out.  The slot that population i pulls from, opp(i) at x - c_i,
// lies in the row that population opp(i) pushes to, so one row pointer per slot serves
// both.  Same values as the general form.
template <int Q, bool MRT, typename ST>
__device__ __forceinline__ void exchange_inner(const StepArgs &a, const AaRec &r,
                                               const float *tab, ST *pop, int y, int x0,
                                               int lane) {
    constexpr int V = Store<ST>::V;
    // slot s in row y + c_s,y holds h_opp(s), read as g_opp(s), and takes h_s; the pointers
    // are formed again for the stores rather than held across the collision
    ST *const rowp = pop + (long long)y * a.pitch + x0;
    auto slot = [&](int s) { return rowp + s * a.plane + Lat<Q>::cy(s) * a.pitch; };
    uint4 q[Q];
    uint32_t e[Q];
    float med[V];
    medium_load<V>(a, (long long)y * a.pitch + x0, med);
#pragma unroll
    for (int i = 0; i < Q; i++) {  // all loads in flight together
        const ST *src = slot(Lat<Q>::opp(i));
        q[i] = *reinterpret_cast<const uint4 *>(src);
        e[i] = 0u;
        if (Lat<Q>::cx(i) == 1 && lane == 0) e[i] = Store<ST>::bits1(src - 1);
        if (Lat<Q>::cx(i) == -1 && lane == 31) e[i] = Store<ST>::bits1(src + V);
    }
    float g[Q][V];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        float f[V];
        Store<ST>::unpackV(q[i], f);
        if (Lat<Q>::cx(i) == 1) {  // value from x - 1
            float left = __shfl_up_sync(0xffffffffu, f[V - 1], 1);
            if (lane == 0) left = Store<ST>::unbits1(e[i]);
            g[i][0] = left;
#pragma unroll
            for (int k = 1; k < V; k++) g[i][k] = f[k - 1];
        } else if (Lat<Q>::cx(i) == -1) {  // value from x + 1
            float right = __shfl_down_sync(0xffffffffu, f[0], 1);
            if (lane == 31) right = Store<ST>::unbits1(e[i]);
#pragma unroll
            for (int k = 0; k + 1 < V; k++) g[i][k] = f[k + 1];
            g[i][V - 1] = right;
        } else {
#pragma unroll
            for (int k = 0; k < V; k++) g[i][k] = f[k];
        }
    }
    collide_site_vector<Q, MRT, ST>(a, r, tab, g, y, x0, med);
#pragma unroll
    for (int s = 0; s < Q; s++) push_inner<Q, ST>(slot(s) - x0, s, g[s], x0, lane);
}

// CTAs per SM: the FP32 exchange form holds row pointers and shifted vectors across the
// collision and gets one CTA fewer (more registers) than the site-local form.
template <int Q, typename ST, bool EXCHANGE> constexpr int aa_min_ctas() {
    return sizeof(ST) == 4 ? (Q == 5 ? 5 : 4) - (EXCHANGE && Q == 9 ? 1 : 0) : (Q == 5 ? 3 : 2);
}

template <int Q, bool MRT, bool PERIODIC, typename ST, bool EXCHANGE>
__global__ void __launch_bounds__(kThreads, (aa_min_ctas<Q, ST, EXCHANGE>()))
    aa_step_kernel(const StepArgs a, const AaRec r) {
    pdl_trigger_and_wait();
    __shared__ float tab[kThreads];
    if (a.mid) {  // block-uniform
        tab[threadIdx.x] = a.mid_tab[threadIdx.x];
        __syncthreads();
    }
    constexpr int V = Store<ST>::V;
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int y = wid / a.segs;
    if (y >= a.ny) return;  // warp-uniform
    const int x0 = (wid - y * a.segs) * (32 * V) + lane * V;
    const bool active = x0 < a.nx;
    ST *pop = static_cast<ST *>(a.out);  // a.in == a.out
    const long long row = (long long)y * a.pitch;
    float g[Q][V];
    float med[V];
    if constexpr (!EXCHANGE) {
        if (!active) return;  // no shuffles in this form
        medium_load<V>(a, row + x0, med);
#pragma unroll
        for (int i = 0; i < Q; i++) Store<ST>::loadV(pop + i * a.plane + row + x0, g[i]);
    } else {  // g_i(x) = slot opp(i) at x - c_i: the pull of step_kernel from the other slot
        const int sx0 = x0 - lane * V;  // the warp's first site (warp-uniform test)
        if (y > 0 && y + 1 < a.ny && sx0 > 0 && sx0 + 32 * V < a.nx) {
            exchange_inner<Q, MRT, ST>(a, r, tab, pop, y, x0, lane);
            return;
        }
        uint4 q[Q];
        uint32_t e[Q];
        bool absent[Q];
        if (active) medium_load<V>(a, row + x0, med);
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const int rs = row_at<PERIODIC>(y, -Lat<Q>::cy(i), a.ny);
            const ST *src = rs < 0 ? nullptr
                                   : pop + Lat<Q>::opp(i) * a.plane + (long long)rs * a.pitch;
            absent[i] = src == nullptr;
            if (Lat<Q>::cx(i) == 1)
                pull_issue<1, PERIODIC>(src, x0, lane, a.nx, active, q[i], e[i]);
            else if (Lat<Q>::cx(i) == -1)
                pull_issue<-1, PERIODIC>(src, x0, lane, a.nx, active, q[i], e[i]);
            else
                pull_issue<0, PERIODIC>(src, x0, lane, a.nx, active, q[i], e[i]);
        }
#pragma unroll
        for (int i = 0; i < Q; i++) {
            if (Lat<Q>::cx(i) == 1)
                pull_finish<1, PERIODIC, ST>(absent[i], x0, lane, a.nx, q[i], e[i], g[i]);
            else if (Lat<Q>::cx(i) == -1)
                pull_finish<-1, PERIODIC, ST>(absent[i], x0, lane, a.nx, q[i], e[i], g[i]);
            else
                pull_finish<0, PERIODIC, ST>(absent[i], x0, lane, a.nx, q[i], e[i], g[i]);
        }
    }
    // the exchange step keeps inactive lanes for the shuffles of its pushes
    if (active) collide_site_vector<Q, MRT, ST>(a, r, tab, g, y, x0, med);
    if constexpr (!EXCHANGE) {  // h_i(x) into slot opp(i) at x
#pragma unroll
        for (int i = 0; i < Q; i++) Store<ST>::storeV(pop + Lat<Q>::opp(i) * a.plane + row + x0, g[i]);
    } else {
        exchange_stores<Q, PERIODIC, ST>(a, pop, g, y, x0, lane, active);
    }
}

using AaFn = void (*)(const StepArgs, const AaRec);

template <int Q, typename ST, bool EX> AaFn aa_fn(bool mrt, bool per) {
    if (mrt) return per ? aa_step_kernel<Q, true, true, ST, EX> : aa_step_kernel<Q, true, false, ST, EX>;
    return per ? aa_step_kernel<Q, false, true, ST, EX> : aa_step_kernel<Q, false, false, ST, EX>;
}
template <typename ST> AaFn aa_pick(int Q, bool mrt, bool per, bool ex) {
    if (Q == 9) return ex ? aa_fn<9, ST, true>(mrt, per) : aa_fn<9, ST, false>(mrt, per);
    return ex ? aa_fn<5, ST, true>(mrt, per) : aa_fn<5, ST, false>(mrt, per);
}

}  // namespace lbaa

using namespace lbaa;
using namespace lbrt;

// n steps in place.  The buffer's form alternates: g(t) at its own site (ctx->raw) before a
// site-local step, h(t - 1) in the opposite slots (ctx->swap) before an exchange step.
lb_status aa_step(lb_ctx *ctx, int n) {
    const bool mrt = ctx->cfg.collision == LB_MRT, per = ctx->cfg.boundary == LB_PERIODIC;
    const bool bf = ctx->cfg.storage == LB_BF16;
    for (int k = 0; k < n; k++) {
        const bool ex = !ctx->raw;  // the state is h(t - 1) in the opposite slots
        StepArgs a = base_args(ctx);
        a.in = ctx->pop[0];
        a.out = ctx->pop[0];
        a.t = ctx->t;
        const long long row = ctx->t - ctx->t_rec0;
        a.trace_row = (ctx->trace && row >= 0 && row < ctx->trace_cap)
                          ? ctx->trace + row * ctx->nrec
                          : nullptr;
        AaRec r{a.trace_row ? ctx->tb5_off : nullptr, ctx->tb5_x, ctx->tb5_id};
        if (ctx->staged) {  // BF16 on wide rows: the TMA-staged persistent form
            lb_status st = stream_launch_aa(ctx, a, ex, r.row_off, r.rec_x, r.rec_id);
            if (st != LB_OK) return st;
        } else {
            AaFn fn = bf ? aa_pick<__nv_bfloat16>(ctx->Q, mrt, per, ex)
                         : aa_pick<float>(ctx->Q, mrt, per, ex);
            // a warp per row segment of 32 V sites, as step_kernel (base_args: segs, main_blocks)
            cudaError_t e =
                launch_pdl(fn, dim3(a.main_blocks), dim3(kThreads), 0, ctx->stream, a, r);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "in-place step launch");
        }
        ctx->raw = ex;  // after an exchange step: g(t + 1) at its own site
        ctx->swap = !ex;
        ctx->t += 1;
    }
    return LB_OK;
}
