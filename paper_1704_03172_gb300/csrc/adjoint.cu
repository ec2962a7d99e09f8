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
//
// BF16 storage: the checkpoints and replayed states are the BF16 states the
// forward run produced (the replay runs the same kernel on the same inputs, so
// it reproduces them bit for bit); the adjoint state stays FP32.  The result is
// the transpose of the exact linear step taken along the stored trajectory, so
// its distance from the FP32 gradient is of the order of the forward's BF16
// error.  FP16 storage is not supported (its per-step range scales would have
// to be replayed as well).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <utility>
#include <vector>

#include "adjoint_site.cuh"
#include "lb_kernels.cuh"
#include "lb_runtime.h"

using namespace lbk;
using namespace lbrt;
using namespace lbadj;

namespace {

// One adjoint step for 4 consecutive x-sites per thread (16-byte FP32 vectors;
// the +-1 x-shift of the reverse pull is a warp shuffle, as in the forward step).
template <int Q, bool MRT, bool PERIODIC>
__global__ void __launch_bounds__(kThreads, Q == 5 ? 4 : 3) adjoint_kernel(const StepArgs a, const AdjArgs d) {
    pdl_trigger_and_wait();
    constexpr int V = 4;
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int y = wid / d.segs;
    if (y >= a.ny) return;  // warp-uniform
    const int x0 = (wid - y * d.segs) * (32 * V) + lane * V;
    const bool active = x0 < a.nx;
    // mu_i(x) = (1 - sigma(x)) lambda_i^{t+1}(x + c_i): P^T pulls from x + c_i
    // (two phases: every population's loads in flight together, then the shifts)
    uint4 q[Q];
    uint32_t e[Q];
    bool absent[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const float *row = src_row<PERIODIC>(d.lam_in + i * a.plane, y + Lat<Q>::cy(i), a.ny, a.pitch);
        absent[i] = row == nullptr;
        const int cx = Lat<Q>::cx(i);
        if (cx == 1)
            pull_issue<-1, PERIODIC>(row, x0, lane, a.nx, active, q[i], e[i]);
        else if (cx == -1)
            pull_issue<1, PERIODIC>(row, x0, lane, a.nx, active, q[i], e[i]);
        else
            pull_issue<0, PERIODIC>(row, x0, lane, a.nx, active, q[i], e[i]);
    }
    float mu[Q][V];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int cx = Lat<Q>::cx(i);
        if (cx == 1)
            pull_finish<-1, PERIODIC, float>(absent[i], x0, lane, a.nx, q[i], e[i], mu[i]);
        else if (cx == -1)
            pull_finish<1, PERIODIC, float>(absent[i], x0, lane, a.nx, q[i], e[i], mu[i]);
        else
            pull_finish<0, PERIODIC, float>(absent[i], x0, lane, a.nx, q[i], e[i], mu[i]);
    }
    if (!active) return;  // no shuffles below
    const long long base = (long long)y * a.pitch + x0;
    const float4 e4 = *reinterpret_cast<const float4 *>(a.eta2 + base);
    const float4 r4 = *reinterpret_cast<const float4 *>(d.rho + base);
    const float e2s[V] = {e4.x, e4.y, e4.z, e4.w}, rhos[V] = {r4.x, r4.y, r4.z, r4.w};
    const bool edge = a.sponge_w > 0 &&
                      (y < a.sponge_w || y >= a.ny - a.sponge_w || x0 < a.sponge_w ||
                       x0 + V - 1 >= a.nx - a.sponge_w);
    const bool has_src = (y == a.src_y) && (a.src_x >= x0) && (a.src_x < x0 + V) && a.src_tab;
    double gadd[V];
#pragma unroll
    for (int k = 0; k < V; k++) {
        const float f = edge ? sponge_factor(x0 + k, y, a) : 1.f;
        float m[Q];
#pragma unroll
        for (int i = 0; i < Q; i++) m[i] = f * mu[i][k];
        float src_w = 0.f, src_dw = 0.f;
        const bool at_src = has_src && a.src_x == x0 + k;
        if (at_src) adj_src<Q>(m, e2s[k], a, src_w, src_dw);
        const float gsum = adj_site<Q, MRT>(m, e2s[k], a);
        const bool real = x0 + k < a.nx;
#pragma unroll
        for (int i = 0; i < Q; i++) mu[i][k] = real ? m[i] : 0.f;  // becomes lambda^t
        gadd[k] = (double)rhos[k] * (double)gsum;
        if (at_src) {
            if (d.grad_src) d.grad_src[a.t - d.t0] = (double)src_w;
            if (a.t < a.src_nt) gadd[k] += (double)a.src_tab[a.t] * (double)src_dw;
        }
    }
#pragma unroll
    for (int i = 0; i < Q; i++)
        *reinterpret_cast<float4 *>(d.lam_out + i * a.plane + base) =
            make_float4(mu[i][0], mu[i][1], mu[i][2], mu[i][3]);
    double2 *gp = reinterpret_cast<double2 *>(d.grad + base);
    double2 g01 = gp[0], g23 = gp[1];
    g01.x += gadd[0];
    g01.y += gadd[1];
    g23.x += gadd[2];
    g23.y += gadd[3];
    gp[0] = g01;
    gp[1] = g23;
}

// receivers: lambda^t += R^t_r c_s^2(x_r) (every population), dJ/d(eta^2) += R dc_s^2 rho^t
template <int Q>
__global__ void adjoint_receivers(const StepArgs a, const AdjArgs d) {
    pdl_trigger_and_wait();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.nrec) return;
    const int2 xy = a.rec[r];
    const long long idx = (long long)xy.y * a.pitch + xy.x;
    const float R = d.resid[(a.t - d.t0) * d.nrec + r];
    const float c2 = cs2_of<Q>(a.eta2[idx], a);
    for (int i = 0; i < Q; i++) atomicAdd(d.lam_out + i * a.plane + idx, R * c2);
    atomicAdd(d.grad + idx, (double)R * (double)dcs2<Q>(a) * (double)d.rho[idx]);
}

// ---- time-blocked reverse sweep: K adjoint levels per launch
//
// The transpose of the overlapped tiling of tblock.cu.  A CTA owns an OUT x OUT tile
// (OUT = 48 - 2K) and loads lambda^{t_hi+1} on the 48 x 48 region made of the tile and a
// K-site halo; level j (time t = t_hi - j) turns lambda^{t+1} into lambda^t in shared
// memory for every site whose distance to the region edge exceeds j (its pull from
// x + c_i is still valid), adds the receiver terms R^t c_s^2 of the receivers inside the
// region (per-region lists, so that the halo sees them too), and one barrier closes the
// level.  The own tile's medium and source gradients are summed over the K levels in
// registers and added to dJ/d(eta^2) once; rho^t comes from the replay tape at
// rho_hi - j plane.  HBM traffic per site falls from 2Q + 2 FP32 words and an FP64
// read-modify-write per level to (48 / OUT)^2 Q + Q + 1 words, K tape words and one
// FP64 read-modify-write per K levels.
struct AdjTbArgs {
    const float *rho_hi;   // rho(x, t_hi) on the tape; level j reads rho_hi - j plane
    long long t_hi;        // time of level 0; the launch covers t_hi .. t_hi - K + 1
    const int *reg_off;    // [regions + 1] offsets into reg_rec (nullptr: no receivers)
    const int2 *reg_rec;   // {receiver r, region site} for every receiver position in a region
    int tiles_x;
};

template <int Q, bool MRT, bool PERIODIC, int K>
__global__ void __launch_bounds__(kTbThreads) adjoint_tb_kernel(const StepArgs a, const AdjArgs d,
                                                                const AdjTbArgs b) {
    pdl_trigger_and_wait();
    constexpr int W = kTbW, NS = kTbNS, OUT = W - 2 * K, PER = kTbPer;
    extern __shared__ float smem[];  // two copies of [Q][NS]
    float *bufA = smem, *bufB = smem + Q * NS;
    const int X0 = blockIdx.x * OUT - K, Y0 = blockIdx.y * OUT - K;
    const int tid = threadIdx.x;

    // ---- lambda^{t_hi + 1} on the region into copy A (zero outside a zero-ghost domain)
    const bool interior = (K % 4 == 0) && (OUT % 4 == 0) && X0 >= 0 && Y0 >= 0 &&
                          X0 + W <= a.nx && Y0 + W <= a.ny;
    if (interior) {  // 16-byte loads: X0 = OUT bx - K is a multiple of 4
        constexpr int CH = W / 4;
        for (int e = tid; e < Q * W * CH; e += kTbThreads) {
            const int i = e / (W * CH), rem = e - i * (W * CH), r = rem / CH, c = rem - r * CH;
            const float4 v = *reinterpret_cast<const float4 *>(
                d.lam_in + i * a.plane + (long long)(Y0 + r) * a.pitch + X0 + 4 * c);
            *reinterpret_cast<float4 *>(bufA + i * NS + r * W + 4 * c) = v;
        }
    } else {
        for (int e = tid; e < Q * NS; e += kTbThreads) {
            const int i = e / NS, s = e - i * NS, r = s / W, c = s - r * W;
            const int gx = X0 + c, gy = Y0 + r;
            float v = 0.f;
            if (PERIODIC)
                v = d.lam_in[i * a.plane + (long long)wrap_mod(gy, a.ny) * a.pitch + wrap_mod(gx, a.nx)];
            else if (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny)
                v = d.lam_in[i * a.plane + (long long)gy * a.pitch + gx];
            bufA[i * NS + s] = v;
        }
    }
    // ---- per-thread sites: column c = tid mod 48 and rows r0 + 8 m (384 = 8 x 48); ring
    // distance (-1: outside the domain), medium, sponge, source and own-tile flags
    static_assert(kTbThreads % W == 0, "a thread's sites share one column");
    constexpr int RS = kTbThreads / W;  // row step between a thread's sites
    const int c = tid % W, r0 = tid / W;
    int ring[PER];
    float e2[PER], sf[PER];
    unsigned srcmask = 0u, ownmask = 0u;
#pragma unroll
    for (int m = 0; m < PER; m++) {
        const int s = tid + m * kTbThreads, r = r0 + RS * m;
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
        // own sites: inside the tile and, unwrapped, inside the grid (the last tile row or
        // column may reach past nx / ny); each grid site is owned by exactly one CTA
        if (live && r >= K && r < K + OUT && c >= K && c < K + OUT && X0 + c < a.nx &&
            Y0 + r < a.ny) {
            ownmask |= 1u << m;
            if (gx == a.src_x && gy == a.src_y && a.src_tab) srcmask |= 1u << m;
        }
        if (!live)
#pragma unroll
            for (int i = 0; i < Q; i++) bufB[i * NS + s] = 0.f;  // copy A is already 0 there
    }
    // grid index of own site m: own0 + m RS pitch (own sites are unwrapped and in the grid)
    const long long own0 = (long long)(Y0 + r0) * a.pitch + X0 + c;
    bool damp = false;
#pragma unroll
    for (int m = 0; m < PER; m++) damp |= sf[m] != 1.f;
    const bool sp_block = __syncthreads_or(damp);

    // The own sites' gradient terms of the K levels are summed in FP32 (the terms are FP32
    // products of FP32 adjoint quantities) and added to the FP64 gradient once: GB300's
    // FP64 rate would otherwise bound the sweep.  rho of the next level is loaded while
    // the current one computes.
    float acc[PER], rho_n[PER];
#pragma unroll
    for (int m = 0; m < PER; m++) {
        acc[m] = 0.f;
        rho_n[m] = (ownmask & (1u << m)) ? b.rho_hi[own0 + (long long)(m * RS) * a.pitch] : 0.f;
    }
    const int reg = blockIdx.y * b.tiles_x + blockIdx.x;
    const int q0 = b.reg_off ? b.reg_off[reg] : 0, q1 = b.reg_off ? b.reg_off[reg + 1] : 0;
#pragma unroll 1
    for (int j = 0; j < K; j++) {
        const float *src = (j & 1) ? bufB : bufA;
        float *dst = (j & 1) ? bufA : bufB;
        const long long t = b.t_hi - j;
        const float *rho = b.rho_hi - (long long)j * a.plane;
        float rho_j[PER];
#pragma unroll
        for (int m = 0; m < PER; m++) {
            rho_j[m] = rho_n[m];
            if (j + 1 < K && (ownmask & (1u << m)))
                rho_n[m] = rho[own0 + (long long)(m * RS) * a.pitch - a.plane];
        }
        // the sites of one level; SPONGE: the region meets the sponge (block-uniform)
        auto level = [&](auto sponge) {
#pragma unroll
            for (int m = 0; m < PER; m++) {
                if (ring[m] <= j) continue;
                const int s = tid + m * kTbThreads;
                // mu_i(x) = sigma(x) lambda_i^{t+1}(x + c_i)
                float mm[Q];
#pragma unroll
                for (int i = 0; i < Q; i++) {
                    mm[i] = src[i * NS + s + Lat<Q>::cy(i) * W + Lat<Q>::cx(i)];
                    if (decltype(sponge)::value) mm[i] *= sf[m];
                }
                if (srcmask & (1u << m)) {  // own source site
                    float src_w, src_dw;
                    adj_src<Q>(mm, e2[m], a, src_w, src_dw);
                    if (d.grad_src) d.grad_src[t - d.t0] = (double)src_w;
                    if (t < a.src_nt) acc[m] += a.src_tab[t] * src_dw;
                }
                const float gsum = adj_site<Q, MRT>(mm, e2[m], a);
#pragma unroll
                for (int i = 0; i < Q; i++) dst[i * NS + s] = mm[i];
                if (ownmask & (1u << m)) acc[m] += rho_j[m] * gsum;
            }
        };
        if (sp_block)
            level(std::true_type{});
        else
            level(std::false_type{});
        if (q1 > q0) {  // block-uniform: receivers inside the region, at time t
            __syncthreads();
            for (int q = q0 + tid; q < q1; q += kTbThreads) {
                const int2 rs = b.reg_rec[q];
                const int2 xy = a.rec[rs.x];
                const long long idx = (long long)xy.y * a.pitch + xy.x;
                const float R = d.resid[(t - d.t0) * d.nrec + rs.x];
                const float c2 = cs2_of<Q>(a.eta2[idx], a);
#pragma unroll
                for (int i = 0; i < Q; i++) atomicAdd(dst + i * NS + rs.y, R * c2);
                const int r = rs.y / W, c = rs.y - r * W;
                if (r >= K && r < K + OUT && c >= K && c < K + OUT && X0 + c == xy.x &&
                    Y0 + r == xy.y)
                    atomicAdd(d.grad + idx, (double)R * (double)dcs2<Q>(a) * (double)rho[idx]);
            }
        }
        __syncthreads();
    }
    // ---- lambda^{t_hi - K + 1} of the own tile, and the summed gradient
#pragma unroll
    for (int m = 0; m < PER; m++)
        if (ownmask & (1u << m)) d.grad[own0 + (long long)(m * RS) * a.pitch] += (double)acc[m];
    const float *fin = (K % 2 == 0) ? bufA : bufB;
    const int OX = blockIdx.x * OUT, OY = blockIdx.y * OUT;
    const bool full = (K % 4 == 0) && (OUT % 4 == 0) && OX + OUT <= a.nx && OY + OUT <= a.ny;
    if (full) {
        constexpr int CH = OUT / 4;
        for (int e = tid; e < Q * OUT * CH; e += kTbThreads) {
            const int i = e / (OUT * CH), rem = e - i * (OUT * CH), r = rem / CH, c = rem - r * CH;
            const float4 v = *reinterpret_cast<const float4 *>(fin + i * NS + (r + K) * W + K + 4 * c);
            *reinterpret_cast<float4 *>(d.lam_out + i * a.plane + (long long)(OY + r) * a.pitch +
                                        OX + 4 * c) = v;
        }
    } else {
        for (int e = tid; e < Q * OUT * OUT; e += kTbThreads) {
            const int i = e / (OUT * OUT), s = e - i * (OUT * OUT), r = s / OUT, c = s - r * OUT;
            const int gx = OX + c, gy = OY + r;
            if (gy < a.ny && gx < a.pitch)
                d.lam_out[i * a.plane + (long long)gy * a.pitch + gx] =
                    gx < a.nx ? fin[i * NS + (r + K) * W + c + K] : 0.f;
        }
    }
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

AdjFn pick_adj_rec(int Q) { return Q == 9 ? adjoint_receivers<9> : adjoint_receivers<5>; }

using AdjTbFn = void (*)(const StepArgs, const AdjArgs, const AdjTbArgs);

// levels per blocked launch: D2Q5 8 (32 x 32 tiles; two copies of 5 x 48^2 floats, 92 KB of
// shared memory, two CTAs per SM), D2Q9 4 (40 x 40 tiles; 166 KB, one CTA per SM)
constexpr int kAdjLevels5 = 8, kAdjLevels9 = 4;
int adj_tb_levels(int Q) { return Q == 5 ? kAdjLevels5 : kAdjLevels9; }

template <int Q, bool MRT, int K> AdjTbFn adj_tb_fn(bool per) {
    return per ? adjoint_tb_kernel<Q, MRT, true, K> : adjoint_tb_kernel<Q, MRT, false, K>;
}

AdjTbFn pick_adj_tb(int Q, bool mrt, bool per) {
    if (Q == 9)
        return mrt ? adj_tb_fn<9, true, kAdjLevels9>(per) : adj_tb_fn<9, false, kAdjLevels9>(per);
    return mrt ? adj_tb_fn<5, true, kAdjLevels5>(per) : adj_tb_fn<5, false, kAdjLevels5>(per);
}

// Every (region, local coordinate) along one axis at which grid coordinate x appears:
// region b covers the unwrapped coordinates b OUT - K .. b OUT - K + 47; a periodic axis
// also places the images x + k n of x.
void axis_hits(int x, int n, int tiles, int K, bool per, std::vector<std::pair<int, int>> &hits) {
    const int OUT = kTbW - 2 * K, lo = -K, hi = tiles * OUT - K + kTbW;
    hits.clear();
    int xs = x;
    if (per)
        while (xs - n >= lo) xs -= n;
    for (; xs < hi; xs += n) {
        if (xs >= lo) {
            const int num = xs + K - (kTbW - 1);
            const int b0 = num <= 0 ? 0 : (num + OUT - 1) / OUT;
            const int b1 = std::min((xs + K) / OUT, tiles - 1);
            for (int bb = b0; bb <= b1; bb++) hits.emplace_back(bb, xs - (bb * OUT - K));
        }
        if (!per) break;
    }
}

// receivers inside each region of the blocked sweep: offsets [regions + 1] and
// {receiver, region site} entries, grouped by region
void region_lists(const lb_ctx *ctx, int K, bool per, std::vector<int> &off,
                  std::vector<int2> &ent) {
    const int OUT = kTbW - 2 * K;
    const int tx = (ctx->nx + OUT - 1) / OUT, ty = (ctx->ny + OUT - 1) / OUT;
    std::vector<std::pair<int, int>> hx, hy;
    std::vector<std::pair<int, int2>> all;  // (region, entry)
    for (int r = 0; r < ctx->nrec; r++) {
        axis_hits(ctx->rec_xy[2 * r], ctx->nx, tx, K, per, hx);
        axis_hits(ctx->rec_xy[2 * r + 1], ctx->ny, ty, K, per, hy);
        for (const auto &py : hy)
            for (const auto &px : hx)
                all.push_back({py.first * tx + px.first, make_int2(r, py.second * kTbW + px.second)});
    }
    off.assign((size_t)tx * ty + 1, 0);
    for (const auto &e : all) off[e.first + 1]++;
    for (size_t k = 1; k < off.size(); k++) off[k] += off[k - 1];
    std::vector<int> pos(off.begin(), off.end() - 1);
    ent.resize(std::max<size_t>(all.size(), 1));
    for (const auto &e : all) ent[pos[e.first]++] = e.second;
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

void tape_reset(lb_ctx *ctx) { ctx->tape_t0 = ctx->t; }

float *tape_row(const lb_ctx *ctx, long long t) {
    const long long r = t - ctx->tape_t0;
    if (!ctx->rho_tape || r < 0 || r >= ctx->tape_cap) return nullptr;
    return ctx->rho_tape + r * (long long)ctx->ny * ctx->pitch;
}

extern "C" lb_status lb_record_rho(lb_ctx *ctx, int nt_capacity) {
    if (!ctx) return LB_EINVAL;
    if (ctx->slab_nyg) return fail(ctx, LB_ESTATE, "a row slab has no adjoint");
    if (nt_capacity < 0) return fail(ctx, LB_EINVAL, "nt_capacity < 0");
    if (nt_capacity > 0 && ctx->aa)
        return fail(ctx, LB_ESTATE, "no rho tape with in-place streaming (LB_STREAM_AA)");
    if (nt_capacity > 0 && (ctx->Q == 7 || ctx->refined || ctx->cfg.storage == LB_F64))
        return fail(ctx, LB_ESTATE, "the rho tape serves the 2-D adjoint without a patch "
                    "(FP32, BF16 or FP16 storage)");
    cudaError_t e = cudaStreamSynchronize(ctx->stream);  // steps may still write the old tape
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rho tape");
    if (ctx->rho_tape) dev_free(ctx, ctx->rho_tape);
    ctx->rho_tape = nullptr;
    ctx->tape_cap = 0;
    if (nt_capacity == 0) return LB_OK;
    const size_t bytes = (size_t)nt_capacity * ctx->ny * ctx->pitch * 4;
    ctx->rho_tape = static_cast<float *>(dev_alloc(ctx, bytes));
    if (!ctx->rho_tape) return fail(ctx, LB_ENOMEM, "rho tape of %d steps (%zu bytes)", nt_capacity, bytes);
    ctx->tape_cap = nt_capacity;
    tape_reset(ctx);
    return LB_OK;
}

extern "C" lb_status lb_checkpoint_every(lb_ctx *ctx, int every) {
    if (!ctx) return LB_EINVAL;
    if (ctx->slab_nyg) return fail(ctx, LB_ESTATE, "a row slab has no adjoint");
    if (every > 0 && ctx->Q == 7) return fail(ctx, LB_ESTATE, "the adjoint is 2-D (D2Q5 / D2Q9)");
    if (every < 0) return fail(ctx, LB_EINVAL, "every < 0");
    if (every > 0 && ctx->aa)
        return fail(ctx, LB_ESTATE, "no checkpoints with in-place streaming (LB_STREAM_AA)");
    if (every > 0 && (ctx->refined || (ctx->cfg.storage != LB_F32 && ctx->cfg.storage != LB_BF16)))
        return fail(ctx, LB_ESTATE, "the adjoint needs an FP32 or BF16 context without a patch");
    ctx->ckpt_every = every;
    ckpt_reset(ctx);
    return LB_OK;
}

extern "C" lb_status lb_adjoint(lb_ctx *ctx, const float *dJdp, int nt, float *grad_c,
                                double *grad_src, float *grad_g0, int on_device) {
    if (!ctx) return LB_EINVAL;
    if (ctx->slab_nyg) return fail(ctx, LB_ESTATE, "a row slab has no adjoint");
    if (ctx->cfg.storage == LB_F64) return fail(ctx, LB_ESTATE, "no adjoint for LB_F64 (test only)");
    if (ctx->aa) return fail(ctx, LB_ESTATE, "no adjoint with in-place streaming (LB_STREAM_AA)");
    if (nt < 1) return fail(ctx, LB_EINVAL, "nt < 1");
    if (ctx->nrec > 0 && !dJdp) return fail(ctx, LB_EINVAL, "dJdp is NULL");
    // The forward rho tape (lb_record_rho) covers the nt steps: no checkpoints, no replays.
    const bool taped = ctx->rho_tape && nt <= ctx->tape_cap && ctx->t - ctx->tape_t0 >= nt &&
                       (ctx->nrec == 0 || ctx->tape_t0 == ctx->t_rec0);
    const int C = taped ? 0 : ctx->ckpt_every;
    if (!taped) {
        if (C <= 0)
            return fail(ctx, LB_ESTATE,
                        "call lb_checkpoint_every or lb_record_rho (at the receivers' start time) "
                        "before stepping");
        if (ctx->t - ctx->ckpt_t0 < nt || (long long)ctx->ckpt_count * C < nt)
            return fail(ctx, LB_ESTATE, "checkpoints cover %lld steps, %d requested",
                        std::min<long long>(ctx->t - ctx->ckpt_t0, (long long)ctx->ckpt_count * C),
                        nt);
        if (ctx->nrec > 0 && ctx->ckpt_t0 != ctx->t_rec0)
            return fail(ctx, LB_ESTATE, "receivers must be set at the checkpointed start time");
    }
    const int Q = ctx->Q;
    // forward states (checkpoints, replays) in the storage type; adjoint states FP32
    const size_t plane = (size_t)ctx->ny * ctx->pitch, sbytes = (size_t)Q * plane * ctx->ebytes,
                 lbytes = (size_t)Q * plane * 4;
    // replay plan: the rho tape holds T steps; sub-checkpoints every T steps when T < C
    const int T = taped ? 0 : adj_tape_steps(plane * 4, C);
    const int nsub = taped ? 0 : (C + T - 1) / T;
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
    void *X[2] = {nullptr, nullptr};
    std::vector<void *> SC(std::max(nsub, 1), nullptr);  // SC[0] is the segment's checkpoint
    float *tape = ctx->rho_tape;
    if (!taped) {
        for (auto &p : X)
            if (!(p = grab(sbytes))) return release(fail(ctx, LB_ENOMEM, "replay states"));
        for (int j = 1; j < nsub; j++)
            if (!(SC[j] = grab(sbytes))) return release(fail(ctx, LB_ENOMEM, "sub-checkpoints"));
        tape = static_cast<float *>(grab((size_t)T * plane * 4));
        if (!tape) return release(fail(ctx, LB_ENOMEM, "rho tape (%d steps)", T));
    }
    float *L[2];
    for (auto &p : L)
        if (!(p = static_cast<float *>(grab(lbytes)))) return release(fail(ctx, LB_ENOMEM, "adjoint state"));
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
    cudaMemsetAsync(L[0], 0, lbytes, ctx->stream);
    cudaMemsetAsync(L[1], 0, lbytes, ctx->stream);
    cudaMemsetAsync(grad, 0, plane * 8, ctx->stream);
    cudaMemsetAsync(gsrc, 0, (size_t)nt * 8, ctx->stream);

    const bool mrt = ctx->cfg.collision == LB_MRT, per = ctx->cfg.boundary == LB_PERIODIC;
    StepFn fwd = pick_step(ctx);
    AdjFn adj = pick_adj(Q, mrt, per), adj_rec = pick_adj_rec(Q);
    // blocked reverse sweep: Ka levels per launch wherever Ka levels of a sub-segment remain
    const int Ka = adj_tb_levels(Q), OUTa = kTbW - 2 * Ka;
    AdjTbFn adj_tb = pick_adj_tb(Q, mrt, per);
    AdjTbArgs tbb;
    tbb.tiles_x = (ctx->nx + OUTa - 1) / OUTa;
    tbb.reg_off = nullptr;
    tbb.reg_rec = nullptr;
    const dim3 tb_grid(tbb.tiles_x, (ctx->ny + OUTa - 1) / OUTa);
    const size_t tb_smem = 2 * (size_t)Q * kTbNS * sizeof(float);
    {
        cudaError_t e = cudaFuncSetAttribute(adj_tb, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tb_smem);
        if (e != cudaSuccess) return release(cuda_fail(ctx, e, "blocked adjoint shared memory"));
    }
    // D2Q5: the wavefront sweep (adjoint5.cu), kAdj5Levels levels per launch, receivers by row
    const bool wave = Q == 5;
    const int *row_off = nullptr, *row_x = nullptr, *row_id = nullptr;
    if (wave && ctx->nrec > 0) {
        std::vector<int> off, xs, ids;
        adj5_row_lists(ctx, off, xs, ids);
        int *o = static_cast<int *>(grab(off.size() * sizeof(int)));
        int *x = static_cast<int *>(grab(xs.size() * sizeof(int)));
        int *i = static_cast<int *>(grab(ids.size() * sizeof(int)));
        if (!o || !x || !i) return release(fail(ctx, LB_ENOMEM, "row receiver lists"));
        cudaMemcpyAsync(o, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
        cudaMemcpyAsync(x, xs.data(), xs.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
        cudaMemcpyAsync(i, ids.data(), ids.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
        // the host vectors go out of scope: the copies must have read them
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return release(cuda_fail(ctx, e, "row receiver lists"));
        row_off = o;
        row_x = x;
        row_id = i;
    }
    std::vector<int> reg_off;
    std::vector<int2> reg_ent;
    if (!wave && ctx->nrec > 0) {
        region_lists(ctx, Ka, per, reg_off, reg_ent);
        int *o = static_cast<int *>(grab(reg_off.size() * sizeof(int)));
        int2 *en = static_cast<int2 *>(grab(reg_ent.size() * sizeof(int2)));
        if (!o || !en) return release(fail(ctx, LB_ENOMEM, "region receiver lists"));
        cudaMemcpyAsync(o, reg_off.data(), reg_off.size() * sizeof(int), cudaMemcpyHostToDevice,
                        ctx->stream);
        cudaMemcpyAsync(en, reg_ent.data(), reg_ent.size() * sizeof(int2), cudaMemcpyHostToDevice,
                        ctx->stream);
        tbb.reg_off = o;
        tbb.reg_rec = en;
    }
    StepArgs base = base_args(ctx);
    base.trace_row = nullptr;  // replays record nothing
    const long long t0 = taped ? ctx->tape_t0 : ctx->ckpt_t0;
    const int segs4 = (ctx->nx + 127) / 128;
    const int adj_blocks = (int)(((long long)ctx->ny * segs4 + kWarps - 1) / kWarps);
    // replay steps t = from .. from + n - 1 starting at state `in`; the state after the
    // last one goes to `last` (when given); rho(t) goes to tape[t - from] (when given).
    // FP32 contexts replay K steps per launch with the time-blocked kernel wherever a whole
    // block of K fits (not from a raw state); other steps run one per launch.
    const int K = ctx->cfg.storage == LB_F32 ? (ctx->Q == 5 ? 8 : ctx->Q == 9 ? 4 : 0) : 0;
    lb_status rst = LB_OK;
    auto replay = [&](const void *in, bool raw, long long from, int n, void *last, bool record) {
        int x = 0;
        for (int m = 0; m < n;) {
            const bool first_raw = raw && m == 0;
            const int len = (K > 0 && !first_raw && n - m >= K) ? K : 1;
            StepArgs a = base;
            a.in = in;
            a.out = (m + len == n && last) ? last : X[x];
            a.raw = first_raw ? 1 : 0;
            a.t = from + m;
            a.rho_out = record ? tape + (size_t)m * plane : nullptr;
            a.rho_stride = (long long)plane;
            if (len > 1) {
                if (rst == LB_OK) rst = tb_launch_args(ctx, a, len);
            } else if (ctx->staged) {
                stream_launch(ctx, a, 0);  // cannot fail once the forward run has stepped
            } else {
                launch_pdl(fwd, dim3(a.main_blocks), dim3(kThreads), 0, ctx->stream, a);
            }
            in = a.out;
            x ^= 1;
            m += len;
        }
    };
    int li = 0;  // L[li] holds lambda^{t+1}
    // the adjoint steps of times sa + len - 1 .. sa; rho(sa + m) at rho0 + m plane
    auto sweep = [&](long long sa, int len, const float *rho0) {
        for (int m = len - 1; m >= 0;) {
            StepArgs a = base;
            a.t = sa + m;
            AdjArgs d;
            d.lam_in = L[li];
            d.lam_out = L[li ^ 1];
            d.rho = rho0 + (size_t)m * plane;
            d.grad = grad;
            d.grad_src = gsrc;
            d.t0 = t0;
            d.resid = resid;
            d.nrec = ctx->nrec;
            d.segs = segs4;
            if (wave && m + 1 >= kAdj5Levels) {  // levels sa + m .. sa + m - K + 1, wavefront
                const cudaError_t e =
                    adj5_launch(ctx, a, d, d.rho, a.t, row_off, row_x, row_id);
                if (e != cudaSuccess && rst == LB_OK) rst = cuda_fail(ctx, e, "wavefront adjoint");
                m -= kAdj5Levels;
            } else if (!wave && m + 1 >= Ka) {  // levels sa + m .. sa + m - Ka + 1 in one launch
                tbb.rho_hi = d.rho;
                tbb.t_hi = a.t;
                launch_pdl(adj_tb, tb_grid, dim3(kTbThreads), tb_smem, ctx->stream, a, d, tbb);
                m -= Ka;
            } else {
                launch_pdl(adj, dim3(adj_blocks), dim3(kThreads), 0, ctx->stream, a, d);
                if (ctx->nrec > 0)
                    launch_pdl(adj_rec, dim3((ctx->nrec + 255) / 256), dim3(256), 0,
                               ctx->stream, a, d);
                m -= 1;
            }
            li ^= 1;
        }
    };
    if (taped) {
        sweep(t0, nt, ctx->rho_tape);
    } else {
        const int nseg = (nt + C - 1) / C;
        for (int k = nseg - 1; k >= 0; k--) {
            const long long ta = t0 + (long long)k * C, tb = std::min<long long>(ta + C, t0 + nt);
            const bool raw_a = (k == 0) && ctx->ckpt_raw0;
            const int nsc = (int)((tb - ta + T - 1) / T);
            SC[0] = ctx->ckpt[k];
            for (int j = 1; j < nsc; j++)  // place the sub-checkpoints
                replay(SC[j - 1], raw_a && j == 1, ta + (long long)(j - 1) * T, T, SC[j], false);
            // sweep the sub-segments backwards: replay recording rho, then the adjoint steps
            for (int j = nsc - 1; j >= 0; j--) {
                const long long sa = ta + (long long)j * T, sb = std::min<long long>(sa + T, tb);
                const int len = (int)(sb - sa);
                replay(SC[j], raw_a && j == 0, sa, len, nullptr, true);
                sweep(sa, len, tape);
            }
        }
    }
    lb_status st = rst != LB_OK ? rst : check_launch(ctx, "adjoint");
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
