// adjoint5.cu -- the D2Q5 reverse sweep of the adjoint as a row wavefront: K adjoint levels
// per launch.
//
// One adjoint level turns lambda^{t+1} into lambda^t (adjoint.cu): it pulls
// mu_i(x) = sigma(x) lambda_i^{t+1}(x + c_i), applies the transposed collision and adds the
// receiver terms.  Written for a_j = lambda_{opp(j)}, the pull is a_j(x - c_j): the forward
// pull of Eq. BGK-LB.  So the sweep of tblock5.cuh carries over unchanged on a: a CTA of 256
// threads owns a strip of 256 columns (256 - 2K output columns) and a chunk of rows that it
// sweeps upward; in iteration r level 0 loads row r of lambda^{t_hi + 1} and level l
// (1 <= l <= K) computes row r - l of lambda^t, t = t_hi - (l - 1), from level l - 1:
//   a_0 (x, y)      this thread, from the previous iteration,
//   a_2 (x, y - 1)  this thread, from two iterations back,
//   a_4 (x, y + 1)  this thread, computed just before in this iteration,
//   a_1 (x - 1, y), a_3 (x + 1, y)  neighbouring threads, through shared memory.
// The medium gradient of a site, sum over the K levels of rho^t(x) (v . dw/d(eta^2)) plus
// the source and receiver terms, travels with the site's row from level to level like the
// populations do (level l adds its term to what level l - 1 left for the same row one
// iteration earlier), and level K adds it to the FP64 gradient once.  HBM sees one read and
// one write of lambda, K reads of the rho tape and one FP64 read-modify-write of the
// gradient per site and K levels.  The per-site arithmetic is adjoint.cu's (adj_site,
// adj_src, the receiver terms), in the same order.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "adjoint_site.cuh"
#include "lb_kernels.cuh"
#include "lb_runtime.h"

namespace lbadj5 {

using namespace lbk;
using namespace lbadj;

constexpr int kWS = 256;  // strip width in columns = threads per CTA

struct Adj5Args {
    const float *rho_hi;  // rho(x, t_hi) on the tape; level l (1-based) reads rho_hi - (l - 1) plane
    long long t_hi;       // time of level 1; the launch covers t_hi .. t_hi - K + 1
    const int *row_off;   // [ny + 1]: receivers of row y are entries row_off[y] .. row_off[y+1]
    const int *rec_x;     // their x, ascending within a row
    const int *rec_id;    // their receiver index
    int H;                // output rows per CTA
    int per;              // periodic boundary
};

// Per-thread constants of one strip and row chunk.
struct Adj5Thread {
    int c, gx, gxw, Y0, Y1;
    bool per, col_in, own_col, pad_col, edgy_cols;
    int dxs;             // distance of this column to the nearest x face
    int spec_lo, spec_hi;  // first and last chunk row that holds the source or a receiver
    float *xs;           // [2][K][2][kWS + 2]: a_1, a_3 of each level's newest row, by parity
};

// Level-0 row r of lambda^{t_hi + 1} as a_j = lambda_{opp(j)}, and eta^2; zero outside a
// zero-ghost domain.
__device__ __forceinline__ void adj5_load(const StepArgs &a, const AdjArgs &d, const Adj5Thread &T,
                                          int r, float (&v)[5], float &e2) {
    int yw = r;
    bool live = T.col_in;
    if (T.per)
        yw = wrap_mod(r, a.ny);
    else
        live = live && r >= 0 && r < a.ny;
    if (!live) {
#pragma unroll
        for (int j = 0; j < 5; j++) v[j] = 0.f;
        e2 = 0.f;
        return;
    }
    const long long o = (long long)yw * a.pitch + T.gxw;
#pragma unroll
    for (int j = 0; j < 5; j++) v[j] = d.lam_in[Lat<5>::opp(j) * a.plane + o];
    e2 = a.eta2[o];
}

// The receivers at site (x, y) at time t: lambda^t_i += R c_s^2 for every population, and the
// gradient term R dc_s^2/d(eta^2) rho^t added to part when the site is this CTA's own.
__device__ __forceinline__ void adj5_receivers(const StepArgs &a, const AdjArgs &d,
                                               const Adj5Args &b, int x, int y, long long t,
                                               float e2, float rho, bool mine, float (&m)[5],
                                               float &part) {
    int lo = b.row_off[y];
    const int hi = b.row_off[y + 1];
    int h = hi;
    while (lo < h) {
        const int mid = (lo + h) >> 1;
        if (b.rec_x[mid] < x)
            lo = mid + 1;
        else
            h = mid;
    }
    for (; lo < hi && b.rec_x[lo] == x; lo++) {
        const float R = d.resid[(t - d.t0) * d.nrec + b.rec_id[lo]];
        const float c2 = cs2_of<5>(e2, a);
#pragma unroll
        for (int i = 0; i < 5; i++) m[i] += R * c2;
        if (mine) part += R * dcs2<5>(a) * rho;
    }
}

// One wavefront iteration r (parity P; the row loop is unrolled by two so that level state
// alternates between register names instead of moving).  FAST: every level's row is an own
// row of the chunk and none holds the source or a receiver; edgy (CTA-uniform): the strip or
// the rows touch the sponge or the outside, so the sites take their sponge factor.
template <bool MRT, int K, int P, bool FAST>
__device__ __forceinline__ void adj5_iter(const StepArgs &a, const AdjArgs &d, const Adj5Args &b,
                                          const Adj5Thread &T, float (&W0)[2][K], float (&EE)[2][K],
                                          float (&G2)[2][K], float (&PA)[2][K], float (&RH)[2][K],
                                          double (&GR)[2], float (&pre)[2][5], float (&pre_e2)[2],
                                          int r, int rend, bool edgy) {
    constexpr int SR = kWS + 2, SL = 2 * SR;  // row and level strides of xs
    float n[5], nE;  // level l's newest row (r - l) in a-labels; level 0: the prefetched row r
#pragma unroll
    for (int j = 0; j < 5; j++) n[j] = pre[P][j];
    nE = pre_e2[P];
    if (r + 1 < rend) adj5_load(a, d, T, r + 1, pre[P ^ 1], pre_e2[P ^ 1]);
    // the tape values and the gradient the next iteration uses, loaded one iteration early
    // (own sites only: only their sums reach the gradient)
    if (T.own_col) {
#pragma unroll
        for (int l = 0; l < K; l++) {
            const int yn = r - l;  // level l's row in the next iteration
            RH[P ^ 1][l] = (yn >= T.Y0 && yn < T.Y1)
                               ? b.rho_hi[-(long long)l * a.plane + (long long)yn * a.pitch + T.gx]
                               : 0.f;
        }
        const int yg = r + 1 - K;  // the row level K stores in the next iteration
        GR[P ^ 1] = (yg >= T.Y0 && yg < T.Y1) ? d.grad[(long long)yg * a.pitch + T.gx] : 0.0;
    }
    float *cur = T.xs + P * K * SL + T.c + 1;        // this iteration's rows, column c
    const float *prv = T.xs + (P ^ 1) * K * SL + T.c;  // last iteration's rows, column c - 1
    float h1[K], h3[K];
#pragma unroll
    for (int l = 0; l < K; l++) {
        h1[l] = prv[l * SL];           // a_1 (x - 1, y)
        h3[l] = prv[l * SL + SR + 2];  // a_3 (x + 1, y)
    }
#pragma unroll
    for (int l = 0; l < K; l++) {
        cur[l * SL] = n[1];
        cur[l * SL + SR] = n[3];
        // pulled a_j(x - c_j); mu_i = a_{opp(i)}(x + c_i)
        const float p0 = W0[P ^ 1][l], p1 = h1[l], p2 = G2[P][l], p3 = h3[l], p4 = n[4];
        const float e2 = EE[P ^ 1][l];
        W0[P][l] = n[0];
        G2[P][l] = n[2];
        EE[P][l] = nE;
        float m[5] = {p0, p3, p4, p1, p2};
        float part = l == 0 ? 0.f : PA[P ^ 1][l - 1];
        const int y = r - l - 1;           // the row level l + 1 computes
        const long long t = b.t_hi - l;    // at this time
        const float rh = RH[P][l];         // rho^t(x, y) of an own site, else 0
        if (FAST) {
            if (edgy) {  // CTA-uniform: sponge columns or rows, or columns outside the domain
                const int yw = T.per ? wrap_mod(y, a.ny) : y;
                const float f = T.col_in ? sponge_of_dist(min(T.dxs, min(yw, a.ny - 1 - yw)), a)
                                         : 0.f;
#pragma unroll
                for (int i = 0; i < 5; i++) m[i] *= f;
            }
            const float gsum = adj_site<5, MRT>(m, e2, a);
            part += rh * gsum;
        } else if (r >= T.Y0 - K + 2 * (l + 1)) {  // its inputs exist (warp-uniform)
            bool live = T.col_in;
            int yw = y;
            if (T.per)
                yw = wrap_mod(y, a.ny);
            else
                live = live && y >= 0 && y < a.ny;
            const bool mine = live && T.own_col && y >= T.Y0 && y < T.Y1;
            if (live) {
                if (a.sponge_w > 0) {
                    const float f = sponge_factor(T.gxw, yw, a);
#pragma unroll
                    for (int i = 0; i < 5; i++) m[i] *= f;
                }
                if (yw == a.src_y && T.gxw == a.src_x && a.src_tab != nullptr) {
                    float src_w, src_dw;
                    adj_src<5>(m, e2, a, src_w, src_dw);
                    if (mine && d.grad_src) d.grad_src[t - d.t0] = (double)src_w;
                    if (t < a.src_nt) part += a.src_tab[t] * src_dw;
                }
                const float gsum = adj_site<5, MRT>(m, e2, a);
                part += rh * gsum;
                if (b.row_off && b.row_off[yw + 1] > b.row_off[yw])  // warp-uniform
                    adj5_receivers(a, d, b, T.gxw, yw, t, e2, rh, mine, m, part);
            } else {
#pragma unroll
                for (int i = 0; i < 5; i++) m[i] = 0.f;
            }
        }
        // back to a-labels for the next level: a_j = lambda_{opp(j)}
        n[0] = m[0];
        n[1] = m[3];
        n[2] = m[4];
        n[3] = m[1];
        n[4] = m[2];
        nE = e2;
        PA[P][l] = part;
    }
    // level K holds row r - K: lambda^{t_hi - K + 1} and the site's summed gradient
    const int yo = r - K;
    if (FAST ? T.own_col : (yo >= T.Y0 && yo < T.Y1 && (T.own_col || T.pad_col))) {
        const long long o = (long long)yo * a.pitch + T.gx;
#pragma unroll
        for (int j = 0; j < 5; j++) d.lam_out[Lat<5>::opp(j) * a.plane + o] = T.own_col ? n[j] : 0.f;
        if (T.own_col) d.grad[o] = GR[P] + (double)PA[P][K - 1];
    }
    __syncthreads();
}

// The strip bx and row chunk by: K adjoint levels over the chunk's rows.
// xs_mem: [2][K][2][kWS + 2] floats of shared memory.
template <bool MRT, int K>
__device__ __forceinline__ void adj5_body(const StepArgs &a, const AdjArgs &d, const Adj5Args &b,
                                          int bx, int by, float *xs_mem) {
    constexpr int OUT = kWS - 2 * K;
    Adj5Thread T;
    T.c = threadIdx.x;
    T.gx = bx * OUT - K + T.c;
    T.per = b.per != 0;
    T.col_in = true;
    T.gxw = T.gx;
    if (T.per)
        T.gxw = wrap_mod(T.gx, a.nx);
    else if (T.gx < 0 || T.gx >= a.nx)
        T.col_in = false, T.gxw = 0;
    T.own_col = T.c >= K && T.c < K + OUT && T.gx < a.nx;
    T.pad_col = T.c >= K && T.c < K + OUT && T.gx >= a.nx && T.gx < a.pitch;
    T.Y0 = by * b.H;
    T.Y1 = min(T.Y0 + b.H, a.ny);
    T.xs = xs_mem;
    if (T.c < 4 * K) {  // the pads either side of every row (the strip's outermost neighbours)
        constexpr int SR = kWS + 2;
        float *row = xs_mem + ((T.c & 1) * K + (T.c >> 1) % K) * 2 * SR + ((T.c >> 1) / K) * SR;
        row[0] = 0.f;
        row[kWS + 1] = 0.f;
    }
    T.dxs = min(T.gxw, a.nx - 1 - T.gxw);
    const bool x_edge = a.sponge_w > 0 && T.col_in && T.dxs < a.sponge_w;
    T.edgy_cols = __syncthreads_or(!T.col_in || x_edge) != 0;
    // the chunk rows that need the general path: the source row, and the rows with receivers
    T.spec_lo = 1;
    T.spec_hi = 0;
    if (a.src_tab != nullptr && a.src_y >= T.Y0 && a.src_y < T.Y1) T.spec_lo = T.spec_hi = a.src_y;
    if (b.row_off && b.row_off[T.Y1] > b.row_off[T.Y0]) {  // first and last receiver rows
        int lo = T.Y0, hi = T.Y1 - 1;
        while (lo < hi) {
            const int m = (lo + hi) >> 1;
            if (b.row_off[m + 1] > b.row_off[T.Y0]) hi = m; else lo = m + 1;
        }
        const int rlo = lo;
        lo = T.Y0;
        hi = T.Y1 - 1;
        while (lo < hi) {
            const int m = (lo + hi + 1) >> 1;
            if (b.row_off[m] < b.row_off[T.Y1]) lo = m; else hi = m - 1;
        }
        if (T.spec_lo > T.spec_hi) {
            T.spec_lo = rlo;
            T.spec_hi = lo;
        } else {
            T.spec_lo = min(T.spec_lo, rlo);
            T.spec_hi = max(T.spec_hi, lo);
        }
    }

    float W0[2][K], EE[2][K], G2[2][K], PA[2][K], RH[2][K], pre[2][5], pre_e2[2];
    double GR[2] = {0.0, 0.0};
#pragma unroll
    for (int l = 0; l < K; l++)
#pragma unroll
        for (int q = 0; q < 2; q++) W0[q][l] = EE[q][l] = G2[q][l] = PA[q][l] = RH[q][l] = 0.f;
    const int rbeg = T.Y0 - K, rend = T.Y1 + K;
    const int fbeg = T.Y0 + K, fend = T.Y1 + 1;  // iterations whose K rows are all own rows
    auto edgy = [&](int r) {  // CTA-uniform
        const int w = a.sponge_w, lo = r - K, hi = r - 1;
        if (T.edgy_cols) return true;
        if (w <= 0) return false;
        if (!T.per) return lo < w || hi > a.ny - 1 - w;
        return true;
    };
    auto fast_ok = [&](int r) {  // CTA-uniform
        if (r < fbeg || r >= fend) return false;
        const int lo = r - K, hi = r - 1;
        return !(T.spec_lo <= hi && T.spec_hi >= lo);
    };
    adj5_load(a, d, T, rbeg, pre[0], pre_e2[0]);
#pragma unroll 1
    for (int r = rbeg; r < rend; r += 2) {
        if (fast_ok(r))
            adj5_iter<MRT, K, 0, true>(a, d, b, T, W0, EE, G2, PA, RH, GR, pre, pre_e2, r, rend, edgy(r));
        else
            adj5_iter<MRT, K, 0, false>(a, d, b, T, W0, EE, G2, PA, RH, GR, pre, pre_e2, r, rend, edgy(r));
        if (r + 1 >= rend) break;
        if (fast_ok(r + 1))
            adj5_iter<MRT, K, 1, true>(a, d, b, T, W0, EE, G2, PA, RH, GR, pre, pre_e2, r + 1,
                                       rend, edgy(r + 1));
        else
            adj5_iter<MRT, K, 1, false>(a, d, b, T, W0, EE, G2, PA, RH, GR, pre, pre_e2, r + 1,
                                        rend, edgy(r + 1));
    }
}

template <bool MRT, int K>
__global__ void __launch_bounds__(kWS, 3) adj5_kernel(const StepArgs a, const AdjArgs d,
                                                      const Adj5Args b) {
    pdl_trigger_and_wait();
    extern __shared__ float xs_mem[];
    adj5_body<MRT, K>(a, d, b, blockIdx.x, blockIdx.y, xs_mem);
}

}  // namespace lbadj5

using namespace lbadj5;
using namespace lbrt;

// Receivers by row for the wavefront sweep: offsets [ny + 1], x ascending within a row.
void adj5_row_lists(const lb_ctx *ctx, std::vector<int> &off, std::vector<int> &xs,
                    std::vector<int> &ids) {
    const int n = ctx->nrec;
    off.assign((size_t)ctx->ny + 1, 0);
    std::vector<int> order(n);
    for (int r = 0; r < n; r++) {
        off[(size_t)ctx->rec_xy[2 * r + 1] + 1]++;
        order[r] = r;
    }
    for (size_t k = 1; k < off.size(); k++) off[k] += off[k - 1];
    const int *xy = ctx->rec_xy.data();
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) {
        return xy[2 * p + 1] != xy[2 * q + 1] ? xy[2 * p + 1] < xy[2 * q + 1] : xy[2 * p] < xy[2 * q];
    });
    xs.assign(std::max(n, 1), 0);
    ids.assign(std::max(n, 1), 0);
    for (int k = 0; k < n; k++) {
        xs[k] = xy[2 * order[k]];
        ids[k] = order[k];
    }
}

// K = kAdj5Levels adjoint levels t_hi .. t_hi - K + 1 from d.lam_in into d.lam_out, with
// rho^t_hi at rho_hi (rho^t at rho_hi - (t_hi - t) plane), on ctx's stream.
cudaError_t adj5_launch(lb_ctx *ctx, const StepArgs &a, const AdjArgs &d, const float *rho_hi,
                        long long t_hi, const int *row_off, const int *rec_x, const int *rec_id) {
    constexpr int K = kAdj5Levels;
    const bool mrt = ctx->cfg.collision == LB_MRT;
    auto fn = mrt ? adj5_kernel<true, K> : adj5_kernel<false, K>;
    const size_t smem = (size_t)2 * K * 2 * (kWS + 2) * sizeof(float);
    static int occ = 0, sms = 0;  // resident CTAs per SM, SMs (the same for both instances)
    if (!occ) {
        int dev = 0, nb = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kWS, smem);
        occ = std::max(1, nb);
    }
    constexpr int OUT = kWS - 2 * K;
    const int strips = (ctx->nx + OUT - 1) / OUT;
    const int chunks = std::max(1, occ * std::max(sms, 1) / strips);  // one wave of CTAs
    Adj5Args b;
    b.rho_hi = rho_hi;
    b.t_hi = t_hi;
    b.row_off = row_off;
    b.rec_x = rec_x;
    b.rec_id = rec_id;
    b.H = std::max(1, (ctx->ny + chunks - 1) / chunks);
    b.per = ctx->cfg.boundary == LB_PERIODIC ? 1 : 0;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid(strips, (ctx->ny + b.H - 1) / b.H);
    return launch_pdl(fn, grid, dim3(kWS), smem, ctx->stream, a, d, b);
}
