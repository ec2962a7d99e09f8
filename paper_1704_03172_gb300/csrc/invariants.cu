// invariants.cu -- FP64 reductions over the LB state: mass sum_x rho(x),
// energy sum_x sum_i g_i^2 / w_i(x) (the quantity a tau = 1/2 step conserves
// on a homogeneous periodic grid, because g^eq is the W^-1-orthogonal
// projection of g and the collision is a reflection), max |g_i|, and the
// number of non-finite values (instability detector).
//
// Two passes with a fixed summation order, so results are bit-reproducible:
// pass 1 reduces each grid row to 4 partials (one block per row, grid-stride
// over rows); pass 2 reduces the row partials in one block.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <string>

#include "lb_kernels.cuh"
#include "lb_runtime.h"

namespace lbinv {

using namespace lbk;

struct InvArgs {
    const void *pop;     // populations
    int raw;             // 1: pop holds g(t) unshifted; 0: post-collision h(t-1) (pull)
    int swap;            // in-place streaming: h(t-1)'s population i in slot opp(i)
    int periodic;
    const float *eta2;   // per-site eta^2 [ny][pitch], or nullptr when c_map is given
    const float *c_map;  // per-site c [ny][nx] (used when eta2 == nullptr)
    double inv_cref;
    int nx, ny, pitch;
    long long plane;
    const float *scale_in;  // per-population scale (16-bit storage) or nullptr
    float w1r, w5r;      // D2Q9 reference weights
};

template <int Q>
__device__ __forceinline__ double weight_d(int i, float e2, const InvArgs &a) {
    if (Q == 5) return i == 0 ? 1.0 - (double)e2 : 0.25 * (double)e2;
    if (i == 0) return 1.0 - 4.0 * (double)e2 * ((double)a.w1r + (double)a.w5r);
    return i < 5 ? (double)e2 * a.w1r : (double)e2 * a.w5r;
}

__device__ __forceinline__ void block_reduce4(double v[4], double *sm) {
    // sm: 4 * 32 doubles; fixed-order tree, so the result is reproducible
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    for (int o = 16; o > 0; o >>= 1) v[3] = fmax(v[3], __shfl_down_sync(0xffffffffu, v[3], o));
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < 4; k++) sm[k * 32 + wid] = v[k];
    __syncthreads();
    if (wid == 0) {
        for (int k = 0; k < 4; k++) v[k] = lane < nw ? sm[k * 32 + lane] : 0.0;
#pragma unroll
        for (int k = 0; k < 3; k++)
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        for (int o = 16; o > 0; o >>= 1)
            v[3] = fmax(v[3], __shfl_down_sync(0xffffffffu, v[3], o));
    }
}

// partial[row] = {sum rho, sum g^2/w, number of non-finite values, max |g|}
template <int Q, typename ST>
__global__ void __launch_bounds__(256) rows_kernel(InvArgs a, double *partial) {
    __shared__ double sm[4 * 32];
    const ST *pop = static_cast<const ST *>(a.pop);
    for (int y = blockIdx.x; y < a.ny; y += gridDim.x) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int x = threadIdx.x; x < a.nx; x += blockDim.x) {
            float e2;
            if (a.eta2) {
                e2 = a.eta2[(long long)y * a.pitch + x];
            } else {
                double eta = (double)a.c_map[(long long)y * a.nx + x] * a.inv_cref;
                e2 = (float)(eta * eta);
            }
#pragma unroll
            for (int i = 0; i < Q; i++) {
                int xs = x, ys = y;
                if (!a.raw) {
                    xs -= Lat<Q>::cx(i);
                    ys -= Lat<Q>::cy(i);
                }
                float g = 0.f;
                bool ok = true;
                if (a.periodic) {
                    xs = (xs + a.nx) % a.nx;
                    ys = (ys + a.ny) % a.ny;
                } else {
                    ok = xs >= 0 && xs < a.nx && ys >= 0 && ys < a.ny;
                }
                const int slot = a.swap ? Lat<Q>::opp(i) : i;
                if (ok) g = Store<ST>::load1(pop + slot * a.plane + (long long)ys * a.pitch + xs) *
                            (a.scale_in ? a.scale_in[i] : 1.f);
                if (!isfinite(g)) {
                    v[2] += 1.0;
                    continue;
                }
                const double gd = g;
                v[0] += gd;
                const double w = weight_d<Q>(i, e2, a);
                if (w > 0.0) v[1] += gd * gd / w;
                v[3] = fmax(v[3], fabs(gd));
            }
        }
        block_reduce4(v, sm);
        if (threadIdx.x == 0)
            for (int k = 0; k < 4; k++) partial[(long long)y * 4 + k] = v[k];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) final_kernel(const double *partial, int ny, double *out) {
    __shared__ double sm[4 * 32];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int y = threadIdx.x; y < ny; y += blockDim.x) {
        v[0] += partial[(long long)y * 4 + 0];
        v[1] += partial[(long long)y * 4 + 1];
        v[2] += partial[(long long)y * 4 + 2];
        v[3] = fmax(v[3], partial[(long long)y * 4 + 3]);
    }
    block_reduce4(v, sm);
    if (threadIdx.x == 0) {
        out[0] = v[0];  // mass
        out[1] = v[1];  // energy
        out[2] = v[3];  // max |g|
        out[3] = v[2];  // non-finite count
    }
}

using RowsFn = void (*)(InvArgs, double *);

template <typename ST> RowsFn rows_fn(int Q) {
    return Q == 9 ? rows_kernel<9, ST> : rows_kernel<5, ST>;
}

RowsFn pick_rows(int Q, int storage) {
    switch (storage) {
        case LB_BF16: return rows_fn<__nv_bfloat16>(Q);
        case LB_F16: return rows_fn<__half>(Q);
        default: return rows_fn<float>(Q);
    }
}

// Queue both passes; partial must hold 4 * ny doubles, out 4 doubles (device).
cudaError_t launch(const InvArgs &a, int Q, int storage, double *partial, double *out,
                   cudaStream_t s) {
    int grid = a.ny < 4096 ? a.ny : 4096;
    pick_rows(Q, storage)<<<grid, 256, 0, s>>>(a, partial);
    final_kernel<<<1, 256, 0, s>>>(partial, a.ny, out);
    return cudaGetLastError();
}

}  // namespace lbinv

// ---------------------------------------------------------------------------
// Allocation-free variant.  Its scratch (the per-row partials of pass 1) is this
// file-scope device array instead of memory from cudaMalloc: every GPU that
// loads the library holds it (512 KiB) until the process exits.  Host code
// must not pass the symbol itself to a kernel -- on the host it names a
// stand-in, not device memory -- so its device address is looked up once per
// device with cudaGetSymbolAddress and cached.
#define LB_NOALLOC_MAX_ROWS 16384
static __device__ __align__(256) double g_noalloc_partial[LB_NOALLOC_MAX_ROWS * 4 + 4];

namespace {
constexpr int kMaxDevices = 64;
std::atomic<double *> g_noalloc_addr[kMaxDevices];

lb_status noalloc_fail(lb_status st, const std::string &msg) {
    lbrt::fail(nullptr, st, "%s", msg.c_str());  // reported by lb_last_error(NULL)
    return st;
}
}  // namespace

extern "C" lb_status lb_invariants_noalloc(const float *g, const float *c_map, int lattice,
                                           int nx, int ny, double c_ref, const double *w_ref,
                                           double *out, void *cuda_stream) {
    if (!g || !c_map || !out) return noalloc_fail(LB_EINVAL, "g, c_map and out must be non-NULL");
    if (lattice != LB_D2Q5 && lattice != LB_D2Q9)
        return noalloc_fail(LB_EINVAL, "lattice must be LB_D2Q5 or LB_D2Q9");
    if (nx < 1 || ny < 1) return noalloc_fail(LB_EINVAL, "nx and ny must be >= 1");
    if (ny > LB_NOALLOC_MAX_ROWS)
        return noalloc_fail(LB_EINVAL, "ny = " + std::to_string(ny) + " exceeds the " +
                                           std::to_string(LB_NOALLOC_MAX_ROWS) +
                                           "-row limit of the static scratch array");
    if ((long long)nx * ny > (1LL << 31)) return noalloc_fail(LB_EINVAL, "nx * ny exceeds 2^31");
    if (!(c_ref > 0.0)) return noalloc_fail(LB_EINVAL, "c_ref must be > 0");
    if (lattice == LB_D2Q9 && !w_ref) return noalloc_fail(LB_EINVAL, "D2Q9 needs w_ref");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(LB_ECUDA, std::string("cudaGetDevice: ") +
                                                            cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(LB_EINVAL, "device ordinal too large");
    double *scratch = g_noalloc_addr[dev].load(std::memory_order_acquire);
    if (!scratch) {  // set-up: once per device, with that device current
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partial);
        if (e != cudaSuccess || !p)
            return noalloc_fail(LB_ECUDA, std::string("cudaGetSymbolAddress: ") +
                                              cudaGetErrorString(e));
        scratch = static_cast<double *>(p);
        g_noalloc_addr[dev].store(scratch, std::memory_order_release);
    }
    // An error that an earlier call left pending on this thread would otherwise be read
    // back after the launches below as if they had failed (and cleared for its owner):
    // report it as such, queue nothing, and leave it pending.
    e = cudaPeekAtLastError();
    if (e != cudaSuccess)
        return noalloc_fail(LB_ECUDA, std::string("an earlier CUDA call left an error pending "
                                                  "on this thread (not cleared): ") +
                                          cudaGetErrorString(e));
    lbinv::InvArgs a;
    memset(&a, 0, sizeof(a));
    a.pop = g;
    a.raw = 1;  // g holds the populations at their own sites
    a.periodic = 0;
    a.eta2 = nullptr;
    a.c_map = c_map;
    a.inv_cref = 1.0 / c_ref;
    a.nx = nx;
    a.ny = ny;
    a.pitch = nx;
    a.plane = (long long)nx * ny;
    a.scale_in = nullptr;
    if (lattice == LB_D2Q9) {
        a.w1r = (float)w_ref[1];
        a.w5r = (float)w_ref[2];
    }
    // every partial that pass 2 reads is written by pass 1 of the same call, so the
    // array needs no clearing between calls
    e = lbinv::launch(a, lattice, LB_F32, scratch, out, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return noalloc_fail(LB_ECUDA, std::string("launch: ") +
                                                            cudaGetErrorString(e));
    return LB_OK;
}

using namespace lbrt;

extern "C" lb_status lb_invariants(lb_ctx *ctx, double *out) {
    if (ctx && ctx->Q == 7) return fail(ctx, LB_ESTATE, "invariants are 2-D (D2Q5 / D2Q9)");
    if (ctx && ctx->cfg.storage == LB_F64)
        return fail(ctx, LB_ESTATE, "invariants read FP32 / 16-bit storage, not LB_F64");
    if (!ctx) return LB_EINVAL;
    if (!out) return fail(ctx, LB_EINVAL, "out is NULL");
    if (ctx->slab_nyg) return fail(ctx, LB_ESTATE, "invariants of a row slab (lb_set_slab)");
    if (!ctx->inv_scratch) {
        ctx->inv_scratch = static_cast<double *>(dev_alloc(ctx, ((size_t)ctx->ny * 4 + 4) * 8));
        if (!ctx->inv_scratch) return fail(ctx, LB_ENOMEM, "invariant scratch");
    }
    lbinv::InvArgs a;
    memset(&a, 0, sizeof(a));
    a.pop = ctx->pop[ctx->cur];
    a.raw = ctx->raw ? 1 : 0;
    a.swap = ctx->swap ? 1 : 0;
    a.periodic = ctx->cfg.boundary == LB_PERIODIC;
    a.eta2 = ctx->eta2;
    a.nx = ctx->nx;
    a.ny = ctx->ny;
    a.pitch = ctx->pitch;
    a.plane = (long long)ctx->ny * ctx->pitch;
    a.scale_in = current_scale(ctx);
    a.w1r = (float)ctx->cfg.w_ref[1];
    a.w5r = (float)ctx->cfg.w_ref[2];
    double *res = ctx->inv_scratch + (size_t)ctx->ny * 4;
    cudaError_t e = lbinv::launch(a, ctx->Q, ctx->cfg.storage, ctx->inv_scratch, res, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "invariants launch");
    e = cudaMemcpyAsync(out, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "invariants");
    if (out[3] > 0) return fail(ctx, LB_EUNSTABLE, "%.0f non-finite population values", out[3]);
    return LB_OK;
}
