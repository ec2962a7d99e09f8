// lbac.cu -- runtime behind the C ABI of include/lbac.h: context, device
// memory, medium preprocessing and the launch loop of the fused LB step.
//
// The method is the linear lattice-Boltzmann scheme of arXiv:1704.03172; the
// per-site arithmetic lives in lb_kernels.cuh.  Nothing here computes on the
// host except parameter validation and launch bookkeeping.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "lbac.h"
#include "lb_kernels.cuh"
#include "lb_runtime.h"

using namespace lbk;

namespace lbrt {

thread_local std::string g_create_error;

lb_status fail(lb_ctx *ctx, lb_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        g_create_error = buf;
    return st;
}

lb_status cuda_fail(lb_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, LB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void *dev_alloc(lb_ctx *ctx, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void *p = nullptr;
    if (ctx->alloc_fn) {
        p = ctx->alloc_fn(bytes, ctx->alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) ctx->allocs.push_back(p);
    return p;
}

void dev_free(lb_ctx *ctx, void *p) {
    if (!p) return;
    auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), p);
    if (it != ctx->allocs.end()) ctx->allocs.erase(it);
    if (ctx->free_fn)
        ctx->free_fn(p, ctx->alloc_user);
    else
        cudaFree(p);
}

int elem_bytes(int storage) { return storage == LB_F32 ? 4 : storage == LB_F64 ? 8 : 2; }

int round_up(int v, int m) { return (v + m - 1) / m * m; }

namespace {

// Host passes over a speed map run on several threads, each over a band of rows: about one
// thread per million sites, at most 16 (small maps stay on the calling thread, where a
// thread's start would cost more than the pass).  The results are merged in band order, so
// they do not depend on timing.
int row_bands(int nrows, int ncols) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const long long per = ((long long)nrows * ncols) >> 20;
    return (int)std::max(1u, std::min({hw, 16u, (unsigned)std::min<long long>(per, nrows / 64) + 1u}));
}

template <class F> void for_row_bands(int nrows, int ncols, F f) {
    const int T = row_bands(nrows, ncols);
    if (T == 1) {
        f(0, nrows, 0);
        return;
    }
    std::vector<std::thread> th;
    int t = 1;
    try {  // a thread that cannot start leaves its band, and the rest, to the calling thread
        for (; t < T; t++)
            th.emplace_back(f, (int)((long long)nrows * t / T),
                            (int)((long long)nrows * (t + 1) / T), t);
    } catch (...) {
    }
    f(0, (int)((long long)nrows / T), 0);
    for (int u = t; u < T; u++)
        f((int)((long long)nrows * u / T), (int)((long long)nrows * (u + 1) / T), u);
    for (auto &x : th) x.join();
}

// Open-addressed set of at most 256 float bit patterns, with their first-seen order.
struct SpeedSet {
    static constexpr unsigned kSlots = 512;  // linear probing
    uint32_t key[kSlots];
    int val[kSlots];
    bool used[kSlots] = {};
    std::vector<uint32_t> order;
    // index of b, inserting it; -1 once a 257th value would be needed
    int find_or_add(uint32_t b) {
        unsigned h = (b * 2654435761u) >> 23;
        while (used[h] && key[h] != b) h = (h + 1) & (kSlots - 1);
        if (!used[h]) {
            if (order.size() == 256) return -1;
            used[h] = true;
            key[h] = b;
            val[h] = (int)order.size();
            order.push_back(b);
        }
        return val[h];
    }
    int find(uint32_t b) const {  // b must be present
        unsigned h = (b * 2654435761u) >> 23;
        while (key[h] != b) h = (h + 1) & (kSlots - 1);
        return val[h];
    }
};

// Medium index: when the host map holds at most 256 distinct speeds, map[y][x]
// (row pitch `pitch`) indexes tab, whose entries are eta^2 formed exactly as
// medium_kernel forms them (so both forms give bit-identical steps).  Returns
// false when a 257th value appears.  Each band of rows collects its distinct values;
// the bands' lists are merged in band order, then every band writes its rows' indices.
bool medium_index(const float *c, int nx, int ny, int pitch, double inv_cref,
                  std::vector<uint8_t> &map, std::vector<float> &tab) {
    const int T = row_bands(ny, nx);
    std::vector<SpeedSet> local(T);
    std::vector<char> over(T, 0);
    for_row_bands(ny, nx, [&](int y0, int y1, int t) {
        SpeedSet &S = local[t];
        uint32_t last = 0;
        bool have = false;
        for (int y = y0; y < y1 && !over[t]; y++) {
            const float *row = c + (size_t)y * nx;
            for (int x = 0; x < nx; x++) {
                uint32_t b;
                memcpy(&b, row + x, 4);
                if (have && b == last) continue;  // runs of equal speeds skip the table
                if (S.find_or_add(b) < 0) {
                    over[t] = 1;
                    break;
                }
                last = b;
                have = true;
            }
        }
    });
    SpeedSet all;
    for (int t = 0; t < T; t++) {
        if (over[t]) return false;
        for (uint32_t b : local[t].order)
            if (all.find_or_add(b) < 0) return false;
    }
    map.assign((size_t)ny * pitch, 0);
    for_row_bands(ny, nx, [&](int y0, int y1, int) {
        uint32_t last = 0;
        int last_i = -1;
        for (int y = y0; y < y1; y++) {
            const float *row = c + (size_t)y * nx;
            uint8_t *mrow = map.data() + (size_t)y * pitch;
            for (int x = 0; x < nx; x++) {
                uint32_t b;
                memcpy(&b, row + x, 4);
                if (last_i < 0 || b != last) {
                    last = b;
                    last_i = all.find(b);
                }
                mrow[x] = (uint8_t)last_i;
            }
        }
    });
    tab.assign(256, 0.f);
    for (size_t i = 0; i < all.order.size(); i++) {
        float cv;
        memcpy(&cv, &all.order[i], 4);
        double eta = (double)cv * inv_cref;
        if (eta > 1.0) eta = 1.0;
        tab[i] = (float)(eta * eta);
    }
    return true;
}

// min and max over the positive finite speeds of a host map, and its distinct speeds while
// there are at most 8 (dv holds 9 once there are more)
void speed_range(const float *c, long long n, int nx, float &mn, float &mx, std::vector<float> &dv) {
    const int ny = (int)(n / nx);
    const int T = row_bands(ny, nx);
    std::vector<float> lmn(T, INFINITY), lmx(T, 0.f);
    std::vector<std::vector<float>> ldv(T);
    for_row_bands(ny, nx, [&](int y0, int y1, int t) {
        float a = INFINITY, b = 0.f, last = -1.f;
        std::vector<float> &d = ldv[t];
        for (long long i = (long long)y0 * nx; i < (long long)y1 * nx; i++) {
            const float v = c[i];
            if (!(v > 0.f) || !std::isfinite(v)) continue;  // refused later, with the medium
            a = std::min(a, v);
            b = std::max(b, v);
            if (v != last && d.size() <= 8 && std::find(d.begin(), d.end(), v) == d.end())
                d.push_back(v);
            last = v;
        }
        lmn[t] = a;
        lmx[t] = b;
    });
    mn = INFINITY;
    mx = 0.f;
    dv.clear();
    for (int t = 0; t < T; t++) {
        mn = std::min(mn, lmn[t]);
        mx = std::max(mx, lmx[t]);
        for (float v : ldv[t])
            if (dv.size() <= 8 && std::find(dv.begin(), dv.end(), v) == dv.end()) dv.push_back(v);
    }
}

}  // namespace

StepArgs base_args(const lb_ctx *c) {
    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.eta2 = c->eta2;
    a.mid = c->mid;
    a.mid_tab = c->mid_tab;
    a.ny3 = c->ny3;
    a.nz = c->nz;
    a.nx = c->nx;
    a.ny = c->ny;
    a.pitch = c->pitch;
    a.plane = (long long)c->ny * c->pitch;
    const int sites_per_warp = 32 * (c->cfg.storage == LB_F32 ? 4 : 8);  // 16-byte vectors
    a.segs = (c->nx + sites_per_warp - 1) / sites_per_warp;
    long long warps = (long long)a.segs * c->ny;
    a.main_blocks = (int)((warps + kWarps - 1) / kWarps);
    a.omega = (float)(1.0 / c->cfg.tau);
    for (int k = 0; k < 9; k++) a.s[k] = mrt_rate_arg(c->Q, k, c->cfg.s[k]);
    a.w1r = (float)c->cfg.w_ref[1];
    a.w5r = (float)c->cfg.w_ref[2];
    double c2r = 2.0 * c->cfg.w_ref[1] + 4.0 * c->cfg.w_ref[2];
    a.c2r = (float)c2r;
    a.a1 = c2r > 0 ? (float)(c->cfg.w_ref[1] / c2r) : 0.f;
    a.a5 = c2r > 0 ? (float)(c->cfg.w_ref[2] / c2r) : 0.f;
    a.sponge_w = c->cfg.sponge_width;
    a.sponge_smax = (float)c->cfg.sponge_sigma_max;
    a.sponge_inv_w = c->cfg.sponge_width > 0 ? 1.f / (float)c->cfg.sponge_width : 0.f;
    a.src_tab = c->src_tab;
    a.src_nt = c->src_nt;
    a.src_x = c->src_x;
    a.src_y = c->src_y;
    a.rec = c->rec;
    a.nrec = c->nrec;
    a.eta2_64 = c->eta2_64;
    a.src64 = c->src64;
    a.coef64 = c->coef64;
    a.y_off = c->slab_y0;
    a.ny_glob = c->slab_nyg;
    a.halo_lo = c->halo_lo;
    a.halo_hi = c->halo_hi;
    a.send_lo = c->send_lo;
    a.send_hi = c->send_hi;
    if (c->lp_scale) a.scale_in = c->lp_scale + c->lp_slot * 9;
    return a;
}

const float *current_scale(const lb_ctx *ctx) {
    return ctx->lp_scale ? ctx->lp_scale + ctx->lp_slot * 9 : nullptr;
}

// ------------------------------------------------------- kernel dispatch --
using SetFn = void (*)(StepArgs, const float *, int);

template <int Q, bool MRT, bool PER, typename ST> StepFn step_fn() {
    return step_kernel<Q, MRT, PER, ST>;
}

template <int Q, bool MRT, typename ST> StepFn step_fn_b(bool per) {
    return per ? step_fn<Q, MRT, true, ST>() : step_fn<Q, MRT, false, ST>();
}
template <int Q, typename ST> StepFn step_fn_c(bool mrt, bool per) {
    return mrt ? step_fn_b<Q, true, ST>(per) : step_fn_b<Q, false, ST>(per);
}
template <typename ST> StepFn step_fn_q(int Q, bool mrt, bool per) {
    if (Q == 7) return step_fn_b<7, false, ST>(per);  // D3Q7: BGK only
    return Q == 9 ? step_fn_c<9, ST>(mrt, per) : step_fn_c<5, ST>(mrt, per);
}

StepFn pick_step_for(int Q, bool mrt, bool per, int storage) {
    switch (storage) {
        case LB_BF16: return step_fn_q<__nv_bfloat16>(Q, mrt, per);
        case LB_F16: return step_fn_q<__half>(Q, mrt, per);
        default: return step_fn_q<float>(Q, mrt, per);
    }
}

// row slabs (lb_set_slab): the step with the halo-row pulls and the cut-row stores
template <int Q, typename ST> StepFn slab_fn(bool mrt, bool per) {
    if (mrt) return per ? step_kernel<Q, true, true, ST, true> : step_kernel<Q, true, false, ST, true>;
    return per ? step_kernel<Q, false, true, ST, true> : step_kernel<Q, false, false, ST, true>;
}

StepFn pick_step(const lb_ctx *c) {
    const bool mrt = c->cfg.collision == LB_MRT, per = c->cfg.boundary == LB_PERIODIC;
    if (c->slab_nyg) {
        const bool bf = c->cfg.storage == LB_BF16;
        if (c->Q == 9) return bf ? slab_fn<9, __nv_bfloat16>(mrt, per) : slab_fn<9, float>(mrt, per);
        return bf ? slab_fn<5, __nv_bfloat16>(mrt, per) : slab_fn<5, float>(mrt, per);
    }
    return pick_step_for(c->Q, mrt, per, c->cfg.storage);
}

template <int Q, typename ST> SetFn set_fn_q(bool per) {
    return per ? set_state_kernel<Q, true, ST> : set_state_kernel<Q, false, ST>;
}
template <typename ST> SetFn set_fn(int Q, bool per) {
    return Q == 9 ? set_fn_q<9, ST>(per) : Q == 7 ? set_fn_q<7, ST>(per) : set_fn_q<5, ST>(per);
}
SetFn pick_set(const lb_ctx *c) {
    bool per = c->cfg.boundary == LB_PERIODIC;
    switch (c->cfg.storage) {
        case LB_BF16: return set_fn<__nv_bfloat16>(c->Q, per);
        case LB_F16: return set_fn<__half>(c->Q, per);
        default: return set_fn<float>(c->Q, per);
    }
}
template <int Q, typename ST> GetFn get_fn_q(bool per) {
    return per ? get_state_kernel<Q, true, ST> : get_state_kernel<Q, false, ST>;
}
template <typename ST> GetFn get_fn(int Q, bool per) {
    return Q == 9 ? get_fn_q<9, ST>(per) : Q == 7 ? get_fn_q<7, ST>(per) : get_fn_q<5, ST>(per);
}
GetFn pick_get_for(int Q, bool per, int storage) {
    switch (storage) {
        case LB_BF16: return get_fn<__nv_bfloat16>(Q, per);
        case LB_F16: return get_fn<__half>(Q, per);
        default: return get_fn<float>(Q, per);
    }
}

GetFn pick_get(const lb_ctx *c) {
    return pick_get_for(c->Q, c->cfg.boundary == LB_PERIODIC, c->cfg.storage);
}

lb_status check_launch(lb_ctx *ctx, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    return LB_OK;
}

// lb_create's linear stability check (stability.cu): LB_EINVAL when the one-step map has an
// eigenvalue of modulus above 1 + 1e-12 at a checked eta on any refinement level.
lb_status stability_check(const lb_config *cfg, double eta_min, double eta_max,
                          const std::vector<double> &distinct) {
    double eta_at = 0;
    int level = 0;
    const double worst =
        stability_worst(cfg, stability_etas(eta_min, eta_max, distinct), &eta_at, &level);
    if (worst > kStableBound)
        return fail(nullptr, LB_EINVAL,
                    "linearly unstable: max |lambda(k)| of the one-step map is %.12g > 1 at "
                    "eta = %.6g%s (refinement level %d); choose other rates or weights",
                    worst, eta_at, worst > 1e299 ? " (no convergence)" : "", level);
    return LB_OK;
}

lb_status validate(const lb_config *cfg) {
    if (!cfg) return fail(nullptr, LB_EINVAL, "cfg is NULL");
    if (cfg->lattice != LB_D2Q5 && cfg->lattice != LB_D2Q9 && cfg->lattice != LB_D3Q7)
        return fail(nullptr, LB_EINVAL, "lattice must be LB_D2Q5, LB_D2Q9 or LB_D3Q7");
    const int nz = std::max(cfg->nz, 1);
    if (nz > 1 && cfg->lattice != LB_D3Q7)
        return fail(nullptr, LB_EINVAL, "nz > 1 needs the LB_D3Q7 lattice");
    if (cfg->lattice == LB_D3Q7) {
        if (cfg->collision != LB_BGK)
            return fail(nullptr, LB_EINVAL, "LB_D3Q7 supports BGK collision only");
        if (cfg->n_patches > 0 || cfg->time_block > 1)
            return fail(nullptr, LB_EINVAL, "LB_D3Q7: no refinement patch or time blocking");
    }
    if (cfg->collision != LB_BGK && cfg->collision != LB_MRT)
        return fail(nullptr, LB_EINVAL, "collision must be LB_BGK or LB_MRT");
    if (cfg->storage != LB_F32 && cfg->storage != LB_BF16 && cfg->storage != LB_F16 &&
        cfg->storage != LB_F64)
        return fail(nullptr, LB_EINVAL, "storage must be LB_F32, LB_BF16, LB_F16 or LB_F64");
    if (cfg->storage == LB_F64 && (cfg->n_patches > 0 || cfg->step_kernel == LB_STEP_STAGED))
        return fail(nullptr, LB_EINVAL, "LB_F64 (test only): no refinement patch, no staged step");
    if (cfg->boundary != LB_ZERO_GHOST && cfg->boundary != LB_PERIODIC)
        return fail(nullptr, LB_EINVAL, "boundary must be LB_ZERO_GHOST or LB_PERIODIC");
    if (cfg->nx < 1 || cfg->ny < 1 || (long long)cfg->nx * cfg->ny * nz > (1LL << 34) ||
        (long long)cfg->ny * nz > (1LL << 30))
        return fail(nullptr, LB_EINVAL, "grid %d x %d x %d out of range", cfg->nx, cfg->ny, nz);
    if (!cfg->c_map) return fail(nullptr, LB_EINVAL, "c_map is NULL");
    if (cfg->collision == LB_BGK && !(cfg->tau >= 0.5 && std::isfinite(cfg->tau)))
        return fail(nullptr, LB_EINVAL, "BGK needs tau >= 1/2 (got %g)", cfg->tau);
    if (cfg->collision == LB_MRT) {
        for (int k = 0; k < cfg->lattice; k++)
            if (!(cfg->s[k] > 0.0 && cfg->s[k] <= 2.0))
                return fail(nullptr, LB_EINVAL, "MRT rate s[%d] = %g outside (0, 2]", k, cfg->s[k]);
    }
    if (cfg->lattice == LB_D2Q9) {
        const double *w = cfg->w_ref;
        if (w[0] < 0 || w[1] < 0 || w[2] < 0 || std::fabs(w[0] + 4 * w[1] + 4 * w[2] - 1.0) > 1e-9)
            return fail(nullptr, LB_EINVAL, "D2Q9 w_ref must be >= 0 with w0 + 4 w1 + 4 w5 = 1");
        if (2 * w[1] + 4 * w[2] <= 0)
            return fail(nullptr, LB_EINVAL, "D2Q9 w_ref gives c_s = 0");
    }
    if (cfg->sponge_width < 0 || cfg->sponge_sigma_max < 0 || cfg->sponge_sigma_max > 1)
        return fail(nullptr, LB_EINVAL, "sponge_width >= 0 and sigma_max in [0, 1] required");
    if (cfg->n_patches < 0 || cfg->n_patches > LB_MAX_PATCHES ||
        (cfg->n_patches > 0 && !cfg->patches))
        return fail(nullptr, LB_EINVAL, "n_patches must be 0 .. %d (nested)", LB_MAX_PATCHES);
    if (cfg->time_block > 1) {
        if (!tb_supported(cfg->lattice, cfg->time_block))
            return fail(nullptr, LB_EINVAL, "time_block %d not supported for D2Q%d (D2Q5: 2, 4, 6, "
                        "8, 16; D2Q9: 2, 4)", cfg->time_block, cfg->lattice);
        if (cfg->n_patches > 0 || !(cfg->storage == LB_F32 ||
                                    (cfg->storage == LB_BF16 && cfg->lattice == LB_D2Q5)))
            return fail(nullptr, LB_EINVAL, "time_block needs FP32 storage (D2Q5: or BF16) and no "
                        "patch");
    }
    if (cfg->step_kernel != LB_STEP_AUTO && cfg->step_kernel != LB_STEP_DIRECT &&
        cfg->step_kernel != LB_STEP_STAGED)
        return fail(nullptr, LB_EINVAL, "step_kernel must be LB_STEP_AUTO, _DIRECT or _STAGED");
    if (cfg->streaming != LB_STREAM_AB && cfg->streaming != LB_STREAM_AA)
        return fail(nullptr, LB_EINVAL, "streaming must be LB_STREAM_AB or LB_STREAM_AA");
    if (cfg->streaming == LB_STREAM_AA &&
        (cfg->lattice == LB_D3Q7 || (cfg->storage != LB_F32 && cfg->storage != LB_BF16) ||
         cfg->n_patches > 0 || cfg->time_block > 1 ||
         (cfg->step_kernel == LB_STEP_STAGED && cfg->storage != LB_BF16)))
        return fail(nullptr, LB_EINVAL, "LB_STREAM_AA: D2Q5 or D2Q9, FP32 or BF16 storage, no "
                    "patch, no time blocking, a staged step with BF16 storage only");
    if (stability_needed(cfg) && !cfg->c_map_on_device) {
        // linear stability at the medium's eta (a device c_map is checked in lb_create, once
        // its range is known): the distinct speeds when there are at most 8, else a spread
        const long long n = (long long)cfg->nx * cfg->ny * nz;
        float mn, mx;
        std::vector<float> dv;
        speed_range(cfg->c_map, n, cfg->nx, mn, mx, dv);
        const double cref = cfg->c_ref > 0 ? cfg->c_ref : (double)mx;
        if (mx > 0.f && cref > 0) {
            std::vector<double> de;
            for (float c : dv) de.push_back(std::min(1.0, (double)c / cref));
            if (de.size() > 8) de.clear();
            lb_status st = stability_check(cfg, std::min(1.0, mn / cref), std::min(1.0, mx / cref), de);
            if (st != LB_OK) return st;
        }
    }
    return LB_OK;
}

}  // namespace lbrt

using namespace lbrt;

extern "C" {

lb_status lb_config_default(lb_config *cfg) {
    if (!cfg) return LB_EINVAL;
    memset(cfg, 0, sizeof(*cfg));
    cfg->lattice = LB_D2Q5;
    cfg->collision = LB_BGK;
    cfg->storage = LB_F32;
    cfg->boundary = LB_ZERO_GHOST;
    cfg->tau = 0.5;
    for (int k = 0; k < 9; k++) cfg->s[k] = 1.0;
    cfg->w_ref[0] = 4.0 / 9.0;
    cfg->w_ref[1] = 1.0 / 9.0;
    cfg->w_ref[2] = 1.0 / 36.0;
    cfg->time_block = 1;
    return LB_OK;
}

lb_status lb_footprint(const lb_config *cfg, int nt, int nrec, int want_adjoint, size_t *bytes) {
    if (!cfg || !bytes) return LB_EINVAL;
    size_t pitch = (size_t)round_up(std::max(cfg->nx, 1), 32);
    size_t plane = pitch * (size_t)std::max(cfg->ny, 1) * (size_t)std::max(cfg->nz, 1);
    size_t q = cfg->lattice == LB_D2Q9 ? 9 : cfg->lattice == LB_D3Q7 ? 7 : 5;
    // populations (two buffers; one in place), eta^2 and, for piecewise-constant media, the
    // medium index
    const size_t nbuf = cfg->streaming == LB_STREAM_AA ? 1 : 2;
    size_t b = nbuf * q * plane * elem_bytes(cfg->storage) + plane * 4 + plane + 1024;
    if (cfg->storage == LB_F64) b += plane * 8 + (size_t)std::max(nt, 0) * 8 + 256;
    if (nrec > 0 && nt > 0) b += (size_t)nt * nrec * 4 + (size_t)nrec * 8;
    if (nt > 0) b += (size_t)nt * 4;
    // refinement levels (refine.cu): per patch, two population buffers with a ghost ring and
    // its eta^2 plane, the interface lists and three snapshot slots, the nested patch's
    // medium and initial pressure when one follows, and the peek copies of a nested level
    for (int k = 0; cfg->patches && k < cfg->n_patches && k < LB_MAX_PATCHES; k++) {
        const size_t nxf = 2 * (size_t)std::max(cfg->patches[k].nx_c, 0) + 1;
        const size_t nyf = 2 * (size_t)std::max(cfg->patches[k].ny_c, 0) + 1;
        const size_t fplane = (nyf + 2) * (size_t)round_up((int)nxf + 2, 32);
        const size_t nI = 2 * ((size_t)cfg->patches[k].nx_c + cfg->patches[k].ny_c);
        const size_t nIf = 2 * (nxf + nyf);
        b += 2 * q * fplane * 4 + fplane * 4 + nI * 8 + nIf * 16 + 3 * nI * q * 4 + 4096;
        if (k + 1 < cfg->n_patches) b += 2 * nxf * nyf * 4;
        if (k >= 1) b += q * fplane * 4 + 2 * nI * q * 4;
        if (nrec > 0) b += (size_t)nrec * 12 + 1024;
    }
    if (want_adjoint < 0) {  // the forward rho tape, the adjoint pair, the FP64 gradient,
                             // dJ/dS and the region receiver lists
        const size_t tiles = ((size_t)std::max(cfg->nx, 1) + 31) / 32 *
                             (((size_t)std::max(cfg->ny, 1) + 31) / 32);
        b += (size_t)std::max(nt, 0) * plane * 4 + 2 * q * plane * 4 + plane * 8 +
             (size_t)std::max(nt, 0) * 8 + (tiles + 1) * 4 + (size_t)std::max(nrec, 0) * 4 * 8;
    } else if (want_adjoint) {
        // lb_adjoint: checkpoints every C steps and, in the storage type, the two replay
        // states and the sub-checkpoints; the FP32 rho tape (T planes), the FP32 adjoint
        // pair, the FP64 gradient and dJ/dS; the receiver lists of the blocked reverse
        // sweep (one offset per 32 x 32 tile or larger, up to four entries per receiver)
        const int C = want_adjoint > 1 ? want_adjoint : 200;
        const int T = adj_tape_steps(plane * 4, C);
        const size_t nsub = (size_t)((C + T - 1) / T);
        const size_t states = (nt > 0 ? ((size_t)nt + C - 1) / C : 1) + 2 + (nsub - 1);
        b += states * q * plane * elem_bytes(cfg->storage) + (size_t)T * plane * 4 +
             2 * q * plane * 4 + plane * 8 + (size_t)std::max(nt, 0) * 8;
        const size_t tiles = ((size_t)std::max(cfg->nx, 1) + 31) / 32 *
                             (((size_t)std::max(cfg->ny, 1) + 31) / 32);
        b += (tiles + 1) * 4 + (size_t)std::max(nrec, 0) * 4 * 8;
    }
    *bytes = b;
    return LB_OK;
}

lb_status lb_create(const lb_config *cfg, lb_ctx **out) {
    if (!out) return fail(nullptr, LB_EINVAL, "out is NULL");
    *out = nullptr;
    lb_status st = validate(cfg);
    if (st != LB_OK) return st;
    lb_ctx *c = new (std::nothrow) lb_ctx();
    if (!c) return fail(nullptr, LB_ENOMEM, "host allocation failed");
    c->cfg = *cfg;
    c->cfg.c_map = nullptr;
    c->cfg.patches = nullptr;
    c->Q = cfg->lattice;
    c->nx = cfg->nx;
    c->nz = std::max(cfg->nz, 1);
    c->ny3 = cfg->ny;
    c->ny = cfg->ny * c->nz;  // rows of all z-planes
    c->pitch = round_up(cfg->nx, 32);
    c->ebytes = elem_bytes(cfg->storage);
    c->alloc_fn = cfg->dev_alloc;
    c->free_fn = cfg->dev_free;
    c->alloc_user = cfg->alloc_user;
    if (cfg->cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return cuda_fail(nullptr, e, "cudaStreamCreate");
        }
        c->own_stream = true;
    }
    auto bail = [&](lb_status s) {
        std::string msg = c->err;
        lb_destroy(c);
        if (!msg.empty()) g_create_error = msg;
        return s;
    };
    const size_t plane = (size_t)c->ny * c->pitch;
    c->aa = cfg->streaming == LB_STREAM_AA;
    for (int b = 0; b < (c->aa ? 1 : 2); b++) {
        c->pop[b] = dev_alloc(c, (size_t)c->Q * plane * c->ebytes);
        if (!c->pop[b]) return bail(fail(c, LB_ENOMEM, "population buffer (%zu bytes)",
                                         (size_t)c->Q * plane * c->ebytes));
        cudaError_t e = cudaMemsetAsync(c->pop[b], 0, (size_t)c->Q * plane * c->ebytes, c->stream);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemsetAsync"));
    }
    if (c->aa) {  // one buffer, holding g(t) at its own site (zero) until the first step
        c->pop[1] = c->pop[0];
        c->raw = true;
    }
    c->eta2 = static_cast<float *>(dev_alloc(c, plane * 4));
    unsigned *flags = static_cast<unsigned *>(dev_alloc(c, 256));
    c->fault = static_cast<unsigned *>(dev_alloc(c, 256));
    if (!c->eta2 || !flags || !c->fault) return bail(fail(c, LB_ENOMEM, "medium buffer"));
    cudaMemsetAsync(c->fault, 0, 4, c->stream);
    // 16-bit storage: the TMA-staged persistent step (faster there); FP32: register-streaming
    // TMA-staged persistent step: forced, or automatic for 16-bit storage on rows of at least
    // 1024 sites (a task is one row segment of 2048 16-bit sites: narrower rows idle most
    // threads, and for FP32 the register-streaming step is faster)
    // (in place: BF16 only, the form the staged kernel has)
    c->staged = cfg->n_patches == 0 && (!c->aa || cfg->storage == LB_BF16) &&
                (cfg->step_kernel == LB_STEP_STAGED ||
                 (cfg->step_kernel == LB_STEP_AUTO && (cfg->storage == LB_BF16 ||
                                                       cfg->storage == LB_F16) && cfg->nx >= 1024));
    if (cfg->storage == LB_F16) {  // FP16 range scales (BF16 has FP32's range and needs none)
        c->lp_scale = static_cast<float *>(dev_alloc(c, 3 * 9 * sizeof(float)));
        c->lp_max = static_cast<unsigned *>(dev_alloc(c, (3 * 9 * kMaxCopies + 1) * sizeof(unsigned)));
        if (!c->lp_scale || !c->lp_max) return bail(fail(c, LB_ENOMEM, "scale buffers"));
        std::vector<float> ones(27, 1.f);
        cudaMemcpyAsync(c->lp_scale, ones.data(), 27 * sizeof(float), cudaMemcpyHostToDevice,
                        c->stream);
        cudaMemsetAsync(c->lp_max, 0, (3 * 9 * kMaxCopies + 1) * sizeof(unsigned), c->stream);
    }
    // medium: c_map -> eta^2 (Eq. 0th lattice weight), on the device
    const float *cmap_dev = cfg->c_map;
    float *staging = nullptr;
    double cref = cfg->c_ref;
    if (!cfg->c_map_on_device) {
        if (!(cref > 0)) {
            std::vector<float> bmx(row_bands(c->ny, c->nx), 0.f);
            for_row_bands(c->ny, c->nx, [&](int y0, int y1, int t) {
                float m = 0.f;
                for (long long i = (long long)y0 * c->nx; i < (long long)y1 * c->nx; i++)
                    m = std::max(m, cfg->c_map[i]);
                bmx[t] = m;
            });
            float mx = 0.f;
            for (float m : bmx) mx = std::max(mx, m);
            cref = mx;
        }
        staging = static_cast<float *>(dev_alloc(c, (size_t)c->nx * c->ny * 4));
        if (!staging) return bail(fail(c, LB_ENOMEM, "c_map staging"));
        cudaError_t e = cudaMemcpyAsync(staging, cfg->c_map, (size_t)c->nx * c->ny * 4,
                                        cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "c_map upload"));
        cmap_dev = staging;
    } else if (!(cref > 0)) {
        return bail(fail(c, LB_EINVAL, "c_ref must be given when c_map is on the device"));
    }
    c->cfg.c_ref = cref;
    const unsigned flags0[3] = {0u, 0x7f800000u, 0u};  // fault bits, min and max eta^2 (bits)
    cudaMemcpyAsync(flags, flags0, sizeof(flags0), cudaMemcpyHostToDevice, c->stream);
    {
        long long total = (long long)c->ny * c->pitch;
        int blocks = (int)((total + 255) / 256);
        medium_kernel<<<blocks, 256, 0, c->stream>>>(cmap_dev, c->eta2, c->nx, c->ny, c->pitch,
                                                      1.0 / cref, flags);
        if ((st = check_launch(c, "medium_kernel")) != LB_OK) return bail(st);
    }
    unsigned hf[3] = {0u, 0u, 0u};
    cudaError_t e = cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "medium setup"));
    dev_free(c, flags);
    if (hf[0] & 1u) return bail(fail(c, LB_EINVAL, "c_map must be finite and > 0"));
    if (hf[0] & 2u) return bail(fail(c, LB_EINVAL, "c_map exceeds c_ref (eta > 1)"));
    if (stability_needed(cfg) && cfg->c_map_on_device) {  // checked over the medium's range
        float e2min, e2max;
        memcpy(&e2min, &hf[1], 4);
        memcpy(&e2max, &hf[2], 4);
        if ((st = stability_check(cfg, std::sqrt((double)e2min), std::sqrt((double)e2max), {})) !=
            LB_OK) {
            c->err = g_create_error;
            return bail(st);
        }
    }
    if (cfg->storage == LB_F64) {
        if ((st = f64_setup(c, cmap_dev, cref)) != LB_OK) return bail(st);
    } else if (!cfg->c_map_on_device) {  // piecewise-constant media: 1-byte medium index
        std::vector<uint8_t> map;
        std::vector<float> tab;
        if (medium_index(cfg->c_map, c->nx, c->ny, c->pitch, 1.0 / cref, map, tab)) {
            c->mid = static_cast<uint8_t *>(dev_alloc(c, map.size()));
            c->mid_tab = static_cast<float *>(dev_alloc(c, 256 * sizeof(float)));
            if (!c->mid || !c->mid_tab) return bail(fail(c, LB_ENOMEM, "medium index"));
            cudaMemcpyAsync(c->mid, map.data(), map.size(), cudaMemcpyHostToDevice, c->stream);
            cudaMemcpyAsync(c->mid_tab, tab.data(), 256 * sizeof(float), cudaMemcpyHostToDevice,
                            c->stream);
            e = cudaStreamSynchronize(c->stream);  // the host vectors go out of scope
            if (e != cudaSuccess) return bail(cuda_fail(c, e, "medium index upload"));
            int n = 0;
            for (size_t i = 0; i < 256; i++) n += tab[i] > 0.f;
            c->n_mid = n;
        }
    }
    if (cfg->n_patches > 0) {
        if ((st = refine_setup(c, cfg, cmap_dev)) != LB_OK) return bail(st);
    }
    if (staging) dev_free(c, staging);
    *out = c;
    return LB_OK;
}

lb_status lb_destroy(lb_ctx *ctx) {
    if (!ctx) return LB_EINVAL;
    cudaStreamSynchronize(ctx->stream);
    for (cudaEvent_t &e : ctx->slab_ev)
        if (e) cudaEventDestroy(e);
    refine_destroy(ctx);
    std::vector<void *> all = ctx->allocs;
    for (void *p : all) dev_free(ctx, p);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return LB_OK;
}

static lb_status set_source_row(lb_ctx *ctx, int x, int y, const double *wavelet, int nt);

lb_status lb_set_source(lb_ctx *ctx, int x, int y, const double *wavelet, int nt) {
    if (!ctx) return LB_EINVAL;
    if (ctx->nz > 1) return fail(ctx, LB_EINVAL, "3-D context: use lb_set_source_3d");
    return set_source_row(ctx, x, y, wavelet, nt);
}

lb_status lb_set_source_3d(lb_ctx *ctx, int x, int y, int z, const double *wavelet, int nt) {
    if (!ctx) return LB_EINVAL;
    if (nt > 0 && (y < 0 || y >= ctx->ny3 || z < 0 || z >= ctx->nz))
        return fail(ctx, LB_EINVAL, "source (%d, %d, %d) outside the grid", x, y, z);
    return set_source_row(ctx, x, z * ctx->ny3 + y, wavelet, nt);
}

// y: row index (z ny3 + y for 3-D grids)
static lb_status set_source_row(lb_ctx *ctx, int x, int y, const double *wavelet, int nt) {
    if (nt < 0 || (nt > 0 && !wavelet)) return fail(ctx, LB_EINVAL, "bad wavelet");
    if (nt > 0 && (x < 0 || x >= ctx->nx || y < 0 || y >= ctx->ny))
        return fail(ctx, LB_EINVAL, "source (%d, %d) outside the grid", x, y);
    if (nt > 0 && ctx->refined && refine_contains(ctx, x, y))
        return fail(ctx, LB_EINVAL, "the source must lie outside the refined patch");
    cudaStreamSynchronize(ctx->stream);
    if (ctx->src_tab) dev_free(ctx, ctx->src_tab);
    ctx->src_tab = nullptr;
    ctx->src_nt = 0;
    if (ctx->cfg.storage == LB_F64) {
        lb_status st = f64_set_source(ctx, wavelet, nt);
        if (st != LB_OK) return st;
    }
    if (nt == 0) return LB_OK;
    std::vector<float> tab(wavelet, wavelet + nt);
    ctx->src_tab = static_cast<float *>(dev_alloc(ctx, (size_t)nt * 4));
    if (!ctx->src_tab) return fail(ctx, LB_ENOMEM, "source table");
    cudaError_t e = cudaMemcpyAsync(ctx->src_tab, tab.data(), (size_t)nt * 4,
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "source upload");
    ctx->src_nt = nt;
    ctx->src_x = x;
    ctx->src_y = y;
    return LB_OK;
}

static lb_status set_receivers_rows(lb_ctx *ctx, const int *xy, int nrec, int nt_capacity);

lb_status lb_set_receivers(lb_ctx *ctx, const int *xy, int nrec, int nt_capacity) {
    if (!ctx) return LB_EINVAL;
    if (ctx->nz > 1) return fail(ctx, LB_EINVAL, "3-D context: use lb_set_receivers_3d");
    return set_receivers_rows(ctx, xy, nrec, nt_capacity);
}

lb_status lb_set_receivers_3d(lb_ctx *ctx, const int *xyz, int nrec, int nt_capacity) {
    if (!ctx) return LB_EINVAL;
    if (nrec < 0 || (nrec > 0 && !xyz)) return fail(ctx, LB_EINVAL, "bad receiver arguments");
    std::vector<int> xy(2 * (size_t)std::max(nrec, 0));
    for (int r = 0; r < nrec; r++) {
        const int x = xyz[3 * r], y = xyz[3 * r + 1], z = xyz[3 * r + 2];
        if (y < 0 || y >= ctx->ny3 || z < 0 || z >= ctx->nz)
            return fail(ctx, LB_EINVAL, "receiver %d (%d, %d, %d) outside the grid", r, x, y, z);
        xy[2 * r] = x;
        xy[2 * r + 1] = z * ctx->ny3 + y;
    }
    return set_receivers_rows(ctx, xy.data(), nrec, nt_capacity);
}

// xy[r] = (x, row), row = z ny3 + y for 3-D grids
static lb_status set_receivers_rows(lb_ctx *ctx, const int *xy, int nrec, int nt_capacity) {
    if (nrec < 0 || (nrec > 0 && (!xy || nt_capacity < 0)))
        return fail(ctx, LB_EINVAL, "bad receiver arguments");
    for (int r = 0; r < nrec; r++)
        if (xy[2 * r] < 0 || xy[2 * r] >= ctx->nx || xy[2 * r + 1] < 0 || xy[2 * r + 1] >= ctx->ny)
            return fail(ctx, LB_EINVAL, "receiver %d (%d, %d) outside the grid", r, xy[2 * r],
                        xy[2 * r + 1]);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->rec) dev_free(ctx, ctx->rec);
    if (ctx->trace) dev_free(ctx, ctx->trace);
    ctx->rec = nullptr;
    ctx->trace = nullptr;
    ctx->nrec = 0;
    ctx->rec_xy.clear();
    ctx->trace_cap = 0;
    ctx->t_rec0 = ctx->t;
    if (nrec == 0) return LB_OK;
    ctx->rec = static_cast<int2 *>(dev_alloc(ctx, (size_t)nrec * 8));
    ctx->trace = static_cast<float *>(dev_alloc(ctx, (size_t)std::max(nt_capacity, 1) * nrec * 4));
    if (!ctx->rec || !ctx->trace) return fail(ctx, LB_ENOMEM, "receiver buffers");
    cudaError_t e = cudaMemcpyAsync(ctx->rec, xy, (size_t)nrec * 8, cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctx->trace, 0, (size_t)std::max(nt_capacity, 1) * nrec * 4,
                            ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "receiver upload");
    ctx->nrec = nrec;
    ctx->rec_xy.assign(xy, xy + 2 * (size_t)nrec);
    ctx->trace_cap = nt_capacity;
    if (ctx->refined) return refine_set_receivers(ctx, xy, nrec);
    if (ctx->aa) return tb5_set_receivers(ctx, xy, nrec);  // rows of receivers, x ascending
    if (ctx->cfg.time_block > 1) return tb_set_receivers(ctx, xy, nrec);
    return LB_OK;
}

static lb_status upload_f32(lb_ctx *ctx, const float *src, size_t n, int on_device,
                            const float **dev, float **tmp) {
    *tmp = nullptr;
    if (!src) {
        *dev = nullptr;
        return LB_OK;
    }
    if (on_device) {
        *dev = src;
        return LB_OK;
    }
    *tmp = static_cast<float *>(dev_alloc(ctx, n * 4));
    if (!*tmp) return fail(ctx, LB_ENOMEM, "staging buffer");
    cudaError_t e = cudaMemcpyAsync(*tmp, src, n * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upload");
    *dev = *tmp;
    return LB_OK;
}

static lb_status set_state_common(lb_ctx *ctx, const float *src, int on_device, int mode) {
    if (ctx->cfg.storage == LB_F64) return f64_set(ctx, src, nullptr, on_device, mode);
    size_t n = (size_t)ctx->nx * ctx->ny * (mode == 0 ? 1 : ctx->Q);
    const float *dev = nullptr;
    float *tmp = nullptr;
    lb_status st = upload_f32(ctx, src, n, on_device, &dev, &tmp);
    if (st != LB_OK) return st;
    StepArgs a = base_args(ctx);
    a.out = ctx->pop[ctx->cur];
    ctx->raw = true;
    if (ctx->lp_scale) {
        // FP16: the written state's scale from its own max (slot s0), and the scale
        // the first step will write with (slot s1), whose max slot starts cleared
        const int s0 = ctx->lp_slot, s1 = (s0 + 1) % 3;
        cudaMemsetAsync(ctx->lp_max, 0, (3 * 9 * kMaxCopies + 1) * sizeof(unsigned), ctx->stream);
        a.t = ctx->t;
        a.max_out = ctx->lp_max + s0 * 9 * kMaxCopies;
        a.scale_next = ctx->lp_scale + s0 * 9;
        a.max_next = ctx->lp_max + s1 * 9 * kMaxCopies;
        if (dev) {
            if (ctx->Q == 9)
                source_max_kernel<9><<<1024, 256, 0, ctx->stream>>>(a, dev, mode);
            else if (ctx->Q == 7)
                source_max_kernel<7><<<1024, 256, 0, ctx->stream>>>(a, dev, mode);
            else
                source_max_kernel<5><<<1024, 256, 0, ctx->stream>>>(a, dev, mode);
        }
        init_scale_kernel<<<1, 32, 0, ctx->stream>>>(a, ctx->Q, ctx->lp_scale + s1 * 9);
        a.scale_out = ctx->lp_scale + s0 * 9;  // set_state_kernel writes with it
    }
    long long total = (long long)ctx->ny * ctx->pitch;
    pick_set(ctx)<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(a, dev, mode);
    ctx->swap = false;
    st = check_launch(ctx, "set_state_kernel");
    if (st == LB_OK && ctx->refined) st = refine_after_set_state(ctx, dev);
    if (tmp) {
        cudaStreamSynchronize(ctx->stream);
        dev_free(ctx, tmp);
    }
    return st;
}

lb_status lb_init_pressure(lb_ctx *ctx, const float *p0, int on_device) {
    if (!ctx) return LB_EINVAL;
    ctx->t = 0;
    ctx->t_rec0 = 0;
    ctx->fine_ready = false;
    ckpt_reset(ctx);
    tape_reset(ctx);
    return set_state_common(ctx, p0, on_device, 0);
}

lb_status lb_set_state(lb_ctx *ctx, const float *in, int on_device) {
    if (!ctx) return LB_EINVAL;
    if (!in) return fail(ctx, LB_EINVAL, "state is NULL");
    if (ctx->refined) return fail(ctx, LB_ESTATE, "lb_set_state is not available with a patch");
    ckpt_reset(ctx);  // checkpoints describe one trajectory; a new state starts another
    tape_reset(ctx);
    return set_state_common(ctx, in, on_device, 1);
}

static lb_status get_common(lb_ctx *ctx, float *out, int on_device, int mode) {
    if (!out) return fail(ctx, LB_EINVAL, "out is NULL");
    if (ctx->cfg.storage == LB_F64) return f64_get(ctx, out, nullptr, on_device, mode);
    size_t n = (size_t)ctx->nx * ctx->ny * (mode == 0 ? 1 : ctx->Q);
    float *dst = out;
    if (!on_device) {
        dst = static_cast<float *>(dev_alloc(ctx, n * 4));
        if (!dst) return fail(ctx, LB_ENOMEM, "staging buffer");
    }
    StepArgs a = base_args(ctx);
    a.in = ctx->pop[ctx->cur];
    a.raw = ctx->raw ? 1 : 0;
    a.swap = ctx->swap ? 1 : 0;
    long long total = (long long)ctx->ny * ctx->nx;
    pick_get(ctx)<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(a, dst, mode);
    lb_status st = check_launch(ctx, "get_state_kernel");
    if (st == LB_OK && mode == 0 && ctx->refined) st = refine_overlay_pressure(ctx, dst);
    cudaError_t e = cudaSuccess;
    if (st == LB_OK && !on_device)
        e = cudaMemcpyAsync(out, dst, n * 4, cudaMemcpyDeviceToHost, ctx->stream);
    cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
    if (!on_device) dev_free(ctx, dst);
    if (st != LB_OK) return st;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "download");
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "stream");
    return LB_OK;
}

lb_status lb_get_pressure(lb_ctx *ctx, float *out, int on_device) {
    if (!ctx) return LB_EINVAL;
    return get_common(ctx, out, on_device, 0);
}

lb_status lb_get_state(lb_ctx *ctx, float *out, int on_device) {
    if (!ctx) return LB_EINVAL;
    if (ctx->refined) return fail(ctx, LB_ESTATE, "lb_get_state is not available with a patch");
    return get_common(ctx, out, on_device, 1);
}

}  // extern "C"

namespace lbrt {

// Arguments of the next uniform-grid step (h^{t-1} in pop[cur] -> h^t in
// pop[cur ^ 1]); advances the context's bookkeeping as if the step ran.
StepArgs prepare_step(lb_ctx *ctx) {
    StepArgs a = base_args(ctx);
    a.in = ctx->pop[ctx->cur];
    a.out = ctx->pop[ctx->cur ^ 1];
    a.t = ctx->t;
    a.raw = ctx->raw ? 1 : 0;
    ctx->raw = false;
    a.rho_out = tape_row(ctx, ctx->t);  // forward rho tape for lb_adjoint, if recording
    a.rho_stride = (long long)ctx->ny * ctx->pitch;
    long long row = ctx->t - ctx->t_rec0;
    a.trace_row = (ctx->trace && row >= 0 && row < ctx->trace_cap) ? ctx->trace + row * ctx->nrec
                                                                  : nullptr;
    ctx->cur ^= 1;
    ctx->t += 1;
    return a;
}

// One uniform-grid step: state h^{t-1} in pop[cur] -> h^t in pop[cur ^ 1].
lb_status launch_step(lb_ctx *ctx, StepFn fn, StepArgs &a) {
    a.in = ctx->pop[ctx->cur];
    a.out = ctx->pop[ctx->cur ^ 1];
    a.t = ctx->t;
    if (ctx->lp_scale) {
        const int s0 = ctx->lp_slot, s1 = (s0 + 1) % 3, s2 = (s0 + 2) % 3;
        a.scale_in = ctx->lp_scale + s0 * 9;
        a.scale_out = ctx->lp_scale + s1 * 9;
        a.max_out = ctx->lp_max + s1 * 9 * kMaxCopies;
        a.scale_next = ctx->lp_scale + s2 * 9;
        a.max_next = ctx->lp_max + s2 * 9 * kMaxCopies;
        ctx->lp_slot = s1;
    }
    a.raw = ctx->raw ? 1 : 0;
    ctx->raw = false;
    a.rho_out = tape_row(ctx, ctx->t);  // forward rho tape for lb_adjoint, if recording
    a.rho_stride = (long long)ctx->ny * ctx->pitch;
    long long row = ctx->t - ctx->t_rec0;
    a.trace_row = (ctx->trace && row >= 0 && row < ctx->trace_cap) ? ctx->trace + row * ctx->nrec
                                                                  : nullptr;
    int rec_blocks = a.trace_row ? (ctx->nrec + kThreads - 1) / kThreads : 0;
    if (ctx->staged) {
        lb_status st = stream_launch(ctx, a, rec_blocks);
        if (st != LB_OK) return st;
    } else {  // programmatic dependent launch: the step waits for the grid before it
        cudaError_t e = launch_pdl(fn, dim3(a.main_blocks + rec_blocks), dim3(kThreads), 0,
                                   ctx->stream, a);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "step launch");
    }
    if (ctx->lp_scale) {
        cudaError_t e = launch_pdl(scale_update_kernel, dim3(1), dim3(32), 0, ctx->stream, a, ctx->Q);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "scale update launch");
    }
    ctx->cur ^= 1;
    ctx->t += 1;
    return LB_OK;
}

}  // namespace lbrt

extern "C" {

static lb_status step_n(lb_ctx *ctx, int n);

// lb_watch_stability's check: the FP64 invariants of the current state (lb_invariants
// reports non-finite values as LB_EUNSTABLE), then the energy against the last check's
static lb_status watch_check(lb_ctx *ctx) {
    double v[4];
    lb_status st = lb_invariants(ctx, v);
    if (st != LB_OK) return st;
    if (ctx->watch_growth > 0 && ctx->watch_energy > 0 &&
        v[1] > ctx->watch_growth * ctx->watch_energy)
        return fail(ctx, LB_EUNSTABLE, "energy grew by a factor %.6g in %d steps (bound %.6g) "
                    "at time %lld", v[1] / ctx->watch_energy, ctx->watch_every,
                    ctx->watch_growth, ctx->t);
    ctx->watch_energy = v[1];
    return LB_OK;
}

lb_status lb_watch_stability(lb_ctx *ctx, int every, double max_growth) {
    if (!ctx) return LB_EINVAL;
    if (every < 0 || max_growth < 0 || !std::isfinite(max_growth))
        return fail(ctx, LB_EINVAL, "every >= 0 and a finite max_growth >= 0 required");
    if (every > 0 && (ctx->Q == 7 || ctx->cfg.storage == LB_F64))
        return fail(ctx, LB_ESTATE, "the watch reads the 2-D FP32 / 16-bit invariants");
    ctx->watch_every = every;
    ctx->watch_growth = max_growth;
    ctx->watch_energy = -1;
    ctx->watch_t0 = ctx->t;
    return LB_OK;
}

lb_status lb_step(lb_ctx *ctx, int n) {
    if (!ctx) return LB_EINVAL;
    if (n < 0) return fail(ctx, LB_EINVAL, "n < 0");
    if (ctx->watch_every <= 0) return step_n(ctx, n);
    while (n > 0) {  // steps in chunks that end on the watch's check times
        const int every = ctx->watch_every;
        const long long since = (ctx->t - ctx->watch_t0) % every;
        const int chunk = (int)std::min<long long>(n, every - since);
        lb_status st = step_n(ctx, chunk);
        if (st != LB_OK) return st;
        n -= chunk;
        if ((ctx->t - ctx->watch_t0) % every == 0 && (st = watch_check(ctx)) != LB_OK) return st;
    }
    return LB_OK;
}

static lb_status step_n(lb_ctx *ctx, int n) {
    if (ctx->refined) return refine_step(ctx, n);
    if (ctx->cfg.storage == LB_F64) return f64_step(ctx, n);
    if (ctx->aa) {
        lb_status st = aa_step(ctx, n);
        return st != LB_OK ? st : check_launch(ctx, "aa_step_kernel");
    }
    StepFn fn = pick_step(ctx);
    StepArgs a = base_args(ctx);
    const int K = ctx->cfg.time_block;
    for (int k = 0; k < n;) {
        if (ctx->ckpt_every > 0) {
            lb_status st = ckpt_maybe_save(ctx);
            if (st != LB_OK) return st;
        }
        if (K > 1 && n - k >= K && !ctx->raw) {
            // K fused steps, unless they would straddle a checkpoint time or the end
            // of the trace capacity; then single steps keep both exact
            const long long row = ctx->t - ctx->t_rec0;
            const bool straddle_ckpt =
                ctx->ckpt_every > 0 && (ctx->t - ctx->ckpt_t0) % ctx->ckpt_every + K > ctx->ckpt_every;
            const bool straddle_trace =
                ctx->trace && row < ctx->trace_cap && row + K > ctx->trace_cap;
            const long long trow = ctx->t - ctx->tape_t0;
            // the time-blocked kernel records the rho tape for FP32 storage only
            const bool straddle_tape =
                ctx->rho_tape && trow < ctx->tape_cap &&
                (trow + K > ctx->tape_cap || ctx->cfg.storage != LB_F32);
            if (!straddle_ckpt && !straddle_trace && !straddle_tape) {
                lb_status st = tb_launch(ctx, K);
                if (st != LB_OK) return st;
                k += K;
                continue;
            }
        }
        lb_status st = launch_step(ctx, fn, a);
        if (st != LB_OK) return st;
        k += 1;
    }
    return check_launch(ctx, "step_kernel");
}

lb_status lb_record_receivers(lb_ctx *ctx, float *out, int nt_max, int *nt_out, int on_device) {
    if (!ctx) return LB_EINVAL;
    long long rows = std::min<long long>(ctx->t - ctx->t_rec0, ctx->trace_cap);
    rows = std::max<long long>(0, std::min<long long>(rows, nt_max));
    if (nt_out) *nt_out = (int)rows;
    cudaError_t e = cudaSuccess;
    if (rows > 0 && ctx->nrec > 0) {
        if (!out) return fail(ctx, LB_EINVAL, "out is NULL");
        e = cudaMemcpyAsync(out, ctx->trace, (size_t)rows * ctx->nrec * 4,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            ctx->stream);
    }
    cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "trace download");
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "stream");
    return LB_OK;
}

lb_status lb_get_time(const lb_ctx *ctx, long long *t) {
    if (!ctx || !t) return LB_EINVAL;
    *t = ctx->t;
    return LB_OK;
}

lb_status lb_sync(lb_ctx *ctx) {
    if (!ctx) return LB_EINVAL;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device");
    unsigned fault = 0;
    e = cudaMemcpy(&fault, ctx->fault, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fault flag");
    if (fault) {  // reported once: the flag is cleared for what follows
        e = cudaMemset(ctx->fault, 0, 4);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "fault flag");
        return fail(ctx, LB_ETIMEOUT, "a bounded wait in a kernel gave up");
    }
    return LB_OK;
}

lb_status lb_info(const lb_ctx *ctx, double *info, int n_info) {
    if (!ctx || !info) return LB_EINVAL;
    double v[6];
    v[0] = ctx->Q;
    v[1] = ctx->pitch;
    v[2] = ctx->ebytes;
    double cs_ref = ctx->Q == 7 ? std::sqrt(1.0 / 3.0) : ctx->Q == 5 ? std::sqrt(0.5)
                                : std::sqrt(2 * ctx->cfg.w_ref[1] + 4 * ctx->cfg.w_ref[2]);
    v[3] = (ctx->cfg.dx > 0 && ctx->cfg.c_ref > 0) ? ctx->cfg.dx * cs_ref / ctx->cfg.c_ref : 0.0;
    v[4] = ctx->n_mid;
    v[5] = ctx->staged ? 1.0 : 0.0;
    for (int k = 0; k < n_info && k < 6; k++) info[k] = v[k];
    return LB_OK;
}

const char *lb_last_error(const lb_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

// ------------------------------------------------------ row-slab decomposition --
lb_status lb_set_slab(lb_ctx *ctx, int y_offset, int ny_global, void *send_lo, void *send_hi,
                      const void *recv_lo, const void *recv_hi) {
    if (!ctx) return LB_EINVAL;
    if (ctx->nz > 1 || ctx->refined || ctx->cfg.time_block > 1 || ctx->aa ||
        (ctx->cfg.storage != LB_F32 && ctx->cfg.storage != LB_BF16))
        return fail(ctx, LB_ESTATE, "slabs are 2-D, FP32 or BF16, without patch, time blocking or "
                    "in-place streaming");
    if (y_offset < 0 || ny_global < ctx->ny || y_offset + ctx->ny > ny_global)
        return fail(ctx, LB_EINVAL, "slab rows [%d, %d) outside a grid of %d rows", y_offset,
                    y_offset + ctx->ny, ny_global);
    for (const void *p : {(const void *)send_lo, (const void *)send_hi, recv_lo, recv_hi})
        if (p && (reinterpret_cast<uintptr_t>(p) & 15u))
            return fail(ctx, LB_EINVAL, "slab row buffers must be 16-byte aligned");
    if (ctx->rho_tape || ctx->ckpt_every > 0)
        return fail(ctx, LB_ESTATE, "a slab has no adjoint (checkpoints or rho tape)");
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream");
    for (cudaEvent_t &ev : ctx->slab_ev)
        if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(ctx, e, "slab events");
    ctx->slab_y0 = y_offset;
    ctx->slab_nyg = ny_global;
    ctx->send_lo = send_lo;
    ctx->send_hi = send_hi;
    ctx->halo_lo = recv_lo;
    ctx->halo_hi = recv_hi;
    ctx->staged = false;  // the register-streaming step reads the halo rows
    return LB_OK;
}

lb_status lb_slab_halo_bytes(const lb_ctx *ctx, size_t *bytes) {
    if (!ctx || !bytes) return LB_EINVAL;
    const int nc = ctx->Q == 9 ? cross_count<9>() : cross_count<5>();
    *bytes = (size_t)nc * ctx->pitch * ctx->ebytes;
    return LB_OK;
}

// Copy the cut rows of slab k into the halo rows of its neighbours, each copy on the
// receiving slab's stream after that slab's step and before its next one; the sending slab
// waits for the copies before its next step overwrites its cut rows.
static lb_status slab_exchange(lb_ctx **s, int n, int periodic) {
    for (int k = 0; k < n; k++) {
        cudaError_t e = cudaEventRecord(s[k]->slab_ev[0], s[k]->stream);
        if (e != cudaSuccess) return cuda_fail(s[k], e, "slab event");
    }
    size_t bytes = 0;
    lb_slab_halo_bytes(s[0], &bytes);
    for (int k = 0; k < n; k++) {  // slab k receives from k - 1 (below) and k + 1 (above)
        const int lo = k > 0 ? k - 1 : (periodic ? n - 1 : -1);
        const int hi = k + 1 < n ? k + 1 : (periodic ? 0 : -1);
        for (int side = 0; side < 2; side++) {
            const int src = side == 0 ? lo : hi;
            void *dst = const_cast<void *>(side == 0 ? s[k]->halo_lo : s[k]->halo_hi);
            const void *from = src < 0 ? nullptr : (side == 0 ? s[src]->send_hi : s[src]->send_lo);
            if (src < 0 || !dst || !from) continue;
            cudaError_t e = cudaStreamWaitEvent(s[k]->stream, s[src]->slab_ev[0], 0);
            if (e == cudaSuccess) {
                int d_dst = 0, d_src = 0;
                cudaPointerAttributes at;
                if (cudaPointerGetAttributes(&at, dst) == cudaSuccess) d_dst = at.device;
                if (cudaPointerGetAttributes(&at, from) == cudaSuccess) d_src = at.device;
                e = d_dst == d_src ? cudaMemcpyAsync(dst, from, bytes, cudaMemcpyDeviceToDevice,
                                                     s[k]->stream)
                                   : cudaMemcpyPeerAsync(dst, d_dst, from, d_src, bytes, s[k]->stream);
            }
            if (e != cudaSuccess) return cuda_fail(s[k], e, "slab halo copy");
        }
        cudaError_t e = cudaEventRecord(s[k]->slab_ev[1], s[k]->stream);
        if (e != cudaSuccess) return cuda_fail(s[k], e, "slab event");
    }
    for (int k = 0; k < n; k++) {  // the senders wait for the copies that read their rows
        for (int d = -1; d <= 1; d += 2) {
            int j = k + d;
            if (periodic) j = (j + n) % n;
            if (j < 0 || j >= n || j == k) continue;
            cudaError_t e = cudaStreamWaitEvent(s[k]->stream, s[j]->slab_ev[1], 0);
            if (e != cudaSuccess) return cuda_fail(s[k], e, "slab event wait");
        }
    }
    return LB_OK;
}

lb_status lb_slab_step(lb_ctx **slabs, int n, int steps) {
    if (!slabs || n < 1 || steps < 0) return LB_EINVAL;
    for (int k = 0; k < n; k++) {
        if (!slabs[k]) return LB_EINVAL;
        if (!slabs[k]->slab_nyg) return fail(slabs[k], LB_ESTATE, "not a slab (lb_set_slab)");
        if (slabs[k]->Q != slabs[0]->Q || slabs[k]->pitch != slabs[0]->pitch ||
            slabs[k]->ebytes != slabs[0]->ebytes ||
            slabs[k]->slab_nyg != slabs[0]->slab_nyg ||
            (k > 0 && slabs[k]->slab_y0 != slabs[k - 1]->slab_y0 + slabs[k - 1]->ny))
            return fail(slabs[k], LB_EINVAL, "slabs must tile one grid, in row order");
    }
    const int periodic = slabs[0]->cfg.boundary == LB_PERIODIC;
    for (int t = 0; t < steps; t++) {
        for (int k = 0; k < n; k++) {
            lb_status st = lb_step(slabs[k], 1);
            if (st != LB_OK) return st;
        }
        lb_status st = slab_exchange(slabs, n, periodic);
        if (st != LB_OK) return st;
    }
    return LB_OK;
}

}  // extern "C"
