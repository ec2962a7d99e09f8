// lb_runtime.h -- internal context structure of the C ABI (not installed).
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <string>
#include <utility>
#include <vector>

#include "lbac.h"
#include "lb_kernels.cuh"

struct lb_refine;  // two-level grid refinement state (refine.cu)

struct lb_ctx {
    lb_config cfg;                  // copy; pointer members cleared
    int Q = 5, nx = 0, ny = 0, pitch = 0, ebytes = 4;
    int ny3 = 0, nz = 1;            // 3-D (D3Q7): ny = ny3 * nz rows, row r = z ny3 + y
    void *pop[2] = {nullptr, nullptr};
    int cur = 0;                    // pop[cur] holds the post-collision state of step t-1
    bool raw = false;               // ... or, when raw, the state g(t) itself (unshifted)
    bool aa = false;                // in-place streaming: one buffer, pop[1] == pop[0]
    bool swap = false;              // in-place streaming after a site-local step: h(t-1) at
                                    // its own site, population i in slot opp(i)
    float *eta2 = nullptr;
    uint8_t *mid = nullptr;         // medium index (<= 256 distinct speeds), or nullptr
    float *mid_tab = nullptr;       // [256] eta^2 per index
    int n_mid = 0;
    bool staged = false;            // steps run the TMA-staged persistent kernel
    unsigned *fault = nullptr;      // device flag: a bounded wait in a kernel gave up
    float *lp_scale = nullptr;      // FP16 storage: [3][9] per-population scales (slots)
    unsigned *lp_max = nullptr;     // FP16 storage: [3][9][kMaxCopies] max |value| + counter
    int lp_slot = 0;                // slot describing the current buffer
    double *inv_scratch = nullptr;  // lb_invariants: [ny][4] row partials + [4] result
    int ckpt_every = 0;             // adjoint checkpoints: state copied every ckpt_every steps
    std::vector<void *> ckpt;       // ckpt[k]: stored buffer at time k * ckpt_every
    int ckpt_count = 0;             // valid checkpoints, from time ckpt_t0
    long long ckpt_t0 = 0;
    float *rho_tape = nullptr;      // lb_record_rho: rho(t) [tape_cap][ny][pitch] from tape_t0
    long long tape_t0 = 0;
    int tape_cap = 0;
    int *tb_off = nullptr;          // temporal blocking: per-tile receiver list offsets
    int *tb_rec = nullptr;          // receiver indices grouped by tile
    int *tb5_off = nullptr;         // D2Q5 wavefront blocking: per-row receiver offsets [ny + 2]
    int *tb5_x = nullptr;           // their x (ascending within a row)
    int *tb5_id = nullptr;          // their receiver index
    bool ckpt_raw0 = false;         // raw flag of the time-0 checkpoint
    float *src_tab = nullptr;
    int src_nt = 0, src_x = 0, src_y = 0;
    // LB_F64 (test-only) storage: FP64 eta^2, source table and coefficients (f64.cu)
    double *eta2_64 = nullptr;
    double *src64 = nullptr;
    double *coef64 = nullptr;
    int2 *rec = nullptr;
    int nrec = 0;
    std::vector<int> rec_xy;        // host copy of rec: (x, row) pairs
    float *trace = nullptr;         // [trace_cap][nrec]
    int trace_cap = 0;
    long long t_rec0 = 0;
    long long t = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool refined = false;
    bool fine_ready = false;
    lb_refine *ref = nullptr;
    void *(*alloc_fn)(size_t, void *) = nullptr;
    void (*free_fn)(void *, void *) = nullptr;
    void *alloc_user = nullptr;
    std::vector<void *> allocs;
    std::string err;
    // lb_set_slab: this context is the row slab [slab_y0, slab_y0 + ny) of a grid of
    // slab_nyg rows; halo rows and cut rows in caller-owned device buffers
    int slab_y0 = 0, slab_nyg = 0;
    const void *halo_lo = nullptr, *halo_hi = nullptr;
    void *send_lo = nullptr, *send_hi = nullptr;
    cudaEvent_t slab_ev[2] = {nullptr, nullptr};  // lb_slab_step: step done / cut rows read
    // lb_watch_stability: every `watch_every` steps lb_step checks the invariants
    int watch_every = 0;
    double watch_growth = 0;        // energy ratio between checks above which it fails
    double watch_energy = -1;       // energy at the last check (< 0: none yet)
    long long watch_t0 = 0;
};

namespace lbrt {
// Launch with programmatic stream serialization: the kernel may start while the previous
// kernel in the stream is finishing, and must call lbk::pdl_trigger_and_wait() before it
// touches global memory.
template <typename... ExpTypes, typename... ActTypes>
inline cudaError_t launch_pdl(void (*kernel)(ExpTypes...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, ActTypes &&...args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = grid;
    lc.blockDim = block;
    lc.dynamicSmemBytes = smem;
    lc.stream = stream;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, kernel, std::forward<ActTypes>(args)...);
}

// MRT rates as the collision kernels take them: s_k divided by the squared norm of row k of
// M (App. A), so that the kernels' relaxation d_k = s_k m_k / |row_k|^2 costs one multiply.
// D2Q5: e 20, p_xx 4; D2Q9: e and eps 36, p_xx and p_xy 4, q_x and q_y 12; 1 otherwise.
inline double mrt_norm(int Q, int k) {
    if (Q == 5) return k == 3 ? 20.0 : k == 4 ? 4.0 : 1.0;
    if (Q == 9)
        return (k == 3 || k == 5) ? 36.0 : (k == 4 || k == 8) ? 4.0 : (k == 6 || k == 7) ? 12.0 : 1.0;
    return 1.0;
}
inline float mrt_rate_arg(int Q, int k, double s) { return (float)(s / mrt_norm(Q, k)); }

using StepFn = void (*)(const lbk::StepArgs);
using GetFn = void (*)(lbk::StepArgs, float *, int);
lbk::StepArgs base_args(const lb_ctx *c);
StepFn pick_step_for(int Q, bool mrt, bool periodic, int storage);
StepFn pick_step(const lb_ctx *c);
lbk::StepArgs prepare_step(lb_ctx *ctx);  // FP32 / BF16 storage (no scale slots)
GetFn pick_get_for(int Q, bool periodic, int storage);
lb_status check_launch(lb_ctx *ctx, const char *what);
int round_up(int v, int m);
// scale pointers of the current buffer (nullptr for FP32 storage)
const float *current_scale(const lb_ctx *ctx);
lb_status fail(lb_ctx *ctx, lb_status st, const char *fmt, ...);
lb_status cuda_fail(lb_ctx *ctx, cudaError_t e, const char *what);
void *dev_alloc(lb_ctx *ctx, size_t bytes);
void dev_free(lb_ctx *ctx, void *p);

// Adjoint replay plan: the rho tape of lb_adjoint holds T = min(C, kAdjTapeBytes /
// plane_bytes) steps (at least 1) of one FP32 plane each; when T < C every
// checkpoint segment is first replayed once to place sub-checkpoints every T steps.
constexpr size_t kAdjTapeBytes = size_t(16) << 30;
inline int adj_tape_steps(size_t plane_bytes, int C) {
    size_t t = plane_bytes ? kAdjTapeBytes / plane_bytes : (size_t)C;
    if (t < 1) t = 1;
    return (int)(t < (size_t)C ? t : (size_t)C);
}
}  // namespace lbrt

// adjoint checkpoints (adjoint.cu): copy the state before step t when t % every == 0
lb_status ckpt_maybe_save(lb_ctx *ctx);
// the same, for callers that queue the copy themselves: reserves checkpoint slot
// k if one is due before the next step and returns the copy to make
bool ckpt_reserve(lb_ctx *ctx, void **dst, const void **src, size_t *bytes);
void ckpt_reset(lb_ctx *ctx);
// the forward rho tape (adjoint.cu): restart it at the current time; its row for step t
// (nullptr outside the tape)
void tape_reset(lb_ctx *ctx);
float *tape_row(const lb_ctx *ctx, long long t);

// temporal blocking (tblock.cu)
bool tb_supported(int Q, int K);
// TMA-staged persistent step (stream_step.cu): one LB step of the context's grid
lb_status stream_launch(lb_ctx *ctx, const lbk::StepArgs &a, int rec_blocks);
// its in-place form (BF16, D2Q5 / D2Q9): the site-local step, or the exchange step; receivers
// from the per-row lists of tb5_set_receivers (rec_off nullptr: none this step)
lb_status stream_launch_aa(lb_ctx *ctx, const lbk::StepArgs &a, bool exchange, const int *rec_off,
                           const int *rec_x, const int *rec_id);
lb_status tb_set_receivers(lb_ctx *ctx, const int *xy, int nrec);
lb_status tb_launch(lb_ctx *ctx, int K);
lb_status tb_launch_args(lb_ctx *ctx, const lbk::StepArgs &a, int K);
// in-place streaming (aa.cu): n steps of an LB_STREAM_AA context
lb_status aa_step(lb_ctx *ctx, int n);
// D2Q5 wavefront temporal blocking (tblock5.cu)
bool tb5_supported(int K);
lb_status tb5_set_receivers(lb_ctx *ctx, const int *xy, int nrec);
lb_status tb5_launch_args(lb_ctx *ctx, const lbk::StepArgs &a, int K);
// served batches of D2Q5 shots, K = kServeTb steps per launch (tblock5.cu; 4: the fastest
// wavefront depth, 3 CTAs per SM at 72 registers): staging bytes of one
// launch's descriptors, whether a shot can take K steps now, its strips and its CTAs at H
// output rows per CTA, the CTAs one wave of the batched kernel holds on the current device,
// the fill (advancing the shots) and the launch from the device copy of the staging block
constexpr int kServeTb = 4;
size_t tb5_batch_bytes(int n);
bool tb5_batch_ready(const lb_ctx *ctx, int K);
int tb5_strips(const lb_ctx *ctx, int K);
int tb5_batch_blocks(const lb_ctx *ctx, int K, int H);
int tb5_batch_wave(int K);
int tb5_batch_fill(lb_ctx *const *ctxs, int n, int K, int H, void *h);
cudaError_t tb5_batch_launch(const void *d, int n, int K, int blocks, bool mrt, bool per,
                             int storage, cudaStream_t stream);

// test-only FP64 storage (f64.cu): medium and coefficients, source table, steps, and the
// state transforms (mode 0 pressure, 1 populations; FP32 arrays f or FP64 arrays d)
lb_status f64_setup(lb_ctx *c, const float *cmap_dev, double cref);
lb_status f64_set_source(lb_ctx *c, const double *wavelet, int nt);
lb_status f64_step(lb_ctx *c, int n);
lb_status f64_set(lb_ctx *c, const float *f, const double *d, int on_device, int mode);
lb_status f64_get(lb_ctx *c, float *f, double *d, int on_device, int mode);

// linear stability of a configuration (stability.cu): whether lb_create checks it, the etas
// it checks, and the largest |lambda| of the one-step map over them and every refinement level
namespace lbrt {
bool stability_needed(const lb_config *cfg);
std::vector<double> stability_etas(double eta_min, double eta_max, const std::vector<double> &distinct);
double stability_worst(const lb_config *cfg, const std::vector<double> &etas, double *eta_at,
                       int *level_at);
constexpr double kStableBound = 1.0 + 1e-12;
}  // namespace lbrt

// grid refinement (refine.cu)
lb_status refine_setup(lb_ctx *ctx, const lb_config *cfg, const float *c_map_dev);
void refine_destroy(lb_ctx *ctx);
bool refine_contains(const lb_ctx *ctx, int x, int y);
lb_status refine_set_receivers(lb_ctx *ctx, const int *xy, int nrec);
lb_status refine_after_set_state(lb_ctx *ctx, const float *p0_dev);
lb_status refine_step(lb_ctx *ctx, int n);
lb_status refine_overlay_pressure(lb_ctx *ctx, float *p_dev);
