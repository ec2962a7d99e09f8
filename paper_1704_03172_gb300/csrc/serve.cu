// serve.cu -- continuous batching of independent shots (the serving layer).
//
// Threads and streams:
//   admitter   creates each admitted shot's lb_ctx (medium, source, receivers,
//              initial state) on the server's setup stream, so admission never
//              drains the batch stream;
//   scheduler  owns the batch stream.  Each scheduling pass advances every
//              active shot by up to `rounds_per_pass` steps: in every round one
//              batch_step_kernel launch per (lattice, collision, boundary,
//              storage) group steps all the group's shots once, each shot
//              reading its own StepArgs descriptor (uploaded once per pass), so
//              many small shots share one launch and fill the GPU together.  D2Q5
//              FP32 / BF16 shots that are far enough from their end take their steps
//              kServeTb at a time instead: one time-blocked launch
//              (tb5_batch_kernel, tblock5.cu) per group advances every such shot by
//              kServeTb steps.
//              Shots that finish leave the batch (their traces are copied to
//              pinned host memory), shots that are ready join at the next pass;
//   workers    run the adjoint of gradient requests (lb_adjoint) on their own
//              streams, overlapping the batched forward work of others.
// FP16 shots, whose per-step scale hand-off is per launch, step on their own, on a
// stream of their own (so they neither wait for nor delay the batched launches).
//
// Failures: a CUDA call that fails while a pass is queued (a descriptor copy, a
// batched launch, an FP16 step) fails the shots it concerns with LB_ECUDA (a
// descriptor-buffer allocation failure: LB_ENOMEM); they stop stepping and are
// retired once their queued work has drained or the stream reports the error.
//
// Memory: every device buffer of a served shot comes from one stream-ordered
// pool owned by the server (cudaMallocFromPoolAsync / cudaFreeAsync on the
// stream that uses the shot at that moment), so creating and retiring shots
// never synchronises the device; pinned trace buffers are recycled.  Admission
// is by lb_footprint against the budget, so the pool stays within it.
//
// All waits are bounded: the scheduler sleeps at most 5 ms when idle, the other
// threads poll their queues with a timeout, and lb_server_wait takes a timeout.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "lb_kernels.cuh"
#include "lb_runtime.h"

using namespace lbk;
using namespace lbrt;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum class RS { Pending, Admitting, Ready, Active, Draining, Adjoint, Done };

struct Req {
    lb_server *srv = nullptr;
    std::atomic<cudaStream_t> astream{nullptr};  // stream the shot's memory is ordered on
    long long id = 0;
    lb_config cfg;
    std::vector<float> cmap, obs;
    std::vector<double> wav;
    std::vector<int> rec;
    int src_x = 0, src_y = 0, nt = 0, want_grad = 0, ckpt = 200;
    bool tape = false;  // gradient from the forward rho tape (no checkpoints, no replays)
    size_t fp = 0;
    RS state = RS::Pending;
    lb_ctx *ctx = nullptr;
    int steps = 0;
    float *h_traces = nullptr;  // pinned [nt][nrec], from the server's recycled buffers
    size_t h_cap = 0;
    std::vector<float> grad_c;
    std::vector<double> grad_src;
    cudaEvent_t ev = nullptr;   // forward work and trace copy complete
    double t_submit = 0, t_start = 0, t_done = 0;
    lb_status status = LB_OK;
    std::string err;
    lb_status fail_st = LB_OK;  // set by the scheduler when a queued operation failed
    std::string fail_msg;
    bool fail_event = false;    // its drain event is still to be recorded (retire())
};

__global__ void residual_kernel(const float *p, const float *d, float *r, long long n) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) r[k] = p[k] - d[k];
}

using BatchFn = void (*)(const StepArgs *, const int *, int);

template <typename ST> BatchFn batch_fn(int Q, bool mrt, bool per) {
    if (Q == 9) {
        if (mrt) return per ? batch_step_kernel<9, true, true, ST> : batch_step_kernel<9, true, false, ST>;
        return per ? batch_step_kernel<9, false, true, ST> : batch_step_kernel<9, false, false, ST>;
    }
    if (mrt) return per ? batch_step_kernel<5, true, true, ST> : batch_step_kernel<5, true, false, ST>;
    return per ? batch_step_kernel<5, false, true, ST> : batch_step_kernel<5, false, false, ST>;
}

BatchFn pick_batch(const lb_config &c) {
    const bool mrt = c.collision == LB_MRT, per = c.boundary == LB_PERIODIC;
    return c.storage == LB_BF16 ? batch_fn<__nv_bfloat16>(c.lattice, mrt, per)
                                : batch_fn<float>(c.lattice, mrt, per);
}

}  // namespace

struct lb_server {
    lb_server_config cfg;
    int device = 0;
    cudaStream_t stream = nullptr;   // batch stream (scheduler)
    cudaStream_t stream16 = nullptr; // FP16 shots, stepped one by one (scheduler)
    cudaStream_t setup = nullptr;    // admission (admitter)
    cudaStream_t idle = nullptr;     // retirement of finished shots: nothing else runs on it
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_adj, cv_admit;
    std::deque<Req *> pending, adj_queue, admit_queue, ready;
    int admitting = 0;
    std::vector<Req *> active;  // stepping or draining; touched only by the scheduler
    std::map<long long, Req *> reqs;
    size_t budget = 0, used = 0;
    long long next_id = 1;
    bool stop = false, stop_helpers = false;
    std::thread sched, admitter;
    std::vector<std::thread> workers;
    StepArgs *d_args = nullptr, *h_args = nullptr;
    int *d_first = nullptr, *h_first = nullptr;
    size_t cap = 0;
    void *d_tb = nullptr, *h_tb = nullptr;  // time-blocked launches' descriptor blocks
    size_t tb_cap = 0;
    int tb_wave = 0;  // CTAs one wave of the time-blocked batch kernel holds (0: not asked yet)
    long long l2_bytes = -1;  // the device's L2 size (-1: not asked yet)
    cudaEvent_t staged = nullptr;
    std::mutex pin_mu;
    std::multimap<size_t, void *> pinned;  // free pinned trace buffers by size
    std::atomic<long long> n_done{0}, n_launch{0};
    std::string err;
};

namespace {

// device memory of a served shot: the server's pool, ordered on the stream that
// currently runs the shot
void *pool_alloc(size_t bytes, void *user) {
    Req *r = static_cast<Req *>(user);
    void *p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, r->srv->pool, r->astream.load()) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pool_free(void *p, void *user) {
    Req *r = static_cast<Req *>(user);
    cudaFreeAsync(p, r->astream.load());
}

void *pin_get(lb_server *S, size_t bytes, size_t *cap) {
    bytes = std::max<size_t>(bytes, 256);
    {
        std::lock_guard<std::mutex> lk(S->pin_mu);
        auto it = S->pinned.lower_bound(bytes);
        if (it != S->pinned.end() && it->first <= 2 * bytes) {
            void *p = it->second;
            *cap = it->first;
            S->pinned.erase(it);
            return p;
        }
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    *cap = bytes;
    return p;
}

void pin_put(lb_server *S, void *p, size_t cap) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(S->pin_mu);
    S->pinned.emplace(cap, p);
}

void finish(lb_server *S, Req *r, lb_status st, const std::string &msg) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (st != LB_OK && r->status == LB_OK) {
        r->status = st;
        r->err = msg;
    }
    r->t_done = now_s();
    r->state = RS::Done;
    S->used -= std::min(S->used, r->fp);
    S->n_done++;
    S->cv_done.notify_all();
    S->cv_work.notify_all();
}

void set_err(lb_server *S, const std::string &msg) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->err = msg;
}

// The scheduler gives up on a shot whose queued work failed: it stops stepping and
// retire() releases it once its stream has drained (or reports the error).  The drain
// event is recorded by retire(), after everything of the pass is queued, because later
// launches of the same pass may still name the shot.
void fail_shot(lb_server *, Req *r, lb_status st, const std::string &msg) {
    if (r->fail_st == LB_OK) {
        r->fail_st = st;
        r->fail_msg = msg;
    }
    if (r->state == RS::Active) {
        r->fail_event = true;
        r->state = RS::Draining;
    }
}

// The stream a shot steps on: FP16 shots on their own, the others on the batch stream.
cudaStream_t shot_stream(const lb_server *S, const Req *r) {
    return r->cfg.storage == LB_F16 ? S->stream16 : S->stream;
}

// Runs on the admitter thread: build the shot's context on the setup stream.
// Every call below that touches the device synchronises the setup stream, so
// the context is complete when it is handed to the scheduler.
void admit(lb_server *S, Req *r) {
    r->srv = S;
    r->astream.store(S->setup);
    lb_config c = r->cfg;
    c.c_map = r->cmap.data();
    c.c_map_on_device = 0;
    c.cuda_stream = S->setup;
    c.time_block = 1;
    c.dev_alloc = pool_alloc;
    c.dev_free = pool_free;
    c.alloc_user = r;
    lb_ctx *ctx = nullptr;
    lb_status st = lb_create(&c, &ctx);
    if (st == LB_OK && !r->wav.empty())
        st = lb_set_source(ctx, r->src_x, r->src_y, r->wav.data(), (int)r->wav.size());
    if (st == LB_OK) st = lb_set_receivers(ctx, r->rec.data(), (int)r->rec.size() / 2, r->nt);
    if (st == LB_OK && c.lattice == LB_D2Q5 && (c.storage == LB_F32 || c.storage == LB_BF16) &&
        !r->rec.empty())  // the receiver rows of the time-blocked batches
        st = tb5_set_receivers(ctx, r->rec.data(), (int)r->rec.size() / 2);
    if (st == LB_OK) st = lb_init_pressure(ctx, nullptr, 0);
    if (st == LB_OK && r->want_grad)
        st = r->tape ? lb_record_rho(ctx, r->nt) : lb_checkpoint_every(ctx, r->ckpt);
    if (st == LB_OK &&
        !(r->h_traces = static_cast<float *>(pin_get(S, (size_t)r->nt * (r->rec.size() / 2) * 4, &r->h_cap))))
        st = LB_ENOMEM;
    if (st == LB_OK && cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess)
        st = LB_ECUDA;
    if (st == LB_OK && cudaStreamSynchronize(S->setup) != cudaSuccess) st = LB_ECUDA;
    if (st != LB_OK) {
        std::string msg = ctx ? lb_last_error(ctx) : lb_last_error(nullptr);
        if (ctx) lb_destroy(ctx);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->admitting--;
        }
        finish(S, r, st, msg);
        return;
    }
    ctx->stream = shot_stream(S, r);  // from here on the scheduler runs it
    r->ctx = ctx;
    std::lock_guard<std::mutex> lk(S->mu);
    r->astream.store(shot_stream(S, r));
    r->state = RS::Ready;
    S->admitting--;
    S->ready.push_back(r);
    S->cv_work.notify_all();
}

void admitter(lb_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        Req *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            while (S->admit_queue.empty()) {
                if (S->stop_helpers) return;
                S->cv_admit.wait_for(lk, std::chrono::milliseconds(10));
            }
            r = S->admit_queue.front();
            S->admit_queue.pop_front();
            S->admitting++;
        }
        admit(S, r);
    }
}
bool ensure_tb_capacity(lb_server *S, size_t bytes) {
    if (bytes <= S->tb_cap) return true;
    const size_t cap = std::max(bytes, 2 * S->tb_cap);
    if (S->d_tb) cudaFree(S->d_tb);
    if (S->h_tb) cudaFreeHost(S->h_tb);
    S->d_tb = S->h_tb = nullptr;
    S->tb_cap = 0;
    if (cudaMalloc(&S->d_tb, cap) != cudaSuccess || cudaMallocHost(&S->h_tb, cap) != cudaSuccess)
        return false;
    S->tb_cap = cap;
    return true;
}

bool ensure_capacity(lb_server *S, size_t n) {
    if (n <= S->cap) return true;
    size_t cap = std::max(n, 2 * S->cap);
    if (S->d_args) cudaFree(S->d_args);
    if (S->d_first) cudaFree(S->d_first);
    if (S->h_args) cudaFreeHost(S->h_args);
    if (S->h_first) cudaFreeHost(S->h_first);
    S->d_args = nullptr;
    S->d_first = nullptr;
    S->h_args = nullptr;
    S->h_first = nullptr;
    S->cap = 0;
    if (cudaMalloc(&S->d_args, cap * sizeof(StepArgs)) != cudaSuccess ||
        cudaMalloc(&S->d_first, 2 * cap * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&S->h_args, cap * sizeof(StepArgs)) != cudaSuccess ||
        cudaMallocHost(&S->h_first, 2 * cap * sizeof(int)) != cudaSuccess)
        return false;
    S->cap = cap;
    return true;
}

// One pass: up to R rounds of one step for every stepping shot.
void pass(lb_server *S) {
    const int R = std::max(1, S->cfg.rounds_per_pass);
    std::vector<Req *> shots;
    for (Req *r : S->active)
        if (r->state == RS::Active && r->steps < r->nt) shots.push_back(r);
    if (shots.empty()) return;
    // FP16 shots step on their own (their scale hand-off is per launch)
    std::vector<Req *> batched;
    for (Req *r : shots) {
        if (r->cfg.storage == LB_F16) {
            int n = std::min(R, r->nt - r->steps);
            const lb_status st = lb_step(r->ctx, n);
            if (st != LB_OK) {
                fail_shot(S, r, st, std::string("FP16 step: ") + lb_last_error(r->ctx));
                continue;
            }
            r->steps += n;
        } else {
            batched.push_back(r);
        }
    }
    if (batched.empty()) return;
    using Key = std::tuple<int, int, int, int>;
    auto key = [](const Req *r) {
        return Key(r->cfg.lattice, r->cfg.collision, r->cfg.boundary, r->cfg.storage);
    };
    // wait until the previous pass has consumed the staging buffers
    if (S->staged) cudaEventSynchronize(S->staged);
    // shots that take this pass's steps K at a time: one time-blocked launch per group and
    // block of K steps
    const int KB = kServeTb, nblk = R / KB;
    // Shots that take this pass's steps K at a time.  A wavefront CTA sweeps its rows one
    // after another, so the launch must fill a wave of CTAs with chunks tall enough that
    // the 2K warm-up rows of each cost little.  By default (tb_min_ctas = 0) the pass takes
    // the chunk height (at most 16K rows) that fills one wave with every ready shot: at
    // least 3K rows, and states larger than L2 can hold, else none of them blocks this pass
    // (two-layer 1024^2 alone, K = 8: 112 GLUPS blocked with one-wave chunks of 18 rows
    // against 153 one step per launch; 4096^2: 295 against 160).  All CTAs of the launch
    // then sweep about the same number of rows, whatever their shot's size.  With
    // tb_min_ctas > 0 the shots block at 16K rows when together they make that many CTAs;
    // below 0 never.
    std::vector<Req *> tbs, rest;
    const int H16 = 16 * KB;
    int tb_rows = H16;
    for (Req *r : batched) {
        const bool ok = S->cfg.tb_min_ctas >= 0 && nblk > 0 && r->nt - r->steps >= nblk * KB &&
                        tb5_batch_ready(r->ctx, KB);
        (ok ? tbs : rest).push_back(r);
    }
    if (!tbs.empty()) {
        bool use = true;
        if (S->cfg.tb_min_ctas > 0) {
            long long ctas = 0;
            for (Req *r : tbs) ctas += tb5_batch_blocks(r->ctx, KB, H16);
            use = ctas >= S->cfg.tb_min_ctas;
        } else {  // the chunk height that fills one wave
            if (S->tb_wave == 0) S->tb_wave = tb5_batch_wave(KB);
            if (S->l2_bytes < 0) {
                int v = 0;
                if (cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, S->device) != cudaSuccess) {
                    cudaGetLastError();  // this query's own failure: assume no L2
                    v = 0;
                }
                S->l2_bytes = v;
            }
            long long rows = 0, state = 0;  // sums over the shots of strips x rows, state bytes
            for (Req *r : tbs) {
                rows += (long long)tb5_strips(r->ctx, KB) * r->ctx->ny;
                state += 2LL * r->ctx->Q * r->ctx->ny * r->ctx->pitch * r->ctx->ebytes;
            }
            const long long h = (rows + S->tb_wave - 1) / S->tb_wave;
            tb_rows = (int)std::min<long long>(H16, h);
            // blocking saves HBM traffic; states that fit in three quarters of L2 have none
            // to save (32 shots of 256^2, 84 MB: 3.7x over one by one stepped, 3.0x blocked)
            use = tb_rows >= 3 * KB && 4 * state > 3 * S->l2_bytes;
        }
        if (!use) {
            rest.insert(rest.end(), tbs.begin(), tbs.end());
            tbs.clear();
        }
    }
    batched.swap(rest);
    std::stable_sort(tbs.begin(), tbs.end(),
                     [&](const Req *a, const Req *b) { return key(a) < key(b); });
    struct TbLaunch {
        size_t off;
        int n, blocks;
        bool mrt, per;
        int storage;
        size_t g0, g1;
    };
    std::vector<TbLaunch> tb_launches;
    size_t tb_bytes = 0;
    if (!tbs.empty()) {
        for (size_t g0 = 0; g0 < tbs.size();) {  // staging bytes of every launch
            size_t g1 = g0;
            while (g1 < tbs.size() && key(tbs[g1]) == key(tbs[g0])) g1++;
            tb_bytes += nblk * tb5_batch_bytes((int)(g1 - g0));
            g0 = g1;
        }
        if (!ensure_tb_capacity(S, tb_bytes)) {
            cudaGetLastError();
            set_err(S, "time-blocked descriptor buffers");
            for (Req *r : tbs) fail_shot(S, r, LB_ENOMEM, "time-blocked descriptor buffers");
            tbs.clear();
        }
        size_t off = 0;
        std::vector<lb_ctx *> cs;
        for (int j = 0; j < nblk && !tbs.empty(); j++) {
            for (size_t g0 = 0; g0 < tbs.size();) {
                size_t g1 = g0;
                while (g1 < tbs.size() && key(tbs[g1]) == key(tbs[g0])) g1++;
                cs.clear();
                for (size_t q = g0; q < g1; q++) cs.push_back(tbs[q]->ctx);
                const int n = (int)(g1 - g0);
                const int blocks =
                    tb5_batch_fill(cs.data(), n, KB, tb_rows, static_cast<char *>(S->h_tb) + off);
                const lb_config &c0 = tbs[g0]->cfg;
                tb_launches.push_back({off, n, blocks, c0.collision == LB_MRT,
                                       c0.boundary == LB_PERIODIC, c0.storage, g0, g1});
                off += tb5_batch_bytes(n);
                g0 = g1;
            }
            for (Req *r : tbs) r->steps += KB;
        }
        tb_bytes = off;
    }
    if (batched.empty() && tb_launches.empty()) return;
    // build every round's descriptors: groups of identical kernels, shots sorted by group
    std::stable_sort(batched.begin(), batched.end(),
                     [&](const Req *a, const Req *b) { return key(a) < key(b); });
    struct Launch {
        BatchFn fn;
        size_t arg0, first0;
        int n, blocks, round;
        size_t g0, g1;  // its shots: batched[g0, g1)
    };
    struct Copy {  // adjoint checkpoint, queued just before its round's launches
        int round;
        void *dst;
        const void *src;
        size_t bytes;
    };
    std::vector<Launch> launches;
    std::vector<Copy> copies;
    size_t need = (size_t)R * batched.size();
    if (!ensure_capacity(S, need + 1)) {
        cudaGetLastError();
        set_err(S, "descriptor buffers");
        for (Req *r : batched) fail_shot(S, r, LB_ENOMEM, "batch descriptor buffers");
        return;
    }
    size_t na = 0, nf = 0;
    for (int k = 0; k < R; k++) {
        size_t g0 = 0;
        while (g0 < batched.size()) {
            size_t g1 = g0;
            while (g1 < batched.size() && key(batched[g1]) == key(batched[g0])) g1++;
            Launch L{pick_batch(batched[g0]->cfg), na, nf, 0, 0, k, g0, g1};
            for (size_t q = g0; q < g1; q++) {
                Req *r = batched[q];
                if (r->steps >= r->nt) continue;
                Copy c{k, nullptr, nullptr, 0};
                if (r->ctx->ckpt_every > 0 && ckpt_reserve(r->ctx, &c.dst, &c.src, &c.bytes))
                    copies.push_back(c);
                StepArgs a = prepare_step(r->ctx);
                const int blocks =
                    a.main_blocks + (a.trace_row ? (a.nrec + kThreads - 1) / kThreads : 0);
                S->h_args[na++] = a;
                S->h_first[nf++] = L.blocks;
                L.blocks += blocks;
                L.n++;
                r->steps++;
            }
            if (L.n > 0) {
                S->h_first[nf++] = L.blocks;  // closing prefix entry
                launches.push_back(L);
            }
            g0 = g1;
        }
    }
    cudaError_t e = cudaSuccess;
    if (na > 0)
        e = cudaMemcpyAsync(S->d_args, S->h_args, na * sizeof(StepArgs), cudaMemcpyHostToDevice,
                            S->stream);
    if (e == cudaSuccess && nf > 0)
        e = cudaMemcpyAsync(S->d_first, S->h_first, nf * sizeof(int), cudaMemcpyHostToDevice,
                            S->stream);
    if (e == cudaSuccess && tb_bytes > 0)
        e = cudaMemcpyAsync(S->d_tb, S->h_tb, tb_bytes, cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess && !S->staged)
        e = cudaEventCreateWithFlags(&S->staged, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(S->staged, S->stream);
    if (e != cudaSuccess) {  // nothing of this pass is queued: every batched shot fails
        const std::string msg = std::string("batch descriptors: ") + cudaGetErrorString(e);
        set_err(S, msg);
        for (Req *r : batched) fail_shot(S, r, LB_ECUDA, msg);
        for (Req *r : tbs) fail_shot(S, r, LB_ECUDA, msg);
        return;
    }
    for (const TbLaunch &L : tb_launches) {  // time-blocked blocks of K steps
        e = tb5_batch_launch(static_cast<char *>(S->d_tb) + L.off, L.n, KB, L.blocks, L.mrt, L.per,
                             L.storage, S->stream);
        if (e != cudaSuccess) {
            const std::string msg = std::string("time-blocked batch: ") + cudaGetErrorString(e);
            set_err(S, msg);
            for (size_t q = L.g0; q < L.g1; q++) fail_shot(S, tbs[q], LB_ECUDA, msg);
            e = cudaSuccess;
            continue;
        }
        S->n_launch++;
    }
    // rounds in order; a checkpoint copy reads the state its round starts from
    size_t ci = 0;
    for (const Launch &L : launches) {
        for (; ci < copies.size() && copies[ci].round <= L.round && e == cudaSuccess; ci++)
            e = cudaMemcpyAsync(copies[ci].dst, copies[ci].src, copies[ci].bytes,
                                cudaMemcpyDeviceToDevice, S->stream);
        if (e == cudaSuccess)
            e = launch_pdl(L.fn, dim3(L.blocks), dim3(kThreads), 0, S->stream,
                           (const StepArgs *)(S->d_args + L.arg0),
                           (const int *)(S->d_first + L.first0), L.n);
        if (e != cudaSuccess) {  // this launch's shots, and every later round, stop here
            const std::string msg = std::string("batched step: ") + cudaGetErrorString(e);
            set_err(S, msg);
            for (size_t q = L.g0; q < L.g1; q++) fail_shot(S, batched[q], LB_ECUDA, msg);
            e = cudaSuccess;
            continue;
        }
        S->n_launch++;
    }
}

// Shots that ran all their steps: copy traces out, then finish or hand to an adjoint worker.
void retire(lb_server *S) {
    std::vector<Req *> keep;
    for (Req *r : S->active) {
        if (r->fail_event) {
            r->fail_event = false;
            cudaEventRecord(r->ev, r->ctx->stream);
        }
        if (r->state == RS::Active && r->steps >= r->nt) {
            const size_t bytes = (size_t)r->nt * (r->rec.size() / 2) * 4;
            cudaError_t e = cudaSuccess;
            if (bytes)
                e = cudaMemcpyAsync(r->h_traces, r->ctx->trace, bytes, cudaMemcpyDeviceToHost,
                                    r->ctx->stream);
            if (e != cudaSuccess && r->fail_st == LB_OK) {
                r->fail_st = LB_ECUDA;
                r->fail_msg = std::string("trace copy: ") + cudaGetErrorString(e);
            }
            cudaEventRecord(r->ev, r->ctx->stream);
            if (r->fail_st != LB_OK) r->state = RS::Draining;
            if (r->state == RS::Active && r->want_grad) {
                r->state = RS::Adjoint;
                std::lock_guard<std::mutex> lk(S->mu);
                S->adj_queue.push_back(r);
                S->cv_adj.notify_one();
                continue;  // leaves the active list; memory stays accounted
            }
            if (r->state == RS::Active) r->state = RS::Draining;
        }
        if (r->state == RS::Draining) {
            const cudaError_t q = cudaEventQuery(r->ev);
            if (q != cudaErrorNotReady) {
                // all of the shot's work is complete (or its stream reports an error): free on
                // a stream with nothing queued, so neither lb_destroy's wait nor the frees hold
                // up the batch stream
                if (q != cudaSuccess && r->fail_st == LB_OK) {
                    r->fail_st = LB_ECUDA;
                    r->fail_msg = std::string("shot's queued work: ") + cudaGetErrorString(q);
                }
                r->ctx->stream = S->idle;
                r->astream.store(S->idle);
                lb_destroy(r->ctx);
                r->ctx = nullptr;
                finish(S, r, r->fail_st, r->fail_msg);
                continue;
            }
        }
        keep.push_back(r);
    }
    std::lock_guard<std::mutex> lk(S->mu);  // lb_server_stats reads the size
    S->active.swap(keep);
}

void scheduler(lb_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            const bool busy = !S->pending.empty() || !S->admit_queue.empty() || !S->ready.empty() ||
                              S->admitting > 0;
            if (S->stop && !busy && S->active.empty()) break;
            // shots whose context is built join the batch
            for (Req *r : S->ready) {
                r->state = RS::Active;
                r->t_start = now_s();
                S->active.push_back(r);
            }
            S->ready.clear();
            // admission in arrival order, by slot and device-memory budget
            size_t slots = S->active.size() + S->admit_queue.size() + (size_t)S->admitting;
            for (auto it = S->pending.begin();
                 it != S->pending.end() && slots < (size_t)S->cfg.max_active;) {
                if (S->used + (*it)->fp <= S->budget) {
                    S->used += (*it)->fp;
                    (*it)->state = RS::Admitting;
                    S->admit_queue.push_back(*it);
                    it = S->pending.erase(it);
                    slots++;
                } else {
                    ++it;
                }
            }
            if (!S->admit_queue.empty()) S->cv_admit.notify_one();
            if (S->active.empty()) {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
        }
        pass(S);
        retire(S);
        bool idle = true;
        for (Req *r : S->active)
            if (r->state == RS::Active) idle = false;
        if (idle) std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    cudaStreamSynchronize(S->stream);
    cudaStreamSynchronize(S->stream16);
}

void adjoint_worker(lb_server *S) {
    cudaSetDevice(S->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        Req *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            while (S->adj_queue.empty()) {
                if (S->stop_helpers) {
                    lk.unlock();
                    cudaStreamDestroy(st);
                    return;
                }
                S->cv_adj.wait_for(lk, std::chrono::milliseconds(10));
            }
            r = S->adj_queue.front();
            S->adj_queue.pop_front();
        }
        cudaStreamWaitEvent(st, r->ev, 0);
        lb_ctx *ctx = r->ctx;
        ctx->stream = st;  // the scheduler no longer touches this context
        r->astream.store(st);
        const int nrec = (int)r->rec.size() / 2;
        const long long n = (long long)r->nt * nrec;
        float *d_obs = nullptr, *d_res = nullptr, *d_gc = nullptr;
        double *d_gs = nullptr;
        auto grab = [&](size_t b) { return pool_alloc(b, r); };
        lb_status status = LB_OK;
        if (n > 0 && (!(d_obs = static_cast<float *>(grab(n * 4))) ||
                      !(d_res = static_cast<float *>(grab(n * 4)))))
            status = LB_ENOMEM;
        if (status == LB_OK && n > 0) {
            cudaMemcpyAsync(d_obs, r->obs.data(), n * 4, cudaMemcpyHostToDevice, st);
            residual_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctx->trace, d_obs, d_res, n);
        }
        r->grad_c.assign((size_t)ctx->nx * ctx->ny, 0.f);
        std::vector<double> gs(r->nt, 0.0);
        if (status == LB_OK) {  // dJ/dp and the gradients stay on the device, then one copy out
            if (!(d_gc = static_cast<float *>(grab(r->grad_c.size() * 4))) ||
                !(d_gs = static_cast<double *>(grab(gs.size() * 8)))) {
                status = LB_ENOMEM;
            } else {
                status = lb_adjoint(ctx, d_res, r->nt, d_gc, d_gs, nullptr, 1);
                if (status == LB_OK) {
                    cudaMemcpyAsync(r->grad_c.data(), d_gc, r->grad_c.size() * 4, cudaMemcpyDeviceToHost, st);
                    cudaMemcpyAsync(gs.data(), d_gs, gs.size() * 8, cudaMemcpyDeviceToHost, st);
                    if (cudaStreamSynchronize(st) != cudaSuccess) status = LB_ECUDA;
                }
            }
        }
        std::string msg = status == LB_OK ? "" : lb_last_error(ctx);
        r->grad_src.assign(r->wav.size(), 0.0);
        for (size_t k = 0; k < r->grad_src.size() && k < gs.size(); k++) r->grad_src[k] = gs[k];
        for (void *p : {(void *)d_obs, (void *)d_res, (void *)d_gc, (void *)d_gs})
            if (p) pool_free(p, r);
        lb_destroy(ctx);
        r->ctx = nullptr;
        finish(S, r, status, msg);
    }
}

}  // namespace

extern "C" {

lb_status lb_server_create(const lb_server_config *cfg, lb_server **out) {
    if (!cfg || !out) return LB_EINVAL;
    *out = nullptr;
    if (cfg->max_active < 1 || cfg->rounds_per_pass < 1 || cfg->adjoint_workers < 1)
        return fail(nullptr, LB_EINVAL, "max_active, rounds_per_pass and adjoint_workers must be >= 1");
    lb_server *S = new lb_server();
    S->cfg = *cfg;
    cudaGetDevice(&S->device);
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = S->device;
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->stream16, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->setup, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->idle, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMemPoolCreate(&S->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        for (cudaStream_t s : {S->stream, S->stream16, S->setup, S->idle})
            if (s) cudaStreamDestroy(s);
        delete S;
        return fail(nullptr, LB_ECUDA, "server streams or memory pool");
    }
    // keep freed memory in the pool for the next shots (bounded by the admission budget)
    unsigned long long keep = ~0ull;
    cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    S->budget = cfg->hbm_budget ? cfg->hbm_budget : (size_t)(0.8 * (double)free_b);
    S->sched = std::thread(scheduler, S);
    S->admitter = std::thread(admitter, S);
    for (int k = 0; k < cfg->adjoint_workers; k++) S->workers.emplace_back(adjoint_worker, S);
    *out = S;
    return LB_OK;
}

lb_status lb_server_submit(lb_server *S, const lb_request *q, long long *id) {
    if (!S || !q || !id) return LB_EINVAL;
    if (q->nt < 1 || q->nrec < 0 || (q->nrec > 0 && !q->rec_xy) || !q->cfg.c_map ||
        (q->nt_wavelet > 0 && !q->wavelet) || (q->want_gradient && q->nrec > 0 && !q->observed))
        return fail(nullptr, LB_EINVAL, "incomplete request");
    if (q->cfg.n_patches > 0) return fail(nullptr, LB_EINVAL, "served shots have no patch");
    if (q->cfg.streaming != LB_STREAM_AB)
        return fail(nullptr, LB_EINVAL, "served shots stream between two buffers (LB_STREAM_AB)");
    if (q->cfg.lattice == LB_D3Q7 || q->cfg.nz > 1)
        return fail(nullptr, LB_EINVAL, "served shots are 2-D (D2Q5 / D2Q9)");
    if (q->cfg.storage == LB_F64)
        return fail(nullptr, LB_EINVAL, "served shots store FP32, BF16 or FP16 (LB_F64 is test only)");
    Req *r = new Req();
    r->cfg = q->cfg;
    r->cmap.assign(q->cfg.c_map, q->cfg.c_map + (size_t)q->cfg.nx * q->cfg.ny);
    r->cfg.c_map = nullptr;
    if (q->nt_wavelet > 0) r->wav.assign(q->wavelet, q->wavelet + q->nt_wavelet);
    r->rec.assign(q->rec_xy, q->rec_xy + 2 * q->nrec);
    if (q->want_gradient && q->nrec > 0) r->obs.assign(q->observed, q->observed + (size_t)q->nt * q->nrec);
    r->src_x = q->src_x;
    r->src_y = q->src_y;
    r->nt = q->nt;
    r->want_grad = q->want_gradient ? 1 : 0;
    r->ckpt = q->checkpoint_every > 0 ? q->checkpoint_every : 200;
    if (r->want_grad) {  // the forward rho tape when asked for, or (0) when it is small
        size_t tape_fp = 0;
        lb_footprint(&q->cfg, q->nt, q->nrec, -1, &tape_fp);
        r->tape = q->checkpoint_every < 0 || (q->checkpoint_every == 0 && tape_fp <= S->budget / 2);
    }
    if (r->want_grad && !r->tape && q->cfg.storage != LB_F32 && q->cfg.storage != LB_BF16) {
        delete r;
        return fail(nullptr, LB_EINVAL,
                    "checkpointed gradients need FP32 or BF16 storage (FP16: the rho tape)");
    }
    lb_footprint(&q->cfg, q->nt, q->nrec, r->want_grad ? (r->tape ? -1 : r->ckpt) : 0, &r->fp);
    r->fp += (size_t)q->nt * q->nrec * 4 * (r->want_grad ? 2 : 0);  // observed + residual
    std::lock_guard<std::mutex> lk(S->mu);
    if (r->fp > S->budget) {
        delete r;
        S->err = "request needs more device memory than the budget";
        return fail(nullptr, LB_ENOMEM, "request needs more device memory than the budget");
    }
    r->id = S->next_id++;
    r->t_submit = now_s();
    S->reqs[r->id] = r;
    S->pending.push_back(r);
    S->cv_work.notify_all();
    *id = r->id;
    return LB_OK;
}

lb_status lb_server_poll(lb_server *S, long long id, int *done) {
    if (!S || !done) return LB_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return LB_EINVAL;
    *done = it->second->state == RS::Done;
    return LB_OK;
}

lb_status lb_server_wait(lb_server *S, long long id, int timeout_ms) {
    if (!S) return LB_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return LB_EINVAL;
    Req *r = it->second;
    auto pred = [&] { return r->state == RS::Done; };
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, pred);
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
        return LB_ETIMEOUT;
    }
    return LB_OK;
}

lb_status lb_server_result(lb_server *S, long long id, float *traces, float *grad_c,
                           double *grad_src, double *times) {
    if (!S) return LB_EINVAL;
    Req *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(id);
        if (it == S->reqs.end()) return LB_EINVAL;
        r = it->second;
        if (r->state != RS::Done) return LB_ESTATE;
        S->reqs.erase(it);
    }
    const size_t nrec = r->rec.size() / 2;
    if (traces && r->h_traces && r->status == LB_OK)
        memcpy(traces, r->h_traces, (size_t)r->nt * nrec * 4);
    if (grad_c && !r->grad_c.empty()) memcpy(grad_c, r->grad_c.data(), r->grad_c.size() * 4);
    if (grad_src && !r->grad_src.empty()) memcpy(grad_src, r->grad_src.data(), r->grad_src.size() * 8);
    if (times) {
        times[0] = r->t_submit;
        times[1] = r->t_start;
        times[2] = r->t_done;
    }
    lb_status st = r->status;
    if (st != LB_OK) set_err(S, r->err);
    pin_put(S, r->h_traces, r->h_cap);
    if (r->ev) cudaEventDestroy(r->ev);
    delete r;
    return st;
}

lb_status lb_server_stats(lb_server *S, double *out, int n) {
    if (!S || !out) return LB_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    double v[5] = {(double)S->n_done.load(), (double)S->active.size(), (double)S->pending.size(),
                   (double)S->used, (double)S->n_launch.load()};
    for (int k = 0; k < n && k < 5; k++) out[k] = v[k];
    return LB_OK;
}

lb_status lb_server_destroy(lb_server *S) {
    if (!S) return LB_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->sched.joinable()) S->sched.join();  // returns once nothing is pending, admitting or stepping
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop_helpers = true;  // workers drain their queue first
        S->cv_adj.notify_all();
        S->cv_admit.notify_all();
    }
    if (S->admitter.joinable()) S->admitter.join();
    for (auto &w : S->workers)
        if (w.joinable()) w.join();
    for (auto &kv : S->reqs) {
        Req *r = kv.second;
        pin_put(S, r->h_traces, r->h_cap);
        if (r->ev) cudaEventDestroy(r->ev);
        delete r;
    }
    if (S->d_args) cudaFree(S->d_args);
    if (S->d_first) cudaFree(S->d_first);
    if (S->h_args) cudaFreeHost(S->h_args);
    if (S->h_first) cudaFreeHost(S->h_first);
    if (S->d_tb) cudaFree(S->d_tb);
    if (S->h_tb) cudaFreeHost(S->h_tb);
    for (auto &kv : S->pinned) cudaFreeHost(kv.second);
    if (S->staged) cudaEventDestroy(S->staged);
    for (cudaStream_t s : {S->stream, S->stream16, S->setup, S->idle}) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    cudaMemPoolDestroy(S->pool);
    delete S;
    return LB_OK;
}

// The message is copied under the server's lock into a per-thread buffer, so the pointer
// stays valid (until this thread's next call) while the scheduler records new errors.
const char *lb_server_last_error(const lb_server *S) {
    thread_local std::string copy;
    if (!S) return "";
    std::lock_guard<std::mutex> lk(const_cast<lb_server *>(S)->mu);
    copy = S->err;
    return copy.c_str();
}

}  // extern "C"
