// stream_step.cu -- TMA-staged persistent form of the fused LB step.
//
// Same per-site arithmetic as step_kernel (finish_sites / collide_sites in
// lb_kernels.cuh), different data movement.  A persistent grid (resident CTAs
// x SM count) walks the row segments ("tasks") of the grid: task = W = 256 V
// consecutive sites of one row.  For every task one thread issues, per
// population, a bulk copy (cp.async.bulk, the untiled TMA form) of the source
// row segment with a 16-byte halo on each side, plus the segment's medium
// (1-byte index or FP32 eta^2), into a shared-memory stage, completing on that
// stage's mbarrier.  While a CTA computes task k from stage k mod S, the copies
// of the next S - 1 tasks are in flight, so the loads are decoupled from the
// arithmetic and no register holds data waiting on DRAM.  Outputs go straight
// from registers to HBM with 16-byte stores.  For D2Q5 a dedicated producer
// warp issues the copies and each compute warp releases a stage on its own (an
// "empty" mbarrier per stage), so no block-wide barrier paces the loop.
//
// Addresses and sizes of every bulk copy are multiples of 16 bytes: rows are
// pitch elements apart (pitch a multiple of 32 elements), a task starts at a
// multiple of W elements (W * element size = 4096 bytes) and the halo is 16
// bytes; copies are clipped to [0, pitch) of the row.
//
// Chosen automatically for 16-bit storage on rows of >= 1024 sites, where it beats
// the register-streaming kernel (GB300, 4096^2: BF16 D2Q5 206 -> 271 GLUPS, FP16
// 195 -> 214, BF16 D2Q9 82 -> 134).  For FP32 the register-streaming kernel is
// faster (159 vs 135 GLUPS), and on narrow rows (e.g. a 256^3 D3Q7 grid) most of a
// task's threads would idle.  Any lattice (D2Q5, D2Q9, D3Q7) can force it.
//
// Every wait on an mbarrier is bounded (one second of %globaltimer).  On a
// timeout the block votes to stop, raises the context's fault flag (read by
// lb_sync), waits (bounded again) for the copies it still has in flight and
// returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "aa_sites.cuh"
#include "lb_kernels.cuh"
#include "lb_runtime.h"

using namespace lbk;
using namespace lbrt;

namespace {

constexpr int kSThreads = 256;                       // threads per CTA
constexpr unsigned long long kWaitNs = 1000000000ull;  // bound of every mbarrier wait

template <typename ST> struct Geom {
    static constexpr int V = Store<ST>::V;             // sites per thread
    static constexpr int W = kSThreads * V;            // sites per task
    static constexpr int H = 16 / (int)sizeof(ST);     // halo elements (16 bytes)
    static constexpr int ROWB = (W + 2 * H) * (int)sizeof(ST);  // staged bytes per population
};

// A stage: Q staged population rows, then the medium (W bytes of index or 4W of eta^2).
template <int Q, typename ST> struct Stage {
    static constexpr int kPops = Q * Geom<ST>::ROWB;
    static_assert(kPops % 16 == 0, "16-byte aligned stage layout");
    static constexpr int bytes(bool indexed) { return kPops + Geom<ST>::W * (indexed ? 1 : 4); }
};
constexpr int kMaxStages = 4;

struct SArgs {
    int tasks_per_row;
    int ntasks;
    int ncta;          // persistent CTAs; blocks beyond them gather receivers
    int stages;        // shared-memory stages per CTA (2 .. kMaxStages)
    int stage_bytes;   // bytes per stage (a multiple of 16)
    unsigned *fault;   // raised when a bounded wait gives up
    lbaa::AaRec rec;   // in-place forms: receivers by row (their sums are taken in the step)
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for phase `parity` of *bar; false after `ns` without completion.
__device__ bool mbar_wait_for(uint64_t *bar, unsigned parity, unsigned long long ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > ns) return false;
    return true;
}

__device__ bool mbar_wait(uint64_t *bar, unsigned parity) { return mbar_wait_for(bar, parity, kWaitNs); }

// Bulk copy global -> shared (TMA, untiled), completing `bytes` on *bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace

namespace {

// Source row of population i for output row y (D3Q7: (y3, z) of that row given); -1:
// outside a zero-ghost domain.
template <int Q, bool PERIODIC>
__device__ __forceinline__ int source_row(const StepArgs &a, int i, int y, int y3, int z3) {
    if (a.raw) return y;  // first step after lb_set_state: g(t) is read in place
    return pull_row_yz<Q, PERIODIC>(a, y, y3, z3, i);  // y (and, for D3Q7, z) shift of the row
}

// In-place forms of the step (AA == 1: site-local, 2: exchange; 0: the two-buffer pull).
// The site-local form stages population i's own row; the exchange form stages slot opp(i)
// of the row population i pulls from, which holds h_i(t - 1).  Either way stage slot i
// then holds what g_i(x) is pulled from, as in the two-buffer step.
//
// Thread 0: queue the bulk copies of task `task` into `stage`, completing on *bar.
template <int Q, bool PERIODIC, typename ST, int AA>
__device__ void issue_task(const StepArgs &a, const SArgs &s, int task, unsigned char *stage,
                           uint64_t *bar) {
    using G = Geom<ST>;
    const int y = task / s.tasks_per_row, xs = (task - y * s.tasks_per_row) * G::W;
    const int lo = max(xs - G::H, 0), hi = min(xs + G::W + G::H, a.pitch);
    const unsigned rowb = (unsigned)(hi - lo) * (unsigned)sizeof(ST);
    const unsigned dst = (unsigned)(lo - (xs - G::H)) * (unsigned)sizeof(ST);
    const unsigned medb = (unsigned)min(G::W, a.pitch - xs) * (a.mid ? 1u : 4u);
    int ys[Q];
    unsigned total = medb;
    int y3, z3;
    row_yz<Q>(a, y, y3, z3);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        ys[i] = AA == 1 ? y : source_row<Q, PERIODIC>(a, i, y, y3, z3);
        if (ys[i] >= 0) total += rowb;
    }
    mbar_expect_tx(bar, total);
    const ST *in = static_cast<const ST *>(a.in);
#pragma unroll
    for (int i = 0; i < Q; i++)
        if (ys[i] >= 0)
            bulk_g2s(stage + i * G::ROWB + dst,
                     in + (AA == 2 ? Lat<Q>::opp(i) : i) * a.plane + (long long)ys[i] * a.pitch + lo,
                     rowb, bar);
    const long long m0 = (long long)y * a.pitch + xs;
    const void *msrc = a.mid ? static_cast<const void *>(a.mid + m0)
                             : static_cast<const void *>(a.eta2 + m0);
    bulk_g2s(stage + Stage<Q, ST>::kPops, msrc, medb, bar);  // medb <= W or 4W by form
}

// The pull of a warp for which the task's `inner` test holds: the same values as the
// general pull below, without its tests.
template <int Q, typename ST>
__device__ __forceinline__ void pull_inner(const unsigned char *stage, int tid, int lane,
                                           float (&g)[Q][Store<ST>::V]) {
    using G = Geom<ST>;
    constexpr int V = G::V;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const ST *sp = reinterpret_cast<const ST *>(stage + i * G::ROWB) + G::H + tid * V;
        float f[V];
        Store<ST>::unpackV(*reinterpret_cast<const uint4 *>(sp), f);
        if (Lat<Q>::cx(i) == 0) {
#pragma unroll
            for (int k = 0; k < V; k++) g[i][k] = f[k];
        } else if (Lat<Q>::cx(i) == 1) {  // value from x - 1: the previous lane, or staged
            float left = __shfl_up_sync(0xffffffffu, f[V - 1], 1);
            if (lane == 0) left = Store<ST>::load1(sp - 1);
            g[i][0] = left;
#pragma unroll
            for (int k = 1; k < V; k++) g[i][k] = f[k - 1];
        } else {  // value from x + 1
            float right = __shfl_down_sync(0xffffffffu, f[0], 1);
            if (lane == 31) right = Store<ST>::load1(sp + V);
#pragma unroll
            for (int k = 0; k + 1 < V; k++) g[i][k] = f[k + 1];
            g[i][V - 1] = right;
        }
    }
}

// All threads: one task from its stage.  Thread t owns sites x0 = xs + t V .. + V - 1;
// the +-1 x-shifts come from the neighbouring lane (shuffle) or, at lanes 0 / 31, from
// the staged neighbour element (the 16-byte halo at the task's ends).
template <int Q, bool MRT, bool PERIODIC, typename ST, int AA>
__device__ __forceinline__ void compute_task(const StepArgs &a, const SArgs &s, int task,
                                             const unsigned char *stage, const float *tab,
                                             float tmax[Q]) {
    using G = Geom<ST>;
    constexpr int V = G::V;
    const int tid = threadIdx.x, lane = tid & 31;
    const int y = task / s.tasks_per_row, xs = (task - y * s.tasks_per_row) * G::W;
    const int x0 = xs + tid * V;
    const bool active = x0 < a.nx;
    const ST *in = static_cast<const ST *>(a.in);
    float g[Q][V];
    // the exchange form, warp-uniform: rows y - 1 .. y + 1 exist and the warp's sites have
    // real neighbours on both sides (staged with the task or its halo), so no population is
    // absent, wrapped or past the row's end.  (The same path in the two-buffer step measured
    // 8 % slower for D2Q5 BF16: it stays on the general pull.)
    const bool inner = AA == 2 && y > 0 && y + 1 < a.ny && x0 - lane * V > 0 &&
                       x0 + (32 - lane) * V < a.nx;
    if (inner) {
        pull_inner<Q, ST>(stage, tid, lane, g);
    } else {
        int y3, z3;
        row_yz<Q>(a, y, y3, z3);
    #pragma unroll
        for (int i = 0; i < Q; i++) {
            const int cx = (AA == 1 || (AA == 0 && a.raw)) ? 0 : Lat<Q>::cx(i);
            const int ys = AA == 1 ? y : source_row<Q, PERIODIC>(a, i, y, y3, z3);
            const int pl = AA == 2 ? Lat<Q>::opp(i) : i;  // the plane staged in slot i
            const ST *sp = reinterpret_cast<const ST *>(stage + i * G::ROWB) + G::H + tid * V;
            uint4 q = make_uint4(0u, 0u, 0u, 0u);
            if (ys >= 0 && active) q = *reinterpret_cast<const uint4 *>(sp);
            float f[V];
            Store<ST>::unpackV(q, f);
            if (cx == 0) {
    #pragma unroll
                for (int k = 0; k < V; k++) g[i][k] = f[k];
            } else if (cx == 1) {  // value from x - 1
                float left = __shfl_up_sync(0xffffffffu, f[V - 1], 1);
                if (lane == 0) {
                    if (ys < 0)
                        left = 0.f;
                    else if (x0 > 0)
                        left = Store<ST>::load1(sp - 1);
                    else
                        left = PERIODIC ? Store<ST>::load1(in + pl * a.plane + (long long)ys * a.pitch +
                                                           a.nx - 1)
                                        : 0.f;
                }
                g[i][0] = left;
    #pragma unroll
                for (int k = 1; k < V; k++) g[i][k] = f[k - 1];
            } else {  // cx == -1: value from x + 1
                float right = __shfl_down_sync(0xffffffffu, f[0], 1);
                if (lane == 31) right = (ys >= 0 && x0 + V < a.nx) ? Store<ST>::load1(sp + V) : 0.f;
    #pragma unroll
                for (int k = 0; k + 1 < V; k++) g[i][k] = f[k + 1];
                g[i][V - 1] = right;
                const int last = a.nx - 1 - x0;  // the last real site's image: periodic row[0]
                if (last >= 0 && last < V) {
                    const float b = (PERIODIC && ys >= 0)
                                        ? Store<ST>::load1(in + pl * a.plane + (long long)ys * a.pitch)
                                        : 0.f;
    #pragma unroll
                    for (int j = 0; j < V; j++)
                        if (j == last) g[i][j] = b;
                }
            }
        }
    }
    if (AA != 2 && !active) return;  // no shuffles below (the exchange form's pushes have)
    float e2s[V];
    const unsigned char *mp = stage + Stage<Q, ST>::kPops;
    if (a.mid) {
        uint32_t w[V / 4];
        if (V == 4) {
            w[0] = *reinterpret_cast<const uint32_t *>(mp + tid * V);
        } else {
            const uint2 u = *reinterpret_cast<const uint2 *>(mp + tid * V);
            w[0] = u.x;
            w[V / 4 - 1] = u.y;
        }
#pragma unroll
        for (int k = 0; k < V; k++) e2s[k] = tab[(w[k >> 2] >> (8 * (k & 3))) & 0xffu];
    } else {
        const float *ep = reinterpret_cast<const float *>(mp) + tid * V;
#pragma unroll
        for (int k = 0; k < V; k += 4) {
            const float4 e = *reinterpret_cast<const float4 *>(ep + k);
            e2s[k] = e.x; e2s[k + 1] = e.y; e2s[k + 2] = e.z; e2s[k + 3] = e.w;
        }
    }
    if constexpr (AA == 0) {
        finish_sites<Q, MRT, ST>(a, g, e2s, x0, y, tmax);
    } else {  // the receivers' sums, the collision, and the in-place stores
        if (active) {
            lbaa::aa_receivers<Q, ST>(a, s.rec, g, y, x0);
            lbaa::aa_collide<Q, MRT, V>(a, g, e2s, y, x0);
        }
        ST *pop = static_cast<ST *>(a.out);  // a.in == a.out
        if constexpr (AA == 1) {  // h_i(x) into slot opp(i) at x
#pragma unroll
            for (int i = 0; i < Q; i++)
                Store<ST>::storeV(pop + Lat<Q>::opp(i) * a.plane + (long long)y * a.pitch + x0, g[i]);
        } else if (y > 0 && y + 1 < a.ny && x0 - lane * V > 0 && x0 + (32 - lane) * V < a.nx) {
            // a warp with no site on a face and no padding (warp-uniform)
#pragma unroll
            for (int i = 0; i < Q; i++)
                lbaa::push_inner<Q, ST>(pop + i * a.plane + (long long)(y + Lat<Q>::cy(i)) * a.pitch,
                                        i, g[i], x0, lane);
        } else {  // h_i(x) into slot i at x + c_i, and the ghost's zeros (all lanes)
            lbaa::exchange_stores<Q, PERIODIC, ST>(a, pop, g, y, x0, lane, active);
        }
    }
}

}  // namespace

namespace {

// D2Q5 without range scales runs a dedicated producer warp next to the eight compute warps
// (288 threads; GB300, 4096^2 BF16: 271 GLUPS against 261 with the block barrier).  The
// register-heavier forms (D2Q9, D3Q7, FP16 with its per-population scales) keep all 64 K
// registers for compute warps (256 threads): with a producer warp they lost 10-35 %.
template <int Q, typename ST> constexpr bool stream_dedicated() {
    return Q == 5 && !Scaled<ST>::value;
}
template <int Q, typename ST> constexpr int stream_threads() {
    return kSThreads + (stream_dedicated<Q, ST>() ? 32 : 0);
}

// Resident CTAs per SM the register budget is held to.
template <int Q, typename ST> constexpr int stream_min_ctas() {
    return Q == 5   ? 3
           : Q == 7 ? (sizeof(ST) == 4 ? 4 : 2)
                    : (sizeof(ST) == 4 ? 3 : 2);
}

// register cap that lets stream_min_ctas CTAs share the 64 K registers of an SM
template <int Q, typename ST> constexpr int stream_max_regs() {
    return (65536 / (stream_min_ctas<Q, ST>() * stream_threads<Q, ST>())) / 8 * 8;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait for phase `parity` of *bar that also gives up once *abort is raised.
__device__ bool mbar_wait_or_abort(uint64_t *bar, unsigned parity, volatile int *abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (global_ns() - t0 > kWaitNs) return false;
    }
    return true;
}

// fold a warp's max |output| per population into max_out (FP16 storage)
template <int Q>
__device__ __forceinline__ void fold_max(const StepArgs &a, const float (&tmax)[Q], int slot) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        float m = tmax[i];
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (lane == 0) atomicMax(a.max_out + i * kMaxCopies + slot % kMaxCopies, __float_as_uint(m));
    }
}

// Two pipelines over the same stages and per-site code.
//
// Dedicated producer (D2Q5, FP32 / BF16): warps 0-7 compute (thread t owns sites t V .. t V + V - 1 of a
// task); warp 8 lane 0 issues every copy.  Stage st carries two mbarriers: full[st]
// completes when the bulk copies of the task placed there have landed, empty[st] when all
// eight compute warps have finished reading it.  The producer refills a stage as soon as its
// empty phase completes, so the compute warps never wait for one another.
//
// Block barrier (D2Q9, D3Q7, FP16): thread 0 refills stage st after a block-wide barrier that
// follows every task; all 64 K registers stay with the compute warps.
//
// Every wait is bounded (one second); whoever gives up raises the context's fault flag (and,
// with a producer warp, the block's abort flag), the warps leave, and the issuing thread
// waits (bounded) for the copies still in flight before it returns.
template <int Q, bool MRT, bool PERIODIC, typename ST, int AA>
__global__ void __launch_bounds__((stream_threads<Q, ST>())) __maxnreg__((stream_max_regs<Q, ST>()))
    stream_step_kernel(const StepArgs a, const SArgs s) {
    constexpr bool SC = Scaled<ST>::value;
    constexpr int kWarpsPerCta = kSThreads / 32;  // compute warps
    const int S = s.stages, SB = s.stage_bytes;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kMaxStages];
    __shared__ __align__(8) uint64_t empty[kMaxStages];
    __shared__ float s_tab[kSThreads];
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31;
    pdl_trigger_and_wait();
    if ((int)blockIdx.x >= s.ncta) {  // block-uniform: receiver gather blocks
        if (tid < kSThreads)
            gather_receivers<Q, PERIODIC, ST>(a, ((int)blockIdx.x - s.ncta) * kSThreads + tid);
        return;
    }
    if (tid < kSThreads && a.mid) s_tab[tid] = a.mid_tab[tid];
    float tmax[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) tmax[i] = 0.f;

    if constexpr (stream_dedicated<Q, ST>()) {
        if (tid == kSThreads) {
            abort_flag = 0;
            for (int st = 0; st < S; st++) {
                mbar_init(&full[st], 1);
                mbar_init(&empty[st], kWarpsPerCta);
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (tid >= kSThreads) {  // producer warp: lane 0 issues every copy of this block
            if (tid != kSThreads) return;
            int k = 0;
            for (int task = blockIdx.x; task < s.ntasks; task += s.ncta, k++) {
                const int st = k % S;
                if (k >= S &&
                    !mbar_wait_or_abort(&empty[st], (unsigned)(k / S - 1) & 1u, &abort_flag)) {
                    if (!abort_flag) {
                        abort_flag = 1;
                        atomicExch(s.fault, 1u);
                    }
                    break;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_task<Q, PERIODIC, ST, AA>(a, s, task, smem + st * SB, &full[st]);
            }
            // the block must not retire with copies landing in its shared memory: wait
            // (bounded) for the last (at most S) issued tasks' copies, which the compute
            // warps also await
            for (int j = max(k - S, 0); j < k; j++) mbar_wait(&full[j % S], (unsigned)(j / S) & 1u);
            return;
        }
        int k = 0;
        for (int task = blockIdx.x; task < s.ntasks; task += s.ncta, k++) {
            const int st = k % S;
            // warp-uniform outcome: compute_task shuffles with all 32 lanes
            const bool ok = __all_sync(
                0xffffffffu, mbar_wait_or_abort(&full[st], (unsigned)(k / S) & 1u, &abort_flag));
            if (!ok) {
                if (lane == 0 && !abort_flag) {
                    abort_flag = 1;
                    atomicExch(s.fault, 1u);
                }
                return;
            }
            compute_task<Q, MRT, PERIODIC, ST, AA>(a, s, task, smem + st * SB, s_tab, tmax);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
    } else {
        if (tid == 0) {
            for (int st = 0; st < S; st++) mbar_init(&full[st], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            for (int st = 0; st < S; st++) {  // prologue: the first S tasks in flight
                const int task = (int)blockIdx.x + st * s.ncta;
                if (task < s.ntasks)
                    issue_task<Q, PERIODIC, ST, AA>(a, s, task, smem + st * SB, &full[st]);
            }
        }
        __syncthreads();
        int k = 0;
        bool failed = false;
        for (int task = blockIdx.x; task < s.ntasks; task += s.ncta, k++) {
            const int st = k % S;
            // warp-uniform outcome: compute_task shuffles with all 32 lanes
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&full[st], (unsigned)(k / S) & 1u));
            if (ok) compute_task<Q, MRT, PERIODIC, ST, AA>(a, s, task, smem + st * SB, s_tab, tmax);
            // every thread is done with stage st (and every wait succeeded) before it is refilled
            if (!__syncthreads_and(ok)) {
                failed = true;
                break;
            }
            if (tid == 0) {
                const int next = task + S * s.ncta;
                if (next < s.ntasks) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue_task<Q, PERIODIC, ST, AA>(a, s, next, smem + st * SB, &full[st]);
                }
            }
        }
        if (failed) {  // record, then wait (bounded) for this block's copies still in flight
            if (tid == 0) {
                atomicExch(s.fault, 1u);
                for (int j = 0; j < S; j++) {
                    const int kk = k + j;
                    if ((int)blockIdx.x + kk * s.ncta >= s.ntasks) break;
                    mbar_wait(&full[kk % S], (unsigned)(kk / S) & 1u);
                }
            }
            return;
        }
    }
    if (SC) fold_max<Q>(a, tmax, blockIdx.x * kWarpsPerCta + (tid >> 5));
}

using SFn = void (*)(const StepArgs, const SArgs);

// Stages per CTA: as many as the shared memory of the resident CTAs allows (2 .. kMaxStages).
int stages_for(int stage_bytes, int ctas_per_sm) {
    int dev = 0, per_sm = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    const int statics = 2048;  // barriers, medium table, abort flag (with room to spare)
    const int fit = (per_sm / ctas_per_sm - reserved - statics) / stage_bytes;
    return std::max(2, std::min(kMaxStages, fit));
}

struct SInfo {
    SFn fn = nullptr;
    int stages = 0;
    int stage_bytes = 0;
    int smem = 0;   // dynamic shared memory per CTA
    int ctas = 0;   // resident CTAs on the device
    int W = 0;      // sites per task
    int threads = 0;  // per CTA
};

template <int Q, bool MRT, bool PER, typename ST, int AA = 0> SInfo make_info(bool indexed) {
    SInfo in;
    in.fn = stream_step_kernel<Q, MRT, PER, ST, AA>;
    constexpr int kCtas = stream_min_ctas<Q, ST>();
    in.stage_bytes = Stage<Q, ST>::bytes(indexed);
    in.stages = stages_for(in.stage_bytes, kCtas);
    in.smem = in.stage_bytes * in.stages;
    in.W = Geom<ST>::W;
    in.threads = stream_threads<Q, ST>();
    int dev = 0, sms = 0, per_sm = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // the attribute belongs to the kernel, shared by both medium forms: allow the larger
    const int b1 = Stage<Q, ST>::bytes(true), b4 = Stage<Q, ST>::bytes(false);
    const int smem_max =
        std::min(smem_optin, std::max(b1 * stages_for(b1, kCtas), b4 * stages_for(b4, kCtas)));
    if (in.smem > smem_max ||
        cudaFuncSetAttribute(in.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, in.fn, in.threads, in.smem) !=
            cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
    }
    in.ctas = per_sm * sms;
    return in;
}

template <int Q, bool MRT, typename ST> SInfo info_p(bool per, bool ix) {
    return per ? make_info<Q, MRT, true, ST>(ix) : make_info<Q, MRT, false, ST>(ix);
}

template <typename ST> SInfo info_st(int Q, bool mrt, bool per, bool ix) {
    if (Q == 7) return info_p<7, false, ST>(per, ix);  // D3Q7: BGK only
    if (Q == 9) return mrt ? info_p<9, true, ST>(per, ix) : info_p<9, false, ST>(per, ix);
    return mrt ? info_p<5, true, ST>(per, ix) : info_p<5, false, ST>(per, ix);
}

// Kernel, shared memory and resident CTA count per (Q, MRT, PERIODIC, storage), measured
// once per process (one device).
const SInfo &stream_info(int Q, bool mrt, bool per, int storage, bool ix) {
    static std::mutex mu;
    static SInfo cache[3][2][2][3][2];
    static bool ready[3][2][2][3][2] = {};
    const int q = Q == 9 ? 1 : Q == 7 ? 2 : 0, m = mrt, p = per;
    const int st = storage == LB_BF16 ? 1 : storage == LB_F16 ? 2 : 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!ready[q][m][p][st][ix]) {
        cache[q][m][p][st][ix] = st == 1   ? info_st<__nv_bfloat16>(Q, mrt, per, ix)
                                 : st == 2 ? info_st<__half>(Q, mrt, per, ix)
                                           : info_st<float>(Q, mrt, per, ix);
        ready[q][m][p][st][ix] = true;
    }
    return cache[q][m][p][st][ix];
}

// The in-place forms (BF16 storage, D2Q5 / D2Q9), AA = 1 site-local, 2 exchange.
template <int AA> SInfo info_aa(int Q, bool mrt, bool per, bool ix) {
    using B = __nv_bfloat16;
    if (Q == 9)
        return mrt ? (per ? make_info<9, true, true, B, AA>(ix) : make_info<9, true, false, B, AA>(ix))
                   : (per ? make_info<9, false, true, B, AA>(ix)
                          : make_info<9, false, false, B, AA>(ix));
    return mrt ? (per ? make_info<5, true, true, B, AA>(ix) : make_info<5, true, false, B, AA>(ix))
               : (per ? make_info<5, false, true, B, AA>(ix) : make_info<5, false, false, B, AA>(ix));
}

const SInfo &stream_info_aa(int Q, bool mrt, bool per, bool ix, bool exchange) {
    static std::mutex mu;
    static SInfo cache[2][2][2][2][2];
    static bool ready[2][2][2][2][2] = {};
    const int q = Q == 9, m = mrt, p = per, x = ix, f = exchange;
    std::lock_guard<std::mutex> lk(mu);
    if (!ready[q][m][p][x][f]) {
        cache[q][m][p][x][f] = exchange ? info_aa<2>(Q, mrt, per, ix) : info_aa<1>(Q, mrt, per, ix);
        ready[q][m][p][x][f] = true;
    }
    return cache[q][m][p][x][f];
}

}  // namespace

namespace {

// Self-test of the bounded-wait failure path: one block waits for the first phase of a
// shared-memory mbarrier on which nothing arrives, with the staged step's polling, gives up
// after `ns` and raises the fault flag as the step does.
__global__ void wait_selftest_kernel(unsigned *fault, unsigned long long ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = __all_sync(0xffffffffu, mbar_wait_for(&bar, 0u, ns));
    if (!ok && threadIdx.x == 0) atomicExch(fault, 1u);
}

}  // namespace

extern "C" lb_status lb_wait_selftest(lb_ctx *ctx, int timeout_us) {
    if (!ctx) return LB_EINVAL;
    if (timeout_us < 1 || timeout_us > 1000000)
        return fail(ctx, LB_EINVAL, "timeout_us must be 1 .. 1000000");
    wait_selftest_kernel<<<1, 32, 0, ctx->stream>>>(ctx->fault,
                                                    (unsigned long long)timeout_us * 1000ull);
    return check_launch(ctx, "wait self-test");
}

lb_status stream_launch(lb_ctx *ctx, const StepArgs &a, int rec_blocks) {
    const SInfo &in = stream_info(ctx->Q, ctx->cfg.collision == LB_MRT,
                                  ctx->cfg.boundary == LB_PERIODIC, ctx->cfg.storage,
                                  a.mid != nullptr);
    if (in.ctas < 1) return fail(ctx, LB_ECUDA, "TMA-staged step: no resident CTA fits");
    SArgs s;
    s.tasks_per_row = (ctx->nx + in.W - 1) / in.W;
    s.ntasks = s.tasks_per_row * ctx->ny;
    s.ncta = std::min(s.ntasks, in.ctas);
    s.stages = in.stages;
    s.stage_bytes = in.stage_bytes;
    s.fault = ctx->fault;
    s.rec = lbaa::AaRec{nullptr, nullptr, nullptr};
    cudaError_t e = launch_pdl(in.fn, dim3(s.ncta + rec_blocks), dim3(in.threads),
                               (size_t)in.smem, ctx->stream, a, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "TMA-staged step launch");
    return LB_OK;
}

lb_status stream_launch_aa(lb_ctx *ctx, const StepArgs &a, bool exchange, const int *rec_off,
                           const int *rec_x, const int *rec_id) {
    if (ctx->cfg.storage != LB_BF16 || (ctx->Q != 5 && ctx->Q != 9))
        return fail(ctx, LB_EINVAL, "TMA-staged in-place step: D2Q5 / D2Q9 with BF16 storage");
    const SInfo &in = stream_info_aa(ctx->Q, ctx->cfg.collision == LB_MRT,
                                     ctx->cfg.boundary == LB_PERIODIC, a.mid != nullptr, exchange);
    if (in.ctas < 1) return fail(ctx, LB_ECUDA, "TMA-staged in-place step: no resident CTA fits");
    SArgs s;
    s.tasks_per_row = (ctx->nx + in.W - 1) / in.W;
    s.ntasks = s.tasks_per_row * ctx->ny;
    s.ncta = std::min(s.ntasks, in.ctas);
    s.stages = in.stages;
    s.stage_bytes = in.stage_bytes;
    s.fault = ctx->fault;
    s.rec = lbaa::AaRec{rec_off, rec_x, rec_id};
    StepArgs b = a;
    b.raw = 0;  // the form, not the raw flag, says where g(t) is read
    cudaError_t e = launch_pdl(in.fn, dim3(s.ncta), dim3(in.threads), (size_t)in.smem,
                               ctx->stream, b, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "TMA-staged in-place step launch");
    return LB_OK;
}
