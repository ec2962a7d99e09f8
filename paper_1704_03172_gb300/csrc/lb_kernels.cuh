// lb_kernels.cuh -- fused pull-stream / collide kernels for the linear LB
// acoustic scheme (arXiv:1704.03172) on sm_103a.
//
// State layout (HBM): SoA populations h[Q][ny][pitch], pitch a multiple of 32
// elements, storing the POST-collision populations of the previous step.  One
// launch of step t
//   1. pulls g_i(x, t) = h_i(x - c_i, t-1)                 (streaming, Eq. BGK-LB lhs)
//   2. forms rho, j and the linear equilibrium               (Eq. linear eqm dist)
//   3. collides (BGK, Eq. BGK-LB; or MRT, Eq. MRT-LB basic)
//   4. adds w_i S[t] at the source node                      (Eq. MRT-LB linear acoustic)
//   5. multiplies by (1 - sigma(x)) in the sponge            (Sec. 4, sponge layers)
//   6. stores h_i(x, t) in place of the other buffer.
// Receiver pressures p = c_s^2 rho at time t are gathered by trailing blocks
// of the same launch, which pull from the (read-only) input buffer.
// After lb_set_state / lb_init_pressure the buffer holds the state g(t)
// itself, unshifted ("raw"), so that every population of an arbitrary initial
// state survives at zero-ghost edges; the first launch then reads it in place.
//
// Each thread owns 4 consecutive x-sites of one row: aligned 16-byte (FP32)
// or 8-byte (16-bit) vector loads/stores; the +-1 x-shift of the moving
// populations is done with warp shuffles, and only lanes 0 / 31 issue one
// extra scalar load for the neighbouring warp's edge element.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string.h>

namespace lbk {

constexpr int kThreads = 256;            // threads per block (8 warps)
constexpr int kWarps = kThreads / 32;
constexpr int kSitesPerWarp = 128;       // 32 lanes x 4 sites
static_assert(kThreads == 256, "one medium-table entry per thread");

// Time-blocked kernels (tblock.cu forward, adjoint.cu reverse): one CTA of kTbThreads
// threads per kTbW x kTbW region (an output tile plus a K-site halo), each thread
// holding the same kTbPer sites of the region for every level.
constexpr int kTbW = 48;
constexpr int kTbNS = kTbW * kTbW;
constexpr int kTbThreads = 384;
constexpr int kTbPer = kTbNS / kTbThreads;
static_assert(kTbPer * kTbThreads == kTbNS, "region must split evenly over the threads");

__host__ __device__ __forceinline__ int wrap_mod(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// Programmatic dependent launch: a step kernel lets the next step's blocks launch at once
// (they become resident as this grid's blocks retire) and, before touching global memory,
// waits until the grid it depends on has completed and its writes are visible.  Without the
// launch attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger_and_wait() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <int Q> struct Lat;
// opp(i): the population with velocity -c_i
template <> struct Lat<5> {
    __host__ __device__ static constexpr int cx(int i) { return i == 1 ? 1 : (i == 3 ? -1 : 0); }
    __host__ __device__ static constexpr int cy(int i) { return i == 2 ? 1 : (i == 4 ? -1 : 0); }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i + 1) % 4 + 1; }
};
template <> struct Lat<9> {
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : (i < 5 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5);
    }
};
// D3Q7, the 3-D extension of D2Q5: c_0 = 0, c_1,3 = +-e_x, c_2,4 = +-e_y, c_5,6 = +-e_z
template <> struct Lat<7> {
    __host__ __device__ static constexpr int cx(int i) { return i == 1 ? 1 : (i == 3 ? -1 : 0); }
    __host__ __device__ static constexpr int cy(int i) { return i == 2 ? 1 : (i == 4 ? -1 : 0); }
    __host__ __device__ static constexpr int cz(int i) { return i == 5 ? 1 : (i == 6 ? -1 : 0); }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : (i < 5 ? (i + 1) % 4 + 1 : 11 - i);
    }
};
static_assert(Lat<5>::opp(1) == 3 && Lat<5>::opp(2) == 4 && Lat<5>::opp(3) == 1 &&
                  Lat<5>::opp(4) == 2, "D2Q5 opposites");
static_assert(Lat<9>::opp(5) == 7 && Lat<9>::opp(6) == 8 && Lat<9>::opp(7) == 5 &&
                  Lat<9>::opp(8) == 6 && Lat<9>::opp(3) == 1, "D2Q9 opposites");
static_assert(Lat<7>::opp(5) == 6 && Lat<7>::opp(6) == 5, "D3Q7 opposites");

// Arguments of one step launch (passed by value).
struct StepArgs {
    const void *in;          // h^{t-1}  [Q][ny][pitch]
    void *out;               // h^{t}
    const float *eta2;       // [ny][pitch] (c / c_ref)^2
    // 3-D grids (D3Q7): ny counts the rows of all z-planes (ny3 rows per plane, nz planes,
    // row r = z ny3 + y); 2-D grids have ny3 = ny and nz = 1
    int ny3, nz;
    // Optional medium index (nullptr: read eta2): when the map holds at most 256
    // distinct speeds, mid[y][x] selects eta^2 = mid_tab[mid] (1 byte per site
    // instead of 4); the step kernels stage mid_tab in shared memory.
    const uint8_t *mid;      // [ny][pitch]
    const float *mid_tab;    // [256]
    int nx, ny, pitch;
    long long plane;         // ny * pitch
    int segs;                // warps per row = ceil(nx / 128)
    int main_blocks;         // blocks doing sites; the rest gather receivers
    // collision
    float omega;             // BGK: 1 / tau
    float s[9];              // MRT: diagonal of S (moment order of App. A), s_k / |row_k of M|^2
    float w1r, w5r, c2r;     // D2Q9 reference weights at eta = 1, c2r = 2 w1r + 4 w5r
    float a1, a5;            // D2Q9 w_i / c_s^2 of axis / diagonal links (eta independent)
    // sponge
    int sponge_w;
    float sponge_smax, sponge_inv_w;
    // source
    const float *src_tab;    // S[n], n < src_nt (device); may be null
    int src_nt, src_x, src_y;
    long long t;             // time of the state being collided
    int raw;                 // 1: `in` holds g(t) itself (set by lb_set_state / lb_init_pressure)
    int ring;                // 1: store nothing on the outermost rows and columns (a refined
                             // patch's ghost ring, whose entering populations the coarse ->
                             // fine transfer of the same launch writes); read by the RING
                             // instances of step_sites only
    int swap;                // in-place streaming: `in` holds h(t-1) at its own site, population
                             // i in slot opp(i), so g_i(x, t) = in[opp(i)](x - c_i)
    // receivers
    const int2 *rec;
    int nrec;
    float *trace_row;        // pressure row for time t, or null
    const int *rec_col;      // column of receiver r in the trace row (nullptr: r)
    // FP16 storage: per-population power-of-two scale, value = stored * scale.
    // Three device slots rotate.  The scale of the input buffer and the one chosen
    // for the output buffer are ready before the launch; every block folds its
    // max |output| into max_out, and a one-block kernel after the step derives the
    // scale the next step will write with (scale_next, from 8 max|out| + |S[t+1]|)
    // and clears max_next for it.  All nullptr for FP32 and BF16 storage (BF16 has
    // the exponent range of FP32 and needs no range scale).
    const float *scale_in;    // [9]
    const float *scale_out;   // [9]
    unsigned *max_out;        // [9][kMaxCopies] float bits of max |value| written
    float *scale_next;        // [9]
    unsigned *max_next;       // [9][kMaxCopies]
    // Adjoint replays only: rho(x, t) of the pulled state g(t), [ny][pitch] FP32
    // (nullptr otherwise); a time-blocked launch writes step j of its K at
    // rho_out + j rho_stride.
    float *rho_out;
    long long rho_stride;
    // LB_F64 (test-only FP64 storage): eta^2 [ny][pitch], the source table S[n] and the
    // collision / sponge coefficients (order of the kCo* indices below) in FP64; nullptr
    // in every other context
    const double *eta2_64;
    const double *src64;
    const double *coef64;
    // Row slabs of one domain (domain decomposition; 2-D, FP32 / BF16 storage): this
    // context's rows are rows y_off .. y_off + ny - 1 of a grid of ny_glob rows (0: not a
    // slab), so the sponge measures distances in the whole grid.  halo_lo / halo_hi hold
    // the stored populations of the row just below / above, written by the neighbouring
    // slab's last step (the crossing populations only, [cross_slot][pitch]; nullptr: the
    // zero ghost or the periodic wrap applies there).  send_lo / send_hi receive the same
    // populations of this slab's first / last output row.
    int y_off, ny_glob;
    const void *halo_lo, *halo_hi;
    void *send_lo, *send_hi;
};

// Slot of population i in a slab halo row: its rank among the populations that cross a
// row cut in the same direction (D2Q5: g2 up, g4 down; D2Q9: g2, g5, g6 up and g4, g7, g8
// down).
template <int Q> __host__ __device__ constexpr int cross_slot(int i) {
    int k = 0;
    for (int j = 0; j < i; j++) k += Lat<Q>::cy(j) == Lat<Q>::cy(i);
    return k;
}
template <int Q> __host__ __device__ constexpr int cross_count() {
    int k = 0;
    for (int j = 0; j < Q; j++) k += Lat<Q>::cy(j) == 1;
    return k;
}

// The stored row population i pulls from for output row r of a 2-D slab when the pull
// crosses into a neighbouring slab (nullptr otherwise: the caller's own rule applies).
template <int Q, typename ST>
__device__ __forceinline__ const ST *slab_halo_row(const StepArgs &a, int r, int i) {
    if (Q == 7) return nullptr;
    const int ys = r - Lat<Q>::cy(i);
    if (ys < 0 && a.halo_lo) return static_cast<const ST *>(a.halo_lo) + cross_slot<Q>(i) * a.pitch;
    if (ys >= a.ny && a.halo_hi)
        return static_cast<const ST *>(a.halo_hi) + cross_slot<Q>(i) * a.pitch;
    return nullptr;
}

// The per-site arithmetic (collision, weights, source, sponge) is written once for an
// arithmetic type R: FP32 in every production kernel, FP64 in the test-only LB_F64 step,
// which takes its coefficients from coef64 instead of the FP32 fields.
enum : int { kCoOmega = 0, kCoS = 1, kCoW1r = 10, kCoW5r, kCoC2r, kCoA1, kCoA5, kCoSmax,
             kCoInvW, kNCo64 };
template <typename R> __device__ __forceinline__ R co(const StepArgs &a, float f, int k);
template <> __device__ __forceinline__ float co<float>(const StepArgs &, float f, int) { return f; }
template <> __device__ __forceinline__ double co<double>(const StepArgs &a, float, int k) {
    return a.coef64[k];
}
template <typename R> __device__ __forceinline__ R src_at(const StepArgs &a);
template <> __device__ __forceinline__ float src_at<float>(const StepArgs &a) {
    return a.src_tab[a.t];
}
template <> __device__ __forceinline__ double src_at<double>(const StepArgs &a) {
    return a.src64[a.t];
}

constexpr int kMaxCopies = 8;          // spread of the per-block atomicMax targets
constexpr float kStoredTarget = 8192.f; // 16-bit: |stored| <= 2^13 for the predicted bound

// smallest power of two >= r (r > 0, finite), clamped to normal floats
__host__ __device__ inline float pow2_ceil(float r) {
    if (!(r > 0.f)) return 1.f;
    unsigned b;
    memcpy(&b, &r, 4);
    int e = (int)((b >> 23) & 0xffu);
    if (b & 0x7fffffu) e += 1;
    if (e < 1) e = 1;
    if (e > 254) e = 254;
    unsigned o = (unsigned)e << 23;
    float f;
    memcpy(&f, &o, 4);
    return f;
}

__device__ __forceinline__ float scale_of(const float *scale, int i) {
    return scale ? scale[i] : 1.f;
}

// ---------------------------------------------------------------- storage --
template <typename ST> struct Store;

// Every storage type moves one 16-byte vector per thread and population:
// V = 4 FP32 sites or V = 8 sites of a 16-bit type.
template <> struct Store<float> {
    static constexpr int kBytes = 4;
    static constexpr int V = 4;
    __device__ static __forceinline__ void loadV(const float *p, float (&v)[V]) {
        float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    __device__ static __forceinline__ void storeV(float *p, const float (&v)[V]) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __device__ static __forceinline__ float load1(const float *p) { return *p; }
    __device__ static __forceinline__ void store1(float *p, float v) { *p = v; }
    // raw forms for the two-phase pull: 16-byte vector and one element as bits
    __device__ static __forceinline__ uint32_t bits1(const float *p) {
        return __float_as_uint(*p);
    }
    __device__ static __forceinline__ float unbits1(uint32_t b) { return __uint_as_float(b); }
    __device__ static __forceinline__ void unpackV(const uint4 &u, float (&v)[V]) {
        v[0] = __uint_as_float(u.x); v[1] = __uint_as_float(u.y);
        v[2] = __uint_as_float(u.z); v[3] = __uint_as_float(u.w);
    }
};

template <> struct Store<__nv_bfloat16> {
    static constexpr int kBytes = 2;
    static constexpr int V = 8;
    __device__ static __forceinline__ void loadV(const __nv_bfloat16 *p, float (&v)[V]) {
        uint4 u = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&w[k]);
            float2 f = __bfloat1622float2(h);
            v[2 * k] = f.x;
            v[2 * k + 1] = f.y;
        }
    }
    __device__ static __forceinline__ void storeV(__nv_bfloat16 *p, const float (&v)[V]) {
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
            w[k] = *reinterpret_cast<uint32_t *>(&h);
        }
        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __device__ static __forceinline__ float load1(const __nv_bfloat16 *p) {
        return __bfloat162float(*p);
    }
    __device__ static __forceinline__ void store1(__nv_bfloat16 *p, float v) {
        *p = __float2bfloat16_rn(v);
    }
    __device__ static __forceinline__ uint32_t bits1(const __nv_bfloat16 *p) {
        return *reinterpret_cast<const unsigned short *>(p);
    }
    __device__ static __forceinline__ float unbits1(uint32_t b) {
        return __uint_as_float(b << 16);  // BF16 is the upper half of an FP32
    }
    __device__ static __forceinline__ void unpackV(const uint4 &u, float (&v)[V]) {
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            v[2 * k] = __uint_as_float(w[k] << 16);
            v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
};

template <> struct Store<__half> {
    static constexpr int kBytes = 2;
    static constexpr int V = 8;
    __device__ static __forceinline__ void loadV(const __half *p, float (&v)[V]) {
        uint4 u = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            __half2 h = *reinterpret_cast<const __half2 *>(&w[k]);
            float2 f = __half22float2(h);
            v[2 * k] = f.x;
            v[2 * k + 1] = f.y;
        }
    }
    __device__ static __forceinline__ void storeV(__half *p, const float (&v)[V]) {
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            __half2 h = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
            w[k] = *reinterpret_cast<uint32_t *>(&h);
        }
        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __device__ static __forceinline__ float load1(const __half *p) { return __half2float(*p); }
    __device__ static __forceinline__ void store1(__half *p, float v) { *p = __float2half_rn(v); }
    __device__ static __forceinline__ uint32_t bits1(const __half *p) {
        return *reinterpret_cast<const unsigned short *>(p);
    }
    __device__ static __forceinline__ float unbits1(uint32_t b) {
        return __half2float(__ushort_as_half((unsigned short)b));
    }
    __device__ static __forceinline__ void unpackV(const uint4 &u, float (&v)[V]) {
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[k]));
            v[2 * k] = f.x;
            v[2 * k + 1] = f.y;
        }
    }
};

// ------------------------------------------------------------------ pulls --
// Pull one population's V values for sites x0..x0+V-1 of this thread's row
// from source row `row` (nullptr: the row lies outside a zero-ghost domain).
// CX is the population's x velocity: the value at site x comes from x - CX.
// Must be called by all 32 lanes of the warp (shuffles).
template <int CX, bool PERIODIC, typename ST>
__device__ __forceinline__ void pullV(const ST *row, int x0, int lane, int nx, bool active,
                                      float scale, float (&v)[Store<ST>::V]) {
    constexpr int V = Store<ST>::V;
    if (row == nullptr) {  // warp-uniform
#pragma unroll
        for (int k = 0; k < V; k++) v[k] = 0.f;
        return;
    }
    float q[V];
    if (active) {
        Store<ST>::loadV(row + x0, q);
    } else {
#pragma unroll
        for (int k = 0; k < V; k++) q[k] = 0.f;
    }
    if (CX == 0) {
#pragma unroll
        for (int k = 0; k < V; k++) v[k] = q[k];
    } else if (CX == 1) {  // value from x - 1
        float left = __shfl_up_sync(0xffffffffu, q[V - 1], 1);
        if (lane == 0) left = (x0 > 0) ? Store<ST>::load1(row + x0 - 1) : 0.f;
        v[0] = left;
#pragma unroll
        for (int k = 1; k < V; k++) v[k] = q[k - 1];
        if (x0 == 0) v[0] = PERIODIC ? Store<ST>::load1(row + nx - 1) : 0.f;
    } else {  // CX == -1: value from x + 1
        float right = __shfl_down_sync(0xffffffffu, q[0], 1);
        if (lane == 31) right = (x0 + V < nx) ? Store<ST>::load1(row + x0 + V) : 0.f;
#pragma unroll
        for (int k = 0; k + 1 < V; k++) v[k] = q[k + 1];
        v[V - 1] = right;
        const int last = nx - 1 - x0;  // local index of the last real site, if in this vector
        if (last >= 0 && last < V) {
            const float b = PERIODIC ? Store<ST>::load1(row) : 0.f;
#pragma unroll
            for (int j = 0; j < V; j++)
                if (j == last) v[j] = b;
        }
    }
    if (scale != 1.f) {
#pragma unroll
        for (int k = 0; k < V; k++) v[k] *= scale;
    }
}

// Two-phase form of pullV for kernels that pull several populations: phase 1
// issues, for every population, the 16-byte vector load and ONE unconditional
// scalar load (lane 0 / 31: the neighbouring warp's edge element, or the
// periodic wrap element; every other lane: the row's first element, a
// broadcast), so that all of a thread's loads are in flight together; phase 2
// shuffles and assembles.  Same values as pullV.
template <int CX, bool PERIODIC, typename ST>
__device__ __forceinline__ void pull_issue(const ST *row, int x0, int lane, int nx, bool active,
                                           uint4 &q, uint32_t &e) {
    constexpr int V = Store<ST>::V;
    q = make_uint4(0u, 0u, 0u, 0u);
    e = 0u;
    if (row == nullptr) return;  // warp-uniform
    if (active) q = *reinterpret_cast<const uint4 *>(row + x0);
    if (CX == 1) {  // lane 0 needs x0 - 1 (or, at x0 == 0, the periodic image nx - 1)
        const ST *ep = row;
        if (lane == 0 && x0 > 0) ep = row + x0 - 1;
        if (PERIODIC && lane == 0 && x0 == 0) ep = row + nx - 1;
        e = Store<ST>::bits1(ep);
    } else if (CX == -1) {  // lane 31 needs x0 + V; the last real site's periodic image is row[0]
        const ST *ep = row;
        if (lane == 31 && x0 + V < nx) ep = row + x0 + V;
        e = Store<ST>::bits1(ep);
    }
}

template <int CX, bool PERIODIC, typename ST>
__device__ __forceinline__ void pull_finish(bool row_null, int x0, int lane, int nx,
                                            const uint4 &q, uint32_t e,
                                            float (&v)[Store<ST>::V]) {
    constexpr int V = Store<ST>::V;
    float f[V];
    Store<ST>::unpackV(q, f);  // zeros for an absent row or an inactive lane
    if (CX == 0) {
#pragma unroll
        for (int k = 0; k < V; k++) v[k] = f[k];
        return;
    }
    const float eb = row_null ? 0.f : Store<ST>::unbits1(e);
    if (CX == 1) {  // value from x - 1
        float left = __shfl_up_sync(0xffffffffu, f[V - 1], 1);
        if (lane == 0) left = (x0 > 0 || PERIODIC) ? eb : 0.f;
        v[0] = left;
#pragma unroll
        for (int k = 1; k < V; k++) v[k] = f[k - 1];
    } else {  // CX == -1: value from x + 1
        float right = __shfl_down_sync(0xffffffffu, f[0], 1);
        if (lane == 31) right = (x0 + V < nx) ? eb : 0.f;
#pragma unroll
        for (int k = 0; k + 1 < V; k++) v[k] = f[k + 1];
        v[V - 1] = right;
        const int last = nx - 1 - x0;  // local index of the last real site, if in this vector
        if (last >= 0 && last < V) {
            const float b = PERIODIC ? eb : 0.f;
#pragma unroll
            for (int j = 0; j < V; j++)
                if (j == last) v[j] = b;
        }
    }
}

template <bool PERIODIC, typename ST>
__device__ __forceinline__ const ST *src_row(const ST *base, int ys, int ny, int pitch) {
    if (ys < 0 || ys >= ny) {
        if (!PERIODIC) return nullptr;
        ys = ys < 0 ? ys + ny : ys - ny;
    }
    return base + (long long)ys * pitch;
}

// Source row of population i for output row r: the pull's y shift (2-D, row = y) or its
// y and z shifts (D3Q7, r = z ny3 + y3, with y3 and z given); -1 outside a zero-ghost
// domain.
template <int Q, bool PERIODIC>
__device__ __forceinline__ int pull_row_yz(const StepArgs &a, int r, int y, int z, int i) {
    if (Q != 7) {
        int ys = r - Lat<Q>::cy(i);
        if (ys < 0 || ys >= a.ny) {
            if (!PERIODIC) return -1;
            ys = ys < 0 ? ys + a.ny : ys - a.ny;
        }
        return ys;
    }
    int ys = y - Lat<Q>::cy(i), zs = z - Lat<Q>::cz(i);
    if (ys < 0 || ys >= a.ny3) {
        if (!PERIODIC) return -1;
        ys = ys < 0 ? ys + a.ny3 : ys - a.ny3;
    }
    if (zs < 0 || zs >= a.nz) {
        if (!PERIODIC) return -1;
        zs = zs < 0 ? zs + a.nz : zs - a.nz;
    }
    return zs * a.ny3 + ys;
}

// (y3, z) of row r of a D3Q7 grid (r itself and 0 for 2-D grids)
template <int Q>
__device__ __forceinline__ void row_yz(const StepArgs &a, int r, int &y, int &z) {
    if (Q != 7) {
        y = r;
        z = 0;
        return;
    }
    z = r / a.ny3;
    y = r - z * a.ny3;
}

template <int Q, bool PERIODIC>
__device__ __forceinline__ int pull_row(const StepArgs &a, int r, int i) {
    int y, z;
    row_yz<Q>(a, r, y, z);
    return pull_row_yz<Q, PERIODIC>(a, r, y, z, i);
}

// ------------------------------------------------------------- collision --
// D2Q5: w_0 = 1 - eta^2, w_1..4 = eta^2 / 4, c_s^2 = eta^2 / 2, so
// g^eq_0 = w_0 rho, g^eq_{1,3} = w_1 rho +- j_x / 2, g^eq_{2,4} = w_1 rho +- j_y / 2.
// g^eq_0 is formed as rho - 4 w_1 rho (= w_0 rho): the equilibrium then carries the mass
// rho up to one unbiased rounding, where fl(1 - eta^2) + eta^2 != 1 would make every
// BGK collision create mass in a fixed ratio that a lossless run keeps forever.
template <bool MRT, typename R>
__device__ __forceinline__ void collide5(R g[5], R e2, const StepArgs &a) {
    const R rho = g[0] + g[1] + g[2] + g[3] + g[4];
    const R jx = g[1] - g[3], jy = g[2] - g[4];
    const R w1 = R(0.25) * e2;
    if (!MRT) {
        const R om = co<R>(a, a.omega, kCoOmega);
        const R b = w1 * rho, eq0 = rho - R(4) * b;
        g[0] += om * (eq0 - g[0]);
        g[1] += om * (b + R(0.5) * jx - g[1]);
        g[2] += om * (b + R(0.5) * jy - g[2]);
        g[3] += om * (b - R(0.5) * jx - g[3]);
        g[4] += om * (b - R(0.5) * jy - g[4]);
    } else {
        // Only e and p_xx are not conserved.  e = -4 g0 + sum_{1..4} g = rho - 5 g0,
        // e^eq = (-4 + 10 c_s^2) rho (Eq. higher moments e), p_xx^eq = 0.
        // g* = g - M^-1 S (m - m^eq), M^-1 = M^T diag(1/5, 1/2, 1/2, 1/20, 1/4).
        const R e_neq = (rho - R(5) * g[0]) - (R(-4) + R(5) * e2) * rho;
        const R pxx = g[1] - g[2] + g[3] - g[4];
        const R de = co<R>(a, a.s[3], kCoS + 3) * e_neq;  // s_e / 20 (rates come normalised)
        const R dp = co<R>(a, a.s[4], kCoS + 4) * pxx;    // s_p / 4
        g[0] += R(4) * de;
        g[1] -= de + dp;
        g[2] -= de - dp;
        g[3] -= de + dp;
        g[4] -= de - dp;
    }
}

// BGK with tau = 1/2 (omega = 2, the paper's lossless choice): g* = 2 g^eq - g, with g^eq
// formed as in collide5.  One fused multiply-add per population instead of three
// operations; the same values up to rounding.
template <typename R>
__device__ __forceinline__ void collide5_lossless(R g[5], R e2) {
    const R rho = g[0] + g[1] + g[2] + g[3] + g[4];
    const R jx = g[1] - g[3], jy = g[2] - g[4];
    const R b = R(0.25) * e2 * rho, eq0 = rho - R(4) * b;
    g[0] = fma(R(2), eq0, -g[0]);
    g[1] = fma(R(2), fma(R(0.5), jx, b), -g[1]);
    g[2] = fma(R(2), fma(R(0.5), jy, b), -g[2]);
    g[3] = fma(R(2), fma(R(-0.5), jx, b), -g[3]);
    g[4] = fma(R(2), fma(R(-0.5), jy, b), -g[4]);
}

// D2Q9 with the eta^2-scaled weights: w_{1..4} = eta^2 w1r, w_{5..8} = eta^2 w5r,
// c_s^2 = eta^2 c2r, so w_i / c_s^2 = a1 or a5 does not depend on eta.
template <bool MRT, typename R>
__device__ __forceinline__ void collide9(R g[9], R e2, const StepArgs &a) {
    if constexpr (!MRT) {
        const R rho = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6] + g[7] + g[8];
        const R jx = g[1] - g[3] + g[5] - g[6] - g[7] + g[8];
        const R jy = g[2] - g[4] + g[5] + g[6] - g[7] - g[8];
        const R w1 = e2 * co<R>(a, a.w1r, kCoW1r), w5 = e2 * co<R>(a, a.w5r, kCoW5r);
        R eq[9];
        const R b1 = w1 * rho, b5 = w5 * rho;
        eq[0] = rho - R(4) * (b1 + b5);  // = w_0 rho, mass-exact as in collide5
        const R ux = co<R>(a, a.a1, kCoA1) * jx, uy = co<R>(a, a.a1, kCoA1) * jy;
        eq[1] = b1 + ux; eq[3] = b1 - ux;
        eq[2] = b1 + uy; eq[4] = b1 - uy;
        const R a5 = co<R>(a, a.a5, kCoA5);
        const R dp = a5 * (jx + jy), dm = a5 * (jx - jy);
        eq[5] = b5 + dp; eq[7] = b5 - dp;
        eq[6] = b5 - dm; eq[8] = b5 + dm;
#pragma unroll
        for (int i = 0; i < 9; i++) g[i] += co<R>(a, a.omega, kCoOmega) * (eq[i] - g[i]);
    } else {
        // The non-conserved moments of g - g^eq (rows 3..8 of M, App. A) straight from g.
        // With b1 = w_1 rho, b5 = w_5 rho and the equilibrium above, the moments of g^eq are
        //   e^eq = -4 rho + 12 b1 + 24 b5,   eps^eq = 4 rho - 24 b1 - 12 b5,
        //   q_x^eq = 4 (a5 - a1) j_x,  q_y^eq = 4 (a5 - a1) j_y,  p_xx^eq = p_xy^eq = 0,
        // and with rho = g_0 + s14 + s58 the g_0 terms cancel:
        //   e - e^eq = 3 s14 + 6 s58 - (12 w1r + 24 w5r) eta^2 rho,
        //   eps - eps^eq = (24 w1r + 12 w5r) eta^2 rho - 6 s14 - 3 s58,
        //   q_x - q_x^eq = -2 X1 + X5 - 4 (a5 - a1) (X1 + X5), with j_x = X1 + X5 (q_y alike).
        const R A = g[1] + g[3], B = g[2] + g[4], C = g[5] + g[7], D = g[6] + g[8];
        const R s14 = A + B, s58 = C + D;
        const R re2 = (g[0] + s14 + s58) * e2;
        const R w1r = co<R>(a, a.w1r, kCoW1r), w5r = co<R>(a, a.w5r, kCoW5r);
        const R kq = R(4) * (co<R>(a, a.a5, kCoA5) - co<R>(a, a.a1, kCoA1));
        const R X1 = g[1] - g[3], Y1 = g[2] - g[4];
        const R u = g[5] - g[7], v = g[6] - g[8];
        const R X5 = u - v, Y5 = u + v;
        // rates arrive divided by the squared row norms: 36, 4, 36, 12, 12, 4
        const R d3 = co<R>(a, a.s[3], kCoS + 3) *
                     (R(3) * s14 + R(6) * s58 - (R(12) * w1r + R(24) * w5r) * re2);
        const R d4 = co<R>(a, a.s[4], kCoS + 4) * (A - B);
        const R d5 = co<R>(a, a.s[5], kCoS + 5) *
                     ((R(24) * w1r + R(12) * w5r) * re2 - R(6) * s14 - R(3) * s58);
        const R d6 = co<R>(a, a.s[6], kCoS + 6) * ((-R(2) - kq) * X1 + (R(1) - kq) * X5);
        const R d7 = co<R>(a, a.s[7], kCoS + 7) * ((-R(2) - kq) * Y1 + (R(1) - kq) * Y5);
        const R d8 = co<R>(a, a.s[8], kCoS + 8) * (C - D);
        // g* = g - M^T (d3..d8)
        g[0] -= -R(4) * d3 + R(4) * d5;
        g[1] -= -d3 + d4 - R(2) * d5 - R(2) * d6;
        g[2] -= -d3 - d4 - R(2) * d5 - R(2) * d7;
        g[3] -= -d3 + d4 - R(2) * d5 + R(2) * d6;
        g[4] -= -d3 - d4 - R(2) * d5 + R(2) * d7;
        const R c5 = R(2) * d3 + d5;
        g[5] -= c5 + d6 + d7 + d8;
        g[6] -= c5 - d6 + d7 - d8;
        g[7] -= c5 - d6 - d7 + d8;
        g[8] -= c5 + d6 - d7 - d8;
    }
}

// D3Q7 BGK with w_0 = 1 - eta^2, w_1..6 = eta^2 / 6, c_s^2 = eta^2 / 3 (the D2Q5 rule of
// Eq. 0th lattice weight carried to three dimensions), so w_i / c_s^2 = 1/2 and
// g^eq_{1,3} = w_1 rho +- j_x / 2, g^eq_{2,4} = w_1 rho +- j_y / 2, g^eq_{5,6} = w_1 rho +- j_z / 2.
template <typename R>
__device__ __forceinline__ void collide7(R g[7], R e2, const StepArgs &a) {
    const R rho = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6];
    const R jx = g[1] - g[3], jy = g[2] - g[4], jz = g[5] - g[6];
    const R om = co<R>(a, a.omega, kCoOmega), b = e2 * (R(1) / R(6)) * rho,
            eq0 = rho - R(6) * b;  // = (1 - eta^2) rho, mass-exact as in collide5
    g[0] += om * (eq0 - g[0]);
    g[1] += om * (b + R(0.5) * jx - g[1]);
    g[2] += om * (b + R(0.5) * jy - g[2]);
    g[3] += om * (b - R(0.5) * jx - g[3]);
    g[4] += om * (b - R(0.5) * jy - g[4]);
    g[5] += om * (b + R(0.5) * jz - g[5]);
    g[6] += om * (b - R(0.5) * jz - g[6]);
}

template <int Q, typename R>
__device__ __forceinline__ R weight_i(int i, R e2, const StepArgs &a) {
    if (Q == 5) return i == 0 ? R(1) - e2 : R(0.25) * e2;
    if (Q == 7) return i == 0 ? R(1) - e2 : e2 * (R(1) / R(6));  // D3Q7: w_0 = 1 - eta^2
    const R w1r = co<R>(a, a.w1r, kCoW1r), w5r = co<R>(a, a.w5r, kCoW5r);
    if (i == 0) return R(1) - R(4) * e2 * (w1r + w5r);
    return i < 5 ? e2 * w1r : e2 * w5r;
}

template <int Q, typename R>
__device__ __forceinline__ R cs2_of(R e2, const StepArgs &a) {
    return Q == 5 ? R(0.5) * e2 : (Q == 7 ? e2 * (R(1) / R(3)) : e2 * co<R>(a, a.c2r, kCoC2r));
}

__device__ __forceinline__ float sponge_factor(int x, int y, const StepArgs &a) {
    int d = min(min(x, a.nx - 1 - x), min(y, a.ny - 1 - y));
    if (d >= a.sponge_w) return 1.f;
    float r = (float)(a.sponge_w - d) * a.sponge_inv_w;
    return 1.f - a.sponge_smax * r * r;
}

// sponge factor at distance d from the nearest face
template <typename R = float>
__device__ __forceinline__ R sponge_of_dist(int d, const StepArgs &a) {
    if (d >= a.sponge_w) return R(1);
    const R q = (R)(a.sponge_w - d) * co<R>(a, a.sponge_inv_w, kCoInvW);
    return R(1) - co<R>(a, a.sponge_smax, kCoSmax) * q * q;
}

// distance from row r to the nearest y face (D3Q7: y or z face)
template <int Q>
__device__ __forceinline__ int row_face_dist(int r, const StepArgs &a) {
    if (Q != 7) {  // slabs: the distance in the whole grid
        const int yg = r + a.y_off, nyg = a.ny_glob > 0 ? a.ny_glob : a.ny;
        return min(yg, nyg - 1 - yg);
    }
    int y, z;
    row_yz<Q>(a, r, y, z);
    return min(min(y, a.ny3 - 1 - y), min(z, a.nz - 1 - z));
}

// sponge factor at row r (D3Q7: distance to the nearest of the six faces)
template <int Q>
__device__ __forceinline__ float sponge_at(int x, int r, const StepArgs &a) {
    return sponge_of_dist(min(min(x, a.nx - 1 - x), row_face_dist<Q>(r, a)), a);
}

// --------------------------------------------------------------- receivers --
template <int Q, bool PERIODIC, typename ST>
__device__ __forceinline__ void gather_receivers(const StepArgs &a, int r) {
    if (r >= a.nrec || a.trace_row == nullptr) return;
    const int2 xy = a.rec[r];
    const ST *in = static_cast<const ST *>(a.in);
    float rho = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        int xs = xy.x - (a.raw ? 0 : Lat<Q>::cx(i));
        const int ys = a.raw ? xy.y : pull_row<Q, PERIODIC>(a, xy.y, i);  // xy.y: row
        const ST *halo = a.raw ? nullptr : slab_halo_row<Q, ST>(a, xy.y, i);
        if (PERIODIC) {
            xs = (xs + a.nx) % a.nx;
        } else if (xs < 0 || xs >= a.nx || (ys < 0 && !halo)) {
            continue;
        }
        rho += Store<ST>::load1(halo ? halo + xs : in + i * a.plane + (long long)ys * a.pitch + xs) *
               scale_of(a.scale_in, i);
    }
    a.trace_row[a.rec_col ? a.rec_col[r] : r] =
        cs2_of<Q>(a.eta2[(long long)xy.y * a.pitch + xy.x], a) * rho;
}

// -------------------------------------------------------------------- step --
// FP16 keeps a per-population scale; BF16 (FP32's exponent range) and FP32 do not.
template <typename ST> struct Scaled {
    static constexpr bool value = false;
};
template <> struct Scaled<__half> {
    static constexpr bool value = true;
};

// Scale that keeps the predicted bound |out| <= 8 max|in| + |S| at or below
// kStoredTarget (8x headroom again before FP16 overflows); `keep` if the bound is 0.
__device__ __forceinline__ float next_scale(float maxval, float S, float keep) {
    const float bound = 8.f * maxval + S;
    return bound > 0.f ? pow2_ceil(bound * (1.f / kStoredTarget)) : keep;
}

// Collision, source and sponge for a thread's V sites, in place.  EDGE: some site of
// the warp lies in the sponge or beyond the last column (damped / zeroed per site; dyz is
// the row's distance to the nearest y / z face).
// LOSSLESS: D2Q5 BGK with omega = 2 (collide5_lossless); the caller tests a.omega once.
template <int Q, bool MRT, int V, bool EDGE, typename R, bool LOSSLESS = false>
__device__ __forceinline__ void collide_sites(R (&g)[Q][V], const R (&e2s)[V],
                                              const StepArgs &a, int x0, int dyz, bool has_src) {
#pragma unroll
    for (int k = 0; k < V; k++) {
        R gs[Q];
#pragma unroll
        for (int i = 0; i < Q; i++) gs[i] = g[i][k];
        if (Q == 5 && LOSSLESS)
            collide5_lossless(gs, e2s[k]);
        else if (Q == 5)
            collide5<MRT>(gs, e2s[k], a);
        else if (Q == 9)
            collide9<MRT>(gs, e2s[k], a);
        else
            collide7(gs, e2s[k], a);
        if (has_src && a.src_x == x0 + k) {
            const R S = src_at<R>(a);
#pragma unroll
            for (int i = 0; i < Q; i++) gs[i] += weight_i<Q>(i, e2s[k], a) * S;
        }
        if (EDGE) {
            const int x = x0 + k;
            const R f =
                a.sponge_w > 0 ? sponge_of_dist<R>(min(min(x, a.nx - 1 - x), dyz), a) : R(1);
            const bool real = x0 + k < a.nx;
#pragma unroll
            for (int i = 0; i < Q; i++) g[i][k] = real ? gs[i] * f : R(0);
        } else {
#pragma unroll
            for (int i = 0; i < Q; i++) g[i][k] = gs[i];
        }
    }
}

// collide_sites with the damping variant (edge) and the lossless form chosen once per call.
template <int Q, bool MRT, int V, typename R>
__device__ __forceinline__ void collide_sites_any(R (&g)[Q][V], const R (&e2s)[V],
                                                  const StepArgs &a, int x0, int dyz, bool has_src,
                                                  bool edge) {
    if (!MRT && Q == 5 && a.omega == 2.f) {  // uniform
        if (!edge)
            collide_sites<Q, MRT, V, false, R, true>(g, e2s, a, x0, dyz, has_src);
        else
            collide_sites<Q, MRT, V, true, R, true>(g, e2s, a, x0, dyz, has_src);
    } else {
        if (!edge)
            collide_sites<Q, MRT, V, false, R>(g, e2s, a, x0, dyz, has_src);
        else
            collide_sites<Q, MRT, V, true, R>(g, e2s, a, x0, dyz, has_src);
    }
}

// Everything after the pulls, for a thread's V sites at (x0..x0+V-1, y): FP16
// input scale, the adjoint replay's rho record, collision + source + sponge, and
// the vector store of h(t) (FP16: scaled, with this thread's max |h_i| folded
// into tmax).  Shared by the register-streaming and the TMA-staged kernels.
template <int Q, bool MRT, typename ST, bool SLAB = false, bool RING = false>
__device__ __forceinline__ void finish_sites(const StepArgs &a, float (&g)[Q][Store<ST>::V],
                                             const float (&e2s)[Store<ST>::V], int x0, int y,
                                             float tmax[Q]) {
    constexpr bool SC = Scaled<ST>::value;
    constexpr int V = Store<ST>::V;
    if (SC) {  // one scale per population: applied after the shuffles
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const float sc = a.scale_in[i];
#pragma unroll
            for (int k = 0; k < V; k++) g[i][k] *= sc;
        }
    }

    if (a.rho_out) {  // warp-uniform: adjoint replay records rho(t)
#pragma unroll
        for (int k = 0; k < V; k += 4) {
            float r[4];
#pragma unroll
            for (int m = 0; m < 4; m++) {
                r[m] = 0.f;
#pragma unroll
                for (int i = 0; i < Q; i++) r[m] += g[i][k + m];
            }
            *reinterpret_cast<float4 *>(a.rho_out + (long long)y * a.pitch + x0 + k) =
                make_float4(r[0], r[1], r[2], r[3]);
        }
    }
    // row y (D3Q7: z ny3 + y3): its distance to the nearest y / z face
    const int dyz = row_face_dist<Q>(y, a);
    bool edge = (a.sponge_w > 0 && (dyz < a.sponge_w || x0 < a.sponge_w ||
                                    x0 + V - 1 >= a.nx - a.sponge_w)) ||
                x0 + V > a.nx;
    // one path per warp: on narrow rows (a 256-wide 3-D grid) every warp holds sponge
    // columns, and per-lane paths would run both variants; for sites outside the sponge
    // the EDGE variant gives the same values
    edge = __any_sync(__activemask(), edge);
    const bool has_src = (y == a.src_y) && (a.src_x >= x0) && (a.src_x < x0 + V) &&
                         a.src_tab != nullptr && a.t < a.src_nt;
    // collide site by site, in place: g[i][k] becomes the stored output.  Warps whose
    // sites are all real and outside the sponge (almost all) skip damping and masking.
    collide_sites_any<Q, MRT, V>(g, e2s, a, x0, dyz, has_src, edge);
    ST *o = static_cast<ST *>(a.out) + (long long)y * a.pitch + x0;
    // RING: the instance that honours StepArgs::ring (refined fine steps only; the test
    // costs the register-heavy 16-bit forms up to 15 %)
    const bool ring_row = RING && a.ring && (y == 0 || y == a.ny - 1);  // warp-uniform
    const bool ring_col = RING && a.ring && (x0 == 0 || x0 + V >= a.nx);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        if (SC) {
            const float inv = 1.f / a.scale_out[i];  // exact: a power of two
            float m = 0.f;
#pragma unroll
            for (int k = 0; k < V; k++) {
                m = fmaxf(m, fabsf(g[i][k]));
                g[i][k] *= inv;
            }
            tmax[i] = fmaxf(tmax[i], m);
        }
        if (ring_row) continue;
        if (!ring_col) {
            Store<ST>::storeV(o + i * a.plane, g[i]);
        } else {  // all but the first and last column
#pragma unroll
            for (int k = 0; k < V; k++)
                if (x0 + k >= 1 && x0 + k < a.nx - 1) Store<ST>::store1(o + i * a.plane + k, g[i][k]);
        }
    }
    if (SLAB && Q != 7 && ((a.send_lo && y == 0) || (a.send_hi && y == a.ny - 1))) {
        // slab cut rows: the populations the neighbouring slab pulls across the cut
#pragma unroll
        for (int i = 0; i < Q; i++) {
            if (Lat<Q>::cy(i) == -1 && a.send_lo && y == 0)
                Store<ST>::storeV(static_cast<ST *>(a.send_lo) + cross_slot<Q>(i) * a.pitch + x0, g[i]);
            if (Lat<Q>::cy(i) == 1 && a.send_hi && y == a.ny - 1)
                Store<ST>::storeV(static_cast<ST *>(a.send_hi) + cross_slot<Q>(i) * a.pitch + x0, g[i]);
        }
    }
}

// The sites of one warp row-segment of block `blk`; tmax receives this
// thread's max |out_i|.  SLAB: the context is a row slab (halo rows at the cuts).
template <int Q, bool MRT, bool PERIODIC, typename ST, bool SLAB = false, bool RING = false>
__device__ __forceinline__ void step_sites(const StepArgs &a, int blk, float tmax[Q],
                                           const float *tab) {
#pragma unroll
    for (int i = 0; i < Q; i++) tmax[i] = 0.f;
    const int lane = threadIdx.x & 31;
    const int wid = blk * kWarps + (threadIdx.x >> 5);
    const int y = wid / a.segs;
    if (y >= a.ny) return;  // warp-uniform
    constexpr int V = Store<ST>::V;
    const int x0 = (wid - y * a.segs) * (32 * V) + lane * V;
    const bool active = x0 < a.nx;
    const ST *in = static_cast<const ST *>(a.in);

    // phase 1: every population's loads in flight together
    uint4 q[Q];
    uint32_t e[Q];
    bool absent[Q];
    int y3, z3;
    row_yz<Q>(a, y, y3, z3);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int cx = a.raw ? 0 : Lat<Q>::cx(i);  // raw: read g(t) in place (warp-uniform)
        const int rs = a.raw ? y : pull_row_yz<Q, PERIODIC>(a, y, y3, z3, i);
        const ST *row = rs < 0 ? nullptr : in + i * a.plane + (long long)rs * a.pitch;
        if (SLAB && !a.raw) {  // a pull across a slab cut reads the neighbour's row
            const ST *halo = slab_halo_row<Q, ST>(a, y, i);
            if (halo) row = halo;
        }
        absent[i] = row == nullptr;
        if (cx == 1)
            pull_issue<1, PERIODIC>(row, x0, lane, a.nx, active, q[i], e[i]);
        else if (cx == -1)
            pull_issue<-1, PERIODIC>(row, x0, lane, a.nx, active, q[i], e[i]);
        else
            pull_issue<0, PERIODIC>(row, x0, lane, a.nx, active, q[i], e[i]);
    }
    // the medium (index words or eta^2), loaded with the populations so that a warp waits
    // on memory once (D2Q9 loads it after the pull: its 72 values leave no registers to hold
    // it across)
    constexpr bool kMedEarly = Q != 9;
    float med[V];
    if (kMedEarly && active) {
        const long long mo = (long long)y * a.pitch + x0;
        if (a.mid) {  // warp-uniform: 1-byte medium index
            if (V == 4) {
                med[0] = __uint_as_float(*reinterpret_cast<const uint32_t *>(a.mid + mo));
            } else {
                const uint2 u = *reinterpret_cast<const uint2 *>(a.mid + mo);
                med[0] = __uint_as_float(u.x);
                med[V / 4 - 1] = __uint_as_float(u.y);
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k += 4) {
                const float4 e = *reinterpret_cast<const float4 *>(a.eta2 + mo + k);
                med[k] = e.x; med[k + 1] = e.y; med[k + 2] = e.z; med[k + 3] = e.w;
            }
        }
    }
    // phase 2: shifts and assembly
    float g[Q][V];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int cx = a.raw ? 0 : Lat<Q>::cx(i);
        if (cx == 1)
            pull_finish<1, PERIODIC, ST>(absent[i], x0, lane, a.nx, q[i], e[i], g[i]);
        else if (cx == -1)
            pull_finish<-1, PERIODIC, ST>(absent[i], x0, lane, a.nx, q[i], e[i], g[i]);
        else
            pull_finish<0, PERIODIC, ST>(absent[i], x0, lane, a.nx, q[i], e[i], g[i]);
    }
    if (!active) return;  // no shuffles below
    if (!kMedEarly) {
        const long long mo = (long long)y * a.pitch + x0;
        if (a.mid) {
            if (V == 4) {
                med[0] = __uint_as_float(*reinterpret_cast<const uint32_t *>(a.mid + mo));
            } else {
                const uint2 u = *reinterpret_cast<const uint2 *>(a.mid + mo);
                med[0] = __uint_as_float(u.x);
                med[V / 4 - 1] = __uint_as_float(u.y);
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k += 4) {
                const float4 e = *reinterpret_cast<const float4 *>(a.eta2 + mo + k);
                med[k] = e.x; med[k + 1] = e.y; med[k + 2] = e.z; med[k + 3] = e.w;
            }
        }
    }
    float e2s[V];
    if (a.mid) {  // eta^2 from the shared table
#pragma unroll
        for (int k = 0; k < V; k++)
            e2s[k] = tab[(__float_as_uint(med[k >> 2]) >> (8 * (k & 3))) & 0xffu];
    } else {
#pragma unroll
        for (int k = 0; k < V; k++) e2s[k] = med[k];
    }
    finish_sites<Q, MRT, ST, SLAB, RING>(a, g, e2s, x0, y, tmax);
}

template <int Q, bool MRT, bool PERIODIC, typename ST, bool SLAB = false>
// Minimum resident blocks per SM: enough warps to keep ~100 KB of loads in
// flight per SM (FP32 D2Q5 fits 5 blocks at <= 48 registers; the 8-site 16-bit
// and the 9-population FP32 forms are held to 64 registers for 4 blocks; the
// 9-population 16-bit form holds 72 values per thread and gets 128 registers).
// The 7-population 16-bit form (56 values) spills ~330 bytes at 64 registers and
// still runs faster with 4 blocks than with 3 at 80 registers (GB300, 256^3 BF16:
// 144 against 136 GLUPS; 5 blocks: 110).
__global__ void __launch_bounds__(kThreads, Q == 5   ? (sizeof(ST) == 4 ? 5 : 4)
                                           : Q == 7 ? 4
                                                    : (sizeof(ST) == 4 ? 4 : 2))
    step_kernel(const StepArgs a) {
    constexpr bool SC = Scaled<ST>::value;
    __shared__ float s_wmax[SC ? 9 : 1][kWarps];
    pdl_trigger_and_wait();
    if ((int)blockIdx.x >= a.main_blocks) {  // block-uniform
        gather_receivers<Q, PERIODIC, ST>(a, ((int)blockIdx.x - a.main_blocks) * kThreads +
                                                 (int)threadIdx.x);
        return;
    }
    __shared__ float s_tab[kThreads];
    if (a.mid) {  // block-uniform
        s_tab[threadIdx.x] = a.mid_tab[threadIdx.x];
        __syncthreads();
    }
    float tmax[Q];
    step_sites<Q, MRT, PERIODIC, ST, SLAB>(a, blockIdx.x, tmax, s_tab);
    if (SC) {  // fold this block's max |output| per population into max_out
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            float m = tmax[i];
            for (int off = 16; off > 0; off >>= 1)
                m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
            if (lane == 0) s_wmax[SC ? i : 0][w] = m;
        }
        __syncthreads();
        if ((int)threadIdx.x < Q) {
            float m = 0.f;
#pragma unroll
            for (int k = 0; k < kWarps; k++) m = fmaxf(m, s_wmax[SC ? threadIdx.x : 0][k]);
            atomicMax(a.max_out + threadIdx.x * kMaxCopies + (blockIdx.x % kMaxCopies),
                      __float_as_uint(m));
        }
    }
}

// FP16, after each step (one block): the scale the next step writes with, from
// this step's maxima (8 max|out| + |S[t+1]| at or below kStoredTarget), and a
// cleared max slot for the next step.  Launched as a programmatic dependent of the
// step (it waits for the step's grid before it reads the maxima), so its launch and
// the next step's overlap the step's last blocks.
static __global__ void scale_update_kernel(StepArgs a, int Q) {
    pdl_trigger_and_wait();
    const int i = threadIdx.x;
    if (i >= Q) return;
    float m = 0.f;
    for (int c = 0; c < kMaxCopies; c++) m = fmaxf(m, __uint_as_float(a.max_out[i * kMaxCopies + c]));
    const long long tn = a.t + 1;
    const float S = (a.src_tab && tn < a.src_nt) ? fabsf(a.src_tab[tn]) : 0.f;
    a.scale_next[i] = next_scale(m, S, a.scale_out[i]);
    for (int c = 0; c < kMaxCopies; c++) a.max_next[i * kMaxCopies + c] = 0u;
}

// ------------------------------------------------------------ batched step --
// One launch advances several independent simulations ("shots") by one step
// each: shot k owns blocks [first[k], first[k + 1]) of the grid (its site blocks
// followed by its receiver blocks) and its own StepArgs descriptor.  Used by the
// serving loop for FP32 and BF16 storage (no cross-block scale hand-off).
template <int Q, bool MRT, bool PERIODIC, typename ST>
__global__ void __launch_bounds__(kThreads)
    batch_step_kernel(const StepArgs *__restrict__ args, const int *__restrict__ first, int nshots) {
    __shared__ StepArgs sa;
    __shared__ int s_blk;
    pdl_trigger_and_wait();
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
        s_blk = (int)blockIdx.x - first[lo];
    }
    __syncthreads();
    const int blk = s_blk;
    if (blk >= sa.main_blocks) {
        gather_receivers<Q, PERIODIC, ST>(sa, (blk - sa.main_blocks) * kThreads + (int)threadIdx.x);
        return;
    }
    __shared__ float s_tab[kThreads];
    if (sa.mid) {  // block-uniform
        s_tab[threadIdx.x] = sa.mid_tab[threadIdx.x];
        __syncthreads();
    }
    float tmax[Q];
    step_sites<Q, MRT, PERIODIC, ST>(sa, blk, tmax, s_tab);
}

// -------------------------------------------------------- state transforms --
// Write the state g(t) in place ("raw", unshifted).  mode 0: g from pressure p
// (g_i = (w_i / c_s^2) p, Eq. linear eqm dist with j = 0); mode 1: g given as
// [Q][ny][nx] FP32; src == nullptr: all zero.
template <int Q, bool PERIODIC, typename ST>
__global__ void set_state_kernel(StepArgs a, const float *src, int mode) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = (long long)a.ny * a.pitch;
    if (idx >= total) return;
    int y = (int)(idx / a.pitch), x = (int)(idx - (long long)y * a.pitch);
    ST *o = static_cast<ST *>(a.out);
    for (int i = 0; i < Q; i++) {
        float v = 0.f;
        if (x < a.nx && src) {
            if (mode == 0) {
                float e2 = a.eta2[idx];
                v = weight_i<Q>(i, e2, a) / cs2_of<Q>(e2, a) * src[(long long)y * a.nx + x];
            } else {
                v = src[(long long)i * a.nx * a.ny + (long long)y * a.nx + x];
            }
        }
        Store<ST>::store1(o + i * a.plane + idx, v / scale_of(a.scale_out, i));
    }
}

// mode 0: pressure [ny][nx]; mode 1: populations [Q][ny][nx] (pre-collision, current time)
template <int Q, bool PERIODIC, typename ST>
__global__ void get_state_kernel(StepArgs a, float *dst, int mode) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = (long long)a.ny * a.nx;
    if (idx >= total) return;
    int y = (int)(idx / a.nx), x = (int)(idx - (long long)y * a.nx);
    const ST *in = static_cast<const ST *>(a.in);
    float rho = 0.f;
    for (int i = 0; i < Q; i++) {
        int xs = x - (a.raw ? 0 : Lat<Q>::cx(i));
        const int ys = a.raw ? y : pull_row<Q, PERIODIC>(a, y, i);  // y: row (z ny3 + y in 3-D)
        const ST *halo = a.raw ? nullptr : slab_halo_row<Q, ST>(a, y, i);
        float v = 0.f;
        bool ok = true;
        if (PERIODIC) {
            xs = (xs + a.nx) % a.nx;
        } else {
            ok = xs >= 0 && xs < a.nx && (ys >= 0 || halo);
        }
        const int slot = a.swap ? Lat<Q>::opp(i) : i;
        if (ok)
            v = Store<ST>::load1(halo ? halo + xs : in + slot * a.plane + (long long)ys * a.pitch + xs) *
                scale_of(a.scale_in, i);
        if (mode == 1) dst[(long long)i * total + idx] = v;
        rho += v;
    }
    if (mode == 0) dst[idx] = cs2_of<Q>(a.eta2[(long long)y * a.pitch + x], a) * rho;
}

// 16-bit initial scale: max |g_i| of the state to be written (same value rule as
// set_state_kernel) accumulated into max_out[i][*].
template <int Q>
__global__ void source_max_kernel(StepArgs a, const float *src, int mode) {
    long long total = (long long)a.ny * a.nx;
    float m[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) m[i] = 0.f;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int y = (int)(idx / a.nx), x = (int)(idx - (long long)y * a.nx);
#pragma unroll
        for (int i = 0; i < Q; i++) {
            float v;
            if (mode == 0) {
                float e2 = a.eta2[(long long)y * a.pitch + x];
                v = weight_i<Q>(i, e2, a) / cs2_of<Q>(e2, a) * src[idx];
            } else {
                v = src[(long long)i * total + idx];
            }
            m[i] = fmaxf(m[i], fabsf(v));
        }
    }
#pragma unroll
    for (int i = 0; i < Q; i++) {
        float v = m[i];
        for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
        if ((threadIdx.x & 31) == 0)
            atomicMax(a.max_out + i * kMaxCopies + (blockIdx.x % kMaxCopies), __float_as_uint(v));
    }
}

// FP16 initial scales from max |g_i| of the state being written (accumulated in
// max_out): scale_next[i] for the written state itself, scale_out-style slot
// `scale_first` for the first step's output (8x headroom plus |S[t]|), whose
// max slot max_next is cleared, together with the block counter.
static __global__ void init_scale_kernel(StepArgs a, int Q, float *scale_first) {
    int i = threadIdx.x;
    if (i >= Q) return;
    float m = 0.f;
    for (int c = 0; c < kMaxCopies; c++) m = fmaxf(m, __uint_as_float(a.max_out[i * kMaxCopies + c]));
    const float s0 = m > 0.f ? pow2_ceil(m * (1.f / kStoredTarget)) : 1.f;
    a.scale_next[i] = s0;
    const float S = (a.src_tab && a.t < a.src_nt) ? fabsf(a.src_tab[a.t]) : 0.f;
    scale_first[i] = next_scale(m, S, s0);
    for (int c = 0; c < kMaxCopies; c++) a.max_next[i * kMaxCopies + c] = 0u;
}

// eta^2 = (c / c_ref)^2 per site (pads 0); flags[0]: bit0 c <= 0 or non-finite, bit1
// eta > 1; flags[1] / flags[2]: the bits of the smallest / largest eta^2 over the real sites
// (non-negative floats order as their bit patterns; the caller sets them to +inf and 0).
// Launched with 256 threads per block.
static __global__ void medium_kernel(const float *c_map, float *eta2, int nx, int ny, int pitch,
                              double inv_cref, unsigned *flags) {
    __shared__ unsigned s_lo[8], s_hi[8];
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    unsigned lo = 0x7f800000u, hi = 0u;
    if (idx < (long long)ny * pitch) {
        int y = (int)(idx / pitch), x = (int)(idx - (long long)y * pitch);
        float v = 0.f;
        if (x < nx) {
            float c = c_map[(long long)y * nx + x];
            if (!(c > 0.f) || !isfinite(c)) atomicOr(flags, 1u);
            double eta = (double)c * inv_cref;
            if (eta > 1.0 + 1e-6) atomicOr(flags, 2u);
            if (eta > 1.0) eta = 1.0;
            v = (float)(eta * eta);
            if (v >= 0.f) lo = hi = __float_as_uint(v);
        }
        eta2[idx] = v;
    }
    for (int off = 16; off > 0; off >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            lo = min(lo, s_lo[w]);
            hi = max(hi, s_hi[w]);
        }
        atomicMin(flags + 1, lo);
        atomicMax(flags + 2, hi);
    }
}

}  // namespace lbk
