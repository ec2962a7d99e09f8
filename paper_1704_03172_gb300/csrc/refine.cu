// refine.cu -- grid refinement of Sec. 4 (ratio n = 2 in space and time per
// level) on the GPU: one patch of the context's grid, and optionally patches
// nested inside it ("multiples of 2": ratio 4, 8 to the coarse grid).
//
// The coarse grid is the context's grid; a patch of coarse cells
// [x0, x0 + nxp] x [y0, y0 + nyp] is covered by a fine grid of
// (2 nxp + 1) x (2 nyp + 1) nodes, fine node (a, b) at coarse position
// (x0 + a/2, y0 + b/2), whose sound speed is the coarse sound speed
// interpolated bilinearly.  Every fine grid is stored with a one-node ghost
// ring: the populations that enter it across its interface I (the patch
// boundary) are written into the ghost ring, so the ordinary fused step kernel
// pulls them in.  A nested patch lies inside the fine grid of the level above
// it, in that grid's node coordinates, and is coupled to it exactly as the
// first patch is coupled to the coarse grid.
//
// Coupling (Eq. grid refinement eqm dist, Eq. coarse-fine dist connect), read
// per population: a fine node of I takes from the coarse grid exactly the
// populations whose upstream node lies outside the fine grid,
//   g^f_i = g^eq_i + (g^c_i - g^eq_i) / 2,
// from coarse vectors interpolated linearly along I and in time (midpoint at
// odd fine times); a coarse node of I takes from the fine grid the populations
// whose upstream node lies strictly inside the patch,
//   g^c_i = g^eq_i + 2 (g^f_i - g^eq_i),
// g^eq being formed from the transferred vector's moments with the receiving
// grid's weights.  The factors 1/2 and 2 are those of the paper's lossless
// setting (tau = 1/2, s = 2).  For other rates each level relaxes with
// tau_f - 1/2 = 2 (tau_c - 1/2) per relaxed moment, which keeps the physical
// viscosity continuous, and the non-equilibrium parts scale by tau_f / (2 tau_c)
// (coarse -> fine) and 2 tau_c / tau_f (fine -> coarse), moment by moment;
// at tau = 1/2 these are the paper's factors.  The coarser grid keeps running
// under its patch, which gives the full coarse vector on I (U, kept for two
// coarse times).
//
// One step T of a grid that holds a patch (fused kernels, all on the context
// stream):
//   the grid's step T (pull, collide, store; its own receivers)
//   snapshot U(T) = the grid's populations on I at time T (before correction), fused
//     into the first transfer below
//   [T >= 1] c2f into the patch's ghost ring from (U(T-1) + U(T)) / 2, patch step 2T-1
//   c2f from U(T), patch step 2T (receivers inside the closed patch)
//   f2c: the grid's nodes of I re-pulled, corrected from the patch state at 2T,
//        re-collided and stored over the grid's step output.
// A "patch step" of a level that holds a nested patch is this same procedure one level
// down, so a coarse step of a two-patch hierarchy runs 1 + 2 + 4 step launches and
// 3 + 2 x 3 coupling launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "lb_kernels.cuh"
#include "lb_runtime.h"

using namespace lbk;
using namespace lbrt;

// One refined level: the fine grid of a patch and its coupling to the grid above it.
struct lb_refine {
    int depth = 1;                   // 1: patch of the context's grid; k: patch of level k - 1
    int coupling = LB_COUPLE_BOTH;   // direction of the coupling to the grid above
    int x0n = 0, y0n = 0;            // patch origin, parent grid node coordinates
    int x0 = 0, y0 = 0;              // patch origin, parent grid storage coordinates
    int nxp = 0, nyp = 0, nxf = 0, nyf = 0;  // patch (parent cells) and fine node counts
    int gx = 0, gy = 0, pitch = 0;   // fine grid with its ghost ring
    void *pop[2] = {nullptr, nullptr};
    int cur = 0;
    bool raw = false;
    float *eta2 = nullptr;
    float *cf = nullptr;             // [nyf][nxf] fine sound speed (medium of a nested patch)
    float *pf = nullptr;             // [nyf][nxf] initial fine pressure (for a nested patch)
    int nI = 0;
    int2 *Ic = nullptr;              // parent nodes of I (storage coordinates)
    float *U[3] = {nullptr, nullptr, nullptr};  // [nI][Q]: slots T % 2, plus one for peeks
    int nIf = 0;
    int4 *If = nullptr;              // fine nodes of I: (a, b, k1, k2), k2 < 0 when single
    int2 *rec_c = nullptr, *rec_f = nullptr;  // rec_c: the context grid's (depth 1 only)
    int *col_c = nullptr, *col_f = nullptr;
    int nrec_c = 0, nrec_f = 0;
    // relaxation on this level, and the non-equilibrium rescales written as collisions:
    // g' = geq + F (g - geq) per non-conserved moment is a collision with rates 1 - F
    double tau_f = 0.5, stau_f[9] = {};
    float omega_f = 2.f, s_f[9] = {};
    float c2f_omega = 0.5f, c2f_s[9] = {}, f2c_omega = -1.f, f2c_s[9] = {};
    // coarse node (X, Y), X in [ox0, ox0 + onx), Y in [oy0, oy0 + ony), is this level's
    // node (oA X + obx, oA Y + oby): the context-grid pressure taken from this level
    int oA = 2, obx = 0, oby = 0, ox0 = 0, oy0 = 0, onx = 0, ony = 0;
    lb_refine *sub = nullptr;        // nested patch inside this level's grid
    void *bak = nullptr;             // depth >= 2: input buffer saved around pressure peeks
    float *Ubak[2] = {nullptr, nullptr};
    ~lb_refine() { delete sub; }
};

namespace {


// fine sound speed and eta^2 (with the ghost ring: nearest real node) from the parent's
// sound speed pc [..][pnx] (node coordinates), bilinearly; cf gets the real nodes' speeds
__global__ void ref_medium_kernel(const float *pc, int pnx, int x0n, int y0n, int nxf, int nyf,
                                  int gx, int gy, int pitch, double inv_cref, float *eta2,
                                  float *cf) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)gy * pitch) return;
    int pb = (int)(idx / pitch), pa = (int)(idx - (long long)pb * pitch);
    if (pa >= gx) {
        eta2[idx] = 0.f;
        return;
    }
    int a = min(max(pa - 1, 0), nxf - 1), b = min(max(pb - 1, 0), nyf - 1);
    int X = x0n + a / 2, Y = y0n + b / 2, ox = a & 1, oy = b & 1, cnt = 0;
    double s = 0.0;
    for (int dy = 0; dy <= oy; dy++)
        for (int dx = 0; dx <= ox; dx++) {
            s += (double)pc[(long long)(Y + dy) * pnx + X + dx];
            cnt++;
        }
    float c = (float)(s / cnt);
    double eta = (double)c * inv_cref;
    if (eta > 1.0) eta = 1.0;
    eta2[idx] = (float)(eta * eta);
    if (cf && pa == a + 1 && pb == b + 1) cf[(long long)b * nxf + a] = c;
}

// raw fine state g = g^eq(p / c_s^2, 0), p = bilinear interpolation of the parent's
// pressure pp [..][pnx] (node coordinates; nullptr: zero); pf gets p at the real nodes
template <int Q>
__global__ void ref_init_fine_kernel(StepArgs af, const float *pp, int pnx, int x0n, int y0n,
                                     int nxf, int nyf, float *pf) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= af.plane) return;
    int pb = (int)(idx / af.pitch), pa = (int)(idx - (long long)pb * af.pitch);
    int a = pa - 1, b = pb - 1;
    float p = 0.f;
    bool inside = a >= 0 && a < nxf && b >= 0 && b < nyf;
    if (inside && pp) {
        int X = x0n + a / 2, Y = y0n + b / 2, ox = a & 1, oy = b & 1, cnt = 0;
        double s = 0.0;
        for (int dy = 0; dy <= oy; dy++)
            for (int dx = 0; dx <= ox; dx++) {
                s += (double)pp[(long long)(Y + dy) * pnx + X + dx];
                cnt++;
            }
        p = (float)(s / cnt);
    }
    if (inside && pf) pf[(long long)b * nxf + a] = p;
    float *o = static_cast<float *>(af.out);
    const float e2 = af.eta2[idx];
    for (int i = 0; i < Q; i++)
        o[i * af.plane + idx] = inside ? weight_i<Q>(i, e2, af) / cs2_of<Q>(e2, af) * p : 0.f;
}

template <int Q>
__device__ __forceinline__ float pull1(const float *in, int raw, int periodic, int x, int y,
                                       int i, int nx, int ny, int pitch, long long plane) {
    int xs = x, ys = y;
    if (!raw) {
        xs -= Lat<Q>::cx(i);
        ys -= Lat<Q>::cy(i);
    }
    if (periodic) {
        xs = (xs + nx) % nx;
        ys = (ys + ny) % ny;
    } else if (xs < 0 || xs >= nx || ys < 0 || ys >= ny) {
        return 0.f;
    }
    return in[i * plane + (long long)ys * pitch + xs];
}

template <int Q>
__global__ void ref_snapshot_kernel(StepArgs ac, const int2 *Ic, int nI, float *U) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nI) return;
    const float *in = static_cast<const float *>(ac.in);
    int2 X = Ic[k];  // at least one node from the parent's edges: no wrap needed
    for (int i = 0; i < Q; i++)
        U[(long long)k * Q + i] = pull1<Q>(in, ac.raw, 0, X.x, X.y, i, ac.nx, ac.ny, ac.pitch,
                                           ac.plane);
}

// coarse -> fine: write the entering populations of the fine nodes of I into
// the fine input buffer (at the upstream ghost node, or in place when raw).  The body
// handles interface node j (of nIf); the kernels below and ref_step_kernel call it.
template <int Q, bool MRT>
__device__ __forceinline__ void c2f_node(const StepArgs &af, const StepArgs &rs, const int4 *If,
                                         int j, const float *Ua, const float *Ub, float alpha,
                                         int nxf, int nyf) {
    const int4 e = If[j];
    const int a = e.x, b = e.y;
    float gh[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        float v = (1.f - alpha) * Ua[(long long)e.z * Q + i] + alpha * Ub[(long long)e.z * Q + i];
        if (e.w >= 0) {
            v += (1.f - alpha) * Ua[(long long)e.w * Q + i] + alpha * Ub[(long long)e.w * Q + i];
            v *= 0.5f;
        }
        gh[i] = v;
    }
    const long long node = (long long)(b + 1) * af.pitch + (a + 1);
    // g^eq (fine weights) + factor (g - g^eq): a collision with the rescale rates rs
    if (Q == 5)
        collide5<MRT>(gh, af.eta2[node], rs);
    else
        collide9<MRT>(gh, af.eta2[node], rs);
    float *in = static_cast<float *>(const_cast<void *>(af.in));
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int ua = a - Lat<Q>::cx(i), ub = b - Lat<Q>::cy(i);
        if (ua >= 0 && ua < nxf && ub >= 0 && ub < nyf) continue;  // comes from the fine grid
        const long long pos =
            af.raw ? node : (long long)(ub + 1) * af.pitch + (ua + 1);
        in[i * af.plane + pos] = gh[i];
    }
}

template <int Q, bool MRT>
__global__ void ref_c2f_kernel(StepArgs af, StepArgs rs, const int4 *If, int nIf, const float *Ua,
                               const float *Ub, float alpha, int nxf, int nyf) {
    pdl_trigger_and_wait();  // launched with launch_pdl
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nIf) return;
    c2f_node<Q, MRT>(af, rs, If, j, Ua, Ub, alpha, nxf, nyf);
}

// Fine -> coarse coupling only: nothing enters the fine grid across I.  The entering
// populations of the fine nodes of I, which the fine step left at the upstream ghost
// nodes of its input, are set to zero (a zero-ghost boundary).  Not used on a raw input:
// the state set at time 0 is kept, as the coupling at time 0 would keep it.
template <int Q>
__global__ void ref_zero_in_kernel(StepArgs af, const int4 *If, int nIf, int nxf, int nyf) {
    pdl_trigger_and_wait();  // launched with launch_pdl
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nIf) return;
    const int a = If[j].x, b = If[j].y;
    float *in = static_cast<float *>(const_cast<void *>(af.in));
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int ua = a - Lat<Q>::cx(i), ub = b - Lat<Q>::cy(i);
        if (ua >= 0 && ua < nxf && ub >= 0 && ub < nyf) continue;  // comes from the fine grid
        in[i * af.plane + (long long)(ub + 1) * af.pitch + (ua + 1)] = 0.f;
    }
}

// The first coarse -> fine transfer of the parent's step T with the snapshot fused in: the
// parent's populations on I at time T are pulled here from its step input (ap), each coarse
// node's vector is stored to Ucur by the fine node that coincides with it, and the transfer
// interpolates them with Ua = U(T - 1) (alpha = 1/2) or takes them alone (alpha = 1, T = 0).
// Same values as the snapshot kernel followed by ref_c2f_kernel.
template <int Q, bool MRT>
__device__ __forceinline__ void snap_c2f_node(const StepArgs &ap, const StepArgs &af,
                                              const StepArgs &rs, const int4 *If, int j,
                                              const int2 *Ic, const float *Ua, float *Ucur,
                                              float alpha, int nxf, int nyf) {
    const int4 e = If[j];
    const int a = e.x, b = e.y;
    const float *pin = static_cast<const float *>(ap.in);
    float u1[Q], u2[Q];
    const int2 X1 = Ic[e.z];
#pragma unroll
    for (int i = 0; i < Q; i++)
        u1[i] = pull1<Q>(pin, ap.raw, 0, X1.x, X1.y, i, ap.nx, ap.ny, ap.pitch, ap.plane);
    if (e.w >= 0) {
        const int2 X2 = Ic[e.w];
#pragma unroll
        for (int i = 0; i < Q; i++)
            u2[i] = pull1<Q>(pin, ap.raw, 0, X2.x, X2.y, i, ap.nx, ap.ny, ap.pitch, ap.plane);
    }
    if (!(a & 1) && !(b & 1)) {  // the fine node that coincides with coarse node e.z
#pragma unroll
        for (int i = 0; i < Q; i++) Ucur[(long long)e.z * Q + i] = u1[i];
    }
    float gh[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        float v = alpha < 1.f ? (1.f - alpha) * Ua[(long long)e.z * Q + i] + alpha * u1[i] : u1[i];
        if (e.w >= 0) {
            v += alpha < 1.f ? (1.f - alpha) * Ua[(long long)e.w * Q + i] + alpha * u2[i] : u2[i];
            v *= 0.5f;
        }
        gh[i] = v;
    }
    const long long node = (long long)(b + 1) * af.pitch + (a + 1);
    if (Q == 5)
        collide5<MRT>(gh, af.eta2[node], rs);
    else
        collide9<MRT>(gh, af.eta2[node], rs);
    float *in = static_cast<float *>(const_cast<void *>(af.in));
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int ua = a - Lat<Q>::cx(i), ub = b - Lat<Q>::cy(i);
        if (ua >= 0 && ua < nxf && ub >= 0 && ub < nyf) continue;  // comes from the fine grid
        const long long pos =
            af.raw ? node : (long long)(ub + 1) * af.pitch + (ua + 1);
        in[i * af.plane + pos] = gh[i];
    }
}

template <int Q, bool MRT>
__global__ void ref_snap_c2f_kernel(StepArgs ap, StepArgs af, StepArgs rs, const int4 *If, int nIf,
                                    const int2 *Ic, const float *Ua, float *Ucur, float alpha,
                                    int nxf, int nyf) {
    pdl_trigger_and_wait();  // launched with launch_pdl
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nIf) return;
    snap_c2f_node<Q, MRT>(ap, af, rs, If, j, Ic, Ua, Ucur, alpha, nxf, nyf);
}

// fine -> coarse on I, then collide (+ sponge) and overwrite the parent's step output
// (coarse interface node k of nI)
template <int Q, bool MRT, bool PERIODIC>
__device__ __forceinline__ void f2c_node(const StepArgs &ac, const StepArgs &rs, const float *fin,
                                         int fraw, int fpitch, long long fplane, const int2 *Ic,
                                         int k, int x0, int y0, int nxp, int nyp) {
    const int2 X = Ic[k];
    const float *cin = static_cast<const float *>(ac.in);
    float g[Q], G[Q];
    const int fa = 1 + 2 * (X.x - x0), fb = 1 + 2 * (X.y - y0);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        g[i] = pull1<Q>(cin, ac.raw, PERIODIC, X.x, X.y, i, ac.nx, ac.ny, ac.pitch, ac.plane);
        G[i] = pull1<Q>(fin, fraw, 0, fa, fb, i, 1 << 30, 1 << 30, fpitch, fplane);
    }
    const float e2 = ac.eta2[(long long)X.y * ac.pitch + X.x];
    // g^eq (coarse weights) + factor (G - g^eq): a collision with the rescale rates rs
    if (Q == 5)
        collide5<MRT>(G, e2, rs);
    else
        collide9<MRT>(G, e2, rs);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int ux = X.x - Lat<Q>::cx(i), uy = X.y - Lat<Q>::cy(i);
        if (ux > x0 && ux < x0 + nxp && uy > y0 && uy < y0 + nyp) g[i] = G[i];
    }
    if (Q == 5)
        collide5<MRT>(g, e2, ac);
    else
        collide9<MRT>(g, e2, ac);
    float f = ac.sponge_w > 0 ? sponge_factor(X.x, X.y, ac) : 1.f;
    float *out = static_cast<float *>(ac.out);
#pragma unroll
    for (int i = 0; i < Q; i++) out[i * ac.plane + (long long)X.y * ac.pitch + X.x] = g[i] * f;
}

template <int Q, bool MRT, bool PERIODIC>
__global__ void ref_f2c_kernel(StepArgs ac, StepArgs rs, const float *fin, int fraw, int fpitch,
                               long long fplane, const int2 *Ic, int nI, int x0, int y0, int nxp,
                               int nyp) {
    pdl_trigger_and_wait();  // launched with launch_pdl
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nI) return;
    f2c_node<Q, MRT, PERIODIC>(ac, rs, fin, fraw, fpitch, fplane, Ic, k, x0, y0, nxp, nyp);
}

// One step of a grid (step_kernel's blocks: sites, then receivers) with one or two coupling
// tasks of patches in leading blocks of the same launch, so that their short chains of
// dependent loads start with the first wave.  A task touches nothing the step reads or
// writes:
// - the snapshot transfer reads the step's input and writes the patch's input ring;
// - the transfer at the parent's later time writes the ring of the fine step's output,
//   which that step leaves alone (StepArgs::ring);
// - the fine -> coarse correction reads the fine step's input and rewrites the parent's
//   output, which an earlier launch finished.
enum { kTaskNone = 0, kTaskSnapC2f = 1, kTaskC2f = 2, kTaskF2c = 3 };
struct RefTask {
    int blocks;       // blocks of the task
    int n;            // interface nodes
    StepArgs p, f, rs;  // parent step, fine level and rescale arguments of the task
    const int4 *If;
    const int2 *Ic;
    const float *Ua, *Ub;
    float *Ucur;
    float alpha;
    int nxf, nyf;
    const float *fin;  // f2c: the fine state
    int fraw, fpitch;
    long long fplane;
    int x0, y0, nxp, nyp;
};

template <int Q, bool MRT, int TASK, bool TASK_PER>
__device__ __forceinline__ void run_task(const RefTask &x, int j) {
    if (j >= x.n) return;
    if (TASK == kTaskSnapC2f)
        snap_c2f_node<Q, MRT>(x.p, x.f, x.rs, x.If, j, x.Ic, x.Ua, x.Ucur, x.alpha, x.nxf, x.nyf);
    else if (TASK == kTaskC2f)
        c2f_node<Q, MRT>(x.f, x.rs, x.If, j, x.Ua, x.Ub, x.alpha, x.nxf, x.nyf);
    else if (TASK == kTaskF2c)
        f2c_node<Q, MRT, TASK_PER>(x.p, x.rs, x.fin, x.fraw, x.fpitch, x.fplane, x.Ic, j, x.x0,
                                   x.y0, x.nxp, x.nyp);
}

template <int Q, bool MRT, bool PERIODIC, int T1, bool P1, int T2, bool P2>
__global__ void __launch_bounds__(kThreads, Q == 5 ? 5 : 4)
    ref_step_kernel(const StepArgs a, const RefTask x1, const RefTask x2) {
    pdl_trigger_and_wait();
    __shared__ float s_tab[kThreads];
    const int b0 = (int)blockIdx.x;
    if (b0 < x1.blocks) {  // block-uniform: the first task
        run_task<Q, MRT, T1, P1>(x1, b0 * kThreads + (int)threadIdx.x);
        return;
    }
    const int b1 = b0 - x1.blocks;
    if (T2 != kTaskNone && b1 < x2.blocks) {  // block-uniform: the second task
        run_task<Q, MRT, T2, P2>(x2, b1 * kThreads + (int)threadIdx.x);
        return;
    }
    const int blk = b1 - (T2 != kTaskNone ? x2.blocks : 0);
    if (blk >= a.main_blocks) {  // block-uniform: receivers
        gather_receivers<Q, PERIODIC, float>(a, (blk - a.main_blocks) * kThreads + (int)threadIdx.x);
        return;
    }
    if (a.mid) {  // block-uniform
        s_tab[threadIdx.x] = a.mid_tab[threadIdx.x];
        __syncthreads();
    }
    float tmax[Q];
    // every fused fine step leaves its ring to a transfer; the coarse step has none
    step_sites<Q, MRT, PERIODIC, float, false, T1 != kTaskSnapC2f>(a, blk, tmax, s_tab);
}

// context-grid pressure at the coarse nodes covered by a level, from its coincident nodes:
// coarse (X, Y) -> level node (A X + bx, A Y + by), stored at (+1, +1)
template <int Q>
__global__ void ref_overlay_kernel(StepArgs af, float *p, int nx, int X0, int Y0, int w, int h,
                                   int A, int bx, int by) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= w * h) return;
    const int X = X0 + k % w, Y = Y0 + k / w;
    const int fa = 1 + A * X + bx, fb = 1 + A * Y + by;
    const float *in = static_cast<const float *>(af.in);
    float rho = 0.f;
    for (int i = 0; i < Q; i++)
        rho += pull1<Q>(in, af.raw, 0, fa, fb, i, 1 << 30, 1 << 30, af.pitch, af.plane);
    p[(long long)Y * nx + X] = cs2_of<Q>(af.eta2[(long long)fb * af.pitch + fa], af) * rho;
}

int blocks_for(long long n) { return (int)((n + 255) / 256); }

// step arguments of refined level R: its own eta^2 plane and rates; no sponge, source or
// receivers (the caller adds receivers)
StepArgs level_args(const lb_ctx *ctx, const lb_refine *R) {
    StepArgs a = base_args(ctx);
    a.eta2 = R->eta2;
    a.mid = nullptr;  // refined levels read their own eta^2 plane
    a.mid_tab = nullptr;
    a.omega = R->omega_f;  // viscosity-continuous relaxation of this level
    for (int k = 0; k < 9; k++) a.s[k] = mrt_rate_arg(ctx->Q, k, R->s_f[k]);
    a.nx = R->gx;
    a.ny = R->gy;
    a.ny3 = R->gy;
    a.nz = 1;
    a.pitch = R->pitch;
    a.plane = (long long)R->gy * R->pitch;
    a.segs = (R->gx + kSitesPerWarp - 1) / kSitesPerWarp;
    a.main_blocks = (int)(((long long)a.segs * R->gy + kWarps - 1) / kWarps);
    a.sponge_w = 0;
    a.src_tab = nullptr;
    a.src_nt = 0;
    a.rec = nullptr;
    a.nrec = 0;
    a.trace_row = nullptr;
    a.rec_col = nullptr;
    a.scale_in = nullptr;
    return a;
}

// rates whose collision is the non-equilibrium rescale g^eq + F (g - g^eq)
StepArgs rescale_args(StepArgs a, int Q, float omega, const float *s) {
    a.omega = omega;
    for (int k = 0; k < 9; k++) a.s[k] = mrt_rate_arg(Q, k, s[k]);
    return a;
}

template <int Q, bool MRT>
void c2f_q(lb_ctx *ctx, lb_refine *R, const StepArgs &af, const float *Ua, const float *Ub,
           float alpha) {
    launch_pdl(ref_c2f_kernel<Q, MRT>, dim3(blocks_for(R->nIf)), dim3(256), 0, ctx->stream, af,
               rescale_args(af, Q, R->c2f_omega, R->c2f_s), R->If, R->nIf, Ua, Ub, alpha, R->nxf,
               R->nyf);
}

void launch_c2f(lb_ctx *ctx, lb_refine *R, const float *Ua, const float *Ub, float alpha) {
    StepArgs af = level_args(ctx, R);
    af.in = R->pop[R->cur];
    af.raw = R->raw ? 1 : 0;
    const bool mrt = ctx->cfg.collision == LB_MRT;
    if (ctx->Q == 9) {
        if (mrt) c2f_q<9, true>(ctx, R, af, Ua, Ub, alpha); else c2f_q<9, false>(ctx, R, af, Ua, Ub, alpha);
    } else {
        if (mrt) c2f_q<5, true>(ctx, R, af, Ua, Ub, alpha); else c2f_q<5, false>(ctx, R, af, Ua, Ub, alpha);
    }
}

template <int Q, bool MRT>
void snap_c2f_q(lb_ctx *ctx, const StepArgs &ap, lb_refine *R, const StepArgs &af, const float *Ua,
                float *Ucur, float alpha) {
    launch_pdl(ref_snap_c2f_kernel<Q, MRT>, dim3(blocks_for(R->nIf)), dim3(256), 0, ctx->stream,
               ap, af, rescale_args(af, Q, R->c2f_omega, R->c2f_s), R->If, R->nIf, R->Ic, Ua, Ucur,
               alpha, R->nxf, R->nyf);
}

// snapshot U(T) of the parent's interface into Ucur fused with the first coarse -> fine
// transfer of step T (alpha = 1/2 with Ua = U(T - 1), or alpha = 1)
void launch_snap_c2f(lb_ctx *ctx, const StepArgs &ap, lb_refine *R, const float *Ua, float *Ucur,
                     float alpha) {
    StepArgs af = level_args(ctx, R);
    af.in = R->pop[R->cur];
    af.raw = R->raw ? 1 : 0;
    const bool mrt = ctx->cfg.collision == LB_MRT;
    if (ctx->Q == 9) {
        if (mrt) snap_c2f_q<9, true>(ctx, ap, R, af, Ua, Ucur, alpha); else snap_c2f_q<9, false>(ctx, ap, R, af, Ua, Ucur, alpha);
    } else {
        if (mrt) snap_c2f_q<5, true>(ctx, ap, R, af, Ua, Ucur, alpha); else snap_c2f_q<5, false>(ctx, ap, R, af, Ua, Ucur, alpha);
    }
}

// fine -> coarse coupling only: zero what enters R across I before its next step (a raw
// input keeps its state)
void launch_zero_in(lb_ctx *ctx, lb_refine *R) {
    if (R->raw) return;
    StepArgs af = level_args(ctx, R);
    af.in = R->pop[R->cur];
    if (ctx->Q == 9)
        launch_pdl(ref_zero_in_kernel<9>, dim3(blocks_for(R->nIf)), dim3(256), 0, ctx->stream, af,
                   R->If, R->nIf, R->nxf, R->nyf);
    else
        launch_pdl(ref_zero_in_kernel<5>, dim3(blocks_for(R->nIf)), dim3(256), 0, ctx->stream, af,
                   R->If, R->nIf, R->nxf, R->nyf);
}

// snapshot of the parent's populations on R's interface, from the parent's step input
void launch_snapshot(lb_ctx *ctx, const StepArgs &ap, lb_refine *R, float *U) {
    if (ctx->Q == 9)
        ref_snapshot_kernel<9><<<blocks_for(R->nI), 256, 0, ctx->stream>>>(ap, R->Ic, R->nI, U);
    else
        ref_snapshot_kernel<5><<<blocks_for(R->nI), 256, 0, ctx->stream>>>(ap, R->Ic, R->nI, U);
}

template <int Q, bool MRT>
void f2c_q(lb_ctx *ctx, const StepArgs &ap, bool periodic, lb_refine *R, const float *fin,
           int fraw) {
    long long fplane = (long long)R->gy * R->pitch;
    launch_pdl(periodic ? ref_f2c_kernel<Q, MRT, true> : ref_f2c_kernel<Q, MRT, false>,
               dim3(blocks_for(R->nI)), dim3(256), 0, ctx->stream, ap,
               rescale_args(ap, Q, R->f2c_omega, R->f2c_s), fin, fraw, R->pitch, fplane, R->Ic, R->nI,
               R->x0, R->y0, R->nxp, R->nyp);
}

// correction of the parent's step output on R's interface from R's state fin
void launch_f2c(lb_ctx *ctx, const StepArgs &ap, bool periodic, lb_refine *R, const float *fin,
                int fraw) {
    const bool mrt = ctx->cfg.collision == LB_MRT;
    if (ctx->Q == 9) {
        if (mrt) f2c_q<9, true>(ctx, ap, periodic, R, fin, fraw); else f2c_q<9, false>(ctx, ap, periodic, R, fin, fraw);
    } else {
        if (mrt) f2c_q<5, true>(ctx, ap, periodic, R, fin, fraw); else f2c_q<5, false>(ctx, ap, periodic, R, fin, fraw);
    }
}

void child_steps(lb_ctx *ctx, const StepArgs &ap, bool periodic, lb_refine *R, float *trace_row,
                 long long T);

// one step t of refined level R (pull from pop[cur], store into pop[cur ^ 1]), with every
// level nested in it; receivers of R at trace row `trace_row`
void level_step(lb_ctx *ctx, lb_refine *R, float *trace_row, long long t) {
    StepArgs af = level_args(ctx, R);
    af.in = R->pop[R->cur];
    af.out = R->pop[R->cur ^ 1];
    af.raw = R->raw ? 1 : 0;
    af.t = t;
    int rec_blocks = 0;
    if (trace_row && R->nrec_f > 0) {
        af.rec = R->rec_f;
        af.nrec = R->nrec_f;
        af.rec_col = R->col_f;
        af.trace_row = trace_row;
        rec_blocks = (R->nrec_f + kThreads - 1) / kThreads;
    }
    StepFn fn = pick_step_for(ctx->Q, ctx->cfg.collision == LB_MRT, false, LB_F32);
    launch_pdl(fn, dim3(af.main_blocks + rec_blocks), dim3(kThreads), 0, ctx->stream, af);
    if (R->sub) child_steps(ctx, af, false, R->sub, trace_row, t);
    R->cur ^= 1;
    R->raw = false;
}

// The part of the parent's step T that advances its patch R from 2T - 1 to 2T + 1: snapshot
// U(T), two steps of R with the coarse-to-fine transfers, and the correction of the parent's
// step output (ap: the parent's step arguments, in / out / raw of step T).
void child_steps(lb_ctx *ctx, const StepArgs &ap, bool periodic, lb_refine *R, float *trace_row,
                 long long T) {
    float *Ucur = R->U[T & 1], *Uprev = R->U[(T + 1) & 1];
    if (R->coupling == LB_COUPLE_F2C) {  // nothing enters the patch: no snapshot, no transfer
        if (T >= 1) {
            launch_zero_in(ctx, R);
            level_step(ctx, R, nullptr, 2 * T - 1);
        }
        launch_zero_in(ctx, R);
    } else if (T >= 1) {  // snapshot U(T) fused with the midpoint transfer
        launch_snap_c2f(ctx, ap, R, Uprev, Ucur, 0.5f);
        level_step(ctx, R, nullptr, 2 * T - 1);
        launch_c2f(ctx, R, Ucur, Ucur, 1.0f);
    } else {  // snapshot U(0) fused with the transfer at time 0
        launch_snap_c2f(ctx, ap, R, nullptr, Ucur, 1.0f);
    }
    const float *fin_last = static_cast<const float *>(R->pop[R->cur]);
    const int fraw = R->raw ? 1 : 0;
    level_step(ctx, R, trace_row, 2 * T);
    if (R->coupling != LB_COUPLE_C2F) launch_f2c(ctx, ap, periodic, R, fin_last, fraw);
}

void launch_overlay(lb_ctx *ctx, lb_refine *R, float *p) {
    if (R->onx <= 0 || R->ony <= 0) return;
    StepArgs af = level_args(ctx, R);
    af.in = R->pop[R->cur];
    af.raw = R->raw ? 1 : 0;
    const int cnt = R->onx * R->ony;
    if (ctx->Q == 9)
        ref_overlay_kernel<9><<<blocks_for(cnt), 256, 0, ctx->stream>>>(
            af, p, ctx->nx, R->ox0, R->oy0, R->onx, R->ony, R->oA, R->obx, R->oby);
    else
        ref_overlay_kernel<5><<<blocks_for(cnt), 256, 0, ctx->stream>>>(
            af, p, ctx->nx, R->ox0, R->oy0, R->onx, R->ony, R->oA, R->obx, R->oby);
}

// Bring patch R (of a parent at time T, step arguments ap: in / raw) to time 2T without
// committing, write the context-grid pressure of the nodes it covers, then recurse.
void peek_level(lb_ctx *ctx, const StepArgs &ap, lb_refine *R, long long T, float *p) {
    float *Ucur = R->U[2], *Uprev = R->U[(T + 1) & 1];
    if (R->coupling == LB_COUPLE_F2C) {
        if (T >= 1) {
            launch_zero_in(ctx, R);
            level_step(ctx, R, nullptr, 2 * T - 1);
        }
        launch_zero_in(ctx, R);
    } else {
        launch_snapshot(ctx, ap, R, Ucur);
        if (T >= 1) {
            launch_c2f(ctx, R, Uprev, Ucur, 0.5f);
            level_step(ctx, R, nullptr, 2 * T - 1);
        }
        launch_c2f(ctx, R, Ucur, Ucur, 1.0f);
    }
    launch_overlay(ctx, R, p);
    if (R->sub) {
        StepArgs af = level_args(ctx, R);
        af.in = R->pop[R->cur];
        af.raw = R->raw ? 1 : 0;
        peek_level(ctx, af, R->sub, 2 * T, p);
    }
}

// floor(a / b) for b > 0
int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

}  // namespace

// Sets up one refined level: patch P of the parent grid (the context grid when parent is
// null).  Parent speeds pc [..][pnx] in the parent's node coordinates.
static lb_status setup_level(lb_ctx *ctx, const lb_config *cfg, lb_refine *parent,
                             const lb_patch &P, const float *pc, int pnx, bool has_sub,
                             lb_refine **out) {
    const int pn_x = parent ? parent->nxf : ctx->nx, pn_y = parent ? parent->nyf : ctx->ny;
    if (P.ratio != 2) return fail(ctx, LB_EINVAL, "patch ratio must be 2");
    if (P.coupling != LB_COUPLE_BOTH && P.coupling != LB_COUPLE_C2F && P.coupling != LB_COUPLE_F2C)
        return fail(ctx, LB_EINVAL, "patch coupling must be LB_COUPLE_BOTH, _C2F or _F2C");
    if (P.nx_c < 1 || P.ny_c < 1 || P.x0 < 1 || P.y0 < 1 || P.x0 + P.nx_c > pn_x - 2 ||
        P.y0 + P.ny_c > pn_y - 2)
        return fail(ctx, LB_EINVAL,
                    parent ? "a nested patch must lie inside the fine grid above it with a "
                             "1-node margin"
                           : "patch must lie inside the grid with a 1-node margin");
    lb_refine *R = new lb_refine();
    *out = R;
    R->coupling = P.coupling;
    R->depth = parent ? parent->depth + 1 : 1;
    {  // rates of this level (tau_f - 1/2 = 2 (tau_c - 1/2) per relaxed moment) and rescales
        auto fine_tau = [](double tc) { return 0.5 + 2.0 * (tc - 0.5); };
        const double tc = parent ? parent->tau_f : cfg->tau, tf = fine_tau(tc);
        R->tau_f = tf;
        R->omega_f = (float)(1.0 / tf);
        R->c2f_omega = (float)(1.0 - tf / (2.0 * tc));
        R->f2c_omega = (float)(1.0 - 2.0 * tc / tf);
        for (int k = 0; k < 9; k++) {
            const double tck = parent ? parent->stau_f[k] : 1.0 / cfg->s[k], tfk = fine_tau(tck);
            R->stau_f[k] = tfk;
            R->s_f[k] = (float)(1.0 / tfk);
            R->c2f_s[k] = (float)(1.0 - tfk / (2.0 * tck));
            R->f2c_s[k] = (float)(1.0 - 2.0 * tck / tfk);
        }
    }
    const int off = parent ? 1 : 0;  // parent storage = parent node + off
    R->x0n = P.x0;
    R->y0n = P.y0;
    R->x0 = P.x0 + off;
    R->y0 = P.y0 + off;
    R->nxp = P.nx_c;
    R->nyp = P.ny_c;
    R->nxf = 2 * P.nx_c + 1;
    R->nyf = 2 * P.ny_c + 1;
    R->gx = R->nxf + 2;
    R->gy = R->nyf + 2;
    R->pitch = round_up(R->gx, 32);
    // the coarse nodes this level covers: parent node a_p = A_p X + b_p, own node
    // a = 2 (a_p - x0n)
    {
        const int Ap = parent ? parent->oA : 1, bxp = parent ? parent->obx : 0,
                  byp = parent ? parent->oby : 0;
        R->oA = 2 * Ap;
        R->obx = 2 * (bxp - P.x0);
        R->oby = 2 * (byp - P.y0);
        const int xl = -floordiv(-(P.x0 - bxp), Ap), xh = floordiv(P.x0 + P.nx_c - bxp, Ap);
        const int yl = -floordiv(-(P.y0 - byp), Ap), yh = floordiv(P.y0 + P.ny_c - byp, Ap);
        R->ox0 = xl;
        R->oy0 = yl;
        R->onx = std::max(0, xh - xl + 1);
        R->ony = std::max(0, yh - yl + 1);
    }
    const size_t plane = (size_t)R->gy * R->pitch;
    const int Q = ctx->Q;
    for (int b = 0; b < 2; b++) {
        R->pop[b] = dev_alloc(ctx, (size_t)Q * plane * 4);
        if (!R->pop[b]) return fail(ctx, LB_ENOMEM, "fine population buffer");
        cudaMemsetAsync(R->pop[b], 0, (size_t)Q * plane * 4, ctx->stream);
    }
    R->eta2 = static_cast<float *>(dev_alloc(ctx, plane * 4));
    if (!R->eta2) return fail(ctx, LB_ENOMEM, "fine medium");
    if (has_sub) {
        R->cf = static_cast<float *>(dev_alloc(ctx, (size_t)R->nxf * R->nyf * 4));
        R->pf = static_cast<float *>(dev_alloc(ctx, (size_t)R->nxf * R->nyf * 4));
        if (!R->cf || !R->pf) return fail(ctx, LB_ENOMEM, "nested patch medium");
    }
    if (R->depth >= 2) {
        R->bak = dev_alloc(ctx, (size_t)Q * plane * 4);
        if (!R->bak) return fail(ctx, LB_ENOMEM, "nested patch peek buffer");
    }
    ref_medium_kernel<<<blocks_for((long long)plane), 256, 0, ctx->stream>>>(
        pc, pnx, R->x0n, R->y0n, R->nxf, R->nyf, R->gx, R->gy, R->pitch, 1.0 / ctx->cfg.c_ref,
        R->eta2, R->cf);
    // interface node lists (parent storage coordinates)
    std::vector<int2> Ic;
    std::vector<int> idx((size_t)(R->nxp + 1) * (R->nyp + 1), -1);
    for (int Y = R->y0; Y <= R->y0 + R->nyp; Y++)
        for (int X = R->x0; X <= R->x0 + R->nxp; X++)
            if (X == R->x0 || X == R->x0 + R->nxp || Y == R->y0 || Y == R->y0 + R->nyp) {
                idx[(size_t)(Y - R->y0) * (R->nxp + 1) + (X - R->x0)] = (int)Ic.size();
                Ic.push_back(make_int2(X, Y));
            }
    auto kidx = [&](int X, int Y) { return idx[(size_t)(Y - R->y0) * (R->nxp + 1) + (X - R->x0)]; };
    std::vector<int4> If;
    for (int b = 0; b < R->nyf; b++)
        for (int a = 0; a < R->nxf; a++) {
            if (!(a == 0 || a == R->nxf - 1 || b == 0 || b == R->nyf - 1)) continue;
            int X = R->x0 + a / 2, Y = R->y0 + b / 2;
            int k1 = kidx(X, Y), k2 = -1;
            if (a & 1)
                k2 = kidx(X + 1, Y);
            else if (b & 1)
                k2 = kidx(X, Y + 1);
            If.push_back(make_int4(a, b, k1, k2));
        }
    R->nI = (int)Ic.size();
    R->nIf = (int)If.size();
    R->Ic = static_cast<int2 *>(dev_alloc(ctx, Ic.size() * sizeof(int2)));
    R->If = static_cast<int4 *>(dev_alloc(ctx, If.size() * sizeof(int4)));
    for (int s = 0; s < 3; s++) R->U[s] = static_cast<float *>(dev_alloc(ctx, (size_t)R->nI * Q * 4));
    if (!R->Ic || !R->If || !R->U[0] || !R->U[1] || !R->U[2])
        return fail(ctx, LB_ENOMEM, "interface buffers");
    if (R->depth >= 2) {
        for (int s = 0; s < 2; s++) {
            R->Ubak[s] = static_cast<float *>(dev_alloc(ctx, (size_t)R->nI * Q * 4));
            if (!R->Ubak[s]) return fail(ctx, LB_ENOMEM, "nested patch peek buffer");
        }
    }
    cudaMemcpyAsync(R->Ic, Ic.data(), Ic.size() * sizeof(int2), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(R->If, If.data(), If.size() * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);  // the host vectors go out of scope
    if (e != cudaSuccess) return cuda_fail(ctx, e, "refinement setup");
    return check_launch(ctx, "refinement setup");
}

lb_status refine_setup(lb_ctx *ctx, const lb_config *cfg, const float *c_map_dev) {
    if (cfg->storage != LB_F32) return fail(ctx, LB_EINVAL, "refinement needs FP32 storage");
    lb_refine *parent = nullptr;
    const float *pc = c_map_dev;
    int pnx = ctx->nx;
    for (int k = 0; k < cfg->n_patches; k++) {
        lb_refine *R = nullptr;
        lb_status st = setup_level(ctx, cfg, parent, cfg->patches[k], pc, pnx,
                                   k + 1 < cfg->n_patches, &R);
        if (parent)
            parent->sub = R;
        else
            ctx->ref = R;
        if (st != LB_OK) return st;
        parent = R;
        pc = R->cf;
        pnx = R->nxf;
    }
    ctx->refined = true;
    return LB_OK;
}

void refine_destroy(lb_ctx *ctx) {
    delete ctx->ref;  // device buffers are owned by the context's allocation list
    ctx->ref = nullptr;
}

bool refine_contains(const lb_ctx *ctx, int x, int y) {
    const lb_refine *R = ctx->ref;
    return R && x >= R->x0 && x <= R->x0 + R->nxp && y >= R->y0 && y <= R->y0 + R->nyp;
}

static lb_status upload_list(lb_ctx *ctx, const std::vector<int2> &v, const std::vector<int> &c,
                             int2 **dv, int **dc) {
    *dv = static_cast<int2 *>(dev_alloc(ctx, std::max<size_t>(1, v.size()) * sizeof(int2)));
    *dc = static_cast<int *>(dev_alloc(ctx, std::max<size_t>(1, c.size()) * sizeof(int)));
    if (!*dv || !*dc) return fail(ctx, LB_ENOMEM, "receiver lists");
    if (!v.empty()) {
        cudaMemcpyAsync(*dv, v.data(), v.size() * sizeof(int2), cudaMemcpyHostToDevice, ctx->stream);
        cudaMemcpyAsync(*dc, c.data(), c.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
    }
    return LB_OK;
}

// each receiver is recorded on the deepest level whose closed patch holds its node
lb_status refine_set_receivers(lb_ctx *ctx, const int *xy, int nrec) {
    std::vector<lb_refine *> lv;
    for (lb_refine *R = ctx->ref; R; R = R->sub) lv.push_back(R);
    std::vector<std::vector<int2>> pos(lv.size() + 1);
    std::vector<std::vector<int>> col(lv.size() + 1);
    for (int r = 0; r < nrec; r++) {
        int a = xy[2 * r], b = xy[2 * r + 1];  // node coordinates of the current level
        size_t L = 0;
        while (L < lv.size()) {
            const lb_refine *R = lv[L];
            if (a < R->x0n || a > R->x0n + R->nxp || b < R->y0n || b > R->y0n + R->nyp) break;
            a = 2 * (a - R->x0n);
            b = 2 * (b - R->y0n);
            L++;
        }
        pos[L].push_back(L == 0 ? make_int2(a, b) : make_int2(a + 1, b + 1));
        col[L].push_back(r);
    }
    lb_refine *R1 = lv[0];
    R1->nrec_c = (int)pos[0].size();
    lb_status st = upload_list(ctx, pos[0], col[0], &R1->rec_c, &R1->col_c);
    for (size_t L = 1; st == LB_OK && L <= lv.size(); L++) {
        lv[L - 1]->nrec_f = (int)pos[L].size();
        st = upload_list(ctx, pos[L], col[L], &lv[L - 1]->rec_f, &lv[L - 1]->col_f);
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);  // the host vectors go out of scope
    if (st != LB_OK) return st;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "receiver upload");
    return LB_OK;
}

lb_status refine_after_set_state(lb_ctx *ctx, const float *p0_dev) {
    const float *pp = p0_dev;
    int pnx = ctx->nx;
    for (lb_refine *R = ctx->ref; R; R = R->sub) {
        StepArgs af = level_args(ctx, R);
        R->cur = 0;
        af.out = R->pop[0];
        float *pf = (R->sub && pp) ? R->pf : nullptr;
        if (ctx->Q == 9)
            ref_init_fine_kernel<9><<<blocks_for(af.plane), 256, 0, ctx->stream>>>(
                af, pp, pnx, R->x0n, R->y0n, R->nxf, R->nyf, pf);
        else
            ref_init_fine_kernel<5><<<blocks_for(af.plane), 256, 0, ctx->stream>>>(
                af, pp, pnx, R->x0n, R->y0n, R->nxf, R->nyf, pf);
        R->raw = true;
        pp = pf;
        pnx = R->nxf;
    }
    return check_launch(ctx, "refined initial state");
}

// The task shapes a fused launch takes: the coarse step with the snapshot transfer; a fine
// step with its own midpoint transfer (and, above a nested patch, that patch's snapshot);
// a fine step with its correction of the parent (and the nested patch's snapshot).  The
// correction is periodic only towards a periodic coarse grid.
template <int Q, bool MRT>
cudaError_t launch_tasks_q(lb_ctx *ctx, int t1, int t2, bool per, bool f2c_per, const StepArgs &a,
                           int rec_blocks, RefTask x1, RefTask x2) {
    x1.blocks = blocks_for(x1.n);
    x2.blocks = t2 != kTaskNone ? blocks_for(x2.n) : 0;
    const dim3 grid(x1.blocks + x2.blocks + a.main_blocks + rec_blocks), block(kThreads);
    cudaStream_t st = ctx->stream;
    if (t1 == kTaskSnapC2f && t2 == kTaskNone)  // the coarse step (either boundary)
        return per ? launch_pdl(ref_step_kernel<Q, MRT, true, kTaskSnapC2f, false, kTaskNone, false>,
                                grid, block, 0, st, a, x1, x2)
                   : launch_pdl(ref_step_kernel<Q, MRT, false, kTaskSnapC2f, false, kTaskNone, false>,
                                grid, block, 0, st, a, x1, x2);
    if (t1 == kTaskC2f && t2 == kTaskNone)
        return launch_pdl(ref_step_kernel<Q, MRT, false, kTaskC2f, false, kTaskNone, false>, grid,
                          block, 0, st, a, x1, x2);
    if (t1 == kTaskC2f && t2 == kTaskSnapC2f)
        return launch_pdl(ref_step_kernel<Q, MRT, false, kTaskC2f, false, kTaskSnapC2f, false>, grid,
                          block, 0, st, a, x1, x2);
    if (t1 == kTaskF2c && t2 == kTaskNone)
        return f2c_per ? launch_pdl(ref_step_kernel<Q, MRT, false, kTaskF2c, true, kTaskNone, false>,
                                    grid, block, 0, st, a, x1, x2)
                       : launch_pdl(ref_step_kernel<Q, MRT, false, kTaskF2c, false, kTaskNone, false>,
                                    grid, block, 0, st, a, x1, x2);
    if (t1 == kTaskF2c && t2 == kTaskSnapC2f)
        return f2c_per
                   ? launch_pdl(ref_step_kernel<Q, MRT, false, kTaskF2c, true, kTaskSnapC2f, false>,
                                grid, block, 0, st, a, x1, x2)
                   : launch_pdl(ref_step_kernel<Q, MRT, false, kTaskF2c, false, kTaskSnapC2f, false>,
                                grid, block, 0, st, a, x1, x2);
    return cudaErrorInvalidValue;
}

cudaError_t launch_tasks(lb_ctx *ctx, int t1, int t2, bool per, bool f2c_per, const StepArgs &a,
                         int rec_blocks, const RefTask &x1, const RefTask &x2) {
    const bool mrt = ctx->cfg.collision == LB_MRT;
    if (ctx->Q == 9)
        return mrt ? launch_tasks_q<9, true>(ctx, t1, t2, per, f2c_per, a, rec_blocks, x1, x2)
                   : launch_tasks_q<9, false>(ctx, t1, t2, per, f2c_per, a, rec_blocks, x1, x2);
    return mrt ? launch_tasks_q<5, true>(ctx, t1, t2, per, f2c_per, a, rec_blocks, x1, x2)
               : launch_tasks_q<5, false>(ctx, t1, t2, per, f2c_per, a, rec_blocks, x1, x2);
}

// R's snapshot of its parent's step T (args ap) fused with the midpoint transfer into the
// ring of R's input
RefTask snap_task(lb_ctx *ctx, lb_refine *R, const StepArgs &ap, long long T) {
    RefTask x = {};
    x.n = R->nIf;
    x.p = ap;
    x.f = level_args(ctx, R);
    x.f.in = R->pop[R->cur];
    x.rs = rescale_args(x.f, ctx->Q, R->c2f_omega, R->c2f_s);
    x.If = R->If;
    x.Ic = R->Ic;
    x.Ua = R->U[(T + 1) & 1];
    x.Ucur = R->U[T & 1];
    x.alpha = 0.5f;
    x.nxf = R->nxf;
    x.nyf = R->nyf;
    return x;
}

// R's transfer at the parent's time T into the ring of the output of R's step running now
RefTask c2f_task(lb_ctx *ctx, lb_refine *R, long long T) {
    RefTask x = {};
    x.n = R->nIf;
    x.f = level_args(ctx, R);
    x.f.in = R->pop[R->cur ^ 1];
    x.rs = rescale_args(x.f, ctx->Q, R->c2f_omega, R->c2f_s);
    x.If = R->If;
    x.Ua = R->U[T & 1];
    x.Ub = R->U[T & 1];
    x.alpha = 1.f;
    x.nxf = R->nxf;
    x.nyf = R->nyf;
    return x;
}

// R's correction of its parent's step output (args ap) from R's state at its input now
RefTask f2c_task(lb_ctx *ctx, lb_refine *R, const StepArgs &ap) {
    RefTask x = {};
    x.n = R->nI;
    x.p = ap;
    x.rs = rescale_args(ap, ctx->Q, R->f2c_omega, R->f2c_s);
    x.fin = static_cast<const float *>(R->pop[R->cur]);
    x.fraw = 0;
    x.fpitch = R->pitch;
    x.fplane = (long long)R->gy * R->pitch;
    x.Ic = R->Ic;
    x.x0 = R->x0;
    x.y0 = R->y0;
    x.nxp = R->nxp;
    x.nyp = R->nyp;
    return x;
}

// Arguments of R's step t (pull from pop[cur] into pop[cur ^ 1], ring left alone), with R's
// receivers at trace_row; *rec_blocks gets their gather blocks.
StepArgs ring_step_args(lb_ctx *ctx, lb_refine *R, long long t, float *trace_row, int *rec_blocks) {
    StepArgs a = level_args(ctx, R);
    a.in = R->pop[R->cur];
    a.out = R->pop[R->cur ^ 1];
    a.t = t;
    a.ring = 1;
    *rec_blocks = 0;
    if (trace_row && R->nrec_f > 0) {
        a.rec = R->rec_f;
        a.nrec = R->nrec_f;
        a.rec_col = R->col_f;
        a.trace_row = trace_row;
        *rec_blocks = (R->nrec_f + kThreads - 1) / kThreads;
    }
    return a;
}

// R's two steps within its parent's step T (parent step arguments ap; T >= 1, every level
// coupled both ways and none raw), each coupling task in a step launch whose buffers it does
// not touch:
//   R step 2T - 1 (ring left alone) + R's transfer at T into that step's output ring
//     [+ the nested patch's snapshot of this step];  then the nested patch's two steps;
//   R step 2T (receivers) + R's correction of the parent's output of step T from R's input
//     [+ the nested patch's snapshot];  then the nested patch's two steps.
// The parent's snapshot for R rode in the parent's own step launch.  Same per-node code and
// order of dependence as child_steps (the refined-block workload's 256 receiver traces after
// 4000 coarse steps agree with the six-launch run to every printed digit).  A two-level grid
// takes three launches per coarse step instead of six; two nested patches seven instead of
// sixteen.
cudaError_t fused_pair(lb_ctx *ctx, lb_refine *R, const StepArgs &ap, bool ap_periodic,
                       float *trace_row, long long T) {
    lb_refine *S = R->sub;
    int rb = 0;
    StepArgs a1 = ring_step_args(ctx, R, 2 * T - 1, nullptr, &rb);
    RefTask none = {};
    cudaError_t e = launch_tasks(ctx, kTaskC2f, S ? kTaskSnapC2f : kTaskNone, false, false, a1, rb,
                                 c2f_task(ctx, R, T), S ? snap_task(ctx, S, a1, 2 * T - 1) : none);
    if (e == cudaSuccess && S) e = fused_pair(ctx, S, a1, false, nullptr, 2 * T - 1);
    R->cur ^= 1;
    StepArgs a2 = ring_step_args(ctx, R, 2 * T, trace_row, &rb);
    if (e == cudaSuccess)
        e = launch_tasks(ctx, kTaskF2c, S ? kTaskSnapC2f : kTaskNone, false, ap_periodic, a2, rb,
                         f2c_task(ctx, R, ap), S ? snap_task(ctx, S, a2, 2 * T) : none);
    if (e == cudaSuccess && S) e = fused_pair(ctx, S, a2, false, trace_row, 2 * T);
    R->cur ^= 1;
    R->raw = false;
    return e;
}

lb_status refine_step(lb_ctx *ctx, int n) {
    lb_refine *R = ctx->ref;
    StepFn coarse_fn = pick_step(ctx);
    const bool periodic = ctx->cfg.boundary == LB_PERIODIC;
    for (int k = 0; k < n; k++) {
        const long long T = ctx->t;
        long long row = T - ctx->t_rec0;
        float *trace_row = (ctx->trace && row >= 0 && row < ctx->trace_cap)
                               ? ctx->trace + row * ctx->nrec : nullptr;
        // coarse step T
        StepArgs ac = base_args(ctx);
        ac.in = ctx->pop[ctx->cur];
        ac.out = ctx->pop[ctx->cur ^ 1];
        ac.t = T;
        ac.raw = ctx->raw ? 1 : 0;
        ac.rec = R->rec_c;
        ac.nrec = R->nrec_c;
        ac.rec_col = R->col_c;
        ac.trace_row = R->nrec_c > 0 ? trace_row : nullptr;
        int rec_blocks = ac.trace_row ? (R->nrec_c + kThreads - 1) / kThreads : 0;
        bool fused = T >= 1;
        for (const lb_refine *L = R; L; L = L->sub)
            fused = fused && L->coupling == LB_COUPLE_BOTH && !L->raw;
        if (fused) {  // the coarse step with level 1's snapshot, then the levels' pairs
            cudaError_t e = launch_tasks(ctx, kTaskSnapC2f, kTaskNone, periodic, false, ac,
                                         rec_blocks, snap_task(ctx, R, ac, T), RefTask{});
            if (e == cudaSuccess) e = fused_pair(ctx, R, ac, periodic, trace_row, T);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "refined step launch");
        } else {
            launch_pdl(coarse_fn, dim3(ac.main_blocks + rec_blocks), dim3(kThreads), 0, ctx->stream,
                       ac);
            child_steps(ctx, ac, periodic, R, trace_row, T);
        }
        ctx->cur ^= 1;
        ctx->raw = false;
        ctx->t += 1;
    }
    return check_launch(ctx, "refined step");
}

// Pressure at the current time inside the closed patches.  The fine states at the
// current time do not exist yet between steps, so the coupling and the patch sub-steps of
// step t are replayed into the buffers they will overwrite anyway (the spare buffer of
// each level, its ghost ring, and the third U slot).  A nested level also runs its own
// sub-steps during the replay, which overwrite its input buffer and interface snapshots:
// those are saved before and restored after.
lb_status refine_overlay_pressure(lb_ctx *ctx, float *p_dev) {
    std::vector<lb_refine *> lv;
    for (lb_refine *R = ctx->ref; R; R = R->sub) lv.push_back(R);
    std::vector<int> cur0(lv.size());
    std::vector<char> raw0(lv.size());
    const int Q = ctx->Q;
    cudaError_t e = cudaSuccess;
    for (size_t L = 0; L < lv.size(); L++) {
        lb_refine *R = lv[L];
        cur0[L] = R->cur;
        raw0[L] = R->raw ? 1 : 0;
        if (R->depth < 2 || e != cudaSuccess) continue;
        const size_t bytes = (size_t)Q * R->gy * R->pitch * 4, ub = (size_t)R->nI * Q * 4;
        e = cudaMemcpyAsync(R->bak, R->pop[R->cur], bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        for (int s = 0; s < 2 && e == cudaSuccess; s++)
            e = cudaMemcpyAsync(R->Ubak[s], R->U[s], ub, cudaMemcpyDeviceToDevice, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "refined pressure: save");
    StepArgs ac = base_args(ctx);
    ac.in = ctx->pop[ctx->cur];
    ac.raw = ctx->raw ? 1 : 0;
    peek_level(ctx, ac, ctx->ref, ctx->t, p_dev);
    for (size_t L = 0; L < lv.size(); L++) {  // the replay committed nothing
        lb_refine *R = lv[L];
        R->cur = cur0[L];
        R->raw = raw0[L] != 0;
        if (R->depth < 2 || e != cudaSuccess) continue;
        const size_t bytes = (size_t)Q * R->gy * R->pitch * 4, ub = (size_t)R->nI * Q * 4;
        e = cudaMemcpyAsync(R->pop[R->cur], R->bak, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        for (int s = 0; s < 2 && e == cudaSuccess; s++)
            e = cudaMemcpyAsync(R->U[s], R->Ubak[s], ub, cudaMemcpyDeviceToDevice, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "refined pressure: restore");
    return check_launch(ctx, "refined pressure");
}
