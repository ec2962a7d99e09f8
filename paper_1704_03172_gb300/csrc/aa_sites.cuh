// aa_sites.cuh -- pieces of the in-place ("AA") step shared by the register-streaming
// kernel (aa.cu) and the TMA-staged one (stream_step.cu): receiver lists, the exchange
// step's pushes and its ghost zeros.  The layout and the two step forms are described in
// aa.cu.
#pragma once

#include "lb_kernels.cuh"

namespace lbaa {

using namespace lbk;

struct AaRec {           // receivers by row, x ascending (tb5_set_receivers' lists)
    const int *row_off;  // [ny + 1], or nullptr: no receivers this step
    const int *rec_x;
    const int *rec_id;
};

// Row of a site in direction dy from row y: wrapped, or -1 outside a zero-ghost domain.
template <bool PERIODIC> __device__ __forceinline__ int row_at(int y, int dy, int ny) {
    int r = y + dy;
    if (r < 0 || r >= ny) {
        if (!PERIODIC) return -1;
        r = r < 0 ? r + ny : r - ny;
    }
    return r;
}

// Push a thread's V values of one population one site along x into the target row dst:
// the value of site x goes to x + CX.  A lane stores a 16-byte vector when every element's
// source site is real and held in its warp (the element next to its own sites comes from
// the neighbouring lane by a shuffle), else element by element; the element a warp's edge
// lane cannot get is stored by the neighbouring warp's edge lane, and the periodic images
// by the owners of the first and last site.  Every lane of the warp calls it.
template <int CX, bool PERIODIC, typename ST>
__device__ __forceinline__ void push_x(ST *dst, const float (&v)[Store<ST>::V], int x0, int lane,
                                       int nx, bool active) {
    constexpr int V = Store<ST>::V;
    if (CX == 1) {  // position p takes site p - 1
        const float left = __shfl_up_sync(0xffffffffu, v[V - 1], 1);
        if (!active) return;
        if (lane > 0) {
            float out[V];
            out[0] = left;
#pragma unroll
            for (int k = 1; k < V; k++) out[k] = v[k - 1];
            Store<ST>::storeV(dst + x0, out);  // positions past nx are padding
        } else {  // position x0 is stored by the previous warp's last lane
#pragma unroll
            for (int k = 1; k < V; k++)
                if (x0 + k < nx) Store<ST>::store1(dst + x0 + k, v[k - 1]);
        }
        if (lane == 31 && x0 + V < nx) Store<ST>::store1(dst + x0 + V, v[V - 1]);
        if (PERIODIC) {  // site nx - 1 wraps to position 0
            const int last = nx - 1 - x0;
#pragma unroll
            for (int k = 0; k < V; k++)
                if (k == last) Store<ST>::store1(dst, v[k]);
        }
    } else {  // CX == -1: position p takes site p + 1
        const float right = __shfl_down_sync(0xffffffffu, v[0], 1);
        if (!active) return;
        if (lane < 31 && x0 + V < nx) {
            float out[V];
#pragma unroll
            for (int k = 0; k + 1 < V; k++) out[k] = v[k + 1];
            out[V - 1] = right;
            Store<ST>::storeV(dst + x0, out);
        } else {  // position x0 + V - 1 takes the next warp's site, or none
#pragma unroll
            for (int k = 0; k + 1 < V; k++)
                if (x0 + k + 1 < nx) Store<ST>::store1(dst + x0 + k, v[k + 1]);
        }
        if (lane == 0 && x0 > 0) Store<ST>::store1(dst + x0 - 1, v[0]);
        if (PERIODIC && x0 == 0) Store<ST>::store1(dst + nx - 1, v[0]);  // site 0 wraps
    }
}

// The exchange step's stores: h_i(x) into slot i at x + c_i, and the ghost's zeros.  Every
// lane of the warp calls it (inactive lanes take part in the shuffles only).
template <int Q, bool PERIODIC, typename ST>
__device__ __forceinline__ void exchange_stores(const StepArgs &a, ST *pop,
                                                const float (&g)[Q][Store<ST>::V], int y, int x0,
                                                int lane, bool active) {
    constexpr int V = Store<ST>::V;
    const long long row = (long long)y * a.pitch;
#pragma unroll
    for (int i = 0; i < Q; i++) {  // h_i(x) into slot i at x + c_i
        const int cx = Lat<Q>::cx(i);
        ST *plane = pop + i * a.plane;
        const int rd = row_at<PERIODIC>(y, Lat<Q>::cy(i), a.ny);  // warp-uniform
        if (rd >= 0) {
            ST *dst = plane + (long long)rd * a.pitch;
            if (cx == 0) {
                if (active) Store<ST>::storeV(dst + x0, g[i]);  // padding sites carry zeros
            } else if (cx == 1) {
                push_x<1, PERIODIC, ST>(dst, g[i], x0, lane, a.nx, active);
            } else {
                push_x<-1, PERIODIC, ST>(dst, g[i], x0, lane, a.nx, active);
            }
        }
        if (!PERIODIC && i != 0 && active) {
            // the ghost's zero in slot i of this thread's sites x whose x - c_i lies outside
            // (no site pushes there)
            const bool row_out = row_at<false>(y, -Lat<Q>::cy(i), a.ny) < 0;
            if (row_out) {
                float z[V];
#pragma unroll
                for (int k = 0; k < V; k++) z[k] = 0.f;
                Store<ST>::storeV(plane + row + x0, z);
            } else if (cx == 1 && x0 == 0) {
                Store<ST>::store1(plane + row, 0.f);
            } else if (cx == -1 && a.nx - 1 - x0 < V) {
                Store<ST>::store1(plane + row + a.nx - 1, 0.f);
            }
        }
    }
}

// Receivers among a thread's V sites (x ascending in the row's list): rho times c_s^2 at
// each, from the populations g(t) streamed in, summed in the order step_kernel sums them.
template <int Q, typename ST>
__device__ __forceinline__ void aa_receivers(const StepArgs &a, const AaRec &r,
                                             const float (&g)[Q][Store<ST>::V], int y, int x0) {
    constexpr int V = Store<ST>::V;
    const long long row = (long long)y * a.pitch;
    if (a.trace_row && r.row_off) {  // receivers among this thread's sites (x ascending)
        int lo = r.row_off[y];
        const int hi = r.row_off[y + 1];
        if (lo < hi) {
            int h = hi;
            while (lo < h) {
                const int m = (lo + h) >> 1;
                if (r.rec_x[m] < x0)
                    lo = m + 1;
                else
                    h = m;
            }
            for (; lo < hi && r.rec_x[lo] < x0 + V; lo++) {
                const int k = r.rec_x[lo] - x0;
                float rho = 0.f;
#pragma unroll
                for (int kk = 0; kk < V; kk++)
                    if (kk == k) {
#pragma unroll
                        for (int i = 0; i < Q; i++) rho += g[i][kk];
                    }
                const int q = r.rec_id[lo];
                a.trace_row[a.rec_col ? a.rec_col[q] : q] =
                    cs2_of<Q>(a.eta2[row + x0 + k], a) * rho;
            }
        }
    }
}

// The exchange step's push of h_s for a warp with no site on a face and no padding: h_s(x)
// into slot s at x + c_s, where dst is slot s's target row (row y + c_s,y).  A lane stores
// a 16-byte vector whose element next to its own sites comes from the neighbouring lane;
// the one a warp's edge lane cannot get is stored by the neighbouring warp's edge lane.
// Every lane of the warp calls it.
template <int Q, typename ST>
__device__ __forceinline__ void push_inner(ST *dst, int s, const float (&v)[Store<ST>::V], int x0,
                                           int lane) {
    constexpr int V = Store<ST>::V;
    if (Lat<Q>::cx(s) == 0) {
        Store<ST>::storeV(dst + x0, v);
    } else if (Lat<Q>::cx(s) == 1) {  // position p takes site p - 1
        const float left = __shfl_up_sync(0xffffffffu, v[V - 1], 1);
        if (lane > 0) {
            float out[V];
            out[0] = left;
#pragma unroll
            for (int k = 1; k < V; k++) out[k] = v[k - 1];
            Store<ST>::storeV(dst + x0, out);
        } else {  // position x0 is the previous warp's
#pragma unroll
            for (int k = 1; k < V; k++) Store<ST>::store1(dst + x0 + k, v[k - 1]);
        }
        if (lane == 31) Store<ST>::store1(dst + x0 + V, v[V - 1]);
    } else {  // position p takes site p + 1
        const float right = __shfl_down_sync(0xffffffffu, v[0], 1);
        if (lane < 31) {
            float out[V];
#pragma unroll
            for (int k = 0; k + 1 < V; k++) out[k] = v[k + 1];
            out[V - 1] = right;
            Store<ST>::storeV(dst + x0, out);
        } else {  // position x0 + V - 1 is the next warp's
#pragma unroll
            for (int k = 0; k + 1 < V; k++) Store<ST>::store1(dst + x0 + k, v[k + 1]);
        }
        if (lane == 0) Store<ST>::store1(dst + x0 - 1, v[0]);
    }
}

// Collision, source and sponge of a thread's V sites as finish_sites does them (the damping
// variant for a warp that holds sponge or padding sites; elsewhere both give the same values).
// Every active lane of the warp calls it.
template <int Q, bool MRT, int V>
__device__ __forceinline__ void aa_collide(const StepArgs &a, float (&g)[Q][V],
                                           const float (&e2s)[V], int y, int x0) {
    const int dyz = row_face_dist<Q>(y, a);
    bool edge = (a.sponge_w > 0 && (dyz < a.sponge_w || x0 < a.sponge_w ||
                                    x0 + V - 1 >= a.nx - a.sponge_w)) ||
                x0 + V > a.nx;
    edge = __any_sync(__activemask(), edge);
    const bool has_src = (y == a.src_y) && (a.src_x >= x0) && (a.src_x < x0 + V) &&
                         a.src_tab != nullptr && a.t < a.src_nt;
    collide_sites_any<Q, MRT, V>(g, e2s, a, x0, dyz, has_src, edge);
}

}  // namespace lbaa
