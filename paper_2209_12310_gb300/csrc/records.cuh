// records.cuh -- classification of points into sort records (hull rule),
// shared by the single-hull post pass and the batched path.
#pragma once

#include "ch_internal.cuh"
#include "octagon.cuh"

namespace ch {

// Hull-rule classification: -1 = dropped, else queue.  Fast paths: the inner
// region (dropped), and a point that float edge functions put surely beyond
// quad edge r (the first quad edge it is not surely left of) and surely
// outside octagon edge 2r or 2r+1 (the two octagon edges over quad edge r):
// no closed-octagon point is strictly outside an edge, so the point is queue
// r's.  Everything else takes the exact slow path.
__device__ __forceinline__ int classify_hull(float x, float y, const Octagon& o) {
    const int X = __float2int_rn(x), Y = __float2int_rn(y);
    if (in_inner(o, X, Y)) return -1;
    float e[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) e[r] = edge_float(o.quad[r], x, y);
    const int r = e[0] <= kEdgeTol ? 0 : e[1] <= kEdgeTol ? 1 : e[2] <= kEdgeTol ? 2 : e[3] <= kEdgeTol ? 3 : 4;
    if (r < 4) {
        const float er = r == 0 ? e[0] : r == 1 ? e[1] : r == 2 ? e[2] : e[3];
        if (er < -kEdgeTol) {
            if (o.discard_none) return r;
            const float a = edge_float(o.oct[2 * r], x, y), b = edge_float(o.oct[2 * r + 1], x, y);
            if (fminf(a, b) < -kEdgeTol) return r;
        }
    }
    return classify_hull_slow(x, y, &o);
}

// The same fast paths without branches, for loops that classify several
// points at once (their arithmetic interleaves): -1, a queue, or kUndecided
// when the exact slow path must decide.  (X, Y) = (x, y) as integers.
constexpr int kUndecided = 4;
__device__ __forceinline__ int classify_hull_fast(float x, float y, int X, int Y, const Octagon& o) {
    float e[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) e[r] = edge_float(o.quad[r], x, y);
    const int r = e[0] <= kEdgeTol ? 0 : e[1] <= kEdgeTol ? 1 : e[2] <= kEdgeTol ? 2 : e[3] <= kEdgeTol ? 3 : 4;
    const float er = r == 0 ? e[0] : r == 1 ? e[1] : r == 2 ? e[2] : e[3];
    const int rr = r & 3;   // r = 4 reads edges 0 and 1; the result is unused
    const float a = edge_float(o.oct[2 * rr], x, y), b = edge_float(o.oct[2 * rr + 1], x, y);
    const bool sure = r < 4 && er < -kEdgeTol && (o.discard_none || fminf(a, b) < -kEdgeTol);
    return in_inner(o, X, Y) ? -1 : sure ? r : kUndecided;
}

// Records per queue, counted per lane: an 8-bit field per queue in `packed`,
// folded into the 32-bit counts before any field can reach 256 (every 255
// add() calls at most).
struct QueueTally {
    unsigned packed = 0u;
    unsigned n[4] = {0u, 0u, 0u, 0u};
    __device__ __forceinline__ void add(bool keep, int r) { packed += keep ? 1u << ((r & 3) << 3) : 0u; }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int q = 0; q < 4; ++q) n[q] += (packed >> (8 * q)) & 0xFFu;
        packed = 0u;
    }
    // Warp-collective, after fold(): the warp's records of queue q.
    __device__ __forceinline__ unsigned warp_total(int q) const { return __reduce_add_sync(0xFFFFFFFFu, n[q]); }
};

// Survivors on an axis support line of the true octagon (x = xmin, y = ymin,
// x = xmax, y = ymax) lie on a hull edge; only the two extreme ones per line
// can be hull vertices.  They are reduced into ctl->line_ep (minimum and
// maximum along the line, lowest index on ties) instead of becoming records;
// the last block turns the end points into records.
// Warp-collective: every lane passes its candidate (valid = false for none);
// the warp reduces per line first and issues one atomic pair per line.
// Returns whether this lane's point lies on a support line.  One vote settles
// the common case of a warp with no point on any line.
__device__ __forceinline__ bool reduce_on_line(const Octagon& o, bool valid, int X, int Y, unsigned idx, Ctl* ctl) {
    const bool h[4] = {valid && X == o.vx[W], valid && Y == o.vy[S], valid && X == o.vx[E], valid && Y == o.vy[N]};
    const bool on = h[0] || h[1] || h[2] || h[3];
    if (!__any_sync(0xFFFFFFFFu, on)) return false;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const bool hit = h[l];
        if (__any_sync(0xFFFFFFFFu, hit)) {
            const unsigned along = (l & 1) ? (unsigned)X : (unsigned)Y;
            unsigned long long mn = hit ? ((unsigned long long)along << 32) | idx : ~0ull;
            unsigned long long mx = hit ? ((unsigned long long)along << 32) | (0xFFFFFFFFu - idx) : 0ull;
#pragma unroll
            for (int o2 = 16; o2; o2 >>= 1) {
                const unsigned long long a = __shfl_xor_sync(0xFFFFFFFFu, mn, o2);
                const unsigned long long b = __shfl_xor_sync(0xFFFFFFFFu, mx, o2);
                mn = a < mn ? a : mn;
                mx = b > mx ? b : mx;
            }
            if ((threadIdx.x & 31) == 0) {
                atomicMin(&ctl->line_ep[2 * l], mn);
                atomicMax(&ctl->line_ep[2 * l + 1], mx);
            }
        }
    }
    return on;
}

// Record of support line l's end point (slot t = 2 l + {0: minimum, 1:
// maximum}) from its packed reduction; false when the line has no survivor.
__device__ __forceinline__ bool line_record(const Octagon& o, int t, unsigned long long e, uint32_t& key,
                                            uint64_t& val) {
    if ((t & 1) ? e == 0ull : e == ~0ull) return false;
    const int l = t >> 1;
    const int along = (int)(e >> 32);
    const unsigned idx = (t & 1) ? 0xFFFFFFFFu - (unsigned)e : (unsigned)e;
    int X, Y;
    switch (l) {
        case 0: X = o.vx[W]; Y = along; break;
        case 1: X = along; Y = o.vy[S]; break;
        case 2: X = o.vx[E]; Y = along; break;
        default: X = along; Y = o.vy[N]; break;
    }
    const int r = classify_hull_slow((float)X, (float)Y, &o);
    if (r < 0) return false;   // cannot happen: it was a survivor
    uint32_t u, v;
    queue_frame(r, X, Y, u, v);
    key = make_key(r, u);
    val = make_val(v, idx);
    return true;
}

}  // namespace ch
