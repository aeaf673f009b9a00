// octagon.cuh -- the filter polygon CP(E) of Alg. 1/2 and its point tests.
//
// The octagon has the 8 extreme points as vertices, counter-clockwise
// W, SW, S, SE, E, NE, N, NW.  Point tests:
//   * paper rule (ch_filter labels, Alg. 2): discard p when it is STRICTLY
//     inside the octagon;
//   * hull rule (ch_hull): discard p when it is in the CLOSED octagon.  A point
//     on an edge but not at a vertex lies between two input points and is no
//     strictly convex hull vertex; a point at a vertex is a duplicate of an
//     extreme, whose record carries the lowest index.  The hull is unchanged;
//     collinear boundary points (common when coordinates clamp) are dropped
//     early instead of in the hull stage.
// An octagon of zero area discards nothing under either rule.
//
// Fast path: an inner region I = {x in [xl,xh], y in [yl,yh], x+y in [sl,sh],
// x-y in [dl,dh]} (an octagon with axis and diagonal edges) verified exactly to
// lie in the closed octagon.  Its bounds compare directly against the 8 keys
// that pass 1 already computes, so a whole tile whose key extremes lie in I is
// discarded with 8 comparisons.  Edge functions are evaluated in float with a
// proven error bound (kEdgeTol) and fall back to exact int64 in the band.
#pragma once

#include "ch_internal.cuh"

namespace ch {

__device__ __forceinline__ Edge make_edge(int ax, int ay, int bx, int by) {
    Edge e;
    e.ax = ax; e.ay = ay;
    e.dx = bx - ax; e.dy = by - ay;
    if (e.dx == 0 && e.dy == 0) {
        e.A = 0.0f; e.B = 0.0f; e.C = kHugePositive;
    } else {
        // orient(a, b, p) = dx*py - dy*px + (dy*ax - dx*ay) = A*px + B*py + C.
        // A, B, px, py are exact in fp32 (|.| < 2^24); C (|C| < 2^49) is rounded
        // once; each of the two FMAs adds at most half an ulp of a result below
        // 2^50 and 2^51.  Total error < 2^25 + 2^26 + 2^27 < 2^28 = kEdgeTol.
        e.A = (float)(-e.dy);
        e.B = (float)e.dx;
        e.C = __ll2float_rn((long long)e.dy * ax - (long long)e.dx * ay);
    }
    return e;
}

__device__ __forceinline__ long long edge_exact(const Edge& e, long long px, long long py) {
    return (long long)e.dx * (py - e.ay) - (long long)e.dy * (px - e.ax);
}

__device__ __forceinline__ float edge_float(const Edge& e, float x, float y) {
    return fmaf(e.A, x, fmaf(e.B, y, e.C));
}

__device__ __forceinline__ bool in_closed_octagon_exact(const Octagon& o, long long px, long long py) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const Edge& e = o.oct[k];
        if ((e.dx | e.dy) == 0) continue;
        if (edge_exact(e, px, py) < 0) return false;
    }
    return true;
}

// Inner-region membership from the pass-1 keys (X, Y, S = X + Y, D = X - Y + 2^24).
__device__ __forceinline__ bool in_inner(const Octagon& o, int X, int Y) {
    const int S = X + Y, D = X - Y + kCoordLimit;
    return X >= o.in_lo[0] && X <= o.in_hi[0] && Y >= o.in_lo[1] && Y <= o.in_hi[1] &&
           S >= o.in_lo[2] && S <= o.in_hi[2] && D >= o.in_lo[3] && D <= o.in_hi[3];
}

__device__ __forceinline__ bool in_inner_strict(const Octagon& o, int X, int Y) {
    const int S = X + Y, D = X - Y + kCoordLimit;
    return X > o.in_lo[0] && X < o.in_hi[0] && Y > o.in_lo[1] && Y < o.in_hi[1] &&
           S > o.in_lo[2] && S < o.in_hi[2] && D > o.in_lo[3] && D < o.in_hi[3];
}

// Hull rule: -1 when p is in the closed octagon (or on the quadrilateral),
// else its queue 0..3.  Out of line: the inner-region test settles most points.
static __device__ __noinline__ int classify_hull_slow(float x, float y, const Octagon* op) {
    const Octagon& o = *op;
    if (!o.discard_none) {
        float m = kHugePositive;
#pragma unroll
        for (int k = 0; k < 8; ++k) m = fminf(m, edge_float(o.oct[k], x, y));
        if (m > kEdgeTol) return -1;                            // surely inside
        if (m >= -kEdgeTol && in_closed_octagon_exact(o, (long long)x, (long long)y)) return -1;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const Edge& q = o.quad[r];
        const float e = edge_float(q, x, y);
        if (e < -kEdgeTol) return r;
        if (e <= kEdgeTol && (q.dx | q.dy) != 0 && edge_exact(q, (long long)x, (long long)y) < 0) return r;
    }
    return -1;
}

// Paper rule: -1 when p is strictly inside the octagon (or in no queue).
static __device__ __noinline__ int classify_paper_slow(float x, float y, const Octagon* op) {
    const Octagon& o = *op;
    if (!o.discard_none) {
        float m = kHugePositive;
#pragma unroll
        for (int k = 0; k < 8; ++k) m = fminf(m, edge_float(o.oct[k], x, y));
        if (m > kEdgeTol) return -1;
        if (m >= -kEdgeTol) {
            bool inside = true;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const Edge& e = o.oct[k];
                if ((e.dx | e.dy) == 0) continue;
                if (edge_exact(e, (long long)x, (long long)y) <= 0) inside = false;
            }
            if (inside) return -1;
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const Edge& q = o.quad[r];
        const float e = edge_float(q, x, y);
        if (e < -kEdgeTol) return r;
        if (e <= kEdgeTol && (q.dx | q.dy) != 0 && edge_exact(q, (long long)x, (long long)y) < 0) return r;
    }
    return -1;
}

// Strictly outside the closed octagon (the survivor test against a sample
// octagon; no queue needed).  Degenerate octagons keep everything.
static __device__ __noinline__ bool outside_closed_slow(float x, float y, const Octagon* op) {
    const Octagon& o = *op;
    if (o.discard_none) return true;
    float m = kHugePositive;
#pragma unroll
    for (int k = 0; k < 8; ++k) m = fminf(m, edge_float(o.oct[k], x, y));
    if (m > kEdgeTol) return false;
    if (m < -kEdgeTol) return true;
    return !in_closed_octagon_exact(o, (long long)x, (long long)y);
}

// Inner region I(t): the 8-direction bounds of the octagon's own vertices,
// shrunk about their centre by t/1024.  Its candidate vertices (the
// intersections of consecutive bounding lines, integer points) span a polygon
// that contains I(t), so all candidates in the closed octagon imply I(t) is.
__device__ __forceinline__ void inner_bounds(const int lo0[4], const int hi0[4], int t, int lo[4], int hi[4]) {
    const long long cx = ((long long)lo0[0] + hi0[0]) / 2, cy = ((long long)lo0[1] + hi0[1]) / 2;
    const long long c[4] = {cx, cy, cx + cy, cx - cy + kCoordLimit};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        lo[k] = (int)(c[k] - (c[k] - lo0[k]) * t / 1024);
        hi[k] = (int)(c[k] + (hi0[k] - c[k]) * t / 1024);
    }
}

// Candidate vertex k of the region with bounds lo / hi: the intersection of
// consecutive bounding lines x=xl, x+y=sl, y=yl, x-y=dh, x=xh, x+y=sh, y=yh,
// x-y=dl (in that order).
__device__ __forceinline__ void inner_corner(const int lo[4], const int hi[4], int k, long long& px, long long& py) {
    const long long xl = lo[0], xh = hi[0], yl = lo[1], yh = hi[1];
    const long long sl = lo[2], sh = hi[2], dl = lo[3] - kCoordLimit, dh = hi[3] - kCoordLimit;
    switch (k) {
        case 0: px = xl; py = sl - xl; break;
        case 1: px = sl - yl; py = yl; break;
        case 2: px = dh + yl; py = yl; break;
        case 3: px = xh; py = xh - dh; break;
        case 4: px = xh; py = sh - xh; break;
        case 5: px = sh - yh; py = yh; break;
        case 6: px = dl + yh; py = yh; break;
        default: px = xl; py = xl - dl; break;
    }
}

__device__ __forceinline__ bool inner_fits(const Octagon& o, const int lo[4], const int hi[4]) {
    if (lo[0] > hi[0] || lo[1] > hi[1] || lo[2] > hi[2] || lo[3] > hi[3]) return false;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        long long px, py;
        inner_corner(lo, hi, k, px, py);
        if (!in_closed_octagon_exact(o, px, py)) return false;
    }
    return true;
}

// Fills every field of o (in shared memory) from the 8 vertices.  The whole
// block calls it (all threads, same arguments; blockDim.x >= 64).  Threads
// 0..7 build the edges, 8..11 the quadrilateral; with with_inner, the block
// then searches the inner region's scale t/1024: rounds of a 4-way search in
// which each of up to 3 candidate scales has its 64 (corner, edge) exact
// tests done by 64 threads at once.  Only scales whose test passed are kept,
// so the region is verified whatever the search finds.  Without with_inner
// the inner region is empty (every test takes the exact path).
static __device__ void setup_octagon_block(Octagon& o, const int vx[8], const int vy[8], const int ext[8],
                                           bool with_inner) {
    __shared__ long long s_area[8];
    __shared__ int s_lo, s_hi, s_bad[3];
    const int tid = (int)threadIdx.x;
    if (tid < 8) {
        const int j = (tid + 1) & 7;
        o.vx[tid] = vx[tid];
        o.vy[tid] = vy[tid];
        o.ext[tid] = ext[tid];
        o.oct[tid] = make_edge(vx[tid], vy[tid], vx[j], vy[j]);
        s_area[tid] = (long long)vx[tid] * vy[j] - (long long)vx[j] * vy[tid];
    } else if (tid < 12) {
        const int r = tid - 8, a = 2 * r, b = (2 * r + 2) & 7;
        o.quad[r] = make_edge(vx[a], vy[a], vx[b], vy[b]);
    }
    if (tid == 0) {
        s_lo = 0;      // the largest scale verified so far (0: none)
        s_hi = 1025;   // a scale known not to fit
    }
    __syncthreads();
    long long area2 = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) area2 += s_area[k];
    const bool none = area2 == 0;
    // 8-direction bounds of the octagon's vertices: x, y, x+y, x-y (biased).
    const int lo0[4] = {vx[W], vy[S], vx[SW] + vy[SW], vx[NW] - vy[NW] + kCoordLimit};
    const int hi0[4] = {vx[E], vy[N], vx[NE] + vy[NE], vx[SE] - vy[SE] + kCoordLimit};
    if (with_inner && !none) {
        // thread: candidate j = tid / 64, corner k = (tid / 8) % 8, edge e = tid % 8;
        // nc = 3 (or 1 for blocks below 192 threads) candidates split (lo, hi)
        // into nc + 1 = 2^sh parts (32-bit arithmetic, shifts only)
        const int j = tid >> 6, k = (tid >> 3) & 7, e = tid & 7;
        const int nc = blockDim.x >= 192 ? 3 : 1, sh = blockDim.x >= 192 ? 2 : 1;
        const Edge ed = o.oct[e];
        for (int round = 0; round < 12; ++round) {
            const int lo = s_lo, hi = s_hi;
            if (hi - lo <= 1) break;
            if (tid < 3) s_bad[tid] = 0;
            __syncthreads();
            const int t = lo + (((hi - lo) * (j + 1)) >> sh);
            if (j < nc && t > lo && t < hi) {
                int bl[4], bh[4];
                inner_bounds(lo0, hi0, t, bl, bh);
                bool bad = bl[0] > bh[0] || bl[1] > bh[1] || bl[2] > bh[2] || bl[3] > bh[3];
                if (!bad && (ed.dx | ed.dy) != 0) {
                    long long px, py;
                    inner_corner(bl, bh, k, px, py);
                    bad = edge_exact(ed, px, py) < 0;
                }
                if (bad) s_bad[j] = 1;
            }
            __syncthreads();
            if (tid == 0) {   // the largest passing candidate; the next failing one above it
                int nlo = lo, nhi = hi;
                for (int c = 0; c < nc; ++c) {
                    const int tc = lo + (((hi - lo) * (c + 1)) >> sh);
                    if (tc <= lo || tc >= hi) continue;
                    if (!s_bad[c]) nlo = tc > nlo ? tc : nlo;
                }
                for (int c = nc - 1; c >= 0; --c) {
                    const int tc = lo + (((hi - lo) * (c + 1)) >> sh);
                    if (tc > nlo && tc < nhi && s_bad[c]) nhi = tc;
                }
                s_lo = nlo;
                s_hi = nhi;
            }
            __syncthreads();
        }
    }
    if (tid == 0) {
        o.discard_none = none;
        const int t1 = (with_inner && !none) ? s_lo : 0;
        if (t1 > 0) {
            int lo[4], hi[4];
            inner_bounds(lo0, hi0, t1, lo, hi);
            for (int k = 0; k < 4; ++k) { o.in_lo[k] = lo[k]; o.in_hi[k] = hi[k]; }
        } else {
            for (int k = 0; k < 4; ++k) { o.in_lo[k] = 1; o.in_hi[k] = 0; }   // empty
        }
    }
    __syncthreads();
}

// Surely strictly inside the sample octagon: every edge function above the
// float error bound (zero-length edges evaluate to a huge constant).  The
// sample octagon's vertices are input points, so its interior lies in the
// interior of the hull: such a point is no hull vertex, whatever the true
// octagon turns out to be.  Edges as (A, B, C) triples in shared memory.
__device__ __forceinline__ bool pt_in_sample(float x, float y, const float* e) {
    float m = kHugePositive;
#pragma unroll
    for (int k = 0; k < 8; ++k) m = fminf(m, fmaf(e[3 * k], x, fmaf(e[3 * k + 1], y, e[3 * k + 2])));
    return m > kEdgeTol;
}

// Strictly inside an inner region given as lo = in[0..3], hi = in[4..7]
// (bounds of x, y, x+y, x-y+2^24).
__device__ __forceinline__ bool pt_in_inner(int X, int Y, const int* in) {
    const int S = X + Y, D = X - Y + kCoordLimit;
    return X > in[0] && X < in[4] && Y > in[1] && Y < in[5] && S > in[2] && S < in[6] && D > in[3] && D < in[7];
}

__device__ __forceinline__ void copy_octagon(Octagon* dst, const Octagon* src) {
    const int words = (int)(sizeof(Octagon) / 4);
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < words; i += blockDim.x) d[i] = s[i];
}

}  // namespace ch
