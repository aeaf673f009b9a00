// star.cuh -- a star-shaped filter polygon for dense data, and its point tests.
//
// When most points survive the octagon (points near a circle, the worst case
// of Table V), the octagon leaves a rim of width ~0.08 R that holds almost
// every point.  A polygon with thousands of vertices that are input points
// hugs the hull far closer.  It is built from a sample: around a centre c,
// the sample is split into kStarBins angular bins and each bin keeps its point
// farthest from c (star.cu); every post-pass block then builds the polygon
// in shared memory (star_finish): it gathers the bins' points, drops some
// reflex vertices, which only enlarges the polygon, checks it exactly, and
// builds the lookup tables of the point tests.
//
// Why dropping points strictly inside it is exact: every vertex is an input
// point, and the polygon is star-shaped around c with every wedge
// (c, V_j, V_j+1) turning counter-clockwise by less than pi and the wedges
// winding once around c (checked exactly).  So it is the union of the
// triangles (c, V_j, V_j+1), each inside the hull of the input; a point in its
// interior is in the interior of the hull, no hull vertex, and so are all its
// duplicates.  The tests below drop a point only when they prove that it lies
// strictly inside; any doubt keeps it.
#pragma once

#include "ch_internal.cuh"

namespace ch {

// The finished polygon (shared memory of a post-pass block):
//   v    vertices relative to c (|.| < 2^24: every orientation is exact in
//        int64), counter-clockwise, the first two repeated after the last;
//   tbl  per bin, the last vertex whose bin comes before it (K - 1 if none);
//   rin  per bin, an integer radius no larger than the distance from c to
//        the line of any edge whose wedge meets the bin or its two
//        neighbours on either side: a point of the bin closer to c than that
//        is strictly inside (0 when no bound was found);
//   rmin the smallest line radius of all edges: a point closer to c than
//        that is strictly inside, whatever its bin (it lies in some wedge,
//        on the inner side of that wedge's edge line).
struct StarPoly {
    int2 v[kStarBins + 2];
    unsigned short tbl[kStarBins];
    unsigned rin[kStarBins];
    unsigned rmin;
    unsigned pad[3];
};

// Angular bin of an offset (dx, dy) from c: a pseudo-angle in [0, 4) that
// grows with the angle (|dy| / (|dx| + |dy|) per quadrant), scaled to
// kStarBins bins.  Float rounding may move a point near a bin boundary to the
// neighbouring bin; no test relies on the bin being right to within one bin.
__device__ __forceinline__ int star_bin(int dx, int dy) {
    const float fx = (float)dx, fy = (float)dy;   // exact: |d| < 2^24
    const float ax = fabsf(fx), ay = fabsf(fy), s = ax + ay;
    const float t = s > 0.0f ? __fdividef(ay, s) : 0.0f;
    const float a = fx >= 0.0f ? (fy >= 0.0f ? t : 4.0f - t) : (fy >= 0.0f ? 2.0f - t : 2.0f + t);
    return (int)(a * (float)(kStarBins / 4)) & (kStarBins - 1);
}

// orient(c, v, p) for v, p given relative to c.
__device__ __forceinline__ long long star_orient_c(int2 v, int px, int py) {
    return (long long)v.x * py - (long long)v.y * px;
}

// Exact test: true only when p = c + (px, py) is strictly inside.  The bin's
// table entry j names the last vertex before the bin; p lies in wedge j
// (V_j, V_j+1) or, when it is past V_j+1, in wedge j+1 (V_j+1's bin may be
// p's own).  The chosen wedge is verified on both spokes, then p must be
// strictly left of the wedge's edge.
__device__ __forceinline__ bool star_inside_exact(int px, int py, int b, const StarPoly& P) {
    const int j = P.tbl[b];
    const int2 a = P.v[j], m = P.v[j + 1], z = P.v[j + 2];
    const bool past_m = star_orient_c(m, px, py) > 0;
    const bool spoke_ok = past_m ? star_orient_c(z, px, py) <= 0 : star_orient_c(a, px, py) >= 0;
    const int2 e0 = past_m ? m : a, e1 = past_m ? z : m;
    const long long side =
        (long long)(e1.x - e0.x) * (py - e0.y) - (long long)(e1.y - e0.y) * (px - e0.x);
    return spoke_ok && side > 0;
}

// Fast test, exact in int64: true when p = c + (px, py) lies closer to c than
// its bin's radius bound, hence strictly inside; false says nothing.
__device__ __forceinline__ bool star_inside_fast(int px, int py, int b, const StarPoly& P) {
    const long long r = (long long)P.rin[b];
    return (long long)px * px + (long long)py * py < r * r;
}

// Full test: the bin's radius bound, then the exact wedge test.
__device__ __forceinline__ bool star_inside(int px, int py, const StarPoly& P) {
    const int b = star_bin(px, py);
    return star_inside_fast(px, py, b, P) || star_inside_exact(px, py, b, P);
}

// The largest integer r with r^2 <= o^2 / l2: the distance from c to an edge
// line with orient(c, A, B) = o and |B - A|^2 = l2 (0 < o < 2^50,
// 0 < l2 < 2^52; the distance is below 2^25), rounded down.  A float
// estimate (four roundings of 2^-24 each: off by less than 8) less 8 is
// raised step by step while (r + 1)^2 l2 <= o^2 holds in exact 128-bit
// arithmetic.  Every loop is bounded; leaving one early only lowers the
// result, and 0 means no bound.
__device__ __forceinline__ unsigned star_line_radius(long long o, long long l2) {
    typedef unsigned __int128 u128;
    const unsigned long long ul = (unsigned long long)l2;
    const u128 oo = (u128)(unsigned long long)o * (unsigned long long)o;
    const float rf = (float)o / sqrtf((float)l2);
    unsigned long long r = rf > 8.0f ? (unsigned long long)rf - 8ull : 0ull;
    for (int it = 0; it < 8 && r > 0ull && (u128)(r * r) * ul > oo; ++it) --r;
    if ((u128)(r * r) * ul > oo) return 0u;
    for (int it = 0; it < 24 && (u128)((r + 1ull) * (r + 1ull)) * ul <= oo; ++it) ++r;
    return (unsigned)r;
}

// Block-wide exclusive scan of one count per thread (warp shuffles, then the
// warp totals in s, one word per warp); returns the thread's offset and
// leaves the total in *total.
template <int T>
__device__ __forceinline__ int star_scan(int c, unsigned* s, int* total) {
    constexpr int kWarps = T / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned incl = (unsigned)c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s[warp] = incl;
    __syncthreads();
    unsigned before = 0u, all = 0u;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const unsigned x = s[w];
        before += w < warp ? x : 0u;
        all += x;
    }
    if (threadIdx.x == 0) *total = (int)all;
    __syncthreads();
    return (int)(before + incl - (unsigned)c);
}

constexpr int kStarSweeps = 4;   // reflex-removal sweeps (alternately even and odd positions)

// Builds the polygon in shared memory, all T threads of the block, from the
// star pass's bins (bins[b]: the packed farthest point of bin b, or 0) around
// c = (cx, cy): work area A (va, ba) and the polygon P, whose first bytes
// double as work area B (vb, bb).  Returns the polygon's vertex count (the
// same in every thread) when it passed its checks and P is ready, else 0;
// leaves the bins as they are.  With kSharedBins the bins are in this
// block's shared memory, and they may share their bytes with work area A:
// every bin is read before the first write to A.
//
// Gather: each non-empty bin's point is re-read from the input by its index
// (so every vertex is an input point of this call, whatever the bins held)
// and kept if it is a valid coordinate and falls in that bin again; the kept
// points, in bin order, are the vertices.
//
// Sweeps: a vertex at an even (then odd) position is dropped when it is
// reflex or flat, orient(V_j-1, V_j, V_j+1) <= 0, and its neighbours still
// turn by less than pi around c, orient(c, V_j-1, V_j+1) > 0; same-parity
// vertices are never neighbours (with K odd, the last vertex sits out the
// even sweeps), so every drop sees its neighbours unchanged.  Dropping a
// reflex vertex adds the triangle (V_j-1, V_j, V_j+1) to the polygon.
//
// Threads own contiguous chunks of the vertex list (the compaction keeps the
// order); each lane walks its chunk from a different start, so that the
// lanes of a warp touch different shared-memory banks.
template <int T, bool kSharedBins = false>
__device__ int star_finish(const unsigned long long* bins, const float* __restrict__ pts, long long n,
                            int cx, int cy, int2* va, unsigned short* ba, StarPoly& P, Ctl* ctl) {
    (void)ctl;   // debug timeline only
    static_assert(T % 32 == 0 && T >= 256 && T <= 1024, "block size");
    constexpr int kPer = kStarBins / T;   // bins per thread: at most 32
    static_assert(sizeof(StarPoly) >= sizeof(int2) * kStarBins + sizeof(unsigned short) * kStarBins,
                  "work area B fits in the polygon");
    int2* vb = P.v;
    unsigned short* bb = reinterpret_cast<unsigned short*>(reinterpret_cast<char*>(P.v) +
                                                           sizeof(int2) * kStarBins);
    __shared__ unsigned s_scan[T / 32];
    __shared__ int s_K, s_bad, s_cross;
    const int t = threadIdx.x, lane = t & 31;
    if (t == 0) { s_bad = 0; s_cross = 0; }
    // 1. gather: bins [t kPer, (t + 1) kPer); all their keys, then all their
    // points, in flight at once
    static_assert(kPer <= 16, "gather registers");
    unsigned kept = 0u;
    int2 d[kPer];
    {
        unsigned long long key[kPer];
#pragma unroll
        for (int i = 0; i < kPer; ++i) key[i] = kSharedBins ? bins[t * kPer + i] : __ldcg(bins + t * kPer + i);
        float2 p[kPer];
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const long long idx = (long long)(unsigned)key[i];
            p[i] = (key[i] != 0ull && idx < n) ? __ldcg(reinterpret_cast<const float2*>(pts) + idx)
                                               : make_float2(-1.0f, -1.0f);
        }
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int b = t * kPer + i;
            const int X = __float2int_rn(p[i].x), Y = __float2int_rn(p[i].y);
            const bool valid = key[i] != 0ull && __int2float_rn(X) == p[i].x && __int2float_rn(Y) == p[i].y &&
                               ((unsigned)(X | Y) >> kCoordBits) == 0u;
            d[i] = make_int2(X - cx, Y - cy);
            if (valid && star_bin(X - cx, Y - cy) == b) kept |= 1u << i;
        }
    }
    {
        const int off = star_scan<T>(__popc(kept), s_scan, &s_K);
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            if (!((kept >> i) & 1u)) continue;
            const int o = off + __popc(kept & ((1u << i) - 1u));
            va[o] = d[i];
            ba[o] = (unsigned short)(t * kPer + i);
        }
    }
    __syncthreads();
    CH_TL(ctl, 9, 1);
    if (s_K < 3) return 0;
    // 2. sweeps, A -> B -> A ...
    int2* src = va; int2* dst = vb;
    unsigned short* bsrc = ba; unsigned short* bdst = bb;
    int idle = 0;   // consecutive sweeps that dropped nothing
    for (int sweep = 0; sweep < kStarSweeps && idle < 2; ++sweep) {
        const int k = s_K;
        if (k <= 3) break;
        const int par = sweep & 1;
        const int chunk = (k + T - 1) / T;   // <= kPer
        const int lo = min(k, t * chunk), hi = min(k, lo + chunk), len = hi - lo;
        const int rot = len > 0 ? lane % len : 0;
        unsigned keep = 0u;
        for (int i = 0; i < len; ++i) {
            int jj = i + rot;
            if (jj >= len) jj -= len;
            const int j = lo + jj;
            bool drop = (j & 1) == par && !((k & 1) && j == k - 1);
            if (drop) {
                const int2 a = src[j == 0 ? k - 1 : j - 1], m = src[j], z = src[j + 1 == k ? 0 : j + 1];
                const long long turn = (long long)(m.x - a.x) * (z.y - a.y) - (long long)(m.y - a.y) * (z.x - a.x);
                drop = turn <= 0 && star_orient_c(a, z.x, z.y) > 0;
            }
            if (!drop) keep |= 1u << jj;
        }
        __syncthreads();   // every read of s_K and src of this sweep is done
        const int off = star_scan<T>(__popc(keep), s_scan, &s_K);
        idle = s_K == k ? idle + 1 : 0;
        for (int i = 0; i < len; ++i) {
            int jj = i + rot;
            if (jj >= len) jj -= len;
            if (!((keep >> jj) & 1u)) continue;
            const int o = off + __popc(keep & ((1u << jj) - 1u));
            dst[o] = src[lo + jj];
            bdst[o] = bsrc[lo + jj];
        }
        __syncthreads();
        int2* tv = src; src = dst; dst = tv;
        unsigned short* tb = bsrc; bsrc = bdst; bdst = tb;
    }
    CH_TL(ctl, 10, 1);
    int K = s_K;
    if (src != va) {   // the list must sit in A before P is written over B
        for (int i = t; i < K; i += T) {
            va[i] = vb[i];
            ba[i] = bb[i];
        }
        __syncthreads();
    }
    // 3. checks: every wedge turns counter-clockwise by less than pi, and
    // exactly one edge crosses the ray from c along +x (the wedges wind once)
    int bad = 0, cross = 0;
    for (int j = t; j < K; j += T) {
        const int2 a = va[j], b = va[j + 1 == K ? 0 : j + 1];
        bad |= star_orient_c(a, b.x, b.y) <= 0;
        cross += (a.y < 0 && b.y >= 0) ? 1 : 0;
    }
    if (bad) atomicOr(&s_bad, 1);
    if (cross) atomicAdd(&s_cross, cross);
    __syncthreads();
    const bool ok = K >= 3 && !s_bad && s_cross == 1;
    if (!ok) return 0;
    // 4. the polygon: vertices, the bin table, then the radius bounds
    for (int j = t; j < K + 2; j += T) P.v[j] = va[j < K ? j : j - K];
    for (int j = t; j < K; j += T) {
        const int b0 = ba[j];
        const int b1 = j + 1 < K ? (int)ba[j + 1] : (int)ba[0] + kStarBins;
        for (int b = b0 + 1; b <= b1; ++b) P.tbl[b & (kStarBins - 1)] = (unsigned short)j;
    }
    __syncthreads();
    CH_TL(ctl, 11, 1);
    // each edge's line radius (work area A is free again), then per bin the
    // smallest over the edges whose wedges can hold its points: from the last
    // vertex before bin b - 2 to the first vertex from bin b + 2 on
    unsigned* er = reinterpret_cast<unsigned*>(va);
    if (t == 0) P.rmin = 0xFFFFFFFFu;
    __syncthreads();
    unsigned emin = 0xFFFFFFFFu;
    for (int e = t; e < K; e += T) {
        const int2 a = P.v[e], c2 = P.v[e + 1];
        const long long o = (long long)a.x * c2.y - (long long)a.y * c2.x;   // > 0 (checked above)
        const long long dx = (long long)c2.x - a.x, dy = (long long)c2.y - a.y;
        er[e] = star_line_radius(o, dx * dx + dy * dy);
        emin = min(emin, er[e]);
    }
    emin = __reduce_min_sync(0xFFFFFFFFu, emin);
    if (lane == 0 && emin != 0xFFFFFFFFu) atomicMin(&P.rmin, emin);
    __syncthreads();
    CH_TL(ctl, 12, 1);
    for (int b = t; b < kStarBins; b += T) {
        int e = P.tbl[(b - 2) & (kStarBins - 1)];
        int last = P.tbl[(b + 2) & (kStarBins - 1)] + 1;
        if (last == K) last = 0;
        unsigned m = er[e];
        int steps = 0;
        while (e != last && steps < 8) {
            e = e + 1 == K ? 0 : e + 1;
            m = min(m, er[e]);
            ++steps;
        }
        P.rin[b] = e == last ? m : 0u;   // a window longer than 8 edges gets no bound
    }
    __syncthreads();
    return K;
}

}  // namespace ch
