// star.cuh -- a star-shaped filter polygon for dense data, and its point test.
//
// When most points survive the octagon (points near a circle, the worst case
// of Table V), the octagon leaves a rim of width ~0.08 R that holds almost
// every point.  A polygon with thousands of vertices that are input points
// hugs the hull far closer.  It is built from a sample (star.cu): around a
// centre c strictly inside it, the sample is split into kStarBins angular
// bins and each bin keeps its point farthest from c; the kept points, in
// angular order, are the polygon's vertices (some reflex vertices are then
// dropped, which only enlarges it).
//
// Why dropping points strictly inside it is exact: every vertex is an input
// point, and the polygon is star-shaped around c with every wedge
// (c, V_j, V_j+1) turning counter-clockwise by less than pi and the wedges
// winding once around c (checked exactly when it is built).  So it is the
// union of the triangles (c, V_j, V_j+1), each inside the hull of the input;
// a point in its interior is in the interior of the hull, no hull vertex,
// and so are all its duplicates.  The test below drops a point only when it
// proves, with exact integer orientations, that the point lies in a closed
// wedge and strictly on c's side of that wedge's edge; any doubt keeps it.
#pragma once

#include "ch_internal.cuh"

namespace ch {

// The polygon as the post pass reads it: vertices relative to c (|.| < 2^24,
// so every orientation below is exact in int64), counter-clockwise, with the
// first two repeated after the last so that j + 2 needs no wrap; per angular
// bin, the last vertex whose bin comes before it (K - 1 when none does).
struct StarPoly {
    int2 v[kStarBins + 2];
    unsigned short tbl[kStarBins];
};
constexpr size_t kStarPolyBytes = sizeof(StarPoly);

// Angular bin of an offset (dx, dy) from c: a pseudo-angle in [0, 4) that
// grows with the angle (|dy| / (|dx| + |dy|) per quadrant), scaled to
// kStarBins bins.  Float rounding may move a point near a bin boundary to
// the neighbouring bin; the test never relies on the bin being right.
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

// True only when p = c + (px, py) is strictly inside the polygon.  The bin's
// table entry j names the last vertex before the bin; p lies in wedge j
// (V_j, V_j+1) or, when it is past V_j+1, in wedge j+1 (V_j+1's bin may be
// p's own).  The chosen wedge is verified on both spokes, then p must be
// strictly left of the wedge's edge.
__device__ __forceinline__ bool star_inside(int px, int py, const int2* __restrict__ v,
                                            const unsigned short* __restrict__ tbl) {
    const int j = tbl[star_bin(px, py)];
    const int2 a = v[j], m = v[j + 1], z = v[j + 2];
    const bool past_m = star_orient_c(m, px, py) > 0;
    const bool spoke_ok = past_m ? star_orient_c(z, px, py) <= 0 : star_orient_c(a, px, py) >= 0;
    const int2 e0 = past_m ? m : a, e1 = past_m ? z : m;
    const long long side =
        (long long)(e1.x - e0.x) * (py - e0.y) - (long long)(e1.y - e0.y) * (px - e0.x);
    return spoke_ok && side > 0;
}

}  // namespace ch
