// extremes.cuh -- the 8 directional extremes of a stream of points, per lane
// (findExtremes, Alg. 2; Sec. 3): the keys, their three-input min / max, and
// the tracking of the first warp tile reaching each extreme.  Shared by the
// single hull's main pass and the batched extremes pass.
#pragma once

#include "ch_internal.cuh"

#include <climits>

namespace ch {

__device__ __forceinline__ bool dir_is_max(int d) { return d >= SE && d <= N; }

__device__ __forceinline__ int dir_key(int d, int X, int Y) {
    switch (d) {
        case W: case E: return X;
        case S: case N: return Y;
        case SW: case NE: return X + Y;
        default: return X - Y + kCoordLimit;
    }
}

// Three-input max / min of non-negative int keys through their float bit
// patterns: below 2^26 the patterns are positive finite floats (subnormal
// below 2^23) that order like the integers; max.f32 without .ftz keeps
// subnormals exact.
__device__ __forceinline__ int kmax3(int a, int b, int c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(__int_as_float(a)), "f"(__int_as_float(b)), "f"(__int_as_float(c)));
    return __float_as_int(r);
}
__device__ __forceinline__ int kmin3(int a, int b, int c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(__int_as_float(a)), "f"(__int_as_float(b)), "f"(__int_as_float(c)));
    return __float_as_int(r);
}

// Tracking.  Each lane keeps, per direction, its best key and the first warp
// tile (code) where that key occurred; tiles are visited in increasing index
// order, so strict improvement keeps the earliest tile.  The answer over all
// lanes is the maximum of (key, ~code) packed in 64 bits: the best key and,
// among tiles reaching it, the lowest; a rescan of that tile finds the lowest
// index.  Tile codes: 0 = unaligned head point, t + 1 = body warp tile t,
// ntiles + 1 = ragged tail.
struct Track {
    int best[8];
    unsigned code[8];
    bool bad;
    unsigned orv;
};

__device__ __forceinline__ void track_init(Track& tr) {
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        tr.best[d] = dir_is_max(d) ? INT_MIN : INT_MAX;
        tr.code[d] = 0u;
    }
    tr.bad = false;
    tr.orv = 0u;
}

// Converts one point and folds its validity (integer value in [0, 2^24)).
__device__ __forceinline__ void convert_pt(float x, float y, int& X, int& Y, Track& tr) {
    X = __float2int_rn(x);
    Y = __float2int_rn(y);
    tr.bad |= (__int2float_rn(X) != x) | (__int2float_rn(Y) != y);
    tr.orv |= (unsigned)X | (unsigned)Y;
}

__device__ __forceinline__ void tile_keys2(int (&tk)[8], int X0, int Y0, int X1, int Y1, bool first) {
    const int s0 = X0 + Y0, s1 = X1 + Y1;
    const int d0 = X0 - Y0 + kCoordLimit, d1 = X1 - Y1 + kCoordLimit;
    if (first) {
        tk[W] = min(X0, X1); tk[SW] = min(s0, s1); tk[S] = min(Y0, Y1); tk[SE] = max(d0, d1);
        tk[E] = max(X0, X1); tk[NE] = max(s0, s1); tk[N] = max(Y0, Y1); tk[NW] = min(d0, d1);
    } else {
        tk[W] = kmin3(tk[W], X0, X1); tk[SW] = kmin3(tk[SW], s0, s1);
        tk[S] = kmin3(tk[S], Y0, Y1); tk[SE] = kmax3(tk[SE], d0, d1);
        tk[E] = kmax3(tk[E], X0, X1); tk[NE] = kmax3(tk[NE], s0, s1);
        tk[N] = kmax3(tk[N], Y0, Y1); tk[NW] = kmin3(tk[NW], d0, d1);
    }
}

__device__ __forceinline__ void track_tile(Track& tr, const int (&tk)[8], unsigned code) {
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const bool better = dir_is_max(d) ? (tk[d] > tr.best[d]) : (tk[d] < tr.best[d]);
        tr.best[d] = better ? tk[d] : tr.best[d];
        tr.code[d] = better ? code : tr.code[d];
    }
}

__device__ __forceinline__ unsigned long long pack_best(int d, int best, unsigned code) {
    if (best == INT_MIN || best == INT_MAX) return 0ull;
    const unsigned k = dir_is_max(d) ? (unsigned)best : 0xFFFFFFFFu - (unsigned)best;
    return ((unsigned long long)k << 32) | (unsigned long long)(0xFFFFFFFFu - code);
}

}  // namespace ch
