// filter.cu -- the filtering stage of GPU heaphull (Alg. 2, GPUfilter) on sm_103a.
//
//   init_kernel      reset the per-call control block
//   pass1_kernel     findExtremes (Alg. 2; Sec. 3): one streaming pass computing
//                    all 8 directional extremes (argmin/argmax of x, y, x+y, x-y).
//                    The paper runs two reduction kernels because its corner
//                    points are defined by Manhattan distance to the corners of
//                    the axis-extreme box; that distance is x+y (or x-y) up to a
//                    constant, so one pass finds all eight.
//   finalize_kernel  lowest-index tie-break, octagon CP(E), queue quadrilateral,
//                    inner box, float edge functions; writes the 8 extreme records.
//   pass2_kernel     the loop of Alg. 1/2: drop points strictly inside CP(E),
//                    findQueue by the quadrilateral rule, and compact the
//                    survivors (warp-aggregated) into sort records.
//   labels_kernel    the same loop writing the paper's label array Q (ch_filter).
#include "ch_internal.cuh"
#include "launch.h"

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

// ---------------------------------------------------------------------------
__global__ void init_kernel(Ctl* ctl) {
    const int t = threadIdx.x;
    if (t < 8) ctl->ext_packed[t] = 0ull;
    if (t < 4) { ctl->tile_ctr[t] = 0u; ctl->counts4[t] = 0u; }
    if (t == 0) {
        ctl->status = CH_OK;
        ctl->abort = 0;
        ctl->count = 8u;
        ctl->epoch += 1u;
    }
    unsigned* h = &ctl->digit_hist[0][0];
    for (int i = t; i < kSortPasses * kDigits; i += blockDim.x) h[i] = 0u;
}

// ---------------------------------------------------------------------------
// Pass 1.  Each lane keeps, per direction, its best key and the first warp tile
// (code) where that key occurred; tiles are visited in increasing index order,
// so strict improvement keeps the earliest tile.  The grid-wide answer is the
// maximum of (key, ~code) packed in 64 bits: the best key and, among tiles that
// reach it, the lowest one.  finalize_kernel rescans that single tile (512
// points) for the lowest index.  Tile codes: 0 = unaligned head point,
// t + 1 = body warp tile t, ntiles + 1 = tail.
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

// Convert one point, fold its validity into the tracker, return int coords.
__device__ __forceinline__ void convert_pt(float x, float y, int& X, int& Y, Track& tr) {
    X = __float2int_rn(x);
    Y = __float2int_rn(y);
    tr.bad |= (__int2float_rn(X) != x) | (__int2float_rn(Y) != y);
    tr.orv |= (unsigned)X | (unsigned)Y;
}

__device__ __forceinline__ void tile_first(int (&tk)[8], int X, int Y) {
    const int s = X + Y, d = X - Y + kCoordLimit;
    tk[W] = X; tk[SW] = s; tk[S] = Y; tk[SE] = d;
    tk[E] = X; tk[NE] = s; tk[N] = Y; tk[NW] = d;
}

__device__ __forceinline__ void tile_acc(int (&tk)[8], int X, int Y) {
    const int s = X + Y, d = X - Y + kCoordLimit;
    tk[W] = min(tk[W], X);
    tk[SW] = min(tk[SW], s);
    tk[S] = min(tk[S], Y);
    tk[SE] = max(tk[SE], d);
    tk[E] = max(tk[E], X);
    tk[NE] = max(tk[NE], s);
    tk[N] = max(tk[N], Y);
    tk[NW] = min(tk[NW], d);
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

// Head point and ragged tail (scalar loads), handled by global warp 0.
__device__ void track_scalar_range(const float* __restrict__ pts, long long lo, long long hi,
                                   unsigned code, int lane, Track& tr) {
    int tk[8];
    bool any = false;
    for (long long i = lo + lane; i < hi; i += 32) {
        int X, Y;
        convert_pt(pts[2 * i], pts[2 * i + 1], X, Y, tr);
        if (!any) tile_first(tk, X, Y); else tile_acc(tk, X, Y);
        any = true;
    }
    if (any) track_tile(tr, tk, code);
}

__global__ void __launch_bounds__(256) pass1_kernel(const float* __restrict__ pts, long long n,
                                                    int head, long long ntiles, Ctl* ctl) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    Track tr;
    track_init(tr);
    if (gwarp == 0 && head) track_scalar_range(pts, 0, head, 0u, lane, tr);

    const float4* p4 = reinterpret_cast<const float4*>(pts + 2 * head);
    for (long long t = gwarp; t < ntiles; t += nwarps) {
        const float4* base = p4 + t * kWarpTileF4 + lane;
        float4 v[kLoadsPerLane];
#pragma unroll
        for (int j = 0; j < kLoadsPerLane; ++j) v[j] = ld_stream_f4(base + j * 32);
        int tk[8];
        int X, Y;
        convert_pt(v[0].x, v[0].y, X, Y, tr);
        tile_first(tk, X, Y);
        convert_pt(v[0].z, v[0].w, X, Y, tr);
        tile_acc(tk, X, Y);
#pragma unroll
        for (int j = 1; j < kLoadsPerLane; ++j) {
            convert_pt(v[j].x, v[j].y, X, Y, tr);
            tile_acc(tk, X, Y);
            convert_pt(v[j].z, v[j].w, X, Y, tr);
            tile_acc(tk, X, Y);
        }
        track_tile(tr, tk, (unsigned)(t + 1));
    }
    if (gwarp == 0) {
        const long long ts = head + ntiles * kWarpTilePts;
        if (ts < n) track_scalar_range(pts, ts, n, (unsigned)(ntiles + 1), lane, tr);
    }

    const bool err = tr.bad || (tr.orv >> kCoordBits) != 0u;
    if (__any_sync(0xFFFFFFFFu, err) && lane == 0) set_status(ctl, CH_ERANGE);

    __shared__ unsigned long long s_red[8][8];
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        unsigned long long p = pack_best(d, tr.best[d], tr.code[d]);
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long q = __shfl_xor_sync(0xFFFFFFFFu, p, o);
            p = q > p ? q : p;
        }
        if (lane == 0) s_red[warp][d] = p;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int d = threadIdx.x;
        unsigned long long m = 0ull;
        const int nw = blockDim.x >> 5;
        for (int w = 0; w < nw; ++w) m = s_red[w][d] > m ? s_red[w][d] : m;
        if (m) atomicMax(&ctl->ext_packed[d], m);
    }
}

// ---------------------------------------------------------------------------
// Octagon setup helpers (one warp).
__device__ Edge make_edge(int ax, int ay, int bx, int by) {
    Edge e;
    e.ax = ax; e.ay = ay;
    e.dx = bx - ax; e.dy = by - ay;
    if (e.dx == 0 && e.dy == 0) {
        e.A = 0.0f; e.B = 0.0f; e.C = kHugePositive;
    } else {
        // orient(a, b, p) = dx*py - dy*px + (dy*ax - dx*ay) = A*px + B*py + C.
        // A, B, px, py are exact in fp32 (|.| < 2^24); C (|C| < 2^49) is rounded
        // once.  With two FMAs the total error is below 2^25 + 2^26 + 2^27 < 2^28
        // (= kEdgeTol): outside that band the float sign is the exact sign.
        e.A = (float)(-e.dy);
        e.B = (float)e.dx;
        e.C = __ll2float_rn((long long)e.dy * ax - (long long)e.dx * ay);
    }
    return e;
}

__device__ __forceinline__ bool in_closed_octagon(const Octagon& o, long long px, long long py) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const Edge& e = o.oct[k];
        if ((e.dx | e.dy) == 0) continue;
        if (orient64(e.ax, e.ay, (long long)e.ax + e.dx, (long long)e.ay + e.dy, px, py) < 0) return false;
    }
    return true;
}

__device__ __forceinline__ bool box_fits(const Octagon& o, int cx, int cy, int hw, int hh, int t) {
    const long long a = (long long)hw * t / 1024, b = (long long)hh * t / 1024;
    return in_closed_octagon(o, cx - a, cy - b) && in_closed_octagon(o, cx + a, cy - b) &&
           in_closed_octagon(o, cx + a, cy + b) && in_closed_octagon(o, cx - a, cy + b);
}

__global__ void __launch_bounds__(256) finalize_kernel(const float* __restrict__ pts, long long n,
                                                       int head, Ctl* ctl, uint32_t* keys,
                                                       uint64_t* vals) {
    __shared__ unsigned long long s_ext[8];
    __shared__ int s_G[8];
    __shared__ long long s_lo[8], s_hi[8];
    __shared__ Octagon s_oct;
    if (read_status(ctl) != CH_OK) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 8) {
        const int d = threadIdx.x;
        const unsigned long long pk = ctl->ext_packed[d];
        const unsigned code = 0xFFFFFFFFu - (unsigned)(pk & 0xFFFFFFFFull);
        const unsigned hi32 = (unsigned)(pk >> 32);
        s_G[d] = dir_is_max(d) ? (int)hi32 : (int)(0xFFFFFFFFu - hi32);
        long long lo, hi;
        if (code == 0u) { lo = 0; hi = head; }
        else { lo = head + (long long)(code - 1u) * kWarpTilePts; hi = min(n, lo + kWarpTilePts); }
        s_lo[d] = lo;
        s_hi[d] = hi;
        s_ext[d] = ~0ull;
    }
    __syncthreads();
    // Rescan the winning tile of every direction for its lowest index (all
    // loads issued up front: 8 directions x 2 points per thread).
    {
        float px[8][2], py[8][2];
#pragma unroll
        for (int d = 0; d < 8; ++d) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long i = s_lo[d] + threadIdx.x + h * 256;
                px[d][h] = 0.0f; py[d][h] = 0.0f;
                if (i < s_hi[d]) { px[d][h] = pts[2 * i]; py[d][h] = pts[2 * i + 1]; }
            }
        }
#pragma unroll
        for (int d = 0; d < 8; ++d) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long i = s_lo[d] + threadIdx.x + h * 256;
                if (i < s_hi[d] &&
                    dir_key(d, __float2int_rn(px[d][h]), __float2int_rn(py[d][h])) == s_G[d])
                    atomicMin(&s_ext[d], (unsigned long long)i);
            }
        }
    }
    __syncthreads();
    if (warp != 0) return;
    for (int d = 0; d < 8; ++d) {
        if (s_ext[d] >= (unsigned long long)n) {   // cannot happen for valid input; fail safe
            if (lane == 0) set_status(ctl, CH_ECUDA);
            return;
        }
    }
    if (lane == 0) {
        long long area2 = 0;
        for (int d = 0; d < 8; ++d) {
            const long long i = s_ext[d];
            s_oct.ext[d] = (int)i;
            s_oct.vx[d] = __float2int_rn(pts[2 * i]);
            s_oct.vy[d] = __float2int_rn(pts[2 * i + 1]);
        }
        for (int k = 0; k < 8; ++k) {
            const int j = (k + 1) & 7;
            area2 += (long long)s_oct.vx[k] * s_oct.vy[j] - (long long)s_oct.vx[j] * s_oct.vy[k];
            s_oct.oct[k] = make_edge(s_oct.vx[k], s_oct.vy[k], s_oct.vx[j], s_oct.vy[j]);
        }
        for (int r = 0; r < 4; ++r) {
            const int a = 2 * r, b = (2 * r + 2) & 7;
            s_oct.quad[r] = make_edge(s_oct.vx[a], s_oct.vy[a], s_oct.vx[b], s_oct.vy[b]);
        }
        s_oct.discard_none = (area2 == 0);
        s_oct.pad[0] = s_oct.pad[1] = s_oct.pad[2] = 0;
    }
    __syncwarp();
    // Largest centred box (aspect of the bounding box) inside the closed
    // octagon: two rounds of a 32-way search over t/1024.
    const int cx = (s_oct.vx[W] + s_oct.vx[E]) / 2, cy = (s_oct.vy[S] + s_oct.vy[N]) / 2;
    const int hw = (s_oct.vx[E] - s_oct.vx[W]) / 2, hh = (s_oct.vy[N] - s_oct.vy[S]) / 2;
    int t1 = 0;
    if (!s_oct.discard_none) {
        unsigned ok = __ballot_sync(0xFFFFFFFFu, box_fits(s_oct, cx, cy, hw, hh, (lane + 1) * 32));
        // nested boxes: predicate is monotone, so take the highest passing lane
        t1 = ok ? (32 - __clz(ok)) * 32 : 0;
        const int t2 = t1 + lane + 1;
        ok = __ballot_sync(0xFFFFFFFFu, lane < 31 && t2 <= 1024 && box_fits(s_oct, cx, cy, hw, hh, t2));
        if (ok) t1 += 32 - __clz(ok);
    }
    if (lane == 0) {
        const long long a = (long long)hw * t1 / 1024, b = (long long)hh * t1 / 1024;
        if (t1 > 0) {
            s_oct.bxl = (float)(cx - a); s_oct.bxh = (float)(cx + a);
            s_oct.byl = (float)(cy - b); s_oct.byh = (float)(cy + b);
        } else {
            s_oct.bxl = 1.0f; s_oct.bxh = 0.0f; s_oct.byl = 1.0f; s_oct.byh = 0.0f;
        }
    }
    __syncwarp();
    // Copy the octagon to the control block.
    {
        const int words = (int)(sizeof(Octagon) / 4);
        const int* src = reinterpret_cast<const int*>(&s_oct);
        int* dst = reinterpret_cast<int*>(&ctl->oct);
        for (int i = lane; i < words; i += 32) dst[i] = src[i];
    }
    // The 8 chain end-point records: queue r runs from quad vertex r to r+1.
    if (lane < 8) {
        const int r = lane >> 1;
        const int d = (lane & 1) ? ((2 * r + 2) & 7) : 2 * r;
        uint32_t u, v;
        queue_frame(r, s_oct.vx[d], s_oct.vy[d], u, v);
        const uint32_t key = make_key(r, u);
        keys[lane] = key;
        vals[lane] = make_val(v, (uint32_t)s_oct.ext[d]);
#pragma unroll
        for (int p = 0; p < kSortPasses; ++p)
            atomicAdd(&ctl->digit_hist[p][(key >> (p * kDigitBits)) & (kDigits - 1)], 1u);
    }
}

// ---------------------------------------------------------------------------
// Pass 2: classification of one point.  Returns -1 (discarded) or queue 0..3.
// The octagon and queue tests run out of line: on filter-bound inputs almost
// every point is settled by the inner-box test of classify().
__device__ __noinline__ int classify_slow(float x, float y, const Octagon* op) {
    const Octagon& o = *op;
    if (!o.discard_none) {
        float m = kHugePositive;
#pragma unroll
        for (int k = 0; k < 8; ++k) m = fminf(m, fmaf(o.oct[k].A, x, fmaf(o.oct[k].B, y, o.oct[k].C)));
        if (m > kEdgeTol) return -1;                                      // surely inside
        if (m >= -kEdgeTol) {                                             // ambiguous band
            const long long X = (long long)x, Y = (long long)y;
            bool inside = true;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const Edge& e = o.oct[k];
                if ((e.dx | e.dy) == 0) continue;
                if (orient64(e.ax, e.ay, (long long)e.ax + e.dx, (long long)e.ay + e.dy, X, Y) <= 0)
                    inside = false;
            }
            if (inside) return -1;
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const Edge& q = o.quad[r];
        const float e = fmaf(q.A, x, fmaf(q.B, y, q.C));
        if (e < -kEdgeTol) return r;
        if (e <= kEdgeTol && (q.dx | q.dy) != 0) {
            if (orient64(q.ax, q.ay, (long long)q.ax + q.dx, (long long)q.ay + q.dy,
                         (long long)x, (long long)y) < 0)
                return r;
        }
    }
    return -1;
}

struct Box {
    float xl, xh, yl, yh;
};

__device__ __forceinline__ int classify(float x, float y, const Box& b, const Octagon& o) {
    if (x > b.xl && x < b.xh && y > b.yl && y < b.yh) return -1;   // strictly inside the box
    return classify_slow(x, y, &o);
}

__device__ __forceinline__ void load_octagon_smem(Octagon& s, const Ctl* ctl) {
    const int words = (int)(sizeof(Octagon) / 4);
    const int* src = reinterpret_cast<const int*>(&ctl->oct);
    int* dst = reinterpret_cast<int*>(&s);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

// Writes the records of the survivors held by this lane (bit s of keep = point
// slot s, its queue in bits 2s..2s+1 of regs) with one atomic per warp.
// get(s, idx, x, y) returns slot s; slots are unrolled so get indexes registers.
template <int kSlots, typename Get>
__device__ __forceinline__ void emit_records(unsigned keep, unsigned long long regs, Get get, Ctl* ctl,
                                             uint32_t* keys, uint64_t* vals,
                                             unsigned (*s_hist)[kDigits]) {
    const int lane = threadIdx.x & 31;
    const unsigned c = __popc(keep);
    unsigned incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    const unsigned total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (total == 0u) return;
    unsigned base = 0u;
    if (lane == 31) base = atomicAdd(&ctl->count, total);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    unsigned pos = base + incl - c;
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        if ((keep >> s) & 1u) {
            long long idx;
            float x, y;
            get(s, idx, x, y);
            const int r = (int)((regs >> (2 * s)) & 3ull);
            uint32_t u, v;
            queue_frame(r, (int)x, (int)y, u, v);
            const uint32_t key = make_key(r, u);
            keys[pos] = key;
            vals[pos] = make_val(v, (uint32_t)idx);
            ++pos;
#pragma unroll
            for (int p = 0; p < kSortPasses; ++p)
                atomicAdd(&s_hist[p][(key >> (p * kDigitBits)) & (kDigits - 1)], 1u);
        }
    }
}

__global__ void __launch_bounds__(256) pass2_kernel(const float* __restrict__ pts, long long n,
                                                    int head, long long ntiles, Ctl* ctl,
                                                    uint32_t* keys, uint64_t* vals) {
    __shared__ Octagon s_oct;
    __shared__ unsigned s_hist[kSortPasses][kDigits];
    if (read_status(ctl) != CH_OK) return;
    load_octagon_smem(s_oct, ctl);
    for (int i = threadIdx.x; i < kSortPasses * kDigits; i += blockDim.x) (&s_hist[0][0])[i] = 0u;
    __syncthreads();
    const Octagon& o = s_oct;
    const Box box{o.bxl, o.bxh, o.byl, o.byh};
    const int lane = threadIdx.x & 31;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const float4* p4 = reinterpret_cast<const float4*>(pts + 2 * head);

    for (long long t = gwarp; t < ntiles; t += nwarps) {
        const float4* base = p4 + t * kWarpTileF4 + lane;
        float4 v[kLoadsPerLane];
#pragma unroll
        for (int j = 0; j < kLoadsPerLane; ++j) v[j] = ld_stream_f4(base + j * 32);
        unsigned keep = 0u;
        unsigned long long regs = 0ull;
#pragma unroll
        for (int j = 0; j < kLoadsPerLane; ++j) {
            const int r0 = classify(v[j].x, v[j].y, box, o);
            const int r1 = classify(v[j].z, v[j].w, box, o);
            if (r0 >= 0) { keep |= 1u << (2 * j); regs |= (unsigned long long)r0 << (4 * j); }
            if (r1 >= 0) { keep |= 1u << (2 * j + 1); regs |= (unsigned long long)r1 << (4 * j + 2); }
        }
        if (__any_sync(0xFFFFFFFFu, keep != 0u)) {
            const long long i0 = head + 2 * (t * kWarpTileF4 + lane);
            auto get = [&](int s, long long& idx, float& x, float& y) {
                const int j = s >> 1;
                idx = i0 + 64 * j + (s & 1);
                x = (s & 1) ? v[j].z : v[j].x;
                y = (s & 1) ? v[j].w : v[j].y;
            };
            emit_records<2 * kLoadsPerLane>(keep, regs, get, ctl, keys, vals, s_hist);
        }
    }
    if (gwarp == 0) {   // head point and ragged tail, 16 points per lane per round
        const long long ranges[2][2] = {{0, head}, {head + ntiles * kWarpTilePts, n}};
        for (int rg = 0; rg < 2; ++rg) {
            const long long hi = ranges[rg][1];
            for (long long b = ranges[rg][0]; b < hi; b += 32 * 16) {
                unsigned keep = 0u;
                unsigned long long regs = 0ull;
                float px[16], py[16];
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const long long i = b + s * 32 + lane;
                    px[s] = 0.0f; py[s] = 0.0f;
                    if (i < hi) {
                        px[s] = pts[2 * i]; py[s] = pts[2 * i + 1];
                        const int r = classify(px[s], py[s], box, o);
                        if (r >= 0) { keep |= 1u << s; regs |= (unsigned long long)r << (2 * s); }
                    }
                }
                auto get = [&](int s, long long& idx, float& x, float& y) {
                    idx = b + s * 32 + lane;
                    x = px[s];
                    y = py[s];
                };
                emit_records<16>(keep, regs, get, ctl, keys, vals, s_hist);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSortPasses * kDigits; i += blockDim.x) {
        const unsigned c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&(&ctl->digit_hist[0][0])[i], c);
    }
}

// ---------------------------------------------------------------------------
// ch_filter: the label array Q of Alg. 2 and the queue sizes.
__global__ void __launch_bounds__(256) labels_kernel(const float* __restrict__ pts, long long n,
                                                     Ctl* ctl, uint8_t* labels) {
    __shared__ Octagon s_oct;
    __shared__ unsigned s_cnt[4];
    if (read_status(ctl) != CH_OK) return;
    load_octagon_smem(s_oct, ctl);
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    const Box box{s_oct.bxl, s_oct.bxh, s_oct.byl, s_oct.byh};
    unsigned c[4] = {0u, 0u, 0u, 0u};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float2 p = reinterpret_cast<const float2*>(pts)[i];
        const int r = classify(p.x, p.y, box, s_oct);
        if (labels) labels[i] = (uint8_t)(r + 1);
        if (r >= 0) c[r]++;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        unsigned v = c[r];
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_cnt[r], v);
    }
    __syncthreads();
    if (threadIdx.x < 4 && s_cnt[threadIdx.x]) atomicAdd(&ctl->counts4[threadIdx.x], s_cnt[threadIdx.x]);
}

__global__ void filter_output_kernel(const Ctl* ctl, long long n, int32_t* out_ext8, int64_t* out_counts4) {
    const int t = threadIdx.x;
    const int st = read_status(ctl);
    if (t < 8 && out_ext8) out_ext8[t] = (n == 0 || st != CH_OK) ? -1 : ctl->oct.ext[t];
    if (t < 4 && out_counts4) out_counts4[t] = (st != CH_OK) ? (int64_t)st : (int64_t)ctl->counts4[t];
}

// ---------------------------------------------------------------------------
// Host launchers
void launch_init(Ctl* ctl, cudaStream_t s) { init_kernel<<<1, 256, 0, s>>>(ctl); }

void launch_pass1(const float* pts, long long n, int head, long long ntiles, Ctl* ctl,
                  int grid, cudaStream_t s) {
    pass1_kernel<<<grid, 256, 0, s>>>(pts, n, head, ntiles, ctl);
}

void launch_finalize(const float* pts, long long n, int head, Ctl* ctl, uint32_t* keys,
                     uint64_t* vals, cudaStream_t s) {
    finalize_kernel<<<1, 256, 0, s>>>(pts, n, head, ctl, keys, vals);
}

void launch_pass2(const float* pts, long long n, int head, long long ntiles, Ctl* ctl,
                  uint32_t* keys, uint64_t* vals, int grid, cudaStream_t s) {
    pass2_kernel<<<grid, 256, 0, s>>>(pts, n, head, ntiles, ctl, keys, vals);
}

void launch_labels(const float* pts, long long n, Ctl* ctl, uint8_t* labels, int grid,
                   cudaStream_t s) {
    labels_kernel<<<grid, 256, 0, s>>>(pts, n, ctl, labels);
}

void launch_filter_output(const Ctl* ctl, long long n, int32_t* out_ext8, int64_t* out_counts4,
                          cudaStream_t s) {
    filter_output_kernel<<<1, 32, 0, s>>>(ctl, n, out_ext8, out_counts4);
}


cudaError_t occupancy_filter(int* p1, int* p2, int* lab) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(p1, pass1_kernel, 256, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(p2, pass2_kernel, 256, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(lab, labels_kernel, 256, 0);
    return e;
}

}  // namespace ch
