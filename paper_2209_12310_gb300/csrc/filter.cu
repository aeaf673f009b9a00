// filter.cu -- the filtering stage of GPU heaphull (Alg. 2, GPUfilter) on sm_103a.
//
// Kernels (in launch order):
//   init_kernel     reset the per-call control block.
//   sample_kernel   extremes of an evenly spaced sample of warp tiles; its last
//                   block builds the sample octagon (vertices are input points).
//   main_kernel     findExtremes (Alg. 2; Sec. 3) over every point: all 8
//                   directional extremes in one pass (the paper's second
//                   kernel finds the corner points by Manhattan distance to the
//                   bounding-box corners; that distance is x+y or x-y up to a
//                   constant, so one pass suffices), with the lowest index on
//                   ties.  In fused mode (ch_hull) the same pass also drops the
//                   points in the closed sample octagon and compacts the rest
//                   ("raw" survivors): one streaming read of the input instead
//                   of two.  When the raw survivors grow past a threshold
//                   (adversarial data such as points on a circle), the pass
//                   stops filtering and the second pass does it (two-pass mode).
//                   Its last block builds the octagon of the true extremes,
//                   and when few raw survivors remain it re-classifies them,
//                   and with few records left computes the hull itself.
//   stagec_kernel   two-pass mode: the loop of Alg. 1/2 over every point
//                   against the true octagon (findQueue by the quadrilateral
//                   rule), or the re-classification of many raw survivors;
//                   compaction into sort records (queue | u, v | index).
//   labels_kernel   ch_filter: the label array Q of Alg. 2 (paper rule).
#include "ch_internal.cuh"
#include "hullcore.cuh"
#include "launch.h"
#include "octagon.cuh"
#include "tma.cuh"

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

// ---------------------------------------------------------------------------
__global__ void init_kernel(Ctl* ctl, int mode) {
    const int t = threadIdx.x;
    if (t < 8) {
        ctl->ext_packed[t] = 0ull;
        ctl->samp_packed[t] = 0ull;
        ctl->line_ep[t] = (t & 1) ? 0ull : ~0ull;   // even: minimum slot, odd: maximum slot
    }
    if (t < 4) { ctl->tile_ctr[t] = 0u; ctl->counts4[t] = 0u; ctl->blocks_done[t] = 0u; }
    if (t == 0) {
        ctl->status = CH_OK;
        ctl->abort = 0;
        ctl->count = 8u;
        ctl->count_raw = 0u;
        ctl->epoch += 1u;
        ctl->mode = mode;
        ctl->done = 0;
        ctl->records_ready = 0;
    }
    unsigned* h = &ctl->digit_hist[0][0];
    for (int i = t; i < kSortPasses * kDigits; i += blockDim.x) h[i] = 0u;
}

// Last-arriver election: returns true in exactly one block, after every other
// block of the grid has finished (and made its writes visible).
__device__ __forceinline__ bool last_block(unsigned* counter, int* s_flag) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *s_flag = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!*s_flag) return false;
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// Warp tiles read by the sample pass: about 1/32 of the input, at most
// kSampleTiles, at least min(ntiles, 64).
__host__ __device__ __forceinline__ long long sample_tiles(long long ntiles) {
    long long s = ntiles / 32;
    if (s < 64) s = ntiles < 64 ? ntiles : 64;
    return s < kSampleTiles ? s : kSampleTiles;
}

// ---------------------------------------------------------------------------
// Sample pass: packed (key, other coordinate) maxima per direction; the other
// coordinate recovers the point (no index needed: the sample octagon only
// filters, and its vertices are input points).
__device__ __forceinline__ unsigned long long samp_pack(int d, int X, int Y) {
    const unsigned k = (unsigned)dir_key(d, X, Y);
    const unsigned aux = (d == W || d == E) ? (unsigned)Y : (unsigned)X;
    const unsigned hk = dir_is_max(d) ? k : 0xFFFFFFFFu - k;
    return ((unsigned long long)hk << 32) | aux;
}

__global__ void __launch_bounds__(256) sample_kernel(const float* __restrict__ pts, long long n, int head,
                                                     long long ntiles, Ctl* ctl) {
    __shared__ unsigned long long s_red[8][8];
    __shared__ Octagon s_o;
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long best[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) best[d] = 0ull;
    const long long nsamp = sample_tiles(ntiles);
    const float4* p4 = reinterpret_cast<const float4*>(pts + 2 * head);
    for (long long k = gwarp; k < nsamp; k += nwarps) {
        const long long t = k * ntiles / nsamp;
        const float4* base = p4 + t * kWarpTileF4 + lane;
        float4 v[kLoadsPerLane];
#pragma unroll
        for (int j = 0; j < kLoadsPerLane; ++j) v[j] = ld_stream_f4(base + j * 32);
#pragma unroll
        for (int j = 0; j < kLoadsPerLane; ++j) {
            const int X0 = __float2int_rn(v[j].x), Y0 = __float2int_rn(v[j].y);
            const int X1 = __float2int_rn(v[j].z), Y1 = __float2int_rn(v[j].w);
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                const unsigned long long a = samp_pack(d, X0, Y0), b = samp_pack(d, X1, Y1);
                const unsigned long long m = a > b ? a : b;
                best[d] = m > best[d] ? m : best[d];
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        unsigned long long p = best[d];
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long q = __shfl_xor_sync(0xFFFFFFFFu, p, o);
            p = q > p ? q : p;
        }
        if (lane == 0) s_red[warp][d] = p;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        unsigned long long m = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = s_red[w][threadIdx.x] > m ? s_red[w][threadIdx.x] : m;
        if (m) atomicMax(&ctl->samp_packed[threadIdx.x], m);
    }
    if (!last_block(&ctl->blocks_done[0], &s_last)) return;
    __shared__ int s_v[2][8];
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = nsamp > 0;
    __syncthreads();
    if (threadIdx.x < 8) {
        const int d = threadIdx.x;
        const unsigned long long p = *(volatile unsigned long long*)&ctl->samp_packed[d];
        if (p == 0ull) atomicAnd(&s_ok, 0);
        const unsigned hk = (unsigned)(p >> 32), aux = (unsigned)p;
        const int key = dir_is_max(d) ? (int)hk : (int)(0xFFFFFFFFu - hk);
        int x, y;
        switch (d) {
            case W: case E: x = key; y = (int)aux; break;
            case S: case N: y = key; x = (int)aux; break;
            case SW: case NE: x = (int)aux; y = key - x; break;
            default: x = (int)aux; y = x - (key - kCoordLimit); break;
        }
        s_v[0][d] = x;
        s_v[1][d] = y;
    }
    __syncthreads();
    if (!s_ok) {   // too few points to sample: run the two-pass path
        if (threadIdx.x == 0) ctl->mode = 1;
        return;
    }
    const int ext[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    setup_octagon_block(s_o, s_v[0], s_v[1], ext);
    if (s_o.discard_none) {
        if (threadIdx.x == 0) ctl->mode = 1;
        return;
    }
    copy_octagon(&ctl->oct_s, &s_o);
}

// ---------------------------------------------------------------------------
// Main pass.  Each lane keeps, per direction, its best key and the first warp
// tile (code) where that key occurred; tiles are visited in increasing index
// order, so strict improvement keeps the earliest tile.  The grid-wide answer
// is the maximum of (key, ~code) packed in 64 bits: the best key and, among
// tiles reaching it, the lowest; the last block rescans that tile (512 points)
// for the lowest index.  Tile codes: 0 = unaligned head point, t + 1 = body
// warp tile t, ntiles + 1 = ragged tail.
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

// Strictly inside the inner region of the sample octagon: the tile's key
// extremes (or one point's keys) against the bounds, strict comparisons.
// Bounds are read from shared memory (lo = in[0..3], hi = in[4..7]) to keep
// them out of the streaming loop's registers.
__device__ __forceinline__ bool tile_in_inner(const int (&tk)[8], const int* in) {
    return tk[W] > in[0] && tk[E] < in[4] && tk[S] > in[1] && tk[N] < in[5] &&
           tk[SW] > in[2] && tk[NE] < in[6] && tk[NW] > in[3] && tk[SE] < in[7];
}

__device__ __forceinline__ bool pt_in_inner(int X, int Y, const int* in) {
    const int S = X + Y, D = X - Y + kCoordLimit;
    return X > in[0] && X < in[4] && Y > in[1] && Y < in[5] && S > in[2] && S < in[6] && D > in[3] && D < in[7];
}

__device__ __forceinline__ unsigned long long pack_best(int d, int best, unsigned code) {
    if (best == INT_MIN || best == INT_MAX) return 0ull;
    const unsigned k = dir_is_max(d) ? (unsigned)best : 0xFFFFFFFFu - (unsigned)best;
    return ((unsigned long long)k << 32) | (unsigned long long)(0xFFFFFFFFu - code);
}

// Raw survivors are staged per warp in shared memory and written out in
// batches: one global atomic per batch instead of one per warp tile (a single
// contended counter otherwise serialises at L2).
constexpr int kWarpBuf = 256;
struct RawBuf {
    unsigned long long xy[kWarpBuf];
    unsigned idx[kWarpBuf];
};

// Warp-collective; returns the global raw count after this batch.
__device__ __forceinline__ unsigned flush_raw(RawBuf& b, unsigned& cnt, Ctl* ctl, uint64_t* raw_xy,
                                              uint32_t* raw_idx) {
    const int lane = threadIdx.x & 31;
    if (cnt == 0u) return 0u;
    unsigned base = 0u;
    if (lane == 0) base = atomicAdd(&ctl->count_raw, cnt);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    __syncwarp();
    for (unsigned i = lane; i < cnt; i += 32) {
        raw_xy[base + i] = b.xy[i];
        raw_idx[base + i] = b.idx[i];
    }
    __syncwarp();
    const unsigned after = base + cnt;
    cnt = 0u;
    return after;
}

// Warp-collective compaction of a lane's kept slots into the warp's buffer.
// get(s, idx, x, y) reads slot s; slots are unrolled so get indexes registers.
// Returns the global raw count when a batch was written out, else 0.
template <int kSlots, typename Get>
__device__ __forceinline__ unsigned emit_raw(unsigned keep, Get get, RawBuf& b, unsigned& cnt, Ctl* ctl,
                                             uint64_t* raw_xy, uint32_t* raw_idx) {
    const int lane = threadIdx.x & 31;
    const unsigned c = __popc(keep);
    unsigned incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    const unsigned total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (total == 0u) return 0u;
    unsigned after = 0u;
    if (cnt + total > (unsigned)kWarpBuf) after = flush_raw(b, cnt, ctl, raw_xy, raw_idx);
    const bool direct = total > (unsigned)kWarpBuf;   // a dense tile: straight to global memory
    unsigned base = cnt;
    if (direct) {
        if (lane == 31) base = atomicAdd(&ctl->count_raw, total);
        base = __shfl_sync(0xFFFFFFFFu, base, 31);
        after = base + total;
    }
    unsigned pos = base + incl - c;
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        if ((keep >> s) & 1u) {
            long long idx;
            float x, y;
            get(s, idx, x, y);
            const unsigned long long xy =
                ((unsigned long long)(unsigned)__float2int_rn(x) << 32) | (unsigned)__float2int_rn(y);
            if (direct) { raw_xy[pos] = xy; raw_idx[pos] = (uint32_t)idx; }
            else { b.xy[pos] = xy; b.idx[pos] = (unsigned)idx; }
            ++pos;
        }
    }
    __syncwarp();
    if (!direct) cnt += total;
    return after;
}

// Survivors on an axis support line of the true octagon (x = xmin, y = ymin,
// x = xmax, y = ymax) lie on a hull edge; only the two extreme ones per line
// can be hull vertices.  They are reduced into ctl->line_ep (minimum and
// maximum along the line, lowest index on ties) instead of becoming records;
// emit_line_records turns the end points into records afterwards.
// Warp-collective: every lane passes its candidate (valid = false for none);
// the warp reduces per line first and issues one atomic pair per line.
__device__ __forceinline__ bool reduce_on_line(const Octagon& o, bool valid, int X, int Y, unsigned idx, Ctl* ctl) {
    bool on = false;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const bool hit = valid && ((l == 0) ? X == o.vx[W] : (l == 1) ? Y == o.vy[S] : (l == 2) ? X == o.vx[E] : Y == o.vy[N]);
        on |= hit;
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

template <int kSlots, typename Get>
__device__ __forceinline__ void emit_records(unsigned keep, unsigned long long regs, Get get, Ctl* ctl,
                                             uint32_t* keys, uint64_t* vals, unsigned (*s_hist)[kDigits],
                                             const Octagon* lines = nullptr) {
    const int lane = threadIdx.x & 31;
    if (lines) {   // divert support-line points to the end-point reduction (warp-collective)
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
            const bool kept = (keep >> s) & 1u;
            if (!__any_sync(0xFFFFFFFFu, kept)) continue;
            long long idx = 0;
            float x = 0.0f, y = 0.0f;
            if (kept) get(s, idx, x, y);
            if (reduce_on_line(*lines, kept, __float2int_rn(x), __float2int_rn(y), (unsigned)idx, ctl))
                keep &= ~(1u << s);
        }
    }
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
            queue_frame(r, __float2int_rn(x), __float2int_rn(y), u, v);
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

__device__ __forceinline__ void flush_hist(unsigned (*s_hist)[kDigits], Ctl* ctl) {
    __syncthreads();
    for (int i = threadIdx.x; i < kSortPasses * kDigits; i += blockDim.x) {
        const unsigned c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&(&ctl->digit_hist[0][0])[i], c);
        (&s_hist[0][0])[i] = 0u;
    }
    __syncthreads();
}

// Hull-rule classification: -1 = dropped, else queue.
__device__ __forceinline__ int classify_hull(float x, float y, const Octagon& o) {
    const int X = __float2int_rn(x), Y = __float2int_rn(y);
    if (in_inner(o, X, Y)) return -1;
    return classify_hull_slow(x, y, &o);
}

// Re-classifies raw survivors [0, hi) against the true octagon into sort
// records; thread `start` of `stride` cooperating threads, warp-uniform loop.
__device__ void reclassify_raw(const uint64_t* raw_xy, const uint32_t* raw_idx, unsigned hi, unsigned stride,
                               unsigned start, const Octagon& o, Ctl* ctl, uint32_t* keys, uint64_t* vals,
                               unsigned (*s_hist)[kDigits]) {
    const int lane = threadIdx.x & 31;
    for (unsigned b = start - lane; b < hi; b += stride) {
        const unsigned i = b + lane;
        unsigned keep = 0u;
        unsigned long long regs = 0ull;
        float x = 0.0f, y = 0.0f;
        unsigned idx = 0u;
        if (i < hi) {
            const unsigned long long xy = raw_xy[i];
            x = (float)(unsigned)(xy >> 32);
            y = (float)(unsigned)(xy & 0xFFFFFFFFull);
            idx = raw_idx[i];
            const int r = classify_hull(x, y, o);
            if (r >= 0) { keep = 1u; regs = (unsigned long long)r; }
        }
        auto get = [&](int, long long& id, float& px, float& py) { id = idx; px = x; py = y; };
        emit_records<1>(keep, regs, get, ctl, keys, vals, s_hist, &o);
    }
}

// Records for the end points of the support-line survivors (one thread each).
__device__ void emit_line_records(const Octagon& o, Ctl* ctl, uint32_t* keys, uint64_t* vals) {
    const int t = threadIdx.x;
    if (t >= 8) return;
    const unsigned long long e = *(volatile unsigned long long*)&ctl->line_ep[t];
    if ((t & 1) ? e == 0ull : e == ~0ull) return;   // no survivor on this line
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
    if (r < 0) return;   // cannot happen: it was a survivor
    uint32_t u, v;
    queue_frame(r, X, Y, u, v);
    const uint32_t key = make_key(r, u);
    const unsigned pos = atomicAdd(&ctl->count, 1u);
    keys[pos] = key;
    vals[pos] = make_val(v, idx);
#pragma unroll
    for (int p = 0; p < kSortPasses; ++p)
        atomicAdd(&ctl->digit_hist[p][(key >> (p * kDigitBits)) & (kDigits - 1)], 1u);
}

// Finalize of the main pass (whole block): lowest-index tie-break, octagon of
// the true extremes (-> s_o and ctl->oct), the 8 chain end-point records.
__device__ void finalize_block(const float* __restrict__ pts, long long n, int head, Ctl* ctl, Octagon& s_o,
                               uint32_t* keys, uint64_t* vals) {
    __shared__ unsigned long long s_ext[8];
    __shared__ int s_G[8];
    __shared__ long long s_lo[8], s_hi[8];
    if (threadIdx.x < 8) {
        const int d = threadIdx.x;
        const unsigned long long pk = *(volatile unsigned long long*)&ctl->ext_packed[d];
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
    // One round of independent loads for all 8 directions (a tile has at
    // most kWarpTilePts points; blockDim.x >= kWarpTilePts / 2).
    {
        float2 p[8][2];
        bool valid[8][2];
#pragma unroll
        for (int d = 0; d < 8; ++d) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long i = s_lo[d] + threadIdx.x + (long long)h * blockDim.x;
                valid[d][h] = i < s_hi[d];
                p[d][h] = valid[d][h] ? reinterpret_cast<const float2*>(pts)[i] : make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int d = 0; d < 8; ++d) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long i = s_lo[d] + threadIdx.x + (long long)h * blockDim.x;
                if (valid[d][h] && dir_key(d, __float2int_rn(p[d][h].x), __float2int_rn(p[d][h].y)) == s_G[d])
                    atomicMin(&s_ext[d], (unsigned long long)i);
            }
        }
    }
    __syncthreads();
    bool bad = false;
    for (int d = 0; d < 8; ++d) bad |= s_ext[d] >= (unsigned long long)n;
    if (bad) {   // cannot happen for valid input; fail safe
        if (threadIdx.x == 0) set_status(ctl, CH_ECUDA);
        return;
    }
    __shared__ int s_vx[8], s_vy[8], s_id[8];
    if (threadIdx.x < 8) {
        const long long i = (long long)s_ext[threadIdx.x];
        s_id[threadIdx.x] = (int)i;
        s_vx[threadIdx.x] = __float2int_rn(pts[2 * i]);
        s_vy[threadIdx.x] = __float2int_rn(pts[2 * i + 1]);
    }
    __syncthreads();
    setup_octagon_block(s_o, s_vx, s_vy, s_id);
    if (threadIdx.x < 12) {
        // Threads 0..7: chain end points (queue r runs from quad vertex r to
        // r+1).  Threads 8..11: the diagonal extreme of queue r, when it lies
        // strictly right of the quad edge (the hull rule drops every point of
        // the closed octagon, vertices included, so the vertices that can be
        // hull vertices get their own record; on the edge it cannot be one).
        const int lane = threadIdx.x;
        int r, d;
        bool emit = true;
        if (lane < 8) {
            r = lane >> 1;
            d = (lane & 1) ? ((2 * r + 2) & 7) : 2 * r;
        } else {
            r = lane - 8;
            d = 2 * r + 1;
            const int a = 2 * r, b = (2 * r + 2) & 7;
            emit = orient64(s_vx[a], s_vy[a], s_vx[b], s_vy[b], s_vx[d], s_vy[d]) < 0;
        }
        if (emit) {
            uint32_t u, v;
            queue_frame(r, s_vx[d], s_vy[d], u, v);
            const uint32_t key = make_key(r, u);
            const unsigned pos = lane < 8 ? (unsigned)lane : atomicAdd(&ctl->count, 1u);
            keys[pos] = key;
            vals[pos] = make_val(v, (uint32_t)s_id[d]);
#pragma unroll
            for (int p = 0; p < kSortPasses; ++p)
                atomicAdd(&ctl->digit_hist[p][(key >> (p * kDigitBits)) & (kDigits - 1)], 1u);
        }
    }
    __syncthreads();
    copy_octagon(&ctl->oct, &s_o);
    __syncthreads();
}

// Processes up to 32 queued lane tiles of a warp (one per lane): reloads the
// lane tile's 16 points (just streamed, so served by L2) and keeps those not
// strictly inside the inner region.  Entries are (warp tile << 5) | lane.
// Warp-collective; returns emit_raw's count.
__device__ __forceinline__ unsigned drain_queue(const float* __restrict__ pts, int head, unsigned* q, unsigned& qn,
                                                const int* in, RawBuf& wbuf, unsigned& wcnt, Ctl* ctl,
                                                uint64_t* raw_xy, uint32_t* raw_idx) {
    const int lane = threadIdx.x & 31;
    const unsigned take = qn < 32u ? qn : 32u;
    float4 w[kLoadsPerLane];
    unsigned keep = 0u;
    long long i0 = 0;
    if ((unsigned)lane < take) {
        const unsigned e = q[lane];
        const long long t = e >> 5;
        const int ln = (int)(e & 31u);
        const float4* base = reinterpret_cast<const float4*>(pts + 2 * head) + t * kWarpTileF4 + ln;
#pragma unroll
        for (int j = 0; j < kLoadsPerLane; ++j) w[j] = __ldcg(base + j * 32);
#pragma unroll
        for (int j = 0; j < kLoadsPerLane; ++j) {
            if (!pt_in_inner(__float2int_rn(w[j].x), __float2int_rn(w[j].y), in)) keep |= 1u << (2 * j);
            if (!pt_in_inner(__float2int_rn(w[j].z), __float2int_rn(w[j].w), in)) keep |= 2u << (2 * j);
        }
        i0 = head + 2 * (t * kWarpTileF4 + ln);
    }
    __syncwarp();
    for (unsigned k = take + lane; k < qn; k += 32) q[k - take] = q[k];   // keep the rest
    __syncwarp();
    qn -= take;
    auto get = [&](int s, long long& idx, float& x, float& y) {
        const int j = s >> 1;
        idx = i0 + 64 * j + (s & 1);
        x = (s & 1) ? w[j].z : w[j].x;
        y = (s & 1) ? w[j].w : w[j].y;
    };
    return emit_raw<2 * kLoadsPerLane>(keep, get, wbuf, wcnt, ctl, raw_xy, raw_idx);
}

constexpr size_t kMainSmemBytes = (size_t)8 * kStages * kWarpTileF4 * sizeof(float4);

__global__ void __launch_bounds__(256, 2) main_kernel(const float* __restrict__ pts, long long n, int head,
                                                      long long ntiles, Ctl* ctl, uint64_t* raw_xy,
                                                      uint32_t* raw_idx, unsigned switch_at) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ int s_inner[8];
    __shared__ unsigned long long s_red[8][8];
    __shared__ int s_mode;
    __shared__ RawBuf s_buf[8];
    __shared__ unsigned long long s_bar[8][kStages];
    __shared__ unsigned s_q[8][64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    if (threadIdx.x == 0) s_mode = *(volatile int*)&ctl->mode;   // one read: uniform per block
    if (threadIdx.x < 4) {
        s_inner[threadIdx.x] = ctl->oct_s.in_lo[threadIdx.x];
        s_inner[4 + threadIdx.x] = ctl->oct_s.in_hi[threadIdx.x];
    }
    __syncthreads();
    bool filt = s_mode == 0;
    RawBuf& wbuf = s_buf[warp];
    unsigned wcnt = 0u;
    unsigned qn = 0u;   // queued lane tiles of this warp (warp-uniform)
    Track tr;
    track_init(tr);
    // Scalar ranges (warp 0): the unaligned head point first and the ragged
    // tail last, so every lane visits tile codes in increasing order.
    auto scalar_range = [&](long long lo_i, long long hi_i, unsigned code) {
        int tk[8];
        bool any = false;
        for (long long b = lo_i; b < hi_i; b += 32) {
            const long long i = b + lane;
            unsigned keep = 0u;
            float x = 0.0f, y = 0.0f;
            if (i < hi_i) {
                x = pts[2 * i]; y = pts[2 * i + 1];
                int X, Y;
                convert_pt(x, y, X, Y, tr);
                tile_keys2(tk, X, Y, X, Y, !any);
                any = true;
                if (filt && !pt_in_inner(X, Y, s_inner)) keep = 1u;
            }
            auto get = [&](int, long long& idx, float& px, float& py) { idx = i; px = x; py = y; };
            if (filt) emit_raw<1>(keep, get, wbuf, wcnt, ctl, raw_xy, raw_idx);
        }
        if (any) track_tile(tr, tk, code);
    };
    if (gwarp == 0 && head) scalar_range(0, head, 0u);

    // Warp tiles t = gwarp + k * nwarps stream through a double-buffered
    // shared-memory ring filled by bulk asynchronous copies (TMA).
    WarpStream ws{reinterpret_cast<float4*>(dsm) + warp * kStages * kWarpTileF4, s_bar[warp],
                  reinterpret_cast<const float4*>(pts + 2 * head), gwarp, nwarps, ntiles, lane};
    ws.start();
    for (long long k = 0;; ++k) {
        const long long t = gwarp + k * nwarps;
        if (t >= ntiles) break;
        const float4* cur = ws.acquire(k, ctl);
        if (!cur) {   // a copy never completed: status is CH_ETIMEOUT
            ws.drain(k);
            break;
        }
        int tk[8];
#pragma unroll
        for (int j = 0; j < kLoadsPerLane; ++j) {
            const float4 v = cur[j * 32 + lane];
            int X0, Y0, X1, Y1;
            convert_pt(v.x, v.y, X0, Y0, tr);
            convert_pt(v.z, v.w, X1, Y1, tr);
            tile_keys2(tk, X0, Y0, X1, Y1, j == 0);
        }
        track_tile(tr, tk, (unsigned)(t + 1));
        if (filt) {
            // Points strictly inside the inner region of the sample octagon
            // are strictly inside the hull; every other point is a raw
            // survivor, classified against the true octagon once its extremes
            // are known.  Lanes whose 16 points are not all inside are queued
            // and handled 32 at a time, one per lane, so outliers cost the
            // warp a few instructions instead of a warp-wide slow path.
            const bool inside = tile_in_inner(tk, s_inner);
            const unsigned fail = __ballot_sync(0xFFFFFFFFu, !inside);
            if (fail) {
                if (!inside) s_q[warp][qn + __popc(fail & lanemask_lt())] = ((unsigned)t << 5) | (unsigned)lane;
                qn += __popc(fail);
                __syncwarp();
                if (qn >= 32u) {
                    const unsigned upto = drain_queue(pts, head, s_q[warp], qn, s_inner, wbuf, wcnt, ctl, raw_xy, raw_idx);
                    if (upto > switch_at) {   // dense data: leave filtering to the second pass
                        if (lane == 0) atomicExch(&ctl->mode, 1);
                        filt = false;
                    }
                }
            }
            if ((k & 7) == 7) {
                int m = 0;
                if (lane == 0) m = *(volatile int*)&ctl->mode;
                filt = filt && __shfl_sync(0xFFFFFFFFu, m, 0) == 0;
            }
        }
        ws.release(k);
    }
    if (gwarp == 0 && head + ntiles * kWarpTilePts < n)
        scalar_range(head + ntiles * kWarpTilePts, n, (unsigned)(ntiles + 1));
    while (qn > 0u) drain_queue(pts, head, s_q[warp], qn, s_inner, wbuf, wcnt, ctl, raw_xy, raw_idx);
    flush_raw(wbuf, wcnt, ctl, raw_xy, raw_idx);

    const bool err = tr.bad || (tr.orv >> kCoordBits) != 0u;
    if (__any_sync(0xFFFFFFFFu, err) && lane == 0) set_status(ctl, CH_ERANGE);
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
        unsigned long long m = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = s_red[w][threadIdx.x] > m ? s_red[w][threadIdx.x] : m;
        if (m) atomicMax(&ctl->ext_packed[threadIdx.x], m);
    }

}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 3) stagec_kernel(const float* __restrict__ pts, long long n, int head,
                                                        long long ntiles, Ctl* ctl, const uint64_t* raw_xy,
                                                        const uint32_t* raw_idx, uint32_t* keys, uint64_t* vals) {
    __shared__ Octagon s_o;
    __shared__ unsigned s_hist[kSortPasses][kDigits];
    if (*(volatile int*)&ctl->done || *(volatile int*)&ctl->records_ready) return;
    const int mode = *(volatile int*)&ctl->mode;
    copy_octagon(&s_o, &ctl->oct);
    for (int i = threadIdx.x; i < kSortPasses * kDigits; i += blockDim.x) (&s_hist[0][0])[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    if (mode == 1) {   // second streaming pass over every point
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
                const int r0 = classify_hull(v[j].x, v[j].y, s_o);
                const int r1 = classify_hull(v[j].z, v[j].w, s_o);
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
                emit_records<2 * kLoadsPerLane>(keep, regs, get, ctl, keys, vals, s_hist, &s_o);
            }
        }
        if (gwarp == 0) {
            const long long ranges[2][2] = {{0, head}, {head + ntiles * kWarpTilePts, n}};
            for (int rg = 0; rg < 2; ++rg) {
                for (long long b = ranges[rg][0]; b < ranges[rg][1]; b += 32) {
                    const long long i = b + lane;
                    unsigned keep = 0u;
                    unsigned long long regs = 0ull;
                    float x = 0.0f, y = 0.0f;
                    if (i < ranges[rg][1]) {
                        x = pts[2 * i]; y = pts[2 * i + 1];
                        const int r = classify_hull(x, y, s_o);
                        if (r >= 0) { keep = 1u; regs = (unsigned long long)r; }
                    }
                    auto get = [&](int, long long& idx, float& px, float& py) { idx = i; px = x; py = y; };
                    emit_records<1>(keep, regs, get, ctl, keys, vals, s_hist, &s_o);
                }
            }
        }
    } else {   // many raw survivors of the fused pass: re-classify them
        const unsigned nraw = *(volatile unsigned*)&ctl->count_raw;
        reclassify_raw(raw_xy, raw_idx, nraw, gridDim.x * blockDim.x, blockIdx.x * blockDim.x + threadIdx.x,
                       s_o, ctl, keys, vals, s_hist);
    }
    flush_hist(s_hist, ctl);
}

// ---------------------------------------------------------------------------
// Single-block tail of a streaming pass.
//   phase 0 (after main_kernel): octagon of the true extremes and the chain
//     end-point records; in fused mode with few raw survivors, re-classify them
//     here and, with few records, compute the hull (ctl->done).
//   phase 1 (after stagec_kernel): support-line end-point records, then with
//     few records compute the hull.
// Data errors found by the streaming pass end the call here: out_n = status.
constexpr int kTailThreads = 256;
constexpr size_t kTailSmemBytes = kMidSmemBytes > sizeof(WrapSmem) ? kMidSmemBytes : sizeof(WrapSmem);

__global__ void __launch_bounds__(kTailThreads) tail_kernel(const float* __restrict__ pts, long long n, int head, Ctl* ctl,
                                                    const uint64_t* raw_xy, const uint32_t* raw_idx, uint32_t* keys,
                                                    uint64_t* vals, int phase, int hull, int32_t* out_idx,
                                                    int64_t* out_n) {
    extern __shared__ __align__(16) char dyn[];
    __shared__ Octagon s_o;
    __shared__ unsigned s_hist[kSortPasses][kDigits];
    CH_TRACE_DECL
    CH_TRACE_MARK();
    if (*(volatile int*)&ctl->done) return;
    if (read_status(ctl) != CH_OK) {
        if (hull && threadIdx.x == 0) { *out_n = read_status(ctl); ctl->done = 1; }
        return;
    }
    if (phase == 0) {
        finalize_block(pts, n, head, ctl, s_o, keys, vals);
        CH_TRACE_MARK();
        if (read_status(ctl) != CH_OK) {
            if (hull && threadIdx.x == 0) { *out_n = read_status(ctl); ctl->done = 1; }
            return;
        }
        if (!hull) return;
        const int mode = *(volatile int*)&ctl->mode;
        const unsigned nraw = *(volatile unsigned*)&ctl->count_raw;
        if (mode != 0 || nraw > kRawSmall) { CH_TRACE_PRINT("tail0-final"); return; }
        for (int i = threadIdx.x; i < kSortPasses * kDigits; i += blockDim.x) (&s_hist[0][0])[i] = 0u;
        __syncthreads();
        reclassify_raw(raw_xy, raw_idx, nraw, blockDim.x, (unsigned)threadIdx.x, s_o, ctl, keys, vals, s_hist);
        flush_hist(s_hist, ctl);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) ctl->records_ready = 1;
        CH_TRACE_MARK();
    } else {
        if (*(volatile int*)&ctl->records_ready) return;   // phase 0 produced every record
        copy_octagon(&s_o, &ctl->oct);
        __syncthreads();
    }
    emit_line_records(s_o, ctl, keys, vals);
    __threadfence();
    __syncthreads();
    CH_TRACE_MARK();
    const unsigned cnt = *(volatile unsigned*)&ctl->count;
    if (cnt <= (unsigned)kMidCap) {
        // Few records: gift wrapping (few chain vertices), else sort-based.
        if (!wrap_hull(keys, vals, (int)cnt, n, ctl, out_idx, out_n, *reinterpret_cast<WrapSmem*>(dyn))) {
            __syncthreads();
            mid_hull(keys, vals, (int)cnt, pts, n, ctl, out_idx, out_n, dyn);
        }
        if (threadIdx.x == 0) ctl->done = 1;
    }
    CH_TRACE_MARK();
#ifdef CH_TRACE
    if (threadIdx.x == 0) printf("[tail phase %d] records %u raw %u\n", phase, cnt, ctl->count_raw);
#endif
    CH_TRACE_PRINT("tail");
}

// ---------------------------------------------------------------------------
// ch_filter: the label array Q of Alg. 2 and the queue sizes (paper rule).
__global__ void __launch_bounds__(256) labels_kernel(const float* __restrict__ pts, long long n,
                                                     Ctl* ctl, uint8_t* labels) {
    __shared__ Octagon s_o;
    __shared__ unsigned s_cnt[4];
    if (read_status(ctl) != CH_OK) return;
    copy_octagon(&s_o, &ctl->oct);
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    unsigned c[4] = {0u, 0u, 0u, 0u};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float2 p = reinterpret_cast<const float2*>(pts)[i];
        const int X = __float2int_rn(p.x), Y = __float2int_rn(p.y);
        const int r = in_inner_strict(s_o, X, Y) ? -1 : classify_paper_slow(p.x, p.y, &s_o);
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
void launch_init(Ctl* ctl, int mode, cudaStream_t s) { init_kernel<<<1, 256, 0, s>>>(ctl, mode); }

void launch_sample(const float* pts, long long n, int head, long long ntiles, Ctl* ctl, int grid, cudaStream_t s) {
    sample_kernel<<<grid, 256, 0, s>>>(pts, n, head, ntiles, ctl);
}

void launch_main(const float* pts, long long n, int head, long long ntiles, Ctl* ctl, uint64_t* raw_xy,
                 uint32_t* raw_idx, unsigned switch_at, int grid, cudaStream_t s) {
    main_kernel<<<grid, 256, kMainSmemBytes, s>>>(pts, n, head, ntiles, ctl, raw_xy, raw_idx, switch_at);
}

void launch_tail(const float* pts, long long n, int head, Ctl* ctl, const uint64_t* raw_xy, const uint32_t* raw_idx,
                 uint32_t* keys, uint64_t* vals, int phase, int hull, int32_t* out_idx, int64_t* out_n,
                 cudaStream_t s) {
    tail_kernel<<<1, kTailThreads, kTailSmemBytes, s>>>(pts, n, head, ctl, raw_xy, raw_idx, keys, vals, phase, hull,
                                                        out_idx, out_n);
}

void launch_stagec(const float* pts, long long n, int head, long long ntiles, Ctl* ctl, const uint64_t* raw_xy,
                   const uint32_t* raw_idx, uint32_t* keys, uint64_t* vals, int grid, cudaStream_t s) {
    stagec_kernel<<<grid, 256, 0, s>>>(pts, n, head, ntiles, ctl, raw_xy, raw_idx, keys, vals);
}

void launch_labels(const float* pts, long long n, Ctl* ctl, uint8_t* labels, int grid, cudaStream_t s) {
    labels_kernel<<<grid, 256, 0, s>>>(pts, n, ctl, labels);
}

void launch_filter_output(const Ctl* ctl, long long n, int32_t* out_ext8, int64_t* out_counts4, cudaStream_t s) {
    filter_output_kernel<<<1, 32, 0, s>>>(ctl, n, out_ext8, out_counts4);
}

long long sample_tiles_host(long long ntiles) { return sample_tiles(ntiles); }

cudaError_t configure_filter_kernels() {
    cudaError_t e = cudaFuncSetAttribute(tail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(main_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMainSmemBytes);
    return e;
}

cudaError_t occupancy_filter(int* main_k, int* stagec, int* labels) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(main_k, main_kernel, 256, kMainSmemBytes);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(stagec, stagec_kernel, 256, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(labels, labels_kernel, 256, 0);
    return e;
}

}  // namespace ch
