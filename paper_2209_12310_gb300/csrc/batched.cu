// batched.cu -- k independent hulls packed back to back (ch_hull_batched).
//
// The sets are cut into tiles of at most `tile` points (a tile never spans
// two sets; tile = threads x points per thread of the tile kernels, one of
// the compiled shapes that the autotuner picks per device and batch size)
// and every launch covers all sets at once:
//   bt_init      per-set control blocks and tile counts;
//   bt_scan      tile offsets (exclusive prefix over the sets, one block);
//   bt_extremes  tiles: validation and the 8 extremes of each set as packed
//                (key, lowest local index) maxima (Alg. 2, findExtremes);
//   bt_octagon   one block per set: octagon, inner region, the chain end
//                point records;
//   bt_filter    tiles: the hull-rule classification of every point against
//                its set's octagon, records compacted into the set's region
//                (the loop of Alg. 1/2), support-line end points reduced;
//   bt_hull_small  one block per set: the support-line records, then the
//                hull of a set with few records in a small footprint;
//   bt_star      sets with more records than one block holds: the star
//                polygon of the set's records (star.cuh) drops the records
//                strictly inside it (points near a circle, Table V);
//   bt_hull      one block per set: the hull of its records (quickhull rounds
//                and the stitch, as in the single hull's last block).
// Sets whose records exceed what one block holds go through the bucketed
// large-survivor path together (batched_large.cu); the rare set it cannot
// finish (a bucket chain longer than kBkChain) is flagged and the host runs
// the single-hull path on it.  Each result equals ch_hull on the set alone
// (local indices).  The device work of one call is captured into a CUDA graph
// on a private stream; the executable graph of a (device, stream) is updated
// in place from call to call and launched on the caller's stream.
#include "batched_large.h"
#include "ch_internal.cuh"
#include "extremes.cuh"
#include "host.h"
#include "hullcore.cuh"
#include "launch.h"
#include "octagon.cuh"
#include "records.cuh"
#include "star.cuh"
#include "tma.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace ch {

constexpr int kBTileMin = 2048;        // smallest tile of the compiled shapes
constexpr int kBHullThreads = 512;     // threads of bt_hull (a multiple of 128)
constexpr int kBOctThreads = 256;      // threads of bt_octagon: a warp per direction

struct BArgs {
    const float* pts;
    const int64_t* offsets;   // device, k + 1
    int k;
    Ctl* ctl;                 // k control blocks
    uint32_t* keys;           // records: set i's region starts at offsets[i] + 16 i
    uint64_t* vals;
    int* tile_base;           // k + 1: first tile of each set
    int* tile_map;            // set of every tile
    int32_t* out_idx;
    int64_t* out_n;
    unsigned char* big;       // k: the set needs the single-hull path
    int tile;                 // points per tile (threads x points per thread of the tile kernels)
    long long total;          // points of the batch
    long long nwt;            // warp tiles of the streamed body (bt_extremes)
    int head;                 // points before the body's first 16-byte boundary (0 or 1)
    int wtile;                // points per warp tile of bt_extremes (32 x points per lane)
    unsigned* star_ctr;       // bt_star's work list: [0] sets from the front, [1] from the back, [2] taken
    int* star_list;           // k entries
    uint32_t* kP;             // the bucketed path's scatter buffer (set regions as keys / vals)
    uint64_t* vP;
};

// Sets with more records than this go through bt_star first (the others of
// its list come after them).
constexpr unsigned kBStarHuge = 1u << 18;

__device__ __forceinline__ long long region_base(const BArgs& a, int i) { return a.offsets[i] + 16ll * i; }

// Set of tile t (written by bt_scan).
__device__ __forceinline__ int tile_set(const BArgs& a, int t) { return a.tile_map[t]; }

__global__ void bt_init(BArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.k) return;
    Ctl* c = a.ctl + i;
    for (int d = 0; d < 8; ++d) {
        c->ext_packed[d] = 0ull;
        c->line_ep[d] = (d & 1) ? 0ull : ~0ull;
    }
    c->status = CH_OK;
    c->abort = 0;
    c->count = 8u;
    c->done = 0;
    c->bk_state = 0;
    c->star_k = 0;
    for (int q = 0; q < 4; ++q) {
        c->counts4[q] = 2u;   // the two chain end points of every queue
        c->blocks_done[q] = 0u;
    }
    a.big[i] = 0;
    const long long ni = a.offsets[i + 1] - a.offsets[i];
    a.tile_base[i] = (int)((ni + a.tile - 1) / a.tile);
    if (i == 0) a.star_ctr[0] = a.star_ctr[1] = a.star_ctr[2] = 0u;
}

// Exclusive prefix of the tile counts in place (one block of 1024 threads);
// tile_base[k] = total tiles; then the set of every tile.
__global__ void __launch_bounds__(1024) bt_scan(int* tile_base, int* tile_map, int k) {
    __shared__ int s_part[1024];
    const int tid = threadIdx.x;
    const int per = (k + 1023) / 1024;
    const int lo = tid * per, hi = min(k, lo + per);
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += tile_base[i];
    s_part[tid] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = tid >= o ? s_part[tid - o] : 0;
        __syncthreads();
        s_part[tid] += v;
        __syncthreads();
    }
    int run = s_part[tid] - sum;
    for (int i = lo; i < hi; ++i) {
        const int c = tile_base[i];
        tile_base[i] = run;
        for (int t = 0; t < c; ++t) tile_map[run + t] = i;
        run += c;
    }
    if (tid == 1023) tile_base[k] = s_part[1023];
}

// ---------------------------------------------------------------------------
// Extremes of every set, streamed (findExtremes, Alg. 2).  The batch's points
// are one array; its 16-byte aligned body is cut into warp tiles of 32 P
// points (P per lane), whatever the sets.  Each block takes a contiguous
// chunk of warp tiles and its warps take the chunk's tiles in turn, so they
// move through the same sets together; each warp streams its tiles through a
// double-buffered shared-memory ring filled by bulk copies.  A tile inside
// one set goes through the single hull's per-lane tracking (extremes.cuh:
// three-input min / max of the keys, the first tile code reaching each
// extreme); when the set changes, the warp folds its lanes and raises the
// set's packed (key, ~tile code) maxima.  A tile that meets a set boundary
// is folded set by set.  The unaligned head point and the ragged tail go
// point by point.  bt_octagon then rescans each set's winning tiles for the
// lowest index.
// Tile codes: 0 = head, t + 1 = body tile t, nwt + 1 = tail.

// Set holding point p (warp-uniform): a 32-way search over the offsets.
__device__ __forceinline__ int bt_find_set(const BArgs& a, long long p) {
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = a.k;   // offsets[lo] <= p < offsets[hi]
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) / 32;
        const int probe = lo + lane * step;
        const bool le = probe < hi && __ldg(a.offsets + probe) <= p;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, le);   // a prefix of the lanes (lane 0 always)
        const int last = 31 - __clz((int)m);
        lo = lo + last * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// The warp's lanes folded into the set's packed maxima; validity into its status.
__device__ __forceinline__ void bt_flush_track(const Track& tr, Ctl* c) {
    const int lane = threadIdx.x & 31;
    const bool err = tr.bad || (tr.orv >> kCoordBits) != 0u;
    if (__any_sync(0xFFFFFFFFu, err) && lane == 0) set_status(c, CH_ERANGE);
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        unsigned long long p = pack_best(d, tr.best[d], tr.code[d]);
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long q = __shfl_xor_sync(0xFFFFFFFFu, p, o);
            p = q > p ? q : p;
        }
        if (lane == 0 && p) atomicMax(&c->ext_packed[d], p);
    }
}

// A warp tile meeting a set boundary (point p0 + 2 (32 j + lane) + h in
// float4 j, half h), set by set from set s on.
template <int P>
__device__ __noinline__ void bt_tile_straddle(const BArgs& a, const float4* cur, long long p0, int s, unsigned code) {
    const int lane = threadIdx.x & 31;
    const long long p1 = p0 + 32ll * P;
    for (int q = s; q < a.k; ++q) {
        const long long qb = __ldg(a.offsets + q), qe = __ldg(a.offsets + q + 1);
        Track tr;
        track_init(tr);
        int tk[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) tk[d] = dir_is_max(d) ? INT_MIN : INT_MAX;
#pragma unroll 1
        for (int j = 0; j < P / 2; ++j) {
            const float4 v = cur[j * 32 + lane];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long i = p0 + 2 * (j * 32 + lane) + h;
                if (i < qb || i >= qe) continue;
                int X, Y;
                convert_pt(h ? v.z : v.x, h ? v.w : v.y, X, Y, tr);
#pragma unroll
                for (int d = 0; d < 8; ++d) {
                    const int key = dir_key(d, X, Y);
                    tk[d] = dir_is_max(d) ? max(tk[d], key) : min(tk[d], key);
                }
            }
        }
        track_tile(tr, tk, code);
        bt_flush_track(tr, a.ctl + q);
        if (qe >= p1) break;
    }
}

// Points [lo, hi) one per lane, each with its own set (head and tail).
__device__ void bt_points_scalar(const BArgs& a, long long lo, long long hi, unsigned code) {
    const int lane = threadIdx.x & 31;
    for (long long b = lo; b < hi; b += 32) {
        const long long i = b + lane;
        if (i >= hi) continue;
        int l = 0, r = a.k;   // offsets[l] <= i < offsets[r]
        while (r - l > 1) {
            const int mid = (l + r) >> 1;
            if (__ldg(a.offsets + mid) <= i) l = mid;
            else r = mid;
        }
        Ctl* c = a.ctl + l;
        const float x = a.pts[2 * i], y = a.pts[2 * i + 1];
        const int X = __float2int_rn(x), Y = __float2int_rn(y);
        if (__int2float_rn(X) != x || __int2float_rn(Y) != y || (((unsigned)X | (unsigned)Y) >> kCoordBits) != 0u) {
            set_status(c, CH_ERANGE);
            continue;
        }
#pragma unroll
        for (int d = 0; d < 8; ++d) atomicMax(&c->ext_packed[d], pack_best(d, dir_key(d, X, Y), code));
    }
}

template <int T, int P>
__global__ void __launch_bounds__(T) bt_extremes(BArgs a) {
    constexpr int kWarps = T / 32, kF4 = 16 * P;
    constexpr long long kPts = 32ll * P;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ unsigned long long s_bar[kWarps][kStages];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long nwt = a.nwt;
    const long long per = (nwt + gridDim.x - 1) / gridDim.x;
    const long long c0 = min(nwt, (long long)blockIdx.x * per), c1 = min(nwt, c0 + per);
    if (blockIdx.x == 0 && warp == 0) {
        bt_points_scalar(a, 0, a.head, 0u);
        bt_points_scalar(a, a.head + nwt * kPts, a.total, (unsigned)(nwt + 1));
    }
    if (c0 + warp >= c1) return;
    WarpStreamT<kF4> ws{reinterpret_cast<float4*>(dsm) + warp * kStages * kF4, s_bar[warp],
                        reinterpret_cast<const float4*>(a.pts + 2 * a.head), c0 + warp, kWarps, c1, lane};
    int s = bt_find_set(a, a.head + (c0 + warp) * kPts);
    int ts = -1;   // the set the lanes' tracks belong to
    Track tr;
    track_init(tr);
    ws.start();
    for (long long k = 0;; ++k) {
        const long long t = c0 + warp + k * kWarps;
        if (t >= c1) break;
        const long long p0 = a.head + t * kPts;
        while (__ldg(a.offsets + s + 1) <= p0) ++s;
        const float4* cur = ws.acquire(k, a.ctl + s);
        if (!cur) {   // a copy never completed: every set of the rest of the chunk fails
            ws.drain(k);
            const long long pend = a.head + c1 * kPts;
            for (int q = s + lane; q < a.k && __ldg(a.offsets + q) < pend; q += 32) set_status(a.ctl + q, CH_ETIMEOUT);
            if (ts >= 0 && lane == 0) set_status(a.ctl + ts, CH_ETIMEOUT);
            return;
        }
        if (__ldg(a.offsets + s + 1) >= p0 + kPts) {   // inside set s
            if (s != ts) {
                if (ts >= 0) bt_flush_track(tr, a.ctl + ts);
                track_init(tr);
                ts = s;
            }
            int tk[8];
#pragma unroll
            for (int j = 0; j < P / 2; ++j) {
                const float4 v = cur[j * 32 + lane];
                int X0, Y0, X1, Y1;
                convert_pt(v.x, v.y, X0, Y0, tr);
                convert_pt(v.z, v.w, X1, Y1, tr);
                tile_keys2(tk, X0, Y0, X1, Y1, j == 0);
            }
            track_tile(tr, tk, (unsigned)(t + 1));
        } else {
            if (ts >= 0) bt_flush_track(tr, a.ctl + ts);
            track_init(tr);
            ts = -1;
            bt_tile_straddle<P>(a, cur, p0, s, (unsigned)(t + 1));
        }
        ws.release(k);
    }
    if (ts >= 0) bt_flush_track(tr, a.ctl + ts);
}

// One block per set: the lowest index of each extreme (warp d rescans the
// winning tile of direction d within the set), the octagon of the extremes
// (with the inner region, which settles most points of bt_filter), the chain
// end-point records.
__global__ void __launch_bounds__(kBOctThreads) bt_octagon(BArgs a) {
    __shared__ Octagon s_o;
    __shared__ int s_vx[8], s_vy[8], s_id[8], s_st, s_bad;
    const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Ctl* c = a.ctl + i;
    const long long base = a.offsets[i], ni = a.offsets[i + 1] - base;
    if (tid == 0) {
        s_st = read_status(c);
        s_bad = 0;
    }
    __syncthreads();
    if (ni == 0 || s_st != CH_OK) {
        if (tid == 0) {
            a.out_n[i] = ni == 0 ? 0 : s_st;
            c->done = 1;
        }
        return;
    }
    {
        const int d = warp;
        const unsigned long long pk = c->ext_packed[d];
        const unsigned code = 0xFFFFFFFFu - (unsigned)(pk & 0xFFFFFFFFull);
        const unsigned hk = (unsigned)(pk >> 32);
        const int best = dir_is_max(d) ? (int)hk : (int)(0xFFFFFFFFu - hk);
        long long lo, hi;   // the tile's points, within the set
        if (code == 0u) { lo = 0; hi = a.head; }
        else if ((long long)code <= a.nwt) { lo = a.head + (long long)(code - 1u) * a.wtile; hi = lo + a.wtile; }
        else { lo = a.head + a.nwt * a.wtile; hi = a.total; }
        lo = max(lo, base);
        hi = min(hi, base + ni);
        long long first = LLONG_MAX;
#pragma unroll 4
        for (long long j = lo + lane; j < hi; j += 32) {
            const float2 p = __ldg(reinterpret_cast<const float2*>(a.pts) + j);
            if (j < first && dir_key(d, __float2int_rn(p.x), __float2int_rn(p.y)) == best) first = j;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const long long q = __shfl_xor_sync(0xFFFFFFFFu, first, o);
            first = q < first ? q : first;
        }
        if (lane == 0) {
            if (pk == 0ull || first == LLONG_MAX) {   // cannot happen for a valid set; fail safe
                s_bad = 1;
                first = base;
            }
            s_id[d] = (int)(first - base);
            const float2 p = reinterpret_cast<const float2*>(a.pts)[first];
            s_vx[d] = __float2int_rn(p.x);
            s_vy[d] = __float2int_rn(p.y);
        }
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) {
            set_status(c, CH_ECUDA);
            a.out_n[i] = CH_ECUDA;
            c->done = 1;
        }
        return;
    }
    setup_octagon_block(s_o, s_vx, s_vy, s_id, true);
    copy_octagon(&c->oct, &s_o);
    const long long rb = region_base(a, i);
    if (tid < 12) {
        int r, d;
        bool emit = true;
        if (tid < 8) {
            r = tid >> 1;
            d = (tid & 1) ? ((2 * r + 2) & 7) : 2 * r;
        } else {
            r = tid - 8;
            d = 2 * r + 1;
            const int qa = 2 * r, qb = (2 * r + 2) & 7;
            emit = orient64(s_vx[qa], s_vy[qa], s_vx[qb], s_vy[qb], s_vx[d], s_vy[d]) < 0;
        }
        if (emit) {
            uint32_t u, v;
            queue_frame(r, s_vx[d], s_vy[d], u, v);
            const unsigned pos = tid < 8 ? (unsigned)tid : atomicAdd(&c->count, 1u);
            if (tid >= 8) atomicAdd(&c->counts4[r], 1u);
            a.keys[rb + pos] = make_key(r, u);
            a.vals[rb + pos] = make_val(v, (uint32_t)s_id[d]);
        }
    }
}

// Per tile of T x P points: every thread loads its P points (a batch of at
// most 8 at a time, all loads in flight together), then classifies them.
// Survivors are staged per warp (kBtWarpRecs records) and written out in
// batches: one returning atomic per batch instead of one per 32 points.
constexpr int kBtWarpRecs = 128;
struct BtWarpBuf {
    uint64_t val[kBtWarpRecs];
    uint32_t key[kBtWarpRecs];
};

__device__ __forceinline__ void bt_flush(BtWarpBuf& b, unsigned& cnt, Ctl* c, uint32_t* keys, uint64_t* vals,
                                         long long rb) {
    const int lane = threadIdx.x & 31;
    if (cnt == 0u) return;
    unsigned base = 0u;
    if (lane == 0) base = atomicAdd(&c->count, cnt);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (unsigned j = lane; j < cnt; j += 32) {
        keys[rb + base + j] = b.key[j];
        vals[rb + base + j] = b.val[j];
    }
    __syncwarp();
    cnt = 0u;
}

template <int T, int P>
__global__ void __launch_bounds__(T) bt_filter(BArgs a, int ntiles) {
    constexpr int kBTile = T * P;
    constexpr int kB = P < 8 ? P : 8;   // points loaded together
    __shared__ Octagon s_o;
    __shared__ int s_set, s_skip;
    __shared__ BtWarpBuf s_wb[T / 32];
    const int tid = threadIdx.x, lane = tid & 31;
    BtWarpBuf& wb = s_wb[tid >> 5];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (tid == 0) {
            const int i = tile_set(a, t);
            s_set = i;
            s_skip = *(volatile int*)&a.ctl[i].done;
        }
        __syncthreads();
        const int i = s_set;
        if (!s_skip) {
            copy_octagon(&s_o, &a.ctl[i].oct);
            __syncthreads();
            Ctl* c = a.ctl + i;
            const long long base = a.offsets[i], ni = a.offsets[i + 1] - base;
            const long long p0 = (long long)(t - a.tile_base[i]) * kBTile;
            const long long p1 = min(ni, p0 + kBTile);
            const long long rb = region_base(a, i);
            const float2* p2 = reinterpret_cast<const float2*>(a.pts) + base;
            unsigned wcnt = 0u;                      // records staged in wb
            unsigned qn[4] = {0u, 0u, 0u, 0u};       // records per queue (lane 0)
            for (long long b0 = p0; b0 < p1; b0 += (long long)T * kB) {   // uniform trip counts
                float2 pv[kB];
#pragma unroll
                for (int j = 0; j < kB; ++j) {
                    const long long p = b0 + (long long)j * T + tid;
                    if (p < p1) pv[j] = __ldcs(p2 + p);
                }
#pragma unroll 1
                for (int j = 0; j < kB; ++j) {
                const long long p = b0 + (long long)j * T + tid;
                const bool valid = p < p1;
                int r = -1, X = 0, Y = 0;
                if (valid) {
                    X = __float2int_rn(pv[j].x);
                    Y = __float2int_rn(pv[j].y);
                    r = classify_hull(pv[j].x, pv[j].y, s_o);
                }
                bool keep = r >= 0;
                if (!__any_sync(0xFFFFFFFFu, keep)) continue;
                if (reduce_on_line(s_o, keep, X, Y, (unsigned)p, c)) keep = false;
                const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
                if (!bal) continue;
#pragma unroll
                for (int q = 0; q < 4; ++q) qn[q] += __popc(__ballot_sync(0xFFFFFFFFu, keep && r == q));
                if (wcnt + (unsigned)__popc(bal) > (unsigned)kBtWarpRecs) bt_flush(wb, wcnt, c, a.keys, a.vals, rb);
                if (keep) {
                    uint32_t u, v;
                    queue_frame(r, X, Y, u, v);
                    const unsigned pos = wcnt + __popc(bal & lanemask_lt());
                    wb.key[pos] = make_key(r, u);
                    wb.val[pos] = make_val(v, (uint32_t)p);
                }
                wcnt += __popc(bal);
                __syncwarp();
                }
            }
            // the tile's records and queue counts (a tile never spans two sets)
            bt_flush(wb, wcnt, c, a.keys, a.vals, rb);
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (qn[q]) atomicAdd(&c->counts4[q], qn[q]);
        }
        __syncthreads();
    }
}

// One block per set, in two kernels.  bt_hull_small (every set): the
// support-line records, then the hull of a set of at most kBSmallRec records
// in a small shared-memory footprint (several blocks per SM).  bt_hull (the
// other sets): the hull when one block can hold the records, else the set is
// flagged for the bucketed path.  A small set whose quickhull rounds exceed
// their vertex capacity is flagged the same way.
constexpr int kBSmallRec = 2048;        // records of a small set
constexpr int kBSmallVert = 256;        // quickhull vertices of a small set
constexpr int kBSmallThreads = 256;
using QhSmall = QhSmemT<kBSmallRec, kBSmallVert>;

__global__ void __launch_bounds__(kBSmallThreads) bt_hull_small(BArgs a) {
    __shared__ QhSmall q;
    __shared__ unsigned long long s_lep[8];
    __shared__ uint64_t s_lval[8];
    __shared__ unsigned s_lkey[8];
    __shared__ int s_lpos[8], s_done, s_mv;
    __shared__ unsigned s_m, s_total;
    __shared__ Octagon s_o;
    const int i = blockIdx.x, tid = threadIdx.x;
    Ctl* c = a.ctl + i;
    if (tid == 0) s_done = *(volatile int*)&c->done;
    __syncthreads();
    if (s_done) return;
    copy_octagon(&s_o, &c->oct);
    if (tid < 8) s_lep[tid] = *(volatile unsigned long long*)&c->line_ep[tid];
    if (tid == 8) s_m = *(volatile unsigned*)&c->count;
    __syncthreads();
    if (tid < 8) s_lpos[tid] = line_record(s_o, tid, s_lep[tid], s_lkey[tid], s_lval[tid]) ? 1 : -1;
    __syncthreads();
    if (tid == 0) {
        unsigned m = s_m;
        for (int t = 0; t < 8; ++t)
            if (s_lpos[t] > 0) s_lpos[t] = (int)m++;
        s_total = m;
        c->count = m;
    }
    __syncthreads();
    const unsigned total = s_total;
    const long long rb = region_base(a, i);
    const long long base = a.offsets[i], ni = a.offsets[i + 1] - base;
    if (tid < 8 && s_lpos[tid] >= 0) {
        a.keys[rb + s_lpos[tid]] = s_lkey[tid];
        a.vals[rb + s_lpos[tid]] = s_lval[tid];
        atomicAdd(&c->counts4[s_lkey[tid] >> kKeyBits], 1u);
    }
    if (total > (unsigned)kBSmallRec) {   // bt_hull's, after bt_star's when one block cannot hold them
        if (tid == 0 && total > (unsigned)kMidCap) {
            if (total > kBStarHuge) a.star_list[atomicAdd(&a.star_ctr[0], 1u)] = i;
            else a.star_list[a.k - 1 - (int)atomicAdd(&a.star_ctr[1], 1u)] = i;
        }
        return;
    }
    __syncthreads();   // also makes this block's line records visible to it
    for (unsigned j = tid; j < total; j += blockDim.x) {
        const uint32_t k = __ldcg(a.keys + rb + j);
        const uint64_t w = __ldcg(a.vals + rb + j);
        q.ru[j] = (int)(k & kKeyMask);
        q.rv[j] = (int)(w >> 31);
        q.ri[j] = (int)(w & 0x7FFFFFFFull);
        q.rs[j] = (int)(k >> kKeyBits);
    }
    __syncthreads();
    if (qh_chains(q, (int)total, &s_mv)) {
        stitch_cycle(q.ru, q.rv, q.ri, s_mv, q.rs, c, ni, a.out_idx + base, a.out_n + i);
        if (tid == 0) c->done = 1;
    } else if (tid == 0) {
        a.big[i] = 1;   // too many chain vertices for the small footprint: the bucketed path
        c->done = 1;
    }
}

// ---------------------------------------------------------------------------
// The star polygon of a set whose records one block cannot hold (points near
// a circle, where the octagon keeps almost all of them).  One block per such
// set, persistent over the list that bt_hull_small builds (the sets with
// more than kBStarHuge records first):
//   1. bins: the set's first kBStarBinRec records go to their angular bins
//      around the centre of the octagon's box, in shared memory; each bin
//      keeps its point farthest from the centre.  A set's records come in
//      the order of its points, so these are a sample of them when the
//      points are in random order; any other order only makes the polygon
//      smaller;
//   2. the polygon (star_finish, star.cuh): its vertices are re-read from
//      the input by index and it is checked exactly; without one the set is
//      left as it is;
//   3. the records whose point is not strictly inside the polygon are
//      copied to the set's region of the scatter buffer (free until the
//      bucketed path), then back, with the per-queue counts recounted.
// A point strictly inside the polygon is an interior point of the set's hull
// (star.cuh), so the records left have the same hull.  The sets then take
// bt_hull's one-block path, or the bucketed path when still too many.
//
// Each warp streams a contiguous range of the records with the loads of its
// next step in flight while it works on the current one; no step waits for
// the other warps.
constexpr int kBStarThreads = 512;
constexpr int kBStarU = 8;                    // records per lane and step
constexpr unsigned kBStarBinRec = 1u << 19;   // records binned (64 per bin)
constexpr size_t kBStarAOff = (sizeof(StarPoly) + 15) / 16 * 16;
constexpr size_t kBStarSmem = kBStarAOff + (sizeof(int2) + sizeof(unsigned short)) * kStarBins;
static_assert(sizeof(unsigned long long) * kStarBins <= (sizeof(int2) + sizeof(unsigned short)) * kStarBins,
              "the bins fit in work area A");

// One step of a warp: records [r, r + 32 kBStarU) of a range ending at hi,
// record r + 32 u + lane in slot u.
__device__ __forceinline__ void bt_star_load(const uint32_t* __restrict__ keys, const uint64_t* __restrict__ vals,
                                             long long rb, unsigned r, unsigned hi, uint32_t (&kk)[kBStarU],
                                             uint64_t (&vv)[kBStarU]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int u = 0; u < kBStarU; ++u) {
        const unsigned j = r + 32u * u + lane;
        kk[u] = j < hi ? __ldcg(keys + rb + j) : 0u;
        vv[u] = j < hi ? __ldcg(vals + rb + j) : 0ull;
    }
}

__device__ __forceinline__ void bt_record_xy(uint32_t k, uint64_t v, int& X, int& Y) {
    frame_to_xy((int)(k >> kKeyBits), (int)(k & kKeyMask), (int)(v >> 31), X, Y);
}

__global__ void __launch_bounds__(kBStarThreads, 1) bt_star(BArgs a) {
    extern __shared__ __align__(16) char dyn[];
    StarPoly& P = *reinterpret_cast<StarPoly*>(dyn);
    unsigned long long* bins = reinterpret_cast<unsigned long long*>(dyn + kBStarAOff);
    int2* va = reinterpret_cast<int2*>(dyn + kBStarAOff);
    unsigned short* ba = reinterpret_cast<unsigned short*>(dyn + kBStarAOff + sizeof(int2) * kStarBins);
    constexpr int kWarps = kBStarThreads / 32;
    constexpr unsigned kStep = 32u * kBStarU;
    __shared__ unsigned s_kept, s_q[4];
    __shared__ int s_set, s_cx, s_cy;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned n_front = a.star_ctr[0], n_back = a.star_ctr[1];
    for (;;) {
        if (tid == 0) {
            const unsigned g = atomicAdd(&a.star_ctr[2], 1u);
            s_set = g < n_front ? a.star_list[g]
                                : (g - n_front < n_back ? a.star_list[a.k - 1 - (int)(g - n_front)] : -1);
        }
        __syncthreads();
        const int i = s_set;
        if (i < 0) return;
        Ctl* c = a.ctl + i;
        const long long base = a.offsets[i], ni = a.offsets[i + 1] - base;
        const long long rb = region_base(a, i);
        const unsigned m = c->count;
        if (tid == 0) {
            s_cx = (c->oct.vx[W] + c->oct.vx[E]) / 2;
            s_cy = (c->oct.vy[S] + c->oct.vy[N]) / 2;
            s_kept = 0u;
        }
        if (tid < 4) s_q[tid] = 0u;
        for (int b = tid; b < kStarBins; b += kBStarThreads) bins[b] = 0ull;
        __syncthreads();
        const int cx = s_cx, cy = s_cy;
        // 1. bins: warp w takes [w per, (w + 1) per) of the first mb records
        {
            const unsigned mb = min(m, kBStarBinRec);
            const unsigned per = ((mb + kWarps - 1) / kWarps + kStep - 1) / kStep * kStep;
            const unsigned lo = min(mb, warp * per), hi = min(mb, lo + per);
            uint32_t kk[kBStarU];
            uint64_t vv[kBStarU];
            bt_star_load(a.keys, a.vals, rb, lo, hi, kk, vv);
            for (unsigned r = lo; r < hi; r += kStep) {
                uint32_t nk[kBStarU];
                uint64_t nv[kBStarU];
                bt_star_load(a.keys, a.vals, rb, r + kStep, hi, nk, nv);
#pragma unroll
                for (int u = 0; u < kBStarU; ++u) {
                    if (r + 32u * u + lane >= hi) continue;
                    int X, Y;
                    bt_record_xy(kk[u], vv[u], X, Y);
                    const int dx = X - cx, dy = Y - cy;
                    const unsigned long long d2 = (unsigned long long)((long long)dx * dx + (long long)dy * dy);
                    const unsigned long long key = ((d2 >> 17) << 32) | (vv[u] & 0x7FFFFFFFull);
                    const int b = star_bin(dx, dy);
                    if (key > bins[b]) atomicMax(&bins[b], key);
                }
#pragma unroll
                for (int u = 0; u < kBStarU; ++u) {
                    kk[u] = nk[u];
                    vv[u] = nv[u];
                }
            }
        }
        __syncthreads();
        // 2. the polygon
        const int K = star_finish<kBStarThreads, true>(bins, a.pts + 2 * base, ni, cx, cy, va, ba, P, c);
        if (tid == 0) c->star_k = K;
        if (K == 0) {
            __syncthreads();
            continue;
        }
        // 3. the records not strictly inside go to the scatter buffer
        unsigned t0 = 0u, t1 = 0u, t2 = 0u, t3 = 0u;   // kept per queue (lane counts)
        {
            const unsigned per = ((m + kWarps - 1) / kWarps + kStep - 1) / kStep * kStep;
            const unsigned lo = min(m, warp * per), hi = min(m, lo + per);
            uint32_t kk[kBStarU];
            uint64_t vv[kBStarU];
            bt_star_load(a.keys, a.vals, rb, lo, hi, kk, vv);
            for (unsigned r = lo; r < hi; r += kStep) {
                uint32_t nk[kBStarU];
                uint64_t nv[kBStarU];
                bt_star_load(a.keys, a.vals, rb, r + kStep, hi, nk, nv);
#pragma unroll
                for (int u = 0; u < kBStarU; ++u) {
                    bool keep = r + 32u * u + lane < hi;
                    if (keep) {
                        int X, Y;
                        bt_record_xy(kk[u], vv[u], X, Y);
                        keep = !star_inside(X - cx, Y - cy, P);
                    }
                    const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
                    if (bal == 0u) continue;
                    unsigned pos = 0u;
                    if (lane == 0) pos = atomicAdd(&s_kept, (unsigned)__popc(bal));
                    pos = __shfl_sync(0xFFFFFFFFu, pos, 0) + (unsigned)__popc(bal & lanemask_lt());
                    if (keep) {
                        a.kP[rb + pos] = kk[u];
                        a.vP[rb + pos] = vv[u];
                        const unsigned q = kk[u] >> kKeyBits;
                        t0 += q == 0u;
                        t1 += q == 1u;
                        t2 += q == 2u;
                        t3 += q == 3u;
                    }
                }
#pragma unroll
                for (int u = 0; u < kBStarU; ++u) {
                    kk[u] = nk[u];
                    vv[u] = nv[u];
                }
            }
        }
        t0 = __reduce_add_sync(0xFFFFFFFFu, t0);
        t1 = __reduce_add_sync(0xFFFFFFFFu, t1);
        t2 = __reduce_add_sync(0xFFFFFFFFu, t2);
        t3 = __reduce_add_sync(0xFFFFFFFFu, t3);
        if (lane == 0) {
            atomicAdd(&s_q[0], t0);
            atomicAdd(&s_q[1], t1);
            atomicAdd(&s_q[2], t2);
            atomicAdd(&s_q[3], t3);
        }
        __syncthreads();
        const unsigned w = s_kept;
        for (unsigned j = tid; j < w; j += kBStarThreads) {   // back into the set's records
            a.keys[rb + j] = __ldcg(a.kP + rb + j);
            a.vals[rb + j] = __ldcg(a.vP + rb + j);
        }
        if (tid < 4) c->counts4[tid] = s_q[tid];
        if (tid == 0) c->count = w;
        __syncthreads();
    }
}

constexpr size_t bt_cmax(size_t x, size_t y) { return x > y ? x : y; }
constexpr size_t kBHullSmem = bt_cmax(kMidSmemBytes, sizeof(QhSmem));

__global__ void __launch_bounds__(kBHullThreads, 1) bt_hull(BArgs a) {
    extern __shared__ __align__(16) char dyn[];
    __shared__ int s_done, s_mv;
    const int i = blockIdx.x, tid = threadIdx.x;
    Ctl* c = a.ctl + i;
    if (tid == 0) s_done = *(volatile int*)&c->done;
    __syncthreads();
    if (s_done) return;   // empty or failed, or done by bt_hull_small
    const unsigned total = *(volatile unsigned*)&c->count;   // with the line records
    const long long rb = region_base(a, i);
    const long long base = a.offsets[i], ni = a.offsets[i + 1] - base;
    if (total > (unsigned)kMidCap) {
        if (tid == 0) a.big[i] = 1;
        return;
    }
    QhSmem& q = *reinterpret_cast<QhSmem*>(dyn);
    for (unsigned j = tid; j < total; j += blockDim.x) {
        const uint32_t k = __ldcg(a.keys + rb + j);
        const uint64_t w = __ldcg(a.vals + rb + j);
        q.ru[j] = (int)(k & kKeyMask);
        q.rv[j] = (int)(w >> 31);
        q.ri[j] = (int)(w & 0x7FFFFFFFull);
        q.rs[j] = (int)(k >> kKeyBits);
    }
    __syncthreads();
    if (qh_chains(q, (int)total, &s_mv)) {
        stitch_cycle(q.ru, q.rv, q.ri, s_mv, q.rs, c, ni, a.out_idx + base, a.out_n + i);
    } else {
        __syncthreads();
        mid_hull(a.keys + rb, a.vals + rb, (int)total, a.pts + 2 * base, ni, c, a.out_idx + base, a.out_n + i, dyn);
    }
}

// ---------------------------------------------------------------------------
// Workspace per (device, stream), grow-only.
struct BWork {
    char* base = nullptr;
    size_t bytes = 0;
};
static std::mutex g_bmu;
static std::map<std::pair<int, cudaStream_t>, BWork> g_bws;

static size_t bt_align(size_t x) { return (x + 255) / 256 * 256; }

struct BLayout {
    size_t ctl, keys, vals, tiles, tmap, rmap, big, redo, star_ctr, star_list;
    size_t seg_nb, seg_bbase, seg_lo, seg_scale, seg_tbase, rt_base, totals;
    size_t bcount, bcur, bstart, blen, bu, bv, bi, kP, vP, cu, cv, ci, clen, ctmap, counters;
    size_t zero_from, zero_to;   // bucket counters: cleared before each batch
    size_t total;
    unsigned bcap, tcap, rtcap;
};

// big_pts: points of the sets that can exceed one block (more than kMidCap
// points), big_sets: how many; they bound the buckets and chain tiles.
static BLayout bt_layout(long long total, int k, long long big_pts, long long big_sets, long long tiles) {
    BLayout L;
    const long long cap = total + 16ll * k + 16;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t r = o;
        o = bt_align(o + bytes);
        return r;
    };
    const size_t nseg = 4 * (size_t)k;
    L.bcap = (unsigned)((big_pts + 16 * big_sets) / kBkAvg + big_sets * (4 * kBkMinQ + 4) + 8);
    L.tcap = L.bcap / kBkGroup + (unsigned)(4 * big_sets) + 8;
    L.ctl = take(sizeof(Ctl) * (size_t)k);
    L.keys = take(sizeof(uint32_t) * (size_t)cap);
    L.vals = take(sizeof(uint64_t) * (size_t)cap);
    L.tiles = take(sizeof(int) * ((size_t)k + 1));
    L.tmap = take(sizeof(int) * ((size_t)tiles + 1));
    L.rtcap = (unsigned)((big_pts + 16 * big_sets) / kBLTile + big_sets + 1);
    L.rmap = take(sizeof(int) * (size_t)L.rtcap);
    L.big = take((size_t)k);
    L.redo = take((size_t)k);
    L.star_ctr = take(4 * 4);
    L.star_list = take(sizeof(int) * (size_t)k);
    L.seg_nb = take(4 * nseg);
    L.seg_bbase = take(4 * (nseg + 1));
    L.seg_lo = take(4 * nseg);
    L.seg_scale = take(4 * nseg);
    L.seg_tbase = take(4 * (nseg + 1));
    L.rt_base = take(4 * ((size_t)k + 1));
    L.totals = take(4 * 8);
    // Cleared before every batch: bucket counters and the merge tree's
    // arrival counters (the layout moves with the batch's sizes, so memory
    // that held other data last time can land here).
    L.zero_from = o;
    L.bcount = take(4 * (size_t)L.bcap);
    L.bcur = take(4 * (size_t)L.bcap);
    L.counters = take(4 * (size_t)kMaxLevels * L.tcap);
    L.zero_to = o;
    L.bstart = take(4 * (size_t)L.bcap);
    L.blen = take(4 * (size_t)L.bcap);
    L.bu = take(4 * (size_t)L.bcap * kBkChain);
    L.bv = take(4 * (size_t)L.bcap * kBkChain);
    L.bi = take(4 * (size_t)L.bcap * kBkChain);
    L.kP = take(sizeof(uint32_t) * (size_t)cap);
    L.vP = take(sizeof(uint64_t) * (size_t)cap);
    L.cu = take(4 * (size_t)L.tcap * kChainTile);
    L.cv = take(4 * (size_t)L.tcap * kChainTile);
    L.ci = take(4 * (size_t)L.tcap * kChainTile);
    L.clen = take(4 * (size_t)L.tcap);
    L.ctmap = take(4 * (size_t)L.tcap);
    L.total = o;
    return L;
}

static int bt_workspace(int dev, cudaStream_t s, long long total, int k, long long big_pts, long long big_sets,
                        long long tiles, char** base, BLayout* L) {
    std::lock_guard<std::mutex> lk(g_bmu);
    *L = bt_layout(total, k, big_pts, big_sets, tiles);
    BWork& w = g_bws[std::make_pair(dev, s)];
    if (w.bytes < L->total) {
        if (w.base) {
            cudaStreamSynchronize(s);
            cudaFree(w.base);
            w.base = nullptr;
            w.bytes = 0;
        }
        void* p = nullptr;
        const size_t want = L->total + L->total / 8;
        if (cudaMalloc(&p, want) != cudaSuccess) {
            cudaGetLastError();
            return CH_ENOMEM;
        }
        w.base = (char*)p;
        w.bytes = want;
    }
    *base = w.base;
    return CH_OK;
}

int reserve_batched(int dev, cudaStream_t s, long long n, int k) {
    char* base = nullptr;
    BLayout L;
    return bt_workspace(dev, s, n, std::max(k, 1), n, std::max(k, 1), n / kBTileMin + std::max(k, 1), &base, &L);
}

void release_batched_stream(int dev, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_bmu);
    auto it = g_bws.find(std::make_pair(dev, s));
    if (it == g_bws.end()) return;
    cudaStreamSynchronize(s);
    if (it->second.base) cudaFree(it->second.base);
    g_bws.erase(it);
}

static void drop_all_batched_graphs();

void release_batched() {
    drop_all_batched_graphs();
    std::lock_guard<std::mutex> lk(g_bmu);
    for (auto& kv : g_bws) {
        cudaStreamSynchronize(kv.first.second);
        if (kv.second.base) cudaFree(kv.second.base);
    }
    g_bws.clear();
}

// ---------------------------------------------------------------------------
// Tile shapes of bt_extremes / bt_filter: threads per block x points per
// thread (tile = their product).  The autotuner below picks one per device
// and batch size.
struct BtShape {
    int threads, per;
};
constexpr BtShape kBtShapes[] = {{128, 16}, {256, 8}, {256, 16}, {256, 32}, {512, 8}, {512, 16}};
constexpr int kNumBtShapes = (int)(sizeof(kBtShapes) / sizeof(kBtShapes[0]));

// Dynamic shared memory of bt_extremes: a two-stage ring of warp tiles per warp.
constexpr size_t bt_ext_smem(int threads, int per) { return (size_t)(threads / 32) * kStages * 16 * per * 16; }

template <int T, int P>
static void bt_occupancy(int* occ) {
    int a = 0, b = 0;
    cudaFuncSetAttribute(bt_extremes<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt_ext_smem(T, P));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, bt_extremes<T, P>, T, bt_ext_smem(T, P));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, bt_filter<T, P>, T, 0);
    occ[0] = std::max(1, a);
    occ[1] = std::max(1, b);
}

struct BtDevice {
    int sms = 0;
    std::string name;
    int occ[kNumBtShapes][2] = {};
};

static int bt_configure(int dev, BtDevice* out) {
    static std::mutex mu;
    static std::map<int, BtDevice> done;
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find(dev);
    if (it != done.end()) { *out = it->second; return CH_OK; }
    BtDevice d;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return CH_ECUDA;
    d.sms = prop.multiProcessorCount;
    d.name = prop.name;
    if (cudaFuncSetAttribute(bt_hull, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBHullSmem) != cudaSuccess)
        return CH_ECUDA;
    if (cudaFuncSetAttribute(bt_star, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBStarSmem) != cudaSuccess)
        return CH_ECUDA;
    if (configure_batched_large() != cudaSuccess) return CH_ECUDA;
    bt_occupancy<128, 16>(d.occ[0]);
    bt_occupancy<256, 8>(d.occ[1]);
    bt_occupancy<256, 16>(d.occ[2]);
    bt_occupancy<256, 32>(d.occ[3]);
    bt_occupancy<512, 8>(d.occ[4]);
    bt_occupancy<512, 16>(d.occ[5]);
    if (cudaGetLastError() != cudaSuccess) return CH_ECUDA;
    done[dev] = d;
    *out = d;
    return CH_OK;
}

static void launch_bt_tiles(int shape, bool filter, const BArgs& a, int nt, int grid, cudaStream_t s) {
#define CH_BT_CASE(i, T, P)                                                   \
    case i:                                                                   \
        if (filter) bt_filter<T, P><<<grid, T, 0, s>>>(a, nt);                \
        else bt_extremes<T, P><<<grid, T, bt_ext_smem(T, P), s>>>(a);         \
        break;
    switch (shape) {
        CH_BT_CASE(0, 128, 16)
        CH_BT_CASE(1, 256, 8)
        CH_BT_CASE(2, 256, 16)
        CH_BT_CASE(3, 256, 32)
        CH_BT_CASE(4, 512, 8)
        CH_BT_CASE(5, 512, 16)
        default: break;
    }
#undef CH_BT_CASE
}

// ---------------------------------------------------------------------------
// Autotuner.  Key: device name, SM count, and the batch's size class
// (floor log2 of its total points and of its set count).  On the first batch
// of a key every shape runs the tile kernels (extremes, octagon, filter) on
// that batch twice; the fastest by CUDA events is kept, in memory and, when
// CH_TUNE_CACHE names a file, in that JSON file ({"key": [threads, per,
// microseconds], ...}), read once at the first lookup.  CH_BLOCK with CH_PPT
// (or CH_TILE = threads x per) names a shape directly; a pair that is not one
// of the compiled shapes makes ch_hull_batched return CH_EINVAL.
static std::mutex g_tune_mu;
static std::map<std::string, std::pair<int, double>> g_tune;   // key -> (shape, microseconds)
static bool g_tune_loaded = false;

static int ilog2(long long x) {
    int r = 0;
    while (x > 1) { x >>= 1; ++r; }
    return r;
}

static std::string tune_key(const BtDevice& d, long long total, int k) {
    char buf[64];
    snprintf(buf, sizeof(buf), "|%d|%d|%d", d.sms, ilog2(std::max(1ll, total)), ilog2(std::max(1, k)));
    std::string name;
    for (char c : d.name) name += (c == '"' || c == '\\' || c == '|') ? '_' : c;
    return name + buf;
}

static int shape_index(int threads, int per) {
    for (int i = 0; i < kNumBtShapes; ++i)
        if (kBtShapes[i].threads == threads && kBtShapes[i].per == per) return i;
    return -1;
}

// The shape named by the environment: index, -1 = none named, -2 = invalid.
static int env_shape() {
    const char* b = getenv("CH_BLOCK");
    const char* p = getenv("CH_PPT");
    const char* t = getenv("CH_TILE");
    if (!b && !p && !t) return -1;
    if (!b || (!p && !t)) return -2;
    const int threads = atoi(b);
    int per = p ? atoi(p) : 0;
    if (!p && threads > 0) per = atoi(t) / threads;
    if (p && t && atoi(t) != threads * per) return -2;
    const int i = shape_index(threads, per);
    return i >= 0 ? i : -2;
}

static void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = getenv("CH_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "rb");
    if (!f) return;
    std::string txt;
    char buf[4096];
    size_t r;
    while ((r = fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, r);
    fclose(f);
    // entries "key": [threads, per, us]
    size_t pos = 0;
    while ((pos = txt.find('"', pos)) != std::string::npos) {
        const size_t e = txt.find('"', pos + 1);
        if (e == std::string::npos) break;
        const std::string key = txt.substr(pos + 1, e - pos - 1);
        int threads = 0, per = 0;
        double us = 0.0;
        const size_t lb = txt.find('[', e);
        if (lb == std::string::npos) break;
        if (sscanf(txt.c_str() + lb, "[%d,%d,%lf]", &threads, &per, &us) == 3 ||
            sscanf(txt.c_str() + lb, "[ %d , %d , %lf ]", &threads, &per, &us) == 3) {
            const int i = shape_index(threads, per);
            if (i >= 0) g_tune[key] = {i, us};
        }
        pos = txt.find(']', lb);
        if (pos == std::string::npos) break;
    }
}

static void tune_save_locked() {
    const char* path = getenv("CH_TUNE_CACHE");
    if (!path || !*path) return;
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return;
    fprintf(f, "{\n");
    size_t n = 0;
    for (const auto& kv : g_tune) {
        const BtShape& sh = kBtShapes[kv.second.first];
        fprintf(f, "  \"%s\": [%d, %d, %.3f]%s\n", kv.first.c_str(), sh.threads, sh.per, kv.second.second,
                ++n < g_tune.size() ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

static long long count_tiles(const std::vector<int64_t>& off, int k, int tile) {
    long long t = 0;
    for (int i = 0; i < k; ++i) t += (off[i + 1] - off[i] + tile - 1) / tile;
    return t;
}

// ---------------------------------------------------------------------------
// The device work of one call.
struct BtCall {
    BArgs a;
    BLArgs b;
    int nt, shape, grid_e, grid_f, sms;
    char* base;
    BLayout L;
};

static void bt_enqueue_tiles(const BtCall& c, cudaStream_t s) {
    const BArgs& a = c.a;
    {
        ProfScope p("batched_prep", s);
        bt_init<<<(a.k + 255) / 256, 256, 0, s>>>(a);
        bt_scan<<<1, 1024, 0, s>>>(a.tile_base, a.tile_map, a.k);
    }
    {
        ProfScope p("batched_extremes", s);
        launch_bt_tiles(c.shape, false, a, c.nt, c.grid_e, s);
    }
    { ProfScope p("batched_octagon", s); bt_octagon<<<a.k, kBOctThreads, 0, s>>>(a); }
    {
        ProfScope p("batched_filter", s);
        launch_bt_tiles(c.shape, true, a, c.nt, c.grid_f, s);
    }
}

static int bt_enqueue(const BtCall& c, unsigned char* redo, cudaStream_t s) {
    bt_enqueue_tiles(c, s);
    { ProfScope p("batched_hull_small", s); bt_hull_small<<<c.a.k, kBSmallThreads, 0, s>>>(c.a); }
    { ProfScope p("batched_star", s); bt_star<<<c.sms, kBStarThreads, kBStarSmem, s>>>(c.a); }
    { ProfScope p("batched_hull", s); bt_hull<<<c.a.k, kBHullThreads, kBHullSmem, s>>>(c.a); }
    // Sets with more records than one block holds: all together through the
    // bucketed path.
    if (cudaMemsetAsync(c.base + c.L.zero_from, 0, c.L.zero_to - c.L.zero_from, s) != cudaSuccess) return CH_ECUDA;
    launch_batched_large(c.b, redo, c.sms, s);
    return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ECUDA;
}

// One executable graph per (device, stream), updated in place per call.
struct BtGraphKey {
    int dev;
    cudaStream_t s;
    bool operator<(const BtGraphKey& o) const { return dev != o.dev ? dev < o.dev : s < o.s; }
};
static std::mutex g_bgraph_mu;
static std::map<BtGraphKey, cudaGraphExec_t> g_bgraphs;

static int bt_launch_graph(const BtCall& c, unsigned char* redo, int dev, cudaStream_t s) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (prof_enabled() || cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return bt_enqueue(c, redo, s);
    // capture on a stream of this thread's own (kept per device), so that
    // concurrent callers never share a capture
    thread_local std::map<int, cudaStream_t> t_capture;
    cudaStream_t& cs = t_capture[dev];
    if (!cs && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cs = nullptr;
        cudaGetLastError();
        return bt_enqueue(c, redo, s);
    }
    cudaGraph_t graph = nullptr;
    int st = CH_ECUDA;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        st = bt_enqueue(c, redo, cs);
        if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || !graph) st = CH_ECUDA;
    }
    if (st != CH_OK) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return bt_enqueue(c, redo, s);
    }
    std::lock_guard<std::mutex> lk(g_bgraph_mu);
    cudaGraphExec_t& exec = g_bgraphs[BtGraphKey{dev, s}];
    if (exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(exec, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
    }
    if (!exec && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        exec = nullptr;
        cudaGraphDestroy(graph);
        cudaGetLastError();
        return bt_enqueue(c, redo, s);
    }
    cudaGraphDestroy(graph);
    return cudaGraphLaunch(exec, s) == cudaSuccess ? CH_OK : CH_ECUDA;
}

void drop_batched_graphs(int dev, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_bgraph_mu);
    auto it = g_bgraphs.find(BtGraphKey{dev, s});
    if (it == g_bgraphs.end()) return;
    if (it->second) cudaGraphExecDestroy(it->second);
    g_bgraphs.erase(it);
}

static void drop_all_batched_graphs() {
    std::lock_guard<std::mutex> lk(g_bgraph_mu);
    for (auto& kv : g_bgraphs)
        if (kv.second) cudaGraphExecDestroy(kv.second);
    g_bgraphs.clear();
}

static void bt_set_shape(BtCall& c, const BtDevice& d, const std::vector<int64_t>& off, int shape) {
    const BtShape& sh = kBtShapes[shape];
    c.shape = shape;
    c.a.tile = sh.threads * sh.per;
    c.nt = (int)count_tiles(off, c.a.k, c.a.tile);
    c.a.wtile = 32 * sh.per;
    c.a.nwt = (c.a.total - c.a.head) / c.a.wtile;
    c.grid_e = (int)std::max(1ll, std::min(c.a.nwt, (long long)d.sms * d.occ[shape][0]));
    c.grid_f = std::max(1, std::min(c.nt, d.sms * d.occ[shape][1]));
}

// Times every shape on this batch (tile kernels only, best of two runs).
static int bt_tune(BtCall& c, const BtDevice& d, const std::vector<int64_t>& off, cudaStream_t s, int* best) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CH_ECUDA;
    double best_us = 1e30;
    *best = 2;
    int st = CH_OK;
    for (int i = 0; i < kNumBtShapes && st == CH_OK; ++i) {
        bt_set_shape(c, d, off, i);
        double t_min = 1e30;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, s);
            bt_enqueue_tiles(c, s);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                st = CH_ECUDA;
                break;
            }
            t_min = std::min(t_min, 1e3 * ms);
        }
        if (t_min < best_us) {
            best_us = t_min;
            *best = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == CH_OK) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[tune_key(d, off[c.a.k], c.a.k)] = {*best, best_us};
        tune_save_locked();
    }
    return st;
}

// The tuned shape of the nearest size class of this device (by the distance
// of the log2 sizes) when one lies within two steps, else the middle shape;
// for callers that must not block on tuning (the server).
static int nearest_tuned_locked(const BtDevice& d, long long total, int k) {
    const std::string prefix = tune_key(d, 1, 1);
    const std::string dev = prefix.substr(0, prefix.size() - 4);   // drops "|0|0"
    const int lt = ilog2(std::max(1ll, total)), lk = ilog2(std::max(1, k));
    int best = 2, best_d = 1 << 30;
    for (const auto& kv : g_tune) {
        if (kv.first.compare(0, dev.size(), dev) != 0) continue;
        int t = 0, kk = 0;
        if (sscanf(kv.first.c_str() + dev.size(), "|%d|%d", &t, &kk) != 2) continue;
        const int dist = std::abs(t - lt) + std::abs(kk - lk);
        if (dist <= 2 && dist < best_d) {
            best_d = dist;
            best = kv.second.first;
        }
    }
    return best;
}

}  // namespace ch

extern "C" int ch_hull_batched(const float* pts, const int64_t* offsets, int32_t k, int32_t* out_idx,
                               int64_t* out_n, const int64_t* host_offsets, void* stream) {
    return ch::hull_batched_impl(pts, offsets, k, out_idx, out_n, host_offsets, (cudaStream_t)stream, true,
                                 nullptr);
}

namespace ch {

int hull_batched_redo(const float* pts, const int64_t* host_offsets, int32_t k, int32_t* out_idx, int64_t* out_n,
                      const unsigned char* flags, cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
    for (int i = 0; i < k; ++i) {
        if (!flags[i]) continue;
        const int64_t o = host_offsets[i];
        const int st = enqueue_hull_nograph(pts + 2 * o, host_offsets[i + 1] - o, out_idx + o, out_n + i, s, dev);
        if (st != CH_OK) return st;
    }
    return CH_OK;
}

int hull_batched_impl(const float* pts, const int64_t* offsets, int32_t k, int32_t* out_idx, int64_t* out_n,
                      const int64_t* host_offsets, cudaStream_t s, bool allow_tune, unsigned char* redo_host) {
    if (k < 0 || k > (1 << 20)) return CH_EINVAL;
    if (k == 0) return CH_OK;
    if (!offsets || !out_n) return CH_EINVAL;
    const int forced = env_shape();
    if (forced == -2) return CH_EINVAL;
    std::vector<int64_t> off((size_t)k + 1);
    if (host_offsets) {
        for (int i = 0; i <= k; ++i) off[i] = host_offsets[i];
    } else {
        if (cudaMemcpyAsync(off.data(), offsets, sizeof(int64_t) * ((size_t)k + 1), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
            return CH_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return CH_ECUDA;
    }
    if (off[0] != 0) return CH_EINVAL;
    long long big_pts = 0, big_sets = 0;
    for (int i = 0; i < k; ++i) {
        if (off[i + 1] < off[i] || off[i + 1] - off[i] > CH_MAX_POINTS) return CH_EINVAL;
        if (off[i + 1] - off[i] + 12 > kMidCap) {
            big_pts += off[i + 1] - off[i];
            ++big_sets;
        }
    }
    const long long max_tiles = count_tiles(off, k, kBTileMin);   // the most tiles of any shape
    if (max_tiles > INT32_MAX) return CH_EINVAL;
    const int64_t total = off[k];
    int st = check_points_args(pts, total);
    if (st != CH_OK) return st;
    if (total > 0 && !out_idx) return CH_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
    BtDevice d;
    if ((st = bt_configure(dev, &d)) != CH_OK) return st;
    BtCall c;
    if ((st = bt_workspace(dev, s, total, k, big_pts, big_sets, max_tiles, &c.base, &c.L)) != CH_OK) return st;
    const BLayout& L = c.L;
    char* base = c.base;
    c.sms = d.sms;
    BArgs& a = c.a;
    a.pts = pts;
    a.offsets = offsets;
    a.k = k;
    a.ctl = (Ctl*)(base + L.ctl);
    a.keys = (uint32_t*)(base + L.keys);
    a.vals = (uint64_t*)(base + L.vals);
    a.tile_base = (int*)(base + L.tiles);
    a.tile_map = (int*)(base + L.tmap);
    a.out_idx = out_idx;
    a.out_n = out_n;
    a.big = (unsigned char*)(base + L.big);
    a.total = total;
    // the streamed body starts at the first 16-byte boundary (pts is 8-byte aligned)
    a.head = (total > 0 && (reinterpret_cast<uintptr_t>(pts) & 15u) != 0u) ? 1 : 0;
    a.star_ctr = (unsigned*)(base + L.star_ctr);
    a.star_list = (int*)(base + L.star_list);
    a.kP = (uint32_t*)(base + L.kP);
    a.vP = (uint64_t*)(base + L.vP);
    BLArgs& b = c.b;
    b.pts = pts;
    b.offsets = offsets;
    b.k = k;
    b.ctl = a.ctl;
    b.keys = a.keys;
    b.vals = a.vals;
    b.big = a.big;
    b.out_idx = out_idx;
    b.out_n = out_n;
    b.seg_nb = (unsigned*)(base + L.seg_nb);
    b.seg_bbase = (unsigned*)(base + L.seg_bbase);
    b.seg_lo = (int*)(base + L.seg_lo);
    b.seg_scale = (float*)(base + L.seg_scale);
    b.seg_tbase = (unsigned*)(base + L.seg_tbase);
    b.ct_map = (int*)(base + L.ctmap);
    b.rt_base = (unsigned*)(base + L.rt_base);
    b.rt_map = (int*)(base + L.rmap);
    b.totals = (unsigned*)(base + L.totals);
    b.bcount = (unsigned*)(base + L.bcount);
    b.bcur = (unsigned*)(base + L.bcur);
    b.bstart = (unsigned*)(base + L.bstart);
    b.blen = (int*)(base + L.blen);
    b.bu = (int*)(base + L.bu);
    b.bv = (int*)(base + L.bv);
    b.bi = (int*)(base + L.bi);
    b.kP = (uint32_t*)(base + L.kP);
    b.vP = (uint64_t*)(base + L.vP);
    b.cu = (int*)(base + L.cu);
    b.cv = (int*)(base + L.cv);
    b.ci = (int*)(base + L.ci);
    b.clen = (int*)(base + L.clen);
    b.counters = (int*)(base + L.counters);
    b.bcap = L.bcap;
    b.rtcap = L.rtcap;
    b.tcap = L.tcap;
    unsigned char* redo = (unsigned char*)(base + L.redo);
    // tile shape: named by the environment, else tuned for this device and size class
    int shape = forced;
    if (shape < 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        auto it = g_tune.find(tune_key(d, total, k));
        if (it != g_tune.end()) shape = it->second.first;
        else if (!allow_tune) shape = nearest_tuned_locked(d, total, k);
    }
    if (shape < 0 && (st = bt_tune(c, d, off, s, &shape)) != CH_OK) return st;
    bt_set_shape(c, d, off, shape);
    if ((st = bt_launch_graph(c, redo, dev, s)) != CH_OK) return st;
    // Sets the bucketed path could not finish (a bucket chain too long): the
    // single-hull path, one by one, once their flags are on the host.
    if (redo_host)
        return cudaMemcpyAsync(redo_host, redo, (size_t)k, cudaMemcpyDeviceToHost, s) == cudaSuccess ? CH_OK
                                                                                                    : CH_ECUDA;
    std::vector<unsigned char> big((size_t)k);
    if (cudaMemcpyAsync(big.data(), redo, (size_t)k, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CH_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CH_ECUDA;
    return hull_batched_redo(pts, off.data(), k, out_idx, out_n, big.data(), s);
}

}  // namespace ch

using namespace ch;

// Tile shape that ch_hull_batched uses for a batch of this size class on the
// current device: from the environment, else the tuned choice (0 when the
// class has not been tuned yet).
extern "C" int ch_batched_config(int64_t total_points, int32_t k, int32_t* threads, int32_t* per) {
    if (!threads || !per || total_points < 0 || k < 1) return CH_EINVAL;
    int shape = env_shape();
    if (shape == -2) return CH_EINVAL;
    if (shape < 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
        BtDevice d;
        const int st = bt_configure(dev, &d);
        if (st != CH_OK) return st;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        auto it = g_tune.find(tune_key(d, total_points, k));
        if (it == g_tune.end()) {
            *threads = 0;
            *per = 0;
            return CH_OK;
        }
        shape = it->second.first;
    }
    *threads = kBtShapes[shape].threads;
    *per = kBtShapes[shape].per;
    return CH_OK;
}
