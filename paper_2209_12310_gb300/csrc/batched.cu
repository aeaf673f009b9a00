// batched.cu -- k independent hulls packed back to back (ch_hull_batched).
//
// The batch's points are one array; its 16-byte aligned body is cut into
// warp tiles of 32 x P points whatever the sets (P points per lane and the
// block size are one of the compiled shapes that the autotuner picks per
// device and batch size), and every launch covers all sets at once:
//   bt_init, bt_slots  control blocks; a star slot per set of at least
//                kBStarMinPts points;
//   bt_extremes  streamed warp tiles: validation and the 8 extremes of each
//                set (Alg. 2, findExtremes) as packed (key, ~tile) maxima;
//   bt_octagon   one block per set: the lowest index of each extreme (a
//                rescan of its tile), octagon, inner region, chain end-point
//                records; the density test that lists a set for a polygon;
//   bt_star_bin, bt_star_build  the listed sets' angular bins and star
//                polygons (star.cuh; points near a circle, Table V);
//   bt_dense     the filter of the sets with a polygon: runs of their points
//                against the polygon and the octagon, kept points as records;
//   bt_filter    streamed warp tiles of the other sets: the hull-rule
//                classification against the set's octagon, records compacted
//                into the set's region (the loop of Alg. 1/2), support-line
//                end points reduced;
//   bt_hull_small  one block per set: the support-line records, then the
//                hull of a set with few records in a small footprint;
//   bt_star_refine  sets with more records than one block holds: a second
//                polygon from the set's records drops those strictly inside;
//   bt_hull      persistent over the remaining sets: the hull of a set's
//                records in one block (quickhull rounds and the stitch, as in
//                the single hull's last block).
// Sets whose records exceed what one block holds (or are many and near the
// hull) go through the bucketed large-survivor path together
// (batched_large.cu); the rare set it cannot finish (a bucket chain longer
// than kBkChain) is flagged and the host runs the single-hull path on it.
// Each result equals ch_hull on the set alone (local indices).  The device
// work of one call is captured into a CUDA graph on a private stream; the
// executable graph of a (device, stream) is updated in place from call to
// call and launched on the caller's stream.
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

constexpr int kBHullThreads = 512;     // threads of bt_hull (a multiple of 128)
constexpr int kBWarpTileMin = 256;     // points of the smallest warp tile of the compiled shapes
constexpr int kBOctThreads = 256;      // threads of bt_octagon: a warp per direction

// Star polygon of dense sets (star.cuh): a set of at least kBStarMinPts
// points has a slot of angular bins and a polygon.  The bins are taken
// around the centre of the box of the set's extremes, over a sample of
// kBStarParts evenly spread runs of the set (up to kBStarRun points each).
constexpr long long kBStarMinPts = 32768;
constexpr int kBStarParts = 16;
constexpr int kBStarRun = 16384;
constexpr int kBDenseSample = 2048;   // points of a set's density test
static_assert(kBDenseSample <= kBStarMinPts, "the density sample is spread over the set");


struct BArgs {
    const float* pts;
    const int64_t* offsets;   // device, k + 1
    int k;
    Ctl* ctl;                 // k control blocks
    uint32_t* keys;           // records: set i's region starts at offsets[i] + 16 i
    uint64_t* vals;
    int32_t* out_idx;
    int64_t* out_n;
    unsigned char* big;       // k: the set needs the single-hull path
    long long total;          // points of the batch
    long long nwt;            // warp tiles of the streamed body
    int head;                 // points before the body's first 16-byte boundary (0 or 1)
    int wtile;                // points per warp tile (32 x points per lane)
    int* star_slot;           // k: the set's star slot, or -1
    unsigned long long* star_bins;   // kStarBins per slot (zeroed before every batch)
    StarPoly* star_polys;     // one per slot
    unsigned* star_ctr;       // work lists: [0] dense sets listed, [1] taken by bt_star_build;
                              // [2] / [3] sets for bt_star_refine from the front / back, [4] taken;
                              // [5] sets for bt_hull, [6] taken; [7] bt_dense's units, [8] taken
    int* star_list;           // k entries
    unsigned* unit_base;      // k entries: first bt_dense unit of each listed set
    int* refine_list;         // k entries
    int* hull_list;           // k entries
    uint32_t* kP;             // the bucketed path's scatter buffer (set regions as keys / vals)
    uint64_t* vP;
};

__device__ __forceinline__ long long region_base(const BArgs& a, int i) { return a.offsets[i] + 16ll * i; }

// One warp per set: the control block.
__global__ void __launch_bounds__(256) bt_init(BArgs a) {
    const int lane = threadIdx.x & 31;
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= a.k) return;
    Ctl* c = a.ctl + i;
    if (lane < 8) {
        c->ext_packed[lane] = 0ull;
        c->line_ep[lane] = (lane & 1) ? 0ull : ~0ull;
    }
    if (lane < 4) {
        c->counts4[lane] = 2u;   // the two chain end points of every queue
        c->blocks_done[lane] = 0u;
    }
    if (lane == 0) {
        c->status = CH_OK;
        c->abort = 0;
        c->count = 8u;
        c->done = 0;
        c->bk_state = 0;
        c->star_ok = 0;
        c->star_k = 0;
        c->star_cx = 0;
        c->star_cy = 0;
        a.big[i] = 0;
    }
    if (i == 0 && lane < 16) a.star_ctr[lane] = 0u;
}

// Star slots (one block of 1024 threads): the sets of at least kBStarMinPts
// points numbered in set order, -1 for the others.
__global__ void __launch_bounds__(1024) bt_slots(BArgs a) {
    __shared__ int s_part[1024];
    const int tid = threadIdx.x;
    const int per = (a.k + 1023) / 1024;
    const int lo = tid * per, hi = min(a.k, lo + per);
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += (a.offsets[i + 1] - a.offsets[i] >= kBStarMinPts) ? 1 : 0;
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
        const bool has = a.offsets[i + 1] - a.offsets[i] >= kBStarMinPts;
        a.star_slot[i] = has ? run : -1;
        run += has ? 1 : 0;
    }
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
    // A set with a star slot whose sample (kBDenseSample points spread over
    // it) has more than 1 / 16 outside the inner region is dense: bt_star_bin
    // and bt_star_build make its star polygon.
    if (a.star_slot[i] >= 0) {
        __shared__ unsigned s_out;
        if (tid == 0) s_out = 0u;
        __syncthreads();
        const long long step = ni / kBDenseSample;   // >= 1: ni >= kBStarMinPts
        unsigned out = 0u;
        for (int j = tid; j < kBDenseSample; j += kBOctThreads) {
            const float2 p = __ldg(reinterpret_cast<const float2*>(a.pts) + base + j * step);
            out += in_inner(s_o, __float2int_rn(p.x), __float2int_rn(p.y)) ? 0u : 1u;
        }
        out = __reduce_add_sync(0xFFFFFFFFu, out);
        if (lane == 0 && out) atomicAdd(&s_out, out);
        __syncthreads();
        if (tid == 0 && s_out * 16u > (unsigned)kBDenseSample) {
            c->star_ok = 1;
            c->star_cx = (s_vx[W] + s_vx[E]) / 2;   // the centre of the extremes' box
            c->star_cy = (s_vy[S] + s_vy[N]) / 2;
            a.star_list[atomicAdd(&a.star_ctr[0], 1u)] = i;
        }
    }
}

// ---------------------------------------------------------------------------
// The filter of the sets without a star polygon, streamed (the loop of
// Alg. 1/2): the warp tiles and block chunks of bt_extremes.  A warp keeps
// the octagon of its current set in shared memory.  Per point: the octagon's
// inner region drops it (a whole lane's points at once when their key
// extremes lie in the region); the points it leaves wait in a per-warp queue
// and go 32 at a time through the hull-rule classification, and the kept
// ones become records of their queue, staged per warp and written to the
// set's region with one atomic per batch.  Survivors on a support line of
// the octagon reduce to the lines' end points (reduce_on_line).  The sets
// with a star polygon are bt_dense's: their tiles are streamed and skipped.
constexpr int kBtWarpRecs = 128;
constexpr int kBtQueue = 64;   // < 32 waiting + 32 added per step
struct BtWarpSmem {
    Octagon o;                       // the warp's set's octagon
    uint64_t val[kBtWarpRecs];       // records staged
    uint32_t key[kBtWarpRecs];
    float qx[kBtQueue], qy[kBtQueue];   // points waiting for the exact tests
    unsigned qi[kBtQueue];
    unsigned char lanes[32];         // lanes whose tile the inner region did not settle
    Ctl* c;                          // the warp's set: control block, record region,
    long long rb;
    unsigned cnt;                    // records staged,
    unsigned nq[4];                  // records per queue
};

// A warp's current set: what the streaming loop reads stays in registers
// (warp-uniform); what the classification needs is in the warp's shared
// memory.
struct BtWarpSet {
    int set = -1;
    long long base = 0;
    bool skip = true;              // empty, failed, or bt_dense's: nothing to classify
    unsigned qn = 0u;              // points queued
};

__device__ __forceinline__ void bt_flush_recs(BtWarpSmem& m, uint32_t* keys, uint64_t* vals) {
    const int lane = threadIdx.x & 31;
    const unsigned cnt = m.cnt;
    if (cnt == 0u) return;
    unsigned base = 0u;
    if (lane == 0) base = atomicAdd(&m.c->count, cnt);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (unsigned j = lane; j < cnt; j += 32) {
        keys[m.rb + base + j] = m.key[j];
        vals[m.rb + base + j] = m.val[j];
    }
    __syncwarp();
    if (lane == 0) m.cnt = 0u;
    __syncwarp();
}

// Warp-collective, out of line: one point per lane of the warp's set (valid
// = false for none), local index li.  The hull-rule classification, the
// support-line reduction and the staging of the kept records.
__device__ __noinline__ void bt_classify32(uint32_t* keys, uint64_t* vals, BtWarpSmem& m, bool valid, float x,
                                           float y, unsigned li) {
    const int lane = threadIdx.x & 31;
    const Octagon& so = m.o;
    int r = -1, X = 0, Y = 0;
    if (valid) {
        X = __float2int_rn(x);
        Y = __float2int_rn(y);
        r = classify_hull(x, y, so);
    }
    bool keep = r >= 0;
    if (!__any_sync(0xFFFFFFFFu, keep)) return;
    if (reduce_on_line(so, keep, X, Y, li, m.c)) keep = false;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
    if (!bal) return;
    unsigned nq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) nq[q] = (unsigned)__popc(__ballot_sync(0xFFFFFFFFu, keep && r == q));
    if (m.cnt + (unsigned)__popc(bal) > (unsigned)kBtWarpRecs) bt_flush_recs(m, keys, vals);
    const unsigned cnt = m.cnt;
    if (keep) {
        uint32_t u, v;
        queue_frame(r, X, Y, u, v);
        const unsigned pos = cnt + (unsigned)__popc(bal & lanemask_lt());
        m.key[pos] = make_key(r, u);
        m.val[pos] = make_val(v, li);
    }
    __syncwarp();
    if (lane == 0) {
        m.cnt = cnt + (unsigned)__popc(bal);
#pragma unroll
        for (int q = 0; q < 4; ++q) m.nq[q] += nq[q];
    }
    __syncwarp();
}

// Warp-collective: queues the lanes' points with need = true; full rounds of
// 32 go through bt_classify32.
__device__ __forceinline__ void bt_queue_push(const BArgs& a, BtWarpSet& w, BtWarpSmem& m, bool need, float x, float y,
                                              unsigned li) {
    const int lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, need);
    if (!bal) return;
    if (need) {
        const unsigned pos = w.qn + (unsigned)__popc(bal & lanemask_lt());
        m.qx[pos] = x;
        m.qy[pos] = y;
        m.qi[pos] = li;
    }
    w.qn += (unsigned)__popc(bal);
    __syncwarp();
    while (w.qn >= 32u) {
        w.qn -= 32u;
        const float qx = m.qx[w.qn + lane], qy = m.qy[w.qn + lane];
        const unsigned qi = m.qi[w.qn + lane];
        __syncwarp();
        bt_classify32(a.keys, a.vals, m, true, qx, qy, qi);
    }
}

// Warp-collective: finishes the warp's set (queue, records, queue counts).
__device__ __forceinline__ void bt_warp_done(const BArgs& a, BtWarpSmem& m, BtWarpSet& w) {
    const int lane = threadIdx.x & 31;
    if (w.set < 0) return;
    if (w.qn) {
        const bool valid = (unsigned)lane < w.qn;
        const float qx = valid ? m.qx[lane] : 0.0f, qy = valid ? m.qy[lane] : 0.0f;
        const unsigned qi = valid ? m.qi[lane] : 0u;
        __syncwarp();
        w.qn = 0u;
        bt_classify32(a.keys, a.vals, m, valid, qx, qy, qi);
    }
    bt_flush_recs(m, a.keys, a.vals);
    if (lane < 4 && m.nq[lane]) atomicAdd(&m.c->counts4[lane], m.nq[lane]);
    w.set = -1;
}

// Warp-collective: makes set q the warp's set (the previous one finished).
__device__ __forceinline__ void bt_warp_set(const BArgs& a, int q, BtWarpSet& w, BtWarpSmem& m) {
    const int lane = threadIdx.x & 31;
    bt_warp_done(a, m, w);
    __syncwarp();
    Ctl* c = a.ctl + q;
    w.set = q;
    w.base = a.offsets[q];
    const int slot = a.star_slot[q];
    // empty and failed sets (bt_octagon's verdict), and the sets with a star
    // polygon, which bt_dense filters
    w.skip = *(volatile int*)&c->done != 0 || (slot >= 0 && c->star_k > 0);
    if (lane == 0) {
        m.c = c;
        m.rb = region_base(a, q);
        m.cnt = 0u;
    }
    if (lane < 4) m.nq[lane] = 0u;
    if (!w.skip) {
        const int* src = reinterpret_cast<const int*>(&c->oct);
        int* dst = reinterpret_cast<int*>(&m.o);
        for (int j = lane; j < (int)(sizeof(Octagon) / 4); j += 32) dst[j] = src[j];
    }
    __syncwarp();
}

// Points [lo, hi) of the batch read from global memory, set by set from the
// set holding lo (head and tail).
__device__ void bt_filter_global(const BArgs& a, long long lo, long long hi, BtWarpSet& w, BtWarpSmem& m) {
    const int lane = threadIdx.x & 31;
    if (lo >= hi) return;
    for (int q = bt_find_set(a, lo); q < a.k; ++q) {
        const long long qb = a.offsets[q], qe = a.offsets[q + 1];
        if (qb >= hi) break;
        if (qe <= lo) continue;
        bt_warp_set(a, q, w, m);
        if (w.skip) continue;
        const long long e = min(hi, qe);
        for (long long j0 = max(lo, qb); j0 < e; j0 += 32) {
            const long long j = j0 + lane;
            const bool valid = j < e;
            const float2 p = valid ? reinterpret_cast<const float2*>(a.pts)[j] : make_float2(0.0f, 0.0f);
            bt_classify32(a.keys, a.vals, m, valid, p.x, p.y, (unsigned)(j - qb));
        }
    }
}

template <int T, int P>
__global__ void __launch_bounds__(T, 1) bt_filter(BArgs a) {
    constexpr int kWarps = T / 32, kF4 = 16 * P;
    constexpr long long kPts = 32ll * P;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ unsigned long long s_bar[kWarps][kStages];
    __shared__ BtWarpSmem s_w[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BtWarpSmem& m = s_w[warp];
    BtWarpSet w;
    const long long nwt = a.nwt;
    const long long per = (nwt + gridDim.x - 1) / gridDim.x;
    const long long c0 = min(nwt, (long long)blockIdx.x * per), c1 = min(nwt, c0 + per);
    if (blockIdx.x == 0 && warp == 0) {
        bt_filter_global(a, 0, a.head, w, m);
        bt_filter_global(a, a.head + nwt * kPts, a.total, w, m);
    }
    if (c0 + warp < c1) {
        WarpStreamT<kF4> ws{reinterpret_cast<float4*>(dsm) + warp * kStages * kF4, s_bar[warp],
                            reinterpret_cast<const float4*>(a.pts + 2 * a.head), c0 + warp, kWarps, c1, lane};
        int s = bt_find_set(a, a.head + (c0 + warp) * kPts);
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
                for (int q = s + lane; q < a.k && __ldg(a.offsets + q) < pend; q += 32)
                    set_status(a.ctl + q, CH_ETIMEOUT);
                break;
            }
            const float2* cur2 = reinterpret_cast<const float2*>(cur);
            if (__ldg(a.offsets + s + 1) >= p0 + kPts) {   // inside set s
                if (s != w.set) bt_warp_set(a, s, w, m);
                if (!w.skip) {
                    const Octagon& so = m.o;
                    int tk[8];
#pragma unroll
                    for (int j = 0; j < P / 2; ++j) {
                        const float4 v = cur[j * 32 + lane];
                        tile_keys2(tk, __float2int_rn(v.x), __float2int_rn(v.y), __float2int_rn(v.z),
                                   __float2int_rn(v.w), j == 0);
                    }
                    const bool inside = tk[W] >= so.in_lo[0] && tk[E] <= so.in_hi[0] && tk[S] >= so.in_lo[1] &&
                                        tk[N] <= so.in_hi[1] && tk[SW] >= so.in_lo[2] && tk[NE] <= so.in_hi[2] &&
                                        tk[NW] >= so.in_lo[3] && tk[SE] <= so.in_hi[3];
                    // The points of the lanes whose tile failed are spread over
                    // the warp, 32 at a time (slot s: failing lane of rank
                    // s / P, its point s % P, in float4 (s % P) / 2, half s % 2).
                    // A point outside the inner region waits for the
                    // classification.
                    const unsigned fail = __ballot_sync(0xFFFFFFFFu, !inside);
                    if (fail) {
                        if (!inside) m.lanes[__popc(fail & lanemask_lt())] = (unsigned char)lane;
                        __syncwarp();
                        const unsigned slots = (unsigned)P * (unsigned)__popc(fail);
#pragma unroll 1
                        for (unsigned s0 = 0; s0 < slots; s0 += 32u) {
                            const unsigned sl = s0 + (unsigned)lane;
                            bool need = false;
                            float x = 0.0f, y = 0.0f;
                            unsigned li = 0u;
                            if (sl < slots) {
                                const int ln = m.lanes[sl / P], j = (int)(sl % P);
                                const int f2 = 2 * ((j >> 1) * 32 + ln) + (j & 1);
                                const float2 p = cur2[f2];
                                x = p.x;
                                y = p.y;
                                li = (unsigned)(p0 - w.base) + (unsigned)f2;
                                need = !in_inner(so, __float2int_rn(x), __float2int_rn(y));
                            }
                            bt_queue_push(a, w, m, need, x, y, li);
                        }
                        __syncwarp();
                    }
                }
            } else {   // the tile meets a set boundary: set by set
                for (int q = s; q < a.k; ++q) {
                    const long long qb = __ldg(a.offsets + q), qe = __ldg(a.offsets + q + 1);
                    if (qb >= p0 + kPts) break;
                    if (qe <= p0) continue;
                    if (q != w.set) bt_warp_set(a, q, w, m);
                    if (w.skip) continue;
#pragma unroll 1
                    for (int j = 0; j < P; ++j) {
                        const long long i = p0 + 2 * ((j >> 1) * 32 + lane) + (j & 1);
                        const float2 p = cur2[2 * ((j >> 1) * 32 + lane) + (j & 1)];
                        bt_classify32(a.keys, a.vals, m, i >= qb && i < qe, p.x, p.y, (unsigned)(i - qb));
                    }
                }
            }
            ws.release(k);
        }
    }
    bt_warp_done(a, m, w);
}

// ---------------------------------------------------------------------------
// Bins of the dense sets (bt_octagon's list).  Chunk ch of the work is run
// ch % kBStarParts of listed set ch / kBStarParts: the points
// [base + part * (n / kBStarParts), + min(n / kBStarParts, kBStarRun)).
// Every point outside the octagon's inner region goes to its angular bin
// around the set's centre, where a 64-bit atomicMax keeps the point farthest
// from the centre, packed (squared distance >> 17, local index); a point
// reads its bin first and issues the atomic only when it beats it.
constexpr int kBStarBinThreads = 256;
constexpr int kBStarBinU = 8;   // points per thread in flight

__global__ void __launch_bounds__(kBStarBinThreads) bt_star_bin(BArgs a) {
    const int tid = threadIdx.x;
    const unsigned nchunks = a.star_ctr[0] * (unsigned)kBStarParts;
    for (unsigned ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int i = a.star_list[ch / kBStarParts];
        const int part = (int)(ch % kBStarParts);
        const Ctl* c = a.ctl + i;
        const long long base = a.offsets[i], ni = a.offsets[i + 1] - base;
        const long long step = ni / kBStarParts;
        const long long lo = (long long)part * step;   // local index of the run
        const int len = (int)min(step, (long long)kBStarRun);
        const int cx = c->star_cx, cy = c->star_cy;
        const int xl = c->oct.in_lo[0], yl = c->oct.in_lo[1], sl = c->oct.in_lo[2], dl = c->oct.in_lo[3];
        const int xh = c->oct.in_hi[0], yh = c->oct.in_hi[1], sh = c->oct.in_hi[2], dh = c->oct.in_hi[3];
        unsigned long long* bins = a.star_bins + (size_t)a.star_slot[i] * kStarBins;
        const float2* p2 = reinterpret_cast<const float2*>(a.pts) + base + lo;
        for (int j0 = 0; j0 < len; j0 += kBStarBinThreads * kBStarBinU) {
            float2 p[kBStarBinU];
#pragma unroll
            for (int u = 0; u < kBStarBinU; ++u) {
                const int j = j0 + u * kBStarBinThreads + tid;
                p[u] = j < len ? __ldcs(p2 + j) : make_float2(-1.0f, -1.0f);
            }
            unsigned long long key[kBStarBinU];
            int bin[kBStarBinU];
#pragma unroll
            for (int u = 0; u < kBStarBinU; ++u) {
                const int X = __float2int_rn(p[u].x), Y = __float2int_rn(p[u].y);
                const int S = X + Y, D = X - Y + kCoordLimit;
                const bool inner = X >= xl && X <= xh && Y >= yl && Y <= yh && S >= sl && S <= sh && D >= dl && D <= dh;
                const bool ok = ((unsigned)(X | Y) >> kCoordBits) == 0u && !inner;   // the set's points are valid
                const int dx = X - cx, dy = Y - cy;
                const unsigned long long d2 = (unsigned long long)((long long)dx * dx + (long long)dy * dy);
                const long long li = lo + j0 + u * kBStarBinThreads + tid;
                key[u] = ok ? ((d2 >> 17) << 32) | (unsigned long long)li : 0ull;
                bin[u] = star_bin(dx, dy);
            }
            unsigned long long cur[kBStarBinU];
#pragma unroll
            for (int u = 0; u < kBStarBinU; ++u) cur[u] = key[u] ? __ldcg(bins + bin[u]) : ~0ull;
#pragma unroll
            for (int u = 0; u < kBStarBinU; ++u)
                if (key[u] > cur[u]) atomicMax(&bins[bin[u]], key[u]);
        }
    }
}

// ---------------------------------------------------------------------------
// Star polygons of the dense sets (bt_octagon's list), one block per set,
// persistent over the list: the polygon of the set's bins (star_finish,
// star.cuh: vertices re-read from the input by index, checked exactly) is
// built in shared memory and copied to the set's slot, for bt_filter.  A
// set without one keeps star_k = 0 and is filtered by its octagon alone.
constexpr int kBStarThreads = 512;
constexpr size_t kBStarAOff = (sizeof(StarPoly) + 15) / 16 * 16;
constexpr size_t kBStarSmem = kBStarAOff + (sizeof(int2) + sizeof(unsigned short)) * kStarBins;
static_assert(sizeof(StarPoly) % 16 == 0, "the polygon is copied in 16-byte words");

__global__ void __launch_bounds__(kBStarThreads, 1) bt_star_build(BArgs a) {
    extern __shared__ __align__(16) char dyn[];
    StarPoly& P = *reinterpret_cast<StarPoly*>(dyn);
    int2* va = reinterpret_cast<int2*>(dyn + kBStarAOff);
    unsigned short* ba = reinterpret_cast<unsigned short*>(dyn + kBStarAOff + sizeof(int2) * kStarBins);
    __shared__ int s_set;
    const int tid = threadIdx.x;
    const unsigned listed = a.star_ctr[0];
    for (;;) {
        if (tid == 0) {
            const unsigned g = atomicAdd(&a.star_ctr[1], 1u);
            s_set = g < listed ? a.star_list[g] : -1;
        }
        __syncthreads();
        const int i = s_set;
        if (i < 0) return;
        Ctl* c = a.ctl + i;
        const long long base = a.offsets[i], ni = a.offsets[i + 1] - base;
        const int slot = a.star_slot[i];
        const int K = star_finish<kBStarThreads>(a.star_bins + (size_t)slot * kStarBins, a.pts + 2 * base, ni,
                                                 c->star_cx, c->star_cy, va, ba, P, c);
        if (K) {
            const int4* src = reinterpret_cast<const int4*>(&P);
            int4* dst = reinterpret_cast<int4*>(a.star_polys + slot);
            for (int j = tid; j < (int)(sizeof(StarPoly) / 16); j += kBStarThreads) dst[j] = src[j];
        }
        if (tid == 0) c->star_k = K;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// The filter of the sets with a star polygon (bt_star_build's), which
// bt_filter leaves to this kernel: the single hull's dense post pass per
// set.  Work units are runs of up to kBDenseRun points of a set
// (bt_dense_plan numbers them); a block takes units one at a time, copies the
// set's polygon (all of it, 112 KB, mostly from L2) and octagon into shared
// memory, and streams the run's points with the loads of its next step in
// flight: a point closer to the centre than the polygon's inscribed radius,
// or than its bin's radius bound, is strictly inside the polygon; the others
// wait in a per-warp queue and go 32 at a time through the exact wedge test
// and the hull-rule classification; kept points become records of their
// queue, staged per warp and written to the set's region with one atomic per
// batch.
constexpr int kBDenseThreads = 512;
constexpr int kBDenseRun = 1 << 18;    // points of a work unit
constexpr int kBDenseU = 8;            // points per thread and step
constexpr int kBDenseRecs = 256;       // records staged per warp
constexpr int kBDenseQueue = 32 * kBDenseU + 32;   // < 32 waiting + a step's points
struct BtDenseWarp {
    uint64_t val[kBDenseRecs];
    uint32_t key[kBDenseRecs];
    float qx[kBDenseQueue], qy[kBDenseQueue];
    unsigned qi[kBDenseQueue];
};
constexpr size_t kBDenseWarpOff = (sizeof(StarPoly) + sizeof(Octagon) + 15) / 16 * 16;
constexpr size_t kBDenseSmem = kBDenseWarpOff + (kBDenseThreads / 32) * sizeof(BtDenseWarp);
static_assert(kBDenseSmem <= 227 * 1024, "one block's shared memory");

// Work units of the sets with a polygon: unit_base[j] = first unit of listed
// set j (one block of 1024 threads; star_ctr[7] = total units).
__global__ void __launch_bounds__(1024) bt_dense_plan(BArgs a) {
    __shared__ unsigned s_part[1024];
    const int tid = threadIdx.x;
    const int n = (int)a.star_ctr[0];
    const int per = (n + 1023) / 1024;
    const int lo = tid * per, hi = min(n, lo + per);
    unsigned sum = 0u;
    for (int j = lo; j < hi; ++j) {
        const int i = a.star_list[j];
        const long long ni = a.offsets[i + 1] - a.offsets[i];
        sum += a.ctl[i].star_k > 0 ? (unsigned)((ni + kBDenseRun - 1) / kBDenseRun) : 0u;
    }
    s_part[tid] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const unsigned v = tid >= o ? s_part[tid - o] : 0u;
        __syncthreads();
        s_part[tid] += v;
        __syncthreads();
    }
    unsigned run = s_part[tid] - sum;
    for (int j = lo; j < hi; ++j) {
        const int i = a.star_list[j];
        const long long ni = a.offsets[i + 1] - a.offsets[i];
        a.unit_base[j] = run;
        run += a.ctl[i].star_k > 0 ? (unsigned)((ni + kBDenseRun - 1) / kBDenseRun) : 0u;
    }
    if (tid == 1023) a.star_ctr[7] = s_part[1023];
}

// Warp-collective: the exact tests of one queued point per lane (valid =
// false for none) and the staging of the kept ones.
__device__ __forceinline__ void bt_dense_exact(const BArgs& a, const StarPoly& P, const Octagon& so, Ctl* c,
                                               long long rb, int cx, int cy, BtDenseWarp& wb, unsigned& cnt,
                                               unsigned (&nq)[4], bool valid, float x, float y, unsigned li) {
    const int lane = threadIdx.x & 31;
    int r = -1, X = 0, Y = 0;
    if (valid) {
        X = __float2int_rn(x);
        Y = __float2int_rn(y);
        const int px = X - cx, py = Y - cy;
        if (!star_inside_exact(px, py, star_bin(px, py), P)) r = classify_hull(x, y, so);
    }
    bool keep = r >= 0;
    if (!__any_sync(0xFFFFFFFFu, keep)) return;
    if (reduce_on_line(so, keep, X, Y, li, c)) keep = false;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
    if (!bal) return;
#pragma unroll
    for (int q = 0; q < 4; ++q) nq[q] += (unsigned)__popc(__ballot_sync(0xFFFFFFFFu, keep && r == q));
    if (cnt + (unsigned)__popc(bal) > (unsigned)kBDenseRecs) {   // write the staged records out
        unsigned base = 0u;
        if (lane == 0) base = atomicAdd(&c->count, cnt);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        for (unsigned j = lane; j < cnt; j += 32) {
            a.keys[rb + base + j] = wb.key[j];
            a.vals[rb + base + j] = wb.val[j];
        }
        __syncwarp();
        cnt = 0u;
    }
    if (keep) {
        uint32_t u, v;
        queue_frame(r, X, Y, u, v);
        const unsigned pos = cnt + (unsigned)__popc(bal & lanemask_lt());
        wb.key[pos] = make_key(r, u);
        wb.val[pos] = make_val(v, li);
    }
    cnt += (unsigned)__popc(bal);
    __syncwarp();
}

__global__ void __launch_bounds__(kBDenseThreads, 1) bt_dense(BArgs a) {
    extern __shared__ __align__(16) char dyn[];
    StarPoly& P = *reinterpret_cast<StarPoly*>(dyn);
    Octagon& so = *reinterpret_cast<Octagon*>(dyn + sizeof(StarPoly));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    BtDenseWarp& wb = reinterpret_cast<BtDenseWarp*>(dyn + kBDenseWarpOff)[warp];
    constexpr int kStep = kBDenseThreads * kBDenseU;
    __shared__ int s_set, s_part;
    const unsigned nunits = a.star_ctr[7];
    const int listed = (int)a.star_ctr[0];
    for (;;) {
        if (tid == 0) {
            const unsigned u = atomicAdd(&a.star_ctr[8], 1u);
            int set = -1, part = 0;
            if (u < nunits) {   // the last listed set whose first unit is at or before u
                int l = 0, r = listed;
                while (r - l > 1) {
                    const int mid = (l + r) >> 1;
                    if (a.unit_base[mid] <= u) l = mid;
                    else r = mid;
                }
                set = a.star_list[l];
                part = (int)(u - a.unit_base[l]);
            }
            s_set = set;
            s_part = part;
        }
        __syncthreads();
        const int i = s_set;
        if (i < 0) return;
        Ctl* c = a.ctl + i;
        const long long base = a.offsets[i], ni = a.offsets[i + 1] - base;
        const long long rb = region_base(a, i);
        const long long lo = (long long)s_part * kBDenseRun, hi = min(ni, lo + kBDenseRun);
        {   // the polygon and the octagon into shared memory
            const int4* src = reinterpret_cast<const int4*>(a.star_polys + a.star_slot[i]);
            int4* dst = reinterpret_cast<int4*>(&P);
            for (int j = tid; j < (int)(sizeof(StarPoly) / 16); j += kBDenseThreads) dst[j] = __ldcg(src + j);
            copy_octagon(&so, &c->oct);
        }
        __syncthreads();
        const int cx = c->star_cx, cy = c->star_cy;
        const long long r0 = P.rmin;
        const float2* p2 = reinterpret_cast<const float2*>(a.pts) + base;
        unsigned cnt = 0u, qn = 0u;
        unsigned nq[4] = {0u, 0u, 0u, 0u};
        float2 cur[kBDenseU];
#pragma unroll
        for (int u = 0; u < kBDenseU; ++u) {
            const long long j = lo + u * kBDenseThreads + tid;
            cur[u] = j < hi ? __ldcs(p2 + j) : make_float2(0.0f, 0.0f);
        }
        for (long long s0 = lo; s0 < hi; s0 += kStep) {
            float2 nxt[kBDenseU];
#pragma unroll
            for (int u = 0; u < kBDenseU; ++u) {
                const long long j = s0 + kStep + u * kBDenseThreads + tid;
                nxt[u] = j < hi ? __ldcs(p2 + j) : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int u = 0; u < kBDenseU; ++u) {
                const long long j = s0 + u * kBDenseThreads + tid;
                bool need = false;
                if (j < hi) {
                    const long long px = __float2int_rn(cur[u].x) - cx, py = __float2int_rn(cur[u].y) - cy;
                    const long long d2 = px * px + py * py;
                    if (d2 >= r0 * r0) {
                        const long long rr = P.rin[star_bin((int)px, (int)py)];
                        need = d2 >= rr * rr;
                    }
                }
                const unsigned bal = __ballot_sync(0xFFFFFFFFu, need);
                if (need) {   // queued
                    const unsigned pos = qn + (unsigned)__popc(bal & lanemask_lt());
                    wb.qx[pos] = cur[u].x;
                    wb.qy[pos] = cur[u].y;
                    wb.qi[pos] = (unsigned)j;
                }
                qn += (unsigned)__popc(bal);
            }
            __syncwarp();
            while (qn >= 32u) {   // full rounds of 32 through the exact tests
                qn -= 32u;
                const float qx = wb.qx[qn + lane], qy = wb.qy[qn + lane];
                const unsigned qi = wb.qi[qn + lane];
                __syncwarp();
                bt_dense_exact(a, P, so, c, rb, cx, cy, wb, cnt, nq, true, qx, qy, qi);
            }
#pragma unroll
            for (int u = 0; u < kBDenseU; ++u) cur[u] = nxt[u];
        }
        if (qn) {   // the queue's remainder
            const bool valid = (unsigned)lane < qn;
            const float qx = valid ? wb.qx[lane] : 0.0f, qy = valid ? wb.qy[lane] : 0.0f;
            const unsigned qi = valid ? wb.qi[lane] : 0u;
            __syncwarp();
            bt_dense_exact(a, P, so, c, rb, cx, cy, wb, cnt, nq, valid, qx, qy, qi);
        }
        if (cnt) {
            unsigned b0 = 0u;
            if (lane == 0) b0 = atomicAdd(&c->count, cnt);
            b0 = __shfl_sync(0xFFFFFFFFu, b0, 0);
            for (unsigned j = lane; j < cnt; j += 32) {
                a.keys[rb + b0 + j] = wb.key[j];
                a.vals[rb + b0 + j] = wb.val[j];
            }
        }
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (nq[q]) atomicAdd(&c->counts4[q], nq[q]);
        __syncthreads();   // the polygon's shared memory is reloaded by the next unit
    }
}

// ---------------------------------------------------------------------------
// Second star polygon of a set whose records one block still cannot hold
// (bt_hull_small's list): its records are the points outside the first
// polygon (or, for a sparse set, outside the octagon), so binning all of
// them puts a rim point in nearly every bin.  One block per set, persistent
// over the list (the sets with more than kBRefineHuge records first):
//   1. bins of all the set's records in shared memory, around the centre of
//      the octagon's box (each bin keeps its point farthest from it);
//   2. the polygon (star_finish: vertices re-read from the input by index,
//      checked exactly); without one the set is left as it is;
//   3. the records whose point is not strictly inside it are copied to the
//      set's region of the scatter buffer (free until the bucketed path),
//      then back, and the per-queue counts are recounted.
// Each warp streams a contiguous range of the records with the loads of its
// next step in flight while it works on the current one.
constexpr int kBRefineU = 8;                    // records per lane and step
constexpr unsigned kBRefineHuge = 1u << 16;     // records of the sets taken first
static_assert(sizeof(unsigned long long) * kStarBins <= (sizeof(int2) + sizeof(unsigned short)) * kStarBins,
              "the bins fit in work area A");

// One step of a warp: records [r, r + 32 kBRefineU) of a range ending at hi,
// record r + 32 u + lane in slot u.
__device__ __forceinline__ void bt_refine_load(const uint32_t* __restrict__ keys, const uint64_t* __restrict__ vals,
                                               long long rb, unsigned r, unsigned hi, uint32_t (&kk)[kBRefineU],
                                               uint64_t (&vv)[kBRefineU]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int u = 0; u < kBRefineU; ++u) {
        const unsigned j = r + 32u * u + lane;
        kk[u] = j < hi ? __ldcg(keys + rb + j) : 0u;
        vv[u] = j < hi ? __ldcg(vals + rb + j) : 0ull;
    }
}

__device__ __forceinline__ void bt_record_xy(uint32_t k, uint64_t v, int& X, int& Y) {
    frame_to_xy((int)(k >> kKeyBits), (int)(k & kKeyMask), (int)(v >> 31), X, Y);
}

__global__ void __launch_bounds__(kBStarThreads, 1) bt_star_refine(BArgs a) {
    extern __shared__ __align__(16) char dyn[];
    StarPoly& P = *reinterpret_cast<StarPoly*>(dyn);
    unsigned long long* bins = reinterpret_cast<unsigned long long*>(dyn + kBStarAOff);
    int2* va = reinterpret_cast<int2*>(dyn + kBStarAOff);
    unsigned short* ba = reinterpret_cast<unsigned short*>(dyn + kBStarAOff + sizeof(int2) * kStarBins);
    constexpr int kWarps = kBStarThreads / 32;
    constexpr unsigned kStep = 32u * kBRefineU;
    __shared__ unsigned s_kept, s_q[4];
    __shared__ int s_set, s_cx, s_cy;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned n_front = a.star_ctr[2], n_back = a.star_ctr[3];
    for (;;) {
        if (tid == 0) {
            const unsigned g = atomicAdd(&a.star_ctr[4], 1u);
            s_set = g < n_front ? a.refine_list[g]
                                : (g - n_front < n_back ? a.refine_list[a.k - 1 - (int)(g - n_front)] : -1);
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
        const unsigned per = ((m + kWarps - 1) / kWarps + kStep - 1) / kStep * kStep;
        const unsigned lo = min(m, warp * per), hi = min(m, lo + per);
        {   // 1. bins
            uint32_t kk[kBRefineU];
            uint64_t vv[kBRefineU];
            bt_refine_load(a.keys, a.vals, rb, lo, hi, kk, vv);
            for (unsigned r = lo; r < hi; r += kStep) {
                uint32_t nk[kBRefineU];
                uint64_t nv[kBRefineU];
                bt_refine_load(a.keys, a.vals, rb, r + kStep, hi, nk, nv);
#pragma unroll
                for (int u = 0; u < kBRefineU; ++u) {
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
                for (int u = 0; u < kBRefineU; ++u) {
                    kk[u] = nk[u];
                    vv[u] = nv[u];
                }
            }
        }
        __syncthreads();
        // 2. the polygon
        const int K = star_finish<kBStarThreads, true>(bins, a.pts + 2 * base, ni, cx, cy, va, ba, P, c);
        if (K == 0) {
            __syncthreads();
            continue;
        }
        // 3. the records not strictly inside go to the scatter buffer, then back
        unsigned t0 = 0u, t1 = 0u, t2 = 0u, t3 = 0u;   // kept per queue (lane counts)
        {
            uint32_t kk[kBRefineU];
            uint64_t vv[kBRefineU];
            bt_refine_load(a.keys, a.vals, rb, lo, hi, kk, vv);
            for (unsigned r = lo; r < hi; r += kStep) {
                uint32_t nk[kBRefineU];
                uint64_t nv[kBRefineU];
                bt_refine_load(a.keys, a.vals, rb, r + kStep, hi, nk, nv);
#pragma unroll
                for (int u = 0; u < kBRefineU; ++u) {
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
                for (int u = 0; u < kBRefineU; ++u) {
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
        const unsigned kept = s_kept;
        for (unsigned j = tid; j < kept; j += kBStarThreads) {
            a.keys[rb + j] = __ldcg(a.kP + rb + j);
            a.vals[rb + j] = __ldcg(a.vP + rb + j);
        }
        if (tid < 4) c->counts4[tid] = s_q[tid];
        if (tid == 0) {
            c->count = kept;
            c->star_k = K;
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
    if (tid == 0) {
        s_done = *(volatile int*)&c->done;
        // a filter pass that gave up on a copy (CH_ETIMEOUT) left the set's
        // records incomplete: report the status, compute nothing
        const int st = read_status(c);
        if (!s_done && st != CH_OK) {
            a.out_n[i] = st;
            c->done = 1;
            s_done = 1;
        }
    }
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
    if (total > (unsigned)kBSmallRec) {   // bt_hull's, after bt_star_refine's when one block cannot hold them
        if (tid == 0) {
            a.hull_list[atomicAdd(&a.star_ctr[5], 1u)] = i;
            if (total > (unsigned)kMidCap) {
                if (total > kBRefineHuge) a.refine_list[atomicAdd(&a.star_ctr[2], 1u)] = i;
                else a.refine_list[a.k - 1 - (int)atomicAdd(&a.star_ctr[3], 1u)] = i;
            }
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

constexpr size_t bt_cmax(size_t x, size_t y) { return x > y ? x : y; }
constexpr int kBQhSkip = 2048;
constexpr size_t kBHullSmem = bt_cmax(kMidSmemBytes, sizeof(QhSmem));

// Persistent over bt_hull_small's list of the sets with more records than
// its small footprint holds (one block per set at a time).
__global__ void __launch_bounds__(kBHullThreads, 1) bt_hull(BArgs a) {
    extern __shared__ __align__(16) char dyn[];
    __shared__ int s_set, s_mv;
    const int tid = threadIdx.x;
    const unsigned listed = a.star_ctr[5];
    for (;;) {
        if (tid == 0) {
            const unsigned g = atomicAdd(&a.star_ctr[6], 1u);
            s_set = g < listed ? a.hull_list[g] : -1;
        }
        __syncthreads();
        const int i = s_set;
        if (i < 0) return;
        Ctl* c = a.ctl + i;
        const unsigned total = *(volatile unsigned*)&c->count;   // with the line records
        const long long rb = region_base(a, i);
        const long long base = a.offsets[i], ni = a.offsets[i + 1] - base;
        // More than one block holds, or past kBQhSkip records that are near
        // the hull (a star polygon left them, or more than a quarter of the
        // points survived the octagon), whose chains would outgrow the
        // quickhull rounds' vertex capacity (kQhCap): the bucketed path.
        const bool dense = c->star_k > 0 || 4ll * total > ni;
        if (*(volatile int*)&c->done || total > (unsigned)kMidCap || (dense && total > (unsigned)kBQhSkip)) {
            if (tid == 0 && !*(volatile int*)&c->done) a.big[i] = 1;
            __syncthreads();
            continue;
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
            mid_hull(a.keys + rb, a.vals + rb, (int)total, a.pts + 2 * base, ni, c, a.out_idx + base, a.out_n + i,
                     dyn);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Workspace per (device, stream), grow-only.
struct BWork {
    char* base = nullptr;
    size_t bytes = 0;
    int k = -1;                           // the last call's sets, and where its
    size_t ctl = 0, big = 0, redo = 0;    // control blocks and flags are
};
static std::mutex g_bmu;
static std::map<std::pair<int, cudaStream_t>, BWork> g_bws;

static size_t bt_align(size_t x) { return (x + 255) / 256 * 256; }

struct BLayout {
    size_t ctl, keys, vals, rmap, big, redo, star_ctr, star_list, refine_list, hull_list, unit_base, star_slot, star_bins, star_polys;
    size_t seg_nb, seg_bbase, seg_lo, seg_scale, seg_tbase, rt_base, totals;
    size_t bcount, bcur, bstart, blen, bu, bv, bi, kP, vP, cu, cv, ci, clen, ctmap, counters;
    size_t zero_from, zero_to;   // star bins and bucket counters: cleared before each batch
    size_t total;
    unsigned bcap, tcap, rtcap;
};

// big_pts: points of the sets that can exceed one block (more than kMidCap
// points), big_sets: how many; they bound the buckets and chain tiles.
// slots: sets with a star slot (at least kBStarMinPts points).
static BLayout bt_layout(long long total, int k, long long big_pts, long long big_sets, long long slots) {
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
    L.rtcap = (unsigned)((big_pts + 16 * big_sets) / kBLTile + big_sets + 1);
    L.rmap = take(sizeof(int) * (size_t)L.rtcap);
    L.big = take((size_t)k);
    L.redo = take((size_t)k);
    L.star_ctr = take(4 * 16);
    L.unit_base = take(sizeof(unsigned) * (size_t)k);
    L.refine_list = take(sizeof(int) * (size_t)k);
    L.hull_list = take(sizeof(int) * (size_t)k);
    L.star_list = take(sizeof(int) * (size_t)k);
    L.star_slot = take(sizeof(int) * (size_t)k);
    L.star_polys = take(sizeof(StarPoly) * (size_t)slots);
    L.seg_nb = take(4 * nseg);
    L.seg_bbase = take(4 * (nseg + 1));
    L.seg_lo = take(4 * nseg);
    L.seg_scale = take(4 * nseg);
    L.seg_tbase = take(4 * (nseg + 1));
    L.rt_base = take(4 * ((size_t)k + 1));
    L.totals = take(4 * 8);
    // Cleared before every batch: the star bins, bucket counters and the
    // merge tree's arrival counters (the layout moves with the batch's
    // sizes, so memory that held other data last time can land here).
    L.zero_from = o;
    L.star_bins = take(sizeof(unsigned long long) * kStarBins * (size_t)slots);
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
                        long long slots, char** base, BLayout* L) {
    std::lock_guard<std::mutex> lk(g_bmu);
    *L = bt_layout(total, k, big_pts, big_sets, slots);
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
    w.k = k;
    w.ctl = L->ctl;
    w.big = L->big;
    w.redo = L->redo;
    return CH_OK;
}

int reserve_batched(int dev, cudaStream_t s, long long n, int k) {
    char* base = nullptr;
    BLayout L;
    return bt_workspace(dev, s, n, std::max(k, 1), n, std::max(k, 1), std::min((long long)std::max(k, 1), n / kBStarMinPts),
                        &base, &L);
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
    cudaFuncSetAttribute(bt_filter<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt_ext_smem(T, P));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, bt_filter<T, P>, T, bt_ext_smem(T, P));
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
    if (cudaFuncSetAttribute(bt_star_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBStarSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(bt_star_refine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBStarSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(bt_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBDenseSmem) != cudaSuccess)
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

static void launch_bt_tiles(int shape, bool filter, const BArgs& a, int grid, cudaStream_t s) {
#define CH_BT_CASE(i, T, P)                                                   \
    case i:                                                                   \
        if (filter) bt_filter<T, P><<<grid, T, bt_ext_smem(T, P), s>>>(a);    \
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

// ---------------------------------------------------------------------------
// The device work of one call.
struct BtCall {
    BArgs a;
    BLArgs b;
    int shape, grid_e, grid_f, sms;
    char* base;
    BLayout L;
};

static int bt_enqueue_tiles(const BtCall& c, cudaStream_t s) {
    const BArgs& a = c.a;
    {
        ProfScope p("batched_prep", s);
        if (cudaMemsetAsync(c.base + c.L.zero_from, 0, c.L.zero_to - c.L.zero_from, s) != cudaSuccess) return CH_ECUDA;
        bt_init<<<(a.k + 7) / 8, 256, 0, s>>>(a);
        bt_slots<<<1, 1024, 0, s>>>(a);
    }
    {
        ProfScope p("batched_extremes", s);
        launch_bt_tiles(c.shape, false, a, c.grid_e, s);
    }
    { ProfScope p("batched_octagon", s); bt_octagon<<<a.k, kBOctThreads, 0, s>>>(a); }
    {
        ProfScope p("batched_star", s);
        bt_star_bin<<<c.sms * 8, kBStarBinThreads, 0, s>>>(a);
        bt_star_build<<<c.sms, kBStarThreads, kBStarSmem, s>>>(a);
    }
    {
        ProfScope p("batched_dense", s);
        bt_dense_plan<<<1, 1024, 0, s>>>(a);
        bt_dense<<<c.sms, kBDenseThreads, kBDenseSmem, s>>>(a);
    }
    {
        ProfScope p("batched_filter", s);
        launch_bt_tiles(c.shape, true, a, c.grid_f, s);
    }
    return CH_OK;
}

static int bt_enqueue(const BtCall& c, unsigned char* redo, cudaStream_t s) {
    const int st = bt_enqueue_tiles(c, s);
    if (st != CH_OK) return st;
    { ProfScope p("batched_hull_small", s); bt_hull_small<<<c.a.k, kBSmallThreads, 0, s>>>(c.a); }
    { ProfScope p("batched_refine", s); bt_star_refine<<<c.sms, kBStarThreads, kBStarSmem, s>>>(c.a); }
    { ProfScope p("batched_hull", s); bt_hull<<<c.sms, kBHullThreads, kBHullSmem, s>>>(c.a); }
    // Sets with more records than one block holds: all together through the
    // bucketed path.
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

static void bt_set_shape(BtCall& c, const BtDevice& d, int shape) {
    const BtShape& sh = kBtShapes[shape];
    c.shape = shape;
    c.a.wtile = 32 * sh.per;
    c.a.nwt = (c.a.total - c.a.head) / c.a.wtile;
    c.grid_e = (int)std::max(1ll, std::min(c.a.nwt, (long long)d.sms * d.occ[shape][0]));
    c.grid_f = (int)std::max(1ll, std::min(c.a.nwt, (long long)d.sms * d.occ[shape][1]));
}

// Times every shape on this batch (tile kernels only, best of two runs).
static int bt_tune(BtCall& c, const BtDevice& d, const std::vector<int64_t>& off, cudaStream_t s, int* best) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CH_ECUDA;
    double best_us = 1e30;
    *best = 2;
    int st = CH_OK;
    for (int i = 0; i < kNumBtShapes && st == CH_OK; ++i) {
        bt_set_shape(c, d, i);
        double t_min = 1e30;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, s);
            if (bt_enqueue_tiles(c, s) != CH_OK) {
                st = CH_ECUDA;
                break;
            }
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
    long long big_pts = 0, big_sets = 0, slots = 0;
    for (int i = 0; i < k; ++i) {
        if (off[i + 1] < off[i] || off[i + 1] - off[i] > CH_MAX_POINTS) return CH_EINVAL;
        if (off[i + 1] - off[i] + 12 > kMidCap) {
            big_pts += off[i + 1] - off[i];
            ++big_sets;
        }
        if (off[i + 1] - off[i] >= kBStarMinPts) ++slots;
    }
    const int64_t total = off[k];
    if (total / kBWarpTileMin + 2 > (int64_t)UINT32_MAX) return CH_EINVAL;   // 32-bit tile codes
    int st = check_points_args(pts, total);
    if (st != CH_OK) return st;
    if (total > 0 && !out_idx) return CH_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
    BtDevice d;
    if ((st = bt_configure(dev, &d)) != CH_OK) return st;
    BtCall c;
    if ((st = bt_workspace(dev, s, total, k, big_pts, big_sets, slots, &c.base, &c.L)) != CH_OK) return st;
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
    a.out_idx = out_idx;
    a.out_n = out_n;
    a.big = (unsigned char*)(base + L.big);
    a.total = total;
    // the streamed body starts at the first 16-byte boundary (pts is 8-byte aligned)
    a.head = (total > 0 && (reinterpret_cast<uintptr_t>(pts) & 15u) != 0u) ? 1 : 0;
    a.star_ctr = (unsigned*)(base + L.star_ctr);
    a.star_list = (int*)(base + L.star_list);
    a.star_slot = (int*)(base + L.star_slot);
    a.star_bins = (unsigned long long*)(base + L.star_bins);
    a.star_polys = (StarPoly*)(base + L.star_polys);
    a.refine_list = (int*)(base + L.refine_list);
    a.hull_list = (int*)(base + L.hull_list);
    a.unit_base = (unsigned*)(base + L.unit_base);
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
    bt_set_shape(c, d, shape);
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

extern "C" int ch_batched_counters(void* stream, int32_t k, int64_t* out) {
    if (!out || k < 1) return CH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
    char* base = nullptr;
    size_t o_ctl = 0, o_big = 0, o_redo = 0;
    {
        std::lock_guard<std::mutex> lk(g_bmu);
        auto it = g_bws.find(std::make_pair(dev, s));
        if (it == g_bws.end() || !it->second.base || it->second.k != k) return CH_EINVAL;
        base = it->second.base;
        o_ctl = it->second.ctl;
        o_big = it->second.big;
        o_redo = it->second.redo;
    }
    std::vector<Ctl> ctl((size_t)k);
    std::vector<unsigned char> big((size_t)k), redo((size_t)k);
    if (cudaMemcpyAsync(ctl.data(), base + o_ctl, sizeof(Ctl) * (size_t)k, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(big.data(), base + o_big, (size_t)k, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(redo.data(), base + o_redo, (size_t)k, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return CH_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CH_ECUDA;
    for (int i = 0; i < k; ++i) {
        out[4 * (size_t)i] = (int64_t)ctl[i].count;
        out[4 * (size_t)i + 1] = (int64_t)ctl[i].star_k;
        out[4 * (size_t)i + 2] = (int64_t)ctl[i].status;
        out[4 * (size_t)i + 3] = redo[i] ? 2 : big[i] ? 1 : 0;
    }
    return 4;
}

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
