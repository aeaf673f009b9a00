// ch_internal.cuh -- device-side data layout and helpers shared by the CUDA
// translation units of libconvhull (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "ch.h"

namespace ch {

// ---------------------------------------------------------------------------
// Geometry of the input domain.  Coordinates are integers in [0, 2^24), so
// x + y < 2^25 and every orientation product is below 2^50 (exact in int64).
// ---------------------------------------------------------------------------
constexpr int kCoordBits = 24;
constexpr int kCoordLimit = 1 << kCoordBits;
constexpr int kKeyBits = 25;                  // bits of the per-queue sort key u
constexpr uint32_t kKeyMask = (1u << kKeyBits) - 1;
constexpr int kSortBits = 27;                 // queue (2 bits) | u (25 bits)
constexpr int kDigitBits = 9;                 // 3 LSD passes of 9 bits
constexpr int kDigits = 1 << kDigitBits;
constexpr int kSortPasses = 3;

// Streaming passes: a warp tile is 256 float4 = 512 points (8 float4 / lane).
constexpr int kLoadsPerLane = 8;
constexpr int kWarpTileF4 = 32 * kLoadsPerLane;
constexpr int kWarpTilePts = 2 * kWarpTileF4;

// Onesweep radix sort tile: 256 threads x 16 keys.
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

// Hull stage tile: 256 threads x 16 sorted records.
constexpr int kChainThreads = 256;
constexpr int kChainItems = 16;
constexpr int kChainTile = kChainThreads * kChainItems;
constexpr int kMergeSmemCap = 8192;           // chain points a global merge keeps on chip
// Bucketed large-survivor path (bucket.cu): records per bucket on average,
// chain vertices a bucket may keep, bucket chains per chain-kernel tile.
constexpr int kBkAvg = 256;
constexpr int kBkNearHull = 64;   // records per bucket when a star polygon filtered them
constexpr int kBkChain = 32;
constexpr int kBkGroup = kChainTile / kBkChain;
// Buckets of a queue of cnt records: about kBkAvg records each, and at least
// 7 cnt^(1/3) (at most one per 8 records).  The queue chain of cnt records
// on a thin ring (the ring workload: width 64 at radius 2^23) has about
// 54 cnt^(1/3) vertices, so a bucket holds about 8 of them and its chain
// stays within kBkChain; a queue whose chains still overflow takes the
// radix-sort path.  kBkMinQ bounds the floor (7 cnt^(1/3) - cnt / kBkAvg
// stays below 115), for the workspace bounds.
constexpr int kBkMinQ = 256;
constexpr int kBkCoarseMax = 4096;   // coarse bucket groups of the two-level partition at most

__host__ __device__ __forceinline__ unsigned bk_buckets_for(unsigned cnt) {
    unsigned nb = (cnt + kBkAvg - 1) / kBkAvg;
    unsigned ring = (unsigned)(7.0f * cbrtf((float)cnt)) + 1u;
    ring = ring < (unsigned)kBkMinQ ? ring : (unsigned)kBkMinQ;
    const unsigned lo = (cnt / 8u < ring) ? cnt / 8u : ring;
    nb = nb > lo ? nb : lo;
    return nb > 0u ? nb : 1u;
}
constexpr int kSampleTiles = 1024;            // warp tiles read by the sample pass (512k points)
// Star polygon of dense data (star.cu): angular bins around the sample
// octagon's centre, extra warp tiles read when the sample is dense.
constexpr int kStarBins = 8192;
constexpr int kStarExtraTiles = 2048;
constexpr int kMaxLevels = 32;

// Warp tiles read by the sample pass: about 1/32 of the input, at most
// kSampleTiles, at least min(ntiles, 64).
__host__ __device__ __forceinline__ long long sample_tiles(long long ntiles) {
    long long s = ntiles / 32;
    if (s < 64) s = ntiles < 64 ? ntiles : 64;
    return s < kSampleTiles ? s : kSampleTiles;
}

// Float edge-function error bound: |e_float - e_exact| < 2^28 for every edge
// and query point of the domain (see octagon setup in filter.cu).
constexpr float kEdgeTol = 268435456.0f;      // 2^28
constexpr float kHugePositive = 1.0e30f;      // "always inside" coefficient of a skipped edge

constexpr unsigned kSpinLimit = 1u << 20;     // bounded waits (onesweep look-back)

// Directions of the 8 extremes in counter-clockwise octagon order.
enum Dir { W = 0, SW, S, SE, E, NE, N, NW };

// Edge function  e(p) = A*px + B*py + C  equals orient(a, b, p) (positive when
// p is left of a->b); exact data kept for the ambiguous band |e| <= kEdgeTol.
struct Edge {
    float A, B, C;
    int ax, ay, dx, dy;  // origin and direction (dx = dy = 0: skipped edge)
};

struct Octagon {
    int vx[8], vy[8];    // vertices W, SW, S, SE, E, NE, N, NW
    int ext[8];          // their indices (-1 for a sample octagon)
    Edge oct[8];         // octagon edges V[k] -> V[k+1]
    Edge quad[4];        // W->S, S->E, E->N, N->W (queue rule)
    int in_lo[4], in_hi[4];   // inner region: x, y, x+y, x-y+2^24 bounds (empty if lo > hi)
    int discard_none;    // octagon of zero area: nothing is discarded
    int pad[3];
};

// Small-path limits: the last block of a pass finishes the hull itself when
// the survivors are few.
constexpr int kMidCap = 8192;           // sort records one block turns into the hull

// Per-call control block in device memory.
struct Ctl {
    unsigned long long ext_packed[8];   // (key, ~tile) packed maxima of pass 1
    unsigned long long samp_packed[8];  // (key, other coordinate) maxima of the sample pass
    int status;                         // CH_OK or a negative ch_status
    int abort;                          // set by a timed-out wait; all waits give up
    unsigned int count;                 // sort records (the 8 extreme records first)
    unsigned int count_raw;             // raw survivors of the fused pass
    unsigned int epoch;                 // onesweep status epoch (incremented per call)
    int mode;                           // 0: fused single pass, 1: two streaming passes
    int done;                           // the hull has been written by a small-path block
    int records_ready;                  // sort records complete before the re-classify stage
    unsigned int blocks_done[4];        // last-arriver counters (sample, main, stage C, roots)
    unsigned int tile_ctr[4];           // onesweep tile claim counters
    unsigned int digit_hist[kSortPasses][kDigits];   // sort fallback only (sort_hist_kernel)
    unsigned int rec_q[4];              // records per queue
    unsigned int reg_start[4], reg_end[4];
    unsigned int reg_tile_base[5];      // chain tiles of queue r: [base[r], base[r+1])
    unsigned int counts4[4];            // survivors per queue (ch_filter)
    unsigned long long line_ep[8];      // end points of survivors on the 4 axis support lines
    int bk_state;                       // large-survivor path: 0 unused, 1 buckets, 2 full sort
    unsigned int bk_cursor;             // tiles of the second partition level
    unsigned int bk_nb[4];              // buckets of queue r
    unsigned int bk_base[5];            // first bucket of queue r
    int bk_lo[4];                       // u of queue r's first chain point
    float bk_scale[4];                  // buckets per unit of u in queue r
    int bk_shift;                       // fine buckets per coarse group: 1 << bk_shift
    unsigned int bk_next;               // next bucket for a bk_hull warp
    int samp_ok;                        // oct_s holds this call's sample octagon
    int star_ok;                        // the star pass found dense data: the post pass builds the polygon
    int star_k;                         // the polygon's vertices (post pass)
    int star_final;                     // the post pass built and accepted the polygon
    int star_cx, star_cy;               // its centre (vertices are stored relative to it)
    unsigned int star_pts, star_out;    // points the star pass read / found outside the sample octagon
    unsigned int star_done;             // last-arriver counter of the star pass
    Octagon oct;                        // octagon of the true extremes
    Octagon oct_s;                      // octagon of a sample's extremes
#if defined(CH_TRACE) || defined(CH_TIMELINE)
    unsigned long long tl[14][2];       // debug builds: first start / last end per phase (%globaltimer)
#endif
};

// Optional phase tracing of single-block kernels (debug builds with
// -DCH_TRACE): thread 0 stamps %globaltimer and prints the deltas.
#ifdef CH_TRACE
__shared__ unsigned long long s_trace_t[24];
__shared__ int s_trace_n;
#define CH_TRACE_DECL if (threadIdx.x == 0) s_trace_n = 0;
#define CH_TRACE_MARK() do { if (threadIdx.x == 0 && s_trace_n >= 0 && s_trace_n < 24) { unsigned long long _t; \
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(_t)); s_trace_t[s_trace_n++] = _t; } } while (0)
#define CH_TRACE_PRINT(tag) do { if (threadIdx.x == 0) { printf("[trace %s]", tag); \
    for (int _i = 1; _i < s_trace_n; ++_i) printf(" %llu", s_trace_t[_i] - s_trace_t[_i - 1]); printf("\n"); } } while (0)
#else
#define CH_TRACE_DECL
#define CH_TRACE_MARK() do { } while (0)
#define CH_TRACE_PRINT(tag) do { } while (0)
#endif
// Debug builds (-DCH_TRACE or -DCH_TIMELINE): grid-wide phase timeline, the
// first start and the last end of each phase in ctl->tl.
#if defined(CH_TRACE) || defined(CH_TIMELINE)
#define CH_TL(ctl, slot, end) do { if (threadIdx.x == 0) { unsigned long long _t; \
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(_t)); \
    if (end) atomicMax(&(ctl)->tl[slot][1], _t); else atomicMin(&(ctl)->tl[slot][0], _t); } } while (0)
#else
#define CH_TL(ctl, slot, end) do { } while (0)
#endif

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long orient64(long long ax, long long ay, long long bx,
                                              long long by, long long px, long long py) {
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

// L2 policy for data read once per call (the input points): evicted first,
// so streaming 100s of MB does not flush the workspace, the control block and
// the kernels' code out of L2.
__device__ __forceinline__ unsigned long long l2_evict_first() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ float4 ld_stream_f4(const float4* p, unsigned long long pol) {
    float4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "l"(p), "l"(pol));
    return r;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
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

__device__ __forceinline__ void set_status(Ctl* ctl, int st) {
    atomicCAS(&ctl->status, CH_OK, st);
}

// One poll of a bounded wait on a flag another block sets: false to poll
// again (after a short sleep); true to give up, after kSpinLimit polls or
// when another wait already gave up (then status CH_ETIMEOUT and the abort
// flag are set, and the caller leaves the wait).
__device__ __forceinline__ bool spin_give_up(unsigned& spins, Ctl* ctl) {
    if (++spins > kSpinLimit || ((spins & 63u) == 0u && *(volatile int*)&ctl->abort)) {
        set_status(ctl, CH_ETIMEOUT);
        atomicExch(&ctl->abort, 1);
        return true;
    }
    __nanosleep(64);
    return false;
}

__device__ __forceinline__ int read_status(const Ctl* ctl) {
    return *(volatile const int*)&ctl->status;
}

// Queue-frame coordinates of a survivor.  For queue r the chain from its
// start extreme to its end extreme is strictly increasing in u, and among
// points of equal u only the one of minimum v can be a hull vertex.  Every
// map (x, y) -> (u, v) is a rotation by a multiple of 90 degrees plus 45,
// scaled by sqrt(2): orientation-preserving, so cross products keep their sign.
//   r = 0 (W->S):  u = x - y + 2^24,      v = x + y
//   r = 1 (S->E):  u = x + y,             v = y - x + 2^24
//   r = 2 (E->N):  u = y - x + 2^24,      v = 2^25 - 2 - x - y
//   r = 3 (N->W):  u = 2^25 - 2 - x - y,  v = x - y + 2^24
__device__ __forceinline__ void queue_frame(int r, int x, int y, uint32_t& u, uint32_t& v) {
    const int off = kCoordLimit;
    const int top = 2 * kCoordLimit - 2;
    switch (r) {
        case 0: u = (uint32_t)(x - y + off); v = (uint32_t)(x + y); break;
        case 1: u = (uint32_t)(x + y); v = (uint32_t)(y - x + off); break;
        case 2: u = (uint32_t)(y - x + off); v = (uint32_t)(top - x - y); break;
        default: u = (uint32_t)(top - x - y); v = (uint32_t)(x - y + off); break;
    }
}

__device__ __forceinline__ uint32_t make_key(int r, uint32_t u) { return ((uint32_t)r << kKeyBits) | u; }
__device__ __forceinline__ uint64_t make_val(uint32_t v, uint32_t idx) {
    return ((uint64_t)v << 31) | (uint64_t)idx;
}

}  // namespace ch
