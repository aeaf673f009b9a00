// batched.cu -- k independent hulls packed back to back (ch_hull_batched).
//
// The sets are cut into tiles of at most kBTile points (a tile never spans
// two sets) and every launch covers all sets at once:
//   bt_init      per-set control blocks and tile counts;
//   bt_scan      tile offsets (exclusive prefix over the sets, one block);
//   bt_extremes  tiles: validation and the 8 extremes of each set as packed
//                (key, lowest local index) maxima (Alg. 2, findExtremes);
//   bt_octagon   one block per set: octagon, inner region, the chain end
//                point records;
//   bt_filter    tiles: the hull-rule classification of every point against
//                its set's octagon, records compacted into the set's region
//                (the loop of Alg. 1/2), support-line end points reduced;
//   bt_hull      one block per set: the hull of its records (quickhull rounds
//                and the stitch, as in the single hull's last block).
// Sets whose records exceed what one block holds go through the bucketed
// large-survivor path together (batched_large.cu); the rare set it cannot
// finish (a bucket chain longer than kBkChain) is flagged and the host runs
// the single-hull path on it.  Each result equals ch_hull on the set alone
// (local indices).
#include "batched_large.h"
#include "ch_internal.cuh"
#include "host.h"
#include "hullcore.cuh"
#include "launch.h"
#include "octagon.cuh"
#include "records.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

namespace ch {

constexpr int kBTile = 4096;           // points per tile
constexpr int kBThreads = 256;         // threads of the tile kernels
constexpr int kBHullThreads = 512;     // threads of bt_hull (a multiple of 128)
constexpr int kBOctThreads = 64;       // threads of bt_octagon

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
};

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
    for (int q = 0; q < 4; ++q) {
        c->counts4[q] = 2u;   // the two chain end points of every queue
        c->blocks_done[q] = 0u;
    }
    a.big[i] = 0;
    const long long ni = a.offsets[i + 1] - a.offsets[i];
    a.tile_base[i] = (int)((ni + kBTile - 1) / kBTile);
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

__device__ __forceinline__ bool bt_dir_is_max(int d) { return d >= SE && d <= N; }

__device__ __forceinline__ int bt_key(int d, int X, int Y) {
    switch (d) {
        case W: case E: return X;
        case S: case N: return Y;
        case SW: case NE: return X + Y;
        default: return X - Y + kCoordLimit;
    }
}

// Three-input max / min of non-negative int keys through their float bit
// patterns (below 2^26 the patterns are positive finite floats that order
// like the integers; max.f32 without .ftz keeps subnormals exact).
__device__ __forceinline__ int bt_max3(int a, int b, int c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(__int_as_float(a)), "f"(__int_as_float(b)), "f"(__int_as_float(c)));
    return __float_as_int(r);
}
__device__ __forceinline__ int bt_min3(int a, int b, int c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(__int_as_float(a)), "f"(__int_as_float(b)), "f"(__int_as_float(c)));
    return __float_as_int(r);
}

// Per tile: each thread holds its kBPer points in registers; the block first
// finds the tile's 8 extreme keys (three-input min / max, two points per
// instruction), then the lowest index reaching each of them (every thread
// checks its own points), and one packed (key, lowest index) atomic per
// direction carries it to the set's maximum.
constexpr int kBPer = kBTile / kBThreads;   // points per thread and tile

__global__ void __launch_bounds__(kBThreads) bt_extremes(BArgs a, int ntiles) {
    __shared__ int s_key[kBThreads / 32][8];
    __shared__ int s_best[8];
    __shared__ unsigned s_idx[8];
    __shared__ int s_set;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (tid == 0) s_set = tile_set(a, t);
        if (tid < 8) s_idx[tid] = 0xFFFFFFFFu;
        __syncthreads();
        const int i = s_set;
        const long long base = a.offsets[i], ni = a.offsets[i + 1] - base;
        const long long p0 = (long long)(t - a.tile_base[i]) * kBTile;
        const int cnt = (int)min((long long)kBTile, ni - p0);   // >= 1
        const float2* p2 = reinterpret_cast<const float2*>(a.pts) + base + p0;
        float2 v[kBPer];
#pragma unroll
        for (int j = 0; j < kBPer; ++j) {
            const int q = tid + j * kBThreads;
            v[j] = __ldcs(p2 + (q < cnt ? q : 0));   // a missing point repeats point 0 of the tile
        }
        int tk[8];
        bool bad = false;
#pragma unroll
        for (int j = 0; j < kBPer; j += 2) {
            const int X0 = __float2int_rn(v[j].x), Y0 = __float2int_rn(v[j].y);
            const int X1 = __float2int_rn(v[j + 1].x), Y1 = __float2int_rn(v[j + 1].y);
            bad |= (__int2float_rn(X0) != v[j].x) | (__int2float_rn(Y0) != v[j].y) |
                   (__int2float_rn(X1) != v[j + 1].x) | (__int2float_rn(Y1) != v[j + 1].y) |
                   (((unsigned)X0 | (unsigned)Y0 | (unsigned)X1 | (unsigned)Y1) >> kCoordBits) != 0u;
            if (j == 0) {
#pragma unroll
                for (int d = 0; d < 8; ++d) {
                    const int k0 = bt_key(d, X0, Y0), k1 = bt_key(d, X1, Y1);
                    tk[d] = bt_dir_is_max(d) ? max(k0, k1) : min(k0, k1);
                }
            } else {
#pragma unroll
                for (int d = 0; d < 8; ++d) {
                    const int k0 = bt_key(d, X0, Y0), k1 = bt_key(d, X1, Y1);
                    tk[d] = bt_dir_is_max(d) ? bt_max3(tk[d], k0, k1) : bt_min3(tk[d], k0, k1);
                }
            }
        }
        if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) set_status(a.ctl + i, CH_ERANGE);
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            int k = tk[d];
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const int r = __shfl_xor_sync(0xFFFFFFFFu, k, o);
                k = bt_dir_is_max(d) ? max(k, r) : min(k, r);
            }
            if (lane == 0) s_key[warp][d] = k;
        }
        __syncthreads();
        if (tid < 8) {
            int k = s_key[0][tid];
            for (int w = 1; w < kBThreads / 32; ++w) k = bt_dir_is_max(tid) ? max(k, s_key[w][tid]) : min(k, s_key[w][tid]);
            s_best[tid] = k;
        }
        __syncthreads();
        // lowest index reaching each extreme key (points in increasing index order per thread)
        unsigned first[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) first[d] = 0xFFFFFFFFu;
#pragma unroll
        for (int j = kBPer - 1; j >= 0; --j) {
            const int q = tid + j * kBThreads;
            const int X = __float2int_rn(v[j].x), Y = __float2int_rn(v[j].y);
#pragma unroll
            for (int d = 0; d < 8; ++d)
                if (q < cnt && bt_key(d, X, Y) == s_best[d]) first[d] = (unsigned)(p0 + q);
        }
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const unsigned m = __reduce_min_sync(0xFFFFFFFFu, first[d]);
            if (lane == 0 && m != 0xFFFFFFFFu) atomicMin(&s_idx[d], m);
        }
        __syncthreads();
        if (tid < 8) {
            const int d = tid;
            const unsigned hk = bt_dir_is_max(d) ? (unsigned)s_best[d] : 0xFFFFFFFFu - (unsigned)s_best[d];
            const unsigned long long pk = ((unsigned long long)hk << 32) | (unsigned long long)(0xFFFFFFFFu - s_idx[d]);
            atomicMax(&a.ctl[i].ext_packed[d], pk);
        }
        __syncthreads();
    }
}

// One block per set: octagon of its extremes (with the inner region, which
// settles most points of bt_filter), the chain end-point records.
__global__ void __launch_bounds__(kBOctThreads) bt_octagon(BArgs a) {
    __shared__ Octagon s_o;
    __shared__ int s_vx[8], s_vy[8], s_id[8], s_st;
    const int i = blockIdx.x, tid = threadIdx.x;
    Ctl* c = a.ctl + i;
    const long long base = a.offsets[i], ni = a.offsets[i + 1] - base;
    if (tid == 0) s_st = read_status(c);
    __syncthreads();
    if (ni == 0 || s_st != CH_OK) {
        if (tid == 0) {
            a.out_n[i] = ni == 0 ? 0 : s_st;
            c->done = 1;
        }
        return;
    }
    if (tid < 8) {
        const unsigned long long pk = c->ext_packed[tid];
        const int id = (int)(0xFFFFFFFFu - (unsigned)(pk & 0xFFFFFFFFull));
        s_id[tid] = id;
        s_vx[tid] = __float2int_rn(a.pts[2 * (base + id)]);
        s_vy[tid] = __float2int_rn(a.pts[2 * (base + id) + 1]);
    }
    __syncthreads();
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

__global__ void __launch_bounds__(kBThreads) bt_filter(BArgs a, int ntiles) {
    __shared__ Octagon s_o;
    __shared__ int s_set, s_skip;
    const int tid = threadIdx.x, lane = tid & 31;
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
            for (long long b0 = p0; b0 < p1; b0 += kBThreads) {   // uniform trip count
                const long long p = b0 + tid;
                const bool valid = p < p1;
                int r = -1, X = 0, Y = 0;
                if (valid) {
                    const float2 v = __ldcs(p2 + p);
                    X = __float2int_rn(v.x);
                    Y = __float2int_rn(v.y);
                    r = classify_hull(v.x, v.y, s_o);
                }
                bool keep = r >= 0;
                if (!__any_sync(0xFFFFFFFFu, keep)) continue;
                if (reduce_on_line(s_o, keep, X, Y, (unsigned)p, c)) keep = false;
                const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
                if (!bal) continue;
                unsigned pos0 = 0u;
                if (lane == 0) pos0 = atomicAdd(&c->count, (unsigned)__popc(bal));
                pos0 = __shfl_sync(0xFFFFFFFFu, pos0, 0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const unsigned bq = __ballot_sync(0xFFFFFFFFu, keep && r == q);
                    if (bq && lane == 0) atomicAdd(&c->counts4[q], (unsigned)__popc(bq));
                }
                if (keep) {
                    uint32_t u, v;
                    queue_frame(r, X, Y, u, v);
                    const long long pos = rb + pos0 + __popc(bal & lanemask_lt());
                    a.keys[pos] = make_key(r, u);
                    a.vals[pos] = make_val(v, (uint32_t)p);
                }
            }
        }
        __syncthreads();
    }
}

constexpr size_t bt_cmax(size_t x, size_t y) { return x > y ? x : y; }
constexpr size_t kBHullSmem = bt_cmax(kMidSmemBytes, sizeof(QhSmem));

// One block per set: support-line records, then the hull of the records when
// one block can hold them (else the set is flagged for the single-hull path).
__global__ void __launch_bounds__(kBHullThreads, 1) bt_hull(BArgs a) {
    extern __shared__ __align__(16) char dyn[];
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
    if (total > (unsigned)kMidCap) {
        if (tid == 0) a.big[i] = 1;
        return;
    }
    __syncthreads();
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
    size_t ctl, keys, vals, tiles, tmap, rmap, big, redo;
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
    L.rtcap = (unsigned)((big_pts + 16 * big_sets) / kBTile + big_sets + 1);
    L.rmap = take(sizeof(int) * (size_t)L.rtcap);
    L.big = take((size_t)k);
    L.redo = take((size_t)k);
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
    return bt_workspace(dev, s, n, std::max(k, 1), n, std::max(k, 1), n / kBTile + std::max(k, 1), &base, &L);
}

void release_batched() {
    std::lock_guard<std::mutex> lk(g_bmu);
    for (auto& kv : g_bws) {
        cudaStreamSynchronize(kv.first.second);
        if (kv.second.base) cudaFree(kv.second.base);
    }
    g_bws.clear();
}

static int bt_configure(int dev, int* sms) {
    static std::mutex mu;
    static std::map<int, int> done;
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find(dev);
    if (it != done.end()) { *sms = it->second; return CH_OK; }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CH_ECUDA;
    if (cudaFuncSetAttribute(bt_hull, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBHullSmem) != cudaSuccess)
        return CH_ECUDA;
    if (configure_batched_large() != cudaSuccess) return CH_ECUDA;
    done[dev] = n;
    *sms = n;
    return CH_OK;
}

}  // namespace ch

using namespace ch;

extern "C" int ch_hull_batched(const float* pts, const int64_t* offsets, int32_t k, int32_t* out_idx,
                               int64_t* out_n, const int64_t* host_offsets, void* stream) {
    if (k < 0 || k > (1 << 20)) return CH_EINVAL;
    if (k == 0) return CH_OK;
    if (!offsets || !out_n) return CH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
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
    long long tiles = 0, big_pts = 0, big_sets = 0;
    for (int i = 0; i < k; ++i) {
        if (off[i + 1] < off[i] || off[i + 1] - off[i] > CH_MAX_POINTS) return CH_EINVAL;
        tiles += (off[i + 1] - off[i] + kBTile - 1) / kBTile;
        if (off[i + 1] - off[i] + 12 > kMidCap) {
            big_pts += off[i + 1] - off[i];
            ++big_sets;
        }
    }
    if (tiles > INT32_MAX) return CH_EINVAL;
    const int64_t total = off[k];
    int st = check_points_args(pts, total);
    if (st != CH_OK) return st;
    if (total > 0 && !out_idx) return CH_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
    if ((st = bt_configure(dev, &sms)) != CH_OK) return st;
    char* base = nullptr;
    BLayout L;
    if ((st = bt_workspace(dev, s, total, k, big_pts, big_sets, tiles, &base, &L)) != CH_OK) return st;
    BArgs a;
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
    const int nt = (int)tiles;
    const int grid_t = std::max(1, std::min(nt, sms * 8));
    {
        ProfScope p("batched_prep", s);
        bt_init<<<(k + 255) / 256, 256, 0, s>>>(a);
        bt_scan<<<1, 1024, 0, s>>>(a.tile_base, a.tile_map, k);
    }
    if (nt > 0) {
        ProfScope p("batched_extremes", s);
        bt_extremes<<<grid_t, kBThreads, 0, s>>>(a, nt);
    }
    { ProfScope p("batched_octagon", s); bt_octagon<<<k, kBOctThreads, 0, s>>>(a); }
    if (nt > 0) {
        ProfScope p("batched_filter", s);
        bt_filter<<<grid_t, kBThreads, 0, s>>>(a, nt);
    }
    { ProfScope p("batched_hull", s); bt_hull<<<k, kBHullThreads, kBHullSmem, s>>>(a); }
    // Sets with more records than one block holds: all together through the
    // bucketed path.
    BLArgs b;
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
    if (cudaMemsetAsync(base + L.zero_from, 0, L.zero_to - L.zero_from, s) != cudaSuccess) return CH_ECUDA;
    launch_batched_large(b, redo, sms, s);
    if (cudaGetLastError() != cudaSuccess) return CH_ECUDA;
    // Sets the bucketed path could not finish (a bucket chain too long): the
    // single-hull path, one by one.
    std::vector<unsigned char> big((size_t)k);
    if (cudaMemcpyAsync(big.data(), redo, (size_t)k, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CH_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CH_ECUDA;
    for (int i = 0; i < k; ++i) {
        if (!big[i]) continue;
        st = enqueue_hull_nograph(pts + 2 * off[i], off[i + 1] - off[i], out_idx + off[i], out_n + i, s, dev);
        if (st != CH_OK) return st;
    }
    return CH_OK;
}
