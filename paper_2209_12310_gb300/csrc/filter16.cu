// filter16.cu -- ch_filter16: the filter of Alg. 2 with a 16-direction
// polygon in place of the octagon.
//
// Among related work (Sec. 2) the paper cites a GPU filter over a convex
// polygon of 16 extreme points, without its directions.  Here they are the
// octagon's 8 (multiples of 45 degrees) and the 8 integer directions between
// them, (+-2, +-1) and (+-1, +-2), in counter-clockwise order from W:
//   k  0 W (-1, 0)   1 (-2,-1)   2 SW (-1,-1)   3 (-1,-2)
//      4 S ( 0,-1)   5 ( 1,-2)   6 SE ( 1,-1)   7 ( 2,-1)
//      8 E ( 1, 0)   9 ( 2, 1)  10 NE ( 1, 1)  11 ( 1, 2)
//     12 N ( 0, 1)  13 (-1, 2)  14 NW (-1, 1)  15 (-2, 1)
// V_k = argmax of a_k x + b_k y over the points, lowest index on ties.  A
// point strictly inside the polygon V_0..V_15 (strictly left of every edge of
// non-zero length; a polygon of zero area discards nothing) gets label 0;
// every other point the queue 1..4 of the quadrilateral rule over W = V_0,
// S = V_4, E = V_8, N = V_12 (as ch_filter).
//
// Launches: f16_init, the extremes (one streaming read), the labels (a second
// read), f16_output.  On 16-byte aligned input the extremes are tiled
// (f16_extremes_tiled: min / max of 8 linear forms per warp tile, the
// winning tile rescanned for the lowest index) and the labels take 4 points
// per lane from a bulk-copy-fed shared-memory ring, with the octagon's inner
// region as a fast path (f16_labels_stream);
// otherwise per-point maxima (f16_extremes) and exact labels (f16_labels).
// Everything is exact: |a x + b y| < 3 * 2^24 fits int32 and every
// orientation product (< 2^48) int64.
#include "ch_internal.cuh"
#include "host.h"
#include "octagon.cuh"
#include "tma.cuh"

#include <algorithm>
#include <climits>

namespace ch {
namespace {

constexpr int kF16Threads = 256;
constexpr int kF16Bias = 1 << 26;   // makes every key positive below 2^27

struct F16Ctl {
    unsigned long long packed[16];  // (key + kF16Bias) << 32 | (0xFFFFFFFF - index): maxima
    int status;
    unsigned counts[4];
    // tiled extremes (aligned input): per direction (tile best, ~tile code)
    unsigned long long tile_packed[16];
    unsigned done;                  // last-arriver counter
    int ready;                      // the last block filled the fields below
    int vx[16], vy[16], live[16];   // the 16-gon's vertices, edges of non-zero length
    int none;                       // zero area: nothing is inside
    Octagon oct;                    // octagon of the even directions, with its inner region
};
static_assert(sizeof(F16Ctl) <= 4 * 4 * (size_t)kChainTile, "F16Ctl lives in the chain-tile scratch");

// a_k x + b_k y for direction k (a compile-time constant after unrolling)
__device__ __forceinline__ int key16(int k, int X, int Y) {
    switch (k) {
        case 0: return -X;
        case 1: return -2 * X - Y;
        case 2: return -X - Y;
        case 3: return -X - 2 * Y;
        case 4: return -Y;
        case 5: return X - 2 * Y;
        case 6: return X - Y;
        case 7: return 2 * X - Y;
        case 8: return X;
        case 9: return 2 * X + Y;
        case 10: return X + Y;
        case 11: return X + 2 * Y;
        case 12: return Y;
        case 13: return -X + 2 * Y;
        case 14: return -X + Y;
        default: return -2 * X + Y;
    }
}

__device__ __forceinline__ long long orient64(int ax, int ay, int bx, int by, int px, int py) {
    return (long long)(bx - ax) * (py - ay) - (long long)(by - ay) * (px - ax);
}

__device__ __forceinline__ bool f16_coord_ok(float v) { return v >= 0.0f && v < 16777216.0f && v == rintf(v); }

__device__ __forceinline__ unsigned long long max_u64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// ctl: the stream workspace's control block, whose status and abort flag
// the bounded waits of the streamed label pass use.
__global__ void f16_init(F16Ctl* c, Ctl* ctl) {
    const int t = threadIdx.x;
    if (t < 16) { c->packed[t] = 0ull; c->tile_packed[t] = 0ull; }
    if (t < 4) c->counts[t] = 0u;
    if (t == 0) { c->status = CH_OK; c->done = 0u; c->ready = 0; ctl->status = CH_OK; ctl->abort = 0; }
}

// ---------------------------------------------------------------------------
// Tiled extremes (16-byte aligned input).  The 16 directions are the minima
// and maxima of 8 linear forms, biased to be non-negative below 2^26:
//   f0 = x, f1 = y, f2 = x + y, f3 = x - y + 2^24, f4 = 2x + y,
//   f5 = 2x - y + 2^24, f6 = x + 2y, f7 = x - 2y + 2^25.
// Direction k = (form, is_max): 0 W (f0, min), 1 (f4, min), 2 SW (f2, min),
// 3 (f6, min), 4 S (f1, min), 5 (f7, max), 6 SE (f3, max), 7 (f5, max),
// 8 E (f0, max), 9 (f4, max), 10 NE (f2, max), 11 (f6, max), 12 N (f1, max),
// 13 (f7, min), 14 NW (f3, min), 15 (f5, min).  Each lane keeps, per
// direction, its best tile value and the first warp tile reaching it (tiles
// rise within a lane); three-input float min / max on the bit patterns of
// the non-negative keys (which order like the integers) cut the per-point
// work.  The last block rescans each direction's winning tile for the lowest
// index, then builds what the label pass needs.
__device__ __forceinline__ int f16_form_of(int k) {
    constexpr int kForm[16] = {0, 4, 2, 6, 1, 7, 3, 5, 0, 4, 2, 6, 1, 7, 3, 5};
    return kForm[k];
}
__device__ __forceinline__ bool f16_is_max(int k) { return k >= 5 && k <= 12; }

__device__ __forceinline__ void f16_forms(int X, int Y, int (&f)[8]) {
    const int s = X + Y, d = X - Y + (1 << 24);
    f[0] = X; f[1] = Y; f[2] = s; f[3] = d;
    f[4] = X + s; f[5] = X + d; f[6] = s + Y; f[7] = d - Y + (1 << 24);
}

__device__ __forceinline__ int f16_max3(int a, int b, int c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(__int_as_float(a)), "f"(__int_as_float(b)), "f"(__int_as_float(c)));
    return __float_as_int(r);
}
__device__ __forceinline__ int f16_min3(int a, int b, int c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(__int_as_float(a)), "f"(__int_as_float(b)), "f"(__int_as_float(c)));
    return __float_as_int(r);
}

// One lane's 16 points of a warp tile (8 float4): per form the minimum and
// maximum; validity folded into *bad.
__device__ __forceinline__ void f16_tile_minmax(const float4 (&v)[kLoadsPerLane], int (&mn)[8], int (&mx)[8],
                                                bool& bad) {
#pragma unroll
    for (int j = 0; j < kLoadsPerLane; ++j) {
        const int X0 = __float2int_rn(v[j].x), Y0 = __float2int_rn(v[j].y);
        const int X1 = __float2int_rn(v[j].z), Y1 = __float2int_rn(v[j].w);
        bad |= (__int2float_rn(X0) != v[j].x) | (__int2float_rn(Y0) != v[j].y) |
               (__int2float_rn(X1) != v[j].z) | (__int2float_rn(Y1) != v[j].w) |
               ((((unsigned)X0 | (unsigned)Y0 | (unsigned)X1 | (unsigned)Y1) >> kCoordBits) != 0u);
        int a[8], b[8];
        f16_forms(X0 & (kCoordLimit - 1), Y0 & (kCoordLimit - 1), a);   // masked: keys stay in range on bad data
        f16_forms(X1 & (kCoordLimit - 1), Y1 & (kCoordLimit - 1), b);
#pragma unroll
        for (int f = 0; f < 8; ++f) {
            if (j == 0) {
                mn[f] = min(a[f], b[f]);
                mx[f] = max(a[f], b[f]);
            } else {
                mn[f] = f16_min3(mn[f], a[f], b[f]);
                mx[f] = f16_max3(mx[f], a[f], b[f]);
            }
        }
    }
}

__global__ void __launch_bounds__(kF16Threads, 2) f16_extremes_tiled(const float4* __restrict__ p4, long long n,
                                                                     long long ntiles, F16Ctl* c) {
    __shared__ unsigned long long s_m[kF16Threads / 32][16];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    int best[16];
    unsigned code[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        best[k] = f16_is_max(k) ? -1 : INT_MAX;
        code[k] = 0u;
    }
    bool bad = false;
    const unsigned long long pol = l2_evict_first();
    for (long long t = gwarp; t < ntiles; t += nwarps) {
        float4 v[kLoadsPerLane];
#pragma unroll
        for (int j = 0; j < kLoadsPerLane; ++j) v[j] = ld_stream_f4(p4 + t * kWarpTileF4 + j * 32 + lane, pol);
        int mn[8], mx[8];
        f16_tile_minmax(v, mn, mx, bad);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int tv = f16_is_max(k) ? mx[f16_form_of(k)] : mn[f16_form_of(k)];
            const bool better = f16_is_max(k) ? tv > best[k] : tv < best[k];
            best[k] = better ? tv : best[k];
            code[k] = better ? (unsigned)(t + 1) : code[k];
        }
    }
    // the ragged tail (fewer than 512 points) in warp 0 of block 0, as tile code ntiles + 1
    if (blockIdx.x == 0 && warp == 0) {
        for (long long i = ntiles * kWarpTilePts + lane; i < n; i += 32) {
            const float2 p = reinterpret_cast<const float2*>(p4)[i];
            const int X = __float2int_rn(p.x), Y = __float2int_rn(p.y);
            bad |= (__int2float_rn(X) != p.x) | (__int2float_rn(Y) != p.y) |
                   ((((unsigned)X | (unsigned)Y) >> kCoordBits) != 0u);
            int f[8];
            f16_forms(X & (kCoordLimit - 1), Y & (kCoordLimit - 1), f);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int tv = f[f16_form_of(k)];
                const bool better = f16_is_max(k) ? tv > best[k] : tv < best[k];
                best[k] = better ? tv : best[k];
                code[k] = better ? (unsigned)(ntiles + 1) : code[k];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        // packed so that the maximum wins: the best value, then the lowest tile
        const bool any = f16_is_max(k) ? best[k] >= 0 : best[k] != INT_MAX;
        const unsigned hk = f16_is_max(k) ? (unsigned)best[k] : 0xFFFFFFFFu - (unsigned)best[k];
        unsigned long long m = any ? ((unsigned long long)hk << 32) | (0xFFFFFFFFu - code[k]) : 0ull;
#pragma unroll
        for (int o = 16; o; o >>= 1) m = max_u64(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        if (lane == 0) s_m[warp][k] = m;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(&c->status, CH_OK, CH_ERANGE);
    if (threadIdx.x < 16) {
        unsigned long long m = 0ull;
        for (int w = 0; w < kF16Threads / 32; ++w) m = max_u64(m, s_m[w][threadIdx.x]);
        if (m) atomicMax(&c->tile_packed[threadIdx.x], m);
    }
    if (!last_block(&c->done, &s_last)) return;
    if (*(volatile int*)&c->status != CH_OK) return;
    // lowest index of each direction's best value within its winning tile
    __shared__ unsigned long long s_best[16];
    __shared__ int s_val[16];
    __shared__ long long s_lo[16], s_hi[16];
    if (threadIdx.x < 16) {
        const int k = threadIdx.x;
        const unsigned long long pk = *(volatile unsigned long long*)&c->tile_packed[k];
        const unsigned hk = (unsigned)(pk >> 32), cd = 0xFFFFFFFFu - (unsigned)pk;
        s_val[k] = f16_is_max(k) ? (int)hk : (int)(0xFFFFFFFFu - hk);
        s_lo[k] = (long long)(cd - 1u) * kWarpTilePts;
        s_hi[k] = min(n, s_lo[k] + kWarpTilePts);
        s_best[k] = ~0ull;
    }
    __syncthreads();
    for (int k = 0; k < 16; ++k) {
        for (long long i = s_lo[k] + threadIdx.x; i < s_hi[k]; i += blockDim.x) {
            const float2 p = reinterpret_cast<const float2*>(p4)[i];
            int f[8];
            f16_forms(__float2int_rn(p.x), __float2int_rn(p.y), f);
            if (f[f16_form_of(k)] == s_val[k]) atomicMin(&s_best[k], (unsigned long long)i);
        }
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        const int k = threadIdx.x;
        const long long i = (long long)s_best[k];
        const float2 p = reinterpret_cast<const float2*>(p4)[i < n ? i : 0];
        const int key = key16(k, __float2int_rn(p.x), __float2int_rn(p.y));
        c->packed[k] = ((unsigned long long)(unsigned)(key + kF16Bias) << 32) | (0xFFFFFFFFu - (unsigned)i);
        c->vx[k] = __float2int_rn(p.x);
        c->vy[k] = __float2int_rn(p.y);
    }
    __syncthreads();
    // what the label pass needs: live edges, zero area, and the octagon of the
    // even directions with its inner region (inside the 16-gon)
    __shared__ int s_vx[8], s_vy[8], s_id[8];
    __shared__ Octagon s_o;
    if (threadIdx.x < 16) {
        const int k = threadIdx.x, j = (k + 1) & 15;
        c->live[k] = (c->vx[k] != c->vx[j] || c->vy[k] != c->vy[j]) ? 1 : 0;
    }
    if (threadIdx.x < 8) {
        s_vx[threadIdx.x] = c->vx[2 * threadIdx.x];
        s_vy[threadIdx.x] = c->vy[2 * threadIdx.x];
        s_id[threadIdx.x] = (int)(0xFFFFFFFFu - (unsigned)(c->packed[2 * threadIdx.x] & 0xFFFFFFFFull));
    }
    if (threadIdx.x == 0) {
        long long a2 = 0;
        for (int k = 0; k < 16; ++k) {
            const int j = (k + 1) & 15;
            a2 += (long long)c->vx[k] * c->vy[j] - (long long)c->vx[j] * c->vy[k];
        }
        c->none = a2 == 0 ? 1 : 0;
    }
    __syncthreads();
    setup_octagon_block(s_o, s_vx, s_vy, s_id, true);
    copy_octagon(&c->oct, &s_o);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        c->ready = 1;
    }
}

// The label pass on 16-byte aligned points with a 4-byte aligned label
// array, fed by bulk copies as ch_filter's: each warp streams its warp tiles
// through a double-buffered shared-memory ring and labels 4 consecutive
// points per lane and round (one 32-bit store).  Points strictly inside the
// octagon's inner region are settled inline (that octagon lies inside the
// 16-gon), the others by the exact 16-edge test; the ragged tail is labelled
// point by point by the first warp.
// Out of line: the inner-region test settles most points, and the streaming
// loop stays small.
static __device__ __noinline__ int f16_label_exact(int X, int Y, const int* vx, const int* vy, const int* live,
                                                   bool none) {
    bool inside = !none;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int j = (k + 1) & 15;
        if (live[k] && orient64(vx[k], vy[k], vx[j], vy[j], X, Y) <= 0) inside = false;
    }
    int r = -1;
    if (!inside) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {   // W->S, S->E, E->N, N->W
            const int a = 4 * q, b = (4 * q + 4) & 15;
            if (r < 0 && orient64(vx[a], vy[a], vx[b], vy[b], X, Y) < 0) r = q;
        }
    }
    return r;
}

constexpr size_t kF16StreamSmemBytes = (size_t)(kF16Threads / 32) * kStages * kWarpTileF4 * sizeof(float4);

__global__ void __launch_bounds__(kF16Threads) f16_labels_stream(const float4* __restrict__ p4, long long n,
                                                                 long long ntiles, F16Ctl* c, Ctl* ctl,
                                                                 uint32_t* labels4) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ int s_vx[16], s_vy[16], s_live[16];
    __shared__ Octagon s_o;
    __shared__ unsigned s_cnt[4];
    __shared__ unsigned long long s_bar[kF16Threads / 32][kStages];
    if (*(volatile int*)&c->status != CH_OK) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t < 16) { s_vx[t] = c->vx[t]; s_vy[t] = c->vy[t]; s_live[t] = c->live[t]; }
    if (t < 4) s_cnt[t] = 0u;
    copy_octagon(&s_o, &c->oct);
    __syncthreads();
    const bool none = c->none != 0;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + t) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned cnt[4] = {0u, 0u, 0u, 0u};
    WarpStream ws{reinterpret_cast<float4*>(dsm) + warp * kStages * kWarpTileF4, s_bar[warp], p4, gwarp, nwarps,
                  ntiles, lane};
    ws.start();
    for (long long k = 0;; ++k) {
        const long long tile = gwarp + k * nwarps;
        if (tile >= ntiles) break;
        const float4* cur = ws.acquire(k, ctl);
        if (!cur) {   // a copy never completed: the workspace status is CH_ETIMEOUT
            ws.drain(k);
            break;
        }
#pragma unroll
        for (int r = 0; r < kWarpTilePts / 128; ++r) {
            const int q = r * 32 + lane;   // 4 points: float4 2q and 2q + 1 of the tile
            const float4 a = cur[2 * q], b = cur[2 * q + 1];
            const float xs[4] = {a.x, a.z, b.x, b.z}, ys[4] = {a.y, a.w, b.y, b.w};
            uint32_t word = 0u;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int X = __float2int_rn(xs[m]), Y = __float2int_rn(ys[m]);
                int lab = -1;
                if (!in_inner_strict(s_o, X, Y)) lab = f16_label_exact(X, Y, s_vx, s_vy, s_live, none);
                word |= (uint32_t)(lab + 1) << (8 * m);
                if (lab >= 0) cnt[lab]++;
            }
            if (labels4) labels4[tile * (kWarpTilePts / 4) + q] = word;
        }
        ws.release(k);
    }
    if (gwarp == 0) {   // the ragged tail
        for (long long i = ntiles * kWarpTilePts + lane; i < n; i += 32) {
            const float2 p = reinterpret_cast<const float2*>(p4)[i];
            const int X = __float2int_rn(p.x), Y = __float2int_rn(p.y);
            const int lab = in_inner_strict(s_o, X, Y) ? -1 : f16_label_exact(X, Y, s_vx, s_vy, s_live, none);
            if (labels4) reinterpret_cast<uint8_t*>(labels4)[i] = (uint8_t)(lab + 1);
            if (lab >= 0) cnt[lab]++;
        }
    }
#pragma unroll
    for (int qd = 0; qd < 4; ++qd) {
        unsigned v = cnt[qd];
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if (lane == 0 && v) atomicAdd(&s_cnt[qd], v);
    }
    __syncthreads();
    if (t < 4 && s_cnt[t]) atomicAdd(&c->counts[t], s_cnt[t]);
}

__global__ void __launch_bounds__(kF16Threads) f16_extremes(const float2* __restrict__ pts, long long n,
                                                            F16Ctl* c) {
    __shared__ unsigned long long s_m[kF16Threads / 32][16];
    int best[16];
    unsigned arg[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        best[k] = INT_MIN;
        arg[k] = 0u;
    }
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // indices rise within a thread, so a strict improvement keeps the lowest
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float2 p = __ldcs(pts + i);
        const bool ok = f16_coord_ok(p.x) && f16_coord_ok(p.y);
        bad |= !ok;
        const int X = ok ? __float2int_rz(p.x) : 0, Y = ok ? __float2int_rz(p.y) : 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int v = key16(k, X, Y);
            if (v > best[k]) {
                best[k] = v;
                arg[k] = (unsigned)i;
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        // keys exceed -2^26, so INT_MIN marks a thread without points
        unsigned long long m = best[k] == INT_MIN
                                   ? 0ull
                                   : ((unsigned long long)(unsigned)(best[k] + kF16Bias) << 32) | (0xFFFFFFFFu - arg[k]);
#pragma unroll
        for (int o = 16; o; o >>= 1) m = max_u64(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        if (lane == 0) s_m[warp][k] = m;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(&c->status, CH_OK, CH_ERANGE);
    if (threadIdx.x < 16) {
        unsigned long long m = 0ull;
        for (int w = 0; w < kF16Threads / 32; ++w) m = max_u64(m, s_m[w][threadIdx.x]);
        if (m) atomicMax(&c->packed[threadIdx.x], m);
    }
}

__global__ void __launch_bounds__(kF16Threads) f16_labels(const float2* __restrict__ pts, long long n, F16Ctl* c,
                                                          uint8_t* labels) {
    __shared__ int s_vx[16], s_vy[16], s_live[16];
    __shared__ int s_none;
    __shared__ unsigned s_cnt[4];
    if (*(volatile int*)&c->status != CH_OK) return;   // set before this launch: the same for every block
    const int t = threadIdx.x;
    if (t < 16) {
        const unsigned idx = 0xFFFFFFFFu - (unsigned)(c->packed[t] & 0xFFFFFFFFull);
        const float2 v = (long long)idx < n ? pts[idx] : make_float2(0.0f, 0.0f);
        s_vx[t] = __float2int_rz(v.x);
        s_vy[t] = __float2int_rz(v.y);
    }
    if (t < 4) s_cnt[t] = 0u;
    __syncthreads();
    if (t < 16) {
        const int j = (t + 1) & 15;
        s_live[t] = (s_vx[t] != s_vx[j] || s_vy[t] != s_vy[j]) ? 1 : 0;
    }
    if (t == 0) {
        long long a2 = 0;
        for (int k = 0; k < 16; ++k) {
            const int j = (k + 1) & 15;
            a2 += (long long)s_vx[k] * s_vy[j] - (long long)s_vx[j] * s_vy[k];
        }
        s_none = a2 == 0 ? 1 : 0;
    }
    __syncthreads();
    const bool none = s_none != 0;
    unsigned cnt[4] = {0u, 0u, 0u, 0u};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + t; i < n; i += stride) {
        const float2 p = __ldcs(pts + i);
        const int X = __float2int_rz(p.x), Y = __float2int_rz(p.y);
        bool inside = !none;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int j = (k + 1) & 15;
            if (s_live[k] && orient64(s_vx[k], s_vy[k], s_vx[j], s_vy[j], X, Y) <= 0) inside = false;
        }
        int r = -1;
        if (!inside) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {   // W->S, S->E, E->N, N->W
                const int a = 4 * q, b = (4 * q + 4) & 15;
                if (r < 0 && orient64(s_vx[a], s_vy[a], s_vx[b], s_vy[b], X, Y) < 0) r = q;
            }
        }
        if (labels) labels[i] = (uint8_t)(r + 1);
        if (r >= 0) cnt[r]++;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        unsigned v = cnt[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if ((t & 31) == 0 && v) atomicAdd(&s_cnt[q], v);
    }
    __syncthreads();
    if (t < 4 && s_cnt[t]) atomicAdd(&c->counts[t], s_cnt[t]);
}

__global__ void f16_output(const F16Ctl* c, const Ctl* ctl, int32_t* out_ext16, int64_t* out_counts4) {
    const int t = threadIdx.x;
    const int st = c->status != CH_OK ? c->status : ctl->status;
    if (t < 16) out_ext16[t] = st != CH_OK ? -1 : (int32_t)(0xFFFFFFFFu - (unsigned)(c->packed[t] & 0xFFFFFFFFull));
    if (t < 4 && out_counts4) out_counts4[t] = st != CH_OK ? (int64_t)st : (int64_t)c->counts[t];
}

}  // namespace
}  // namespace ch

using namespace ch;

extern "C" int ch_filter16(const float* pts, int64_t n, int32_t* out_ext16, uint8_t* out_labels,
                           int64_t* out_counts4, void* stream) {
    int st = check_points_args(pts, n);
    if (st != CH_OK) return st;
    if (!out_ext16) return CH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        if (cudaMemsetAsync(out_ext16, 0xFF, 16 * sizeof(int32_t), s) != cudaSuccess) return CH_ECUDA;
        if (out_counts4 && cudaMemsetAsync(out_counts4, 0, 4 * sizeof(int64_t), s) != cudaSuccess)
            return CH_ECUDA;
        return CH_OK;
    }
    int dev = 0, sms = 0, occ_e = 0, occ_l = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CH_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_e, f16_extremes, kF16Threads, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_l, f16_labels, kF16Threads, 0) != cudaSuccess)
        return CH_ECUDA;
    static bool s_configured = false;   // the streamed label pass's shared memory (idempotent)
    if (!s_configured) {
        if (cudaFuncSetAttribute(f16_labels_stream, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kF16StreamSmemBytes) != cudaSuccess)
            return CH_ECUDA;
        s_configured = true;
    }
    int occ_s = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, f16_labels_stream, kF16Threads, kF16StreamSmemBytes) !=
        cudaSuccess)
        return CH_ECUDA;
    char* base = nullptr;
    Layout L;
    if ((st = get_workspace(dev, s, n, &base, &L)) != CH_OK) return st;
    F16Ctl* c = reinterpret_cast<F16Ctl*>(base + L.off_cu);
    Ctl* ctl = reinterpret_cast<Ctl*>(base + L.off_ctl);
    const float2* p2 = reinterpret_cast<const float2*>(pts);
    const long long blocks = (n + kF16Threads - 1) / kF16Threads;
    const int grid_e = (int)std::min<long long>(blocks, (long long)sms * std::max(1, occ_e));
    const int grid_l = (int)std::min<long long>(blocks, (long long)sms * std::max(1, occ_l));
    // 16-byte aligned points take the tiled extremes and, with a 4-byte
    // aligned label array, the 4-points-per-thread label pass
    const bool aligned = ((uintptr_t)pts & 15u) == 0u;
    const bool lab4 = aligned && ((uintptr_t)out_labels & 3u) == 0u;
    f16_init<<<1, 32, 0, s>>>(c, ctl);
    {
        ProfScope p("filter16_extremes", s);
        if (aligned) {
            int occ_t = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_t, f16_extremes_tiled, kF16Threads, 0) !=
                cudaSuccess)
                return CH_ECUDA;
            const long long ntiles = n / kWarpTilePts;
            const long long want = (ntiles + kF16Threads / 32 - 1) / (kF16Threads / 32);
            const int grid_t = (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * std::max(1, occ_t)));
            f16_extremes_tiled<<<grid_t, kF16Threads, 0, s>>>(reinterpret_cast<const float4*>(pts), n, ntiles, c);
        } else {
            f16_extremes<<<grid_e, kF16Threads, 0, s>>>(p2, n, c);
        }
    }
    if (out_labels || out_counts4) {
        ProfScope p("filter16_labels", s);
        if (lab4) {
            const int grid_s = (int)std::min<long long>(blocks, (long long)sms * std::max(1, occ_s));
            f16_labels_stream<<<grid_s, kF16Threads, kF16StreamSmemBytes, s>>>(
                reinterpret_cast<const float4*>(pts), n, n / kWarpTilePts, c, ctl,
                reinterpret_cast<uint32_t*>(out_labels));
        } else
            f16_labels<<<grid_l, kF16Threads, 0, s>>>(p2, n, c, out_labels);
    }
    f16_output<<<1, 32, 0, s>>>(c, ctl, out_ext16, out_counts4);
    return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ECUDA;
}
