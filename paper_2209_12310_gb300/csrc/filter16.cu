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
// Launches: f16_init, f16_extremes (one streaming read: per-thread maxima,
// warp shuffles, one 64-bit atomicMax per block and direction), f16_labels (a
// second read: exact int64 orientation against the 16 edges), f16_output.
// Everything is exact: |a x + b y| < 3 * 2^24 fits int32 and every
// orientation product (< 2^48) int64.
#include "ch_internal.cuh"
#include "host.h"

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

__device__ __forceinline__ bool f16_coord_ok(float v) { return v >= 0.0f && v < 16777216.0f && v == rintf(v); }

__device__ __forceinline__ unsigned long long max_u64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

__global__ void f16_init(F16Ctl* c) {
    const int t = threadIdx.x;
    if (t < 16) c->packed[t] = 0ull;
    if (t < 4) c->counts[t] = 0u;
    if (t == 0) c->status = CH_OK;
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

__device__ __forceinline__ long long orient64(int ax, int ay, int bx, int by, int px, int py) {
    return (long long)(bx - ax) * (py - ay) - (long long)(by - ay) * (px - ax);
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

__global__ void f16_output(const F16Ctl* c, int32_t* out_ext16, int64_t* out_counts4) {
    const int t = threadIdx.x;
    const int st = c->status;
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
    char* base = nullptr;
    Layout L;
    if ((st = get_workspace(dev, s, n, &base, &L)) != CH_OK) return st;
    F16Ctl* c = reinterpret_cast<F16Ctl*>(base + L.off_cu);
    const float2* p2 = reinterpret_cast<const float2*>(pts);
    const long long blocks = (n + kF16Threads - 1) / kF16Threads;
    const int grid_e = (int)std::min<long long>(blocks, (long long)sms * std::max(1, occ_e));
    const int grid_l = (int)std::min<long long>(blocks, (long long)sms * std::max(1, occ_l));
    f16_init<<<1, 32, 0, s>>>(c);
    {
        ProfScope p("filter16_extremes", s);
        f16_extremes<<<grid_e, kF16Threads, 0, s>>>(p2, n, c);
    }
    if (out_labels || out_counts4) {
        ProfScope p("filter16_labels", s);
        f16_labels<<<grid_l, kF16Threads, 0, s>>>(p2, n, c, out_labels);
    }
    f16_output<<<1, 32, 0, s>>>(c, out_ext16, out_counts4);
    return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ECUDA;
}
