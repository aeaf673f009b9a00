// manhattan.cu -- ch_filter_manhattan: the paper's two-kernel findExtremes
// (Sec. 3), kept as an ablation of the fused single pass.
//
// The paper finds the extreme points in two steps: a first kernel reduces
// the axis extremes (minimum and maximum x and y: W, E, S, N), which give the
// bounding box; a second kernel then finds, for each corner of that box, the
// point of minimum Manhattan distance to it (SW, SE, NE, NW).  Each kernel
// streams every point once, so the input is read twice (16 bytes a point),
// where the fused main pass of ch_filter reads it once: every point lies in
// the box, so the distance to corner (xmax, ymax) is (xmax - x) + (ymax - y),
// which the fused pass minimises as the maximum of x + y (and likewise for
// the other corners).  Both forms select the same points, ties going to the
// lowest index.  The octagon and the label array are then built exactly as
// for ch_filter.
#include "ch_internal.cuh"
#include "host.h"
#include "launch.h"
#include "octagon.cuh"

#include <algorithm>

namespace ch {
namespace {

constexpr int kMhThreads = 256;
constexpr int kMhUnroll = 4;   // points in flight per thread

// Packed (key, lowest index): the larger packed value wins; minima pass the
// complement of their key, and every index is complemented.
__device__ __forceinline__ unsigned long long mh_pack(unsigned key, bool is_max, unsigned idx) {
    const unsigned hk = is_max ? key : 0xFFFFFFFFu - key;
    return ((unsigned long long)hk << 32) | (unsigned long long)(0xFFFFFFFFu - idx);
}

__device__ __forceinline__ unsigned mh_index(unsigned long long p) { return 0xFFFFFFFFu - (unsigned)p; }

// Block reduction of 4 packed maxima into slots[0..3] of the control block.
__device__ __forceinline__ void mh_reduce4(unsigned long long (&best)[4], unsigned long long* slots) {
    __shared__ unsigned long long s_red[kMhThreads / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        unsigned long long p = best[d];
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long q = __shfl_xor_sync(0xFFFFFFFFu, p, o);
            p = q > p ? q : p;
        }
        if (lane == 0) s_red[warp][d] = p;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        unsigned long long m = 0ull;
        for (int w = 0; w < kMhThreads / 32; ++w) m = s_red[w][threadIdx.x] > m ? s_red[w][threadIdx.x] : m;
        if (m) atomicMax(&slots[threadIdx.x], m);
    }
}

// Kernel 1: axis extremes W (min x), E (max x), S (min y), N (max y) into
// ext_packed[0..3], and the validity of every coordinate.
__global__ void __launch_bounds__(kMhThreads) mh_axis_kernel(const float2* __restrict__ pts, long long n, Ctl* ctl) {
    unsigned long long best[4] = {0ull, 0ull, 0ull, 0ull};
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * kMhUnroll) {
        float2 p[kMhUnroll];
#pragma unroll
        for (int u = 0; u < kMhUnroll; ++u) {
            const long long i = i0 + u * stride;
            p[u] = i < n ? __ldg(pts + i) : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < kMhUnroll; ++u) {
            const long long i = i0 + u * stride;
            if (i >= n) continue;
            const int X = __float2int_rn(p[u].x), Y = __float2int_rn(p[u].y);
            bad |= (__int2float_rn(X) != p[u].x) | (__int2float_rn(Y) != p[u].y) |
                   ((((unsigned)X | (unsigned)Y) >> kCoordBits) != 0u);
            const unsigned idx = (unsigned)i;
            const unsigned long long c[4] = {mh_pack((unsigned)X, false, idx), mh_pack((unsigned)X, true, idx),
                                             mh_pack((unsigned)Y, false, idx), mh_pack((unsigned)Y, true, idx)};
#pragma unroll
            for (int d = 0; d < 4; ++d) best[d] = c[d] > best[d] ? c[d] : best[d];
        }
    }
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) set_status(ctl, CH_ERANGE);
    mh_reduce4(best, ctl->ext_packed);
}

// Kernel 2: per corner of the box from kernel 1, the point of minimum
// Manhattan distance: SW (xmin, ymin), SE (xmax, ymin), NE (xmax, ymax),
// NW (xmin, ymax) into ext_packed[4..7].  The last block builds the octagon
// of the 8 points (in ch_filter's order W, SW, S, SE, E, NE, N, NW).
__global__ void __launch_bounds__(kMhThreads) mh_corner_kernel(const float2* __restrict__ pts, long long n, Ctl* ctl) {
    __shared__ int s_box[4], s_last;
    __shared__ Octagon s_o;
    if (threadIdx.x < 4) {   // xmin, xmax, ymin, ymax from the axis extremes' points
        const unsigned i = mh_index(*(volatile unsigned long long*)&ctl->ext_packed[threadIdx.x]);
        const float2 p = pts[i];
        s_box[threadIdx.x] = __float2int_rn(threadIdx.x < 2 ? p.x : p.y);
    }
    __syncthreads();
    const int xmin = s_box[0], xmax = s_box[1], ymin = s_box[2], ymax = s_box[3];
    unsigned long long best[4] = {0ull, 0ull, 0ull, 0ull};
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (read_status(ctl) == CH_OK) {
        for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * kMhUnroll) {
            float2 p[kMhUnroll];
#pragma unroll
            for (int u = 0; u < kMhUnroll; ++u) {
                const long long i = i0 + u * stride;
                p[u] = i < n ? __ldg(pts + i) : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int u = 0; u < kMhUnroll; ++u) {
                const long long i = i0 + u * stride;
                if (i >= n) continue;
                const int X = __float2int_rn(p[u].x), Y = __float2int_rn(p[u].y);
                const unsigned idx = (unsigned)i;
                // Manhattan distances to the four corners (every point is in the box)
                const unsigned long long c[4] = {mh_pack((unsigned)((X - xmin) + (Y - ymin)), false, idx),
                                                 mh_pack((unsigned)((xmax - X) + (Y - ymin)), false, idx),
                                                 mh_pack((unsigned)((xmax - X) + (ymax - Y)), false, idx),
                                                 mh_pack((unsigned)((X - xmin) + (ymax - Y)), false, idx)};
#pragma unroll
                for (int d = 0; d < 4; ++d) best[d] = c[d] > best[d] ? c[d] : best[d];
            }
        }
    }
    mh_reduce4(best, ctl->ext_packed + 4);
    if (!last_block(&ctl->blocks_done[1], &s_last)) return;
    if (__syncthreads_or(read_status(ctl) != CH_OK)) return;
    __shared__ int s_vx[8], s_vy[8], s_id[8];
    if (threadIdx.x < 8) {
        // slots: 0 W, 1 E, 2 S, 3 N, 4 SW, 5 SE, 6 NE, 7 NW -> octagon order
        const int slot_of_dir[8] = {0, 4, 2, 5, 1, 6, 3, 7};
        const unsigned i = mh_index(*(volatile unsigned long long*)&ctl->ext_packed[slot_of_dir[threadIdx.x]]);
        const float2 p = pts[i];
        s_id[threadIdx.x] = (int)i;
        s_vx[threadIdx.x] = __float2int_rn(p.x);
        s_vy[threadIdx.x] = __float2int_rn(p.y);
    }
    __syncthreads();
    setup_octagon_block(s_o, s_vx, s_vy, s_id, true);   // with the inner region, as ch_filter's label pass uses
    copy_octagon(&ctl->oct, &s_o);
}

__global__ void mh_init_kernel(Ctl* ctl) {
    const int t = threadIdx.x;
    if (t < 8) ctl->ext_packed[t] = 0ull;
    if (t < 4) { ctl->counts4[t] = 0u; ctl->blocks_done[t] = 0u; }
    if (t == 0) { ctl->status = CH_OK; ctl->abort = 0; }
}

}  // namespace
}  // namespace ch

using namespace ch;

extern "C" int ch_filter_manhattan(const float* pts, int64_t n, int32_t* out_ext8, uint8_t* out_labels,
                                   int64_t* out_counts4, void* stream) {
    int st = check_points_args(pts, n);
    if (st != CH_OK) return st;
    if (!out_ext8) return CH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        if (cudaMemsetAsync(out_ext8, 0xFF, 8 * sizeof(int32_t), s) != cudaSuccess) return CH_ECUDA;
        if (out_counts4 && cudaMemsetAsync(out_counts4, 0, 4 * sizeof(int64_t), s) != cudaSuccess) return CH_ECUDA;
        return CH_OK;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CH_ECUDA;
    char* base = nullptr;
    Layout L;
    if ((st = get_workspace(dev, s, n, &base, &L)) != CH_OK) return st;
    Ctl* ctl = (Ctl*)(base + L.off_ctl);
    const float2* p2 = reinterpret_cast<const float2*>(pts);
    const long long want = (n + (long long)kMhThreads * kMhUnroll - 1) / ((long long)kMhThreads * kMhUnroll);
    const int grid = (int)std::max(1ll, std::min(want, (long long)sms * 8));
    mh_init_kernel<<<1, 32, 0, s>>>(ctl);
    { ProfScope p("manhattan_axis", s); mh_axis_kernel<<<grid, kMhThreads, 0, s>>>(p2, n, ctl); }
    { ProfScope p("manhattan_corner", s); mh_corner_kernel<<<grid, kMhThreads, 0, s>>>(p2, n, ctl); }
    if (out_labels || out_counts4) {
        ProfScope p("labels", s);
        int mainb = 1, lab = 1;
        if (occupancy_filter(&mainb, &lab) != cudaSuccess) return CH_ECUDA;
        launch_labels(pts, n, ctl, out_labels, sms * std::max(1, lab), s);
    }
    launch_filter_output(ctl, n, out_ext8, out_counts4, s);
    return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ECUDA;
}
