// star.cu -- the star pass: the angular bins of the star polygon (star.cuh).
//
// star_kernel runs on a branch of its own beside the main pass (it needs only
// the sample octagon) and is small enough to share the SMs with it.  Each warp
// reads warp tiles of the input: first the sample pass's tiles (still in L2),
// then, in blocks whose first tiles showed dense data (more than 1/32 of the
// points outside the sample octagon), kStarExtraTiles more tiles spread over
// the input.  Every point outside the sample octagon goes to its angular bin
// around the sample octagon's centre c, where a 64-bit atomicMax keeps the
// point farthest from c (its squared distance, truncated, above its index);
// a point first reads its bin and issues the atomic only if it beats it.
//
// The block that finishes last decides: when the points seen outside the
// sample octagon are more than 1/32 of those read (the main pass's own
// threshold for dense data), it publishes c and the post pass builds the
// polygon from the bins (star_finish) and clears them; otherwise it clears
// the bins itself.  Nothing here waits for another block.
#include "ch_internal.cuh"
#include "launch.h"
#include "octagon.cuh"
#include "star.cuh"
#include "tma.cuh"

namespace ch {

constexpr int kStarThreads = 128;

// Warp tile of the star pass's k-th read: the sample pass's tiles first, then
// the extra tiles, half a stride away from an even spread.
__device__ __forceinline__ long long star_tile(long long k, long long nsamp, long long nextra, long long ntiles) {
    if (k < nsamp) return k * ntiles / nsamp;
    const long long e = k - nsamp;
    return ((2 * e + 1) * ntiles) / (2 * nextra);
}

// One warp tile: bins the points outside the sample octagon and counts them
// (per lane).
__device__ __forceinline__ void star_tile_pass(const float4* __restrict__ p4, long long t, int head, const int* s_in,
                                               const float* s_edge, int cx, int cy, unsigned long long* bins,
                                               unsigned& nout, unsigned long long pol) {
    const int lane = threadIdx.x & 31;
    const float4* base = p4 + t * kWarpTileF4 + lane;
    constexpr int kHalf = kLoadsPerLane / 2;   // half a tile's loads in flight keeps the registers low
#pragma unroll 1
    for (int j0 = 0; j0 < kLoadsPerLane; j0 += kHalf) {
        float4 v[kHalf];
#pragma unroll
        for (int j = 0; j < kHalf; ++j) v[j] = ld_stream_f4(base + (j0 + j) * 32, pol);
        // the keys of the points outside the sample octagon, then one load of
        // each point's bin: only a point that beats the bin's current value
        // issues the atomicMax (after a bin's first few points that is rare,
        // so far fewer atomics meet at each bin)
        unsigned long long key[2 * kHalf];
        int bin[2 * kHalf];
#pragma unroll
        for (int j = 0; j < kHalf; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float x = h ? v[j].z : v[j].x, y = h ? v[j].w : v[j].y;
                const int X = __float2int_rn(x), Y = __float2int_rn(y);
                const bool out = !pt_in_inner(X, Y, s_in) && !pt_in_sample(x, y, s_edge);
                const int dx = X - cx, dy = Y - cy;
                const unsigned long long d2 = (unsigned long long)((long long)dx * dx + (long long)dy * dy);
                const unsigned idx = (unsigned)(head + t * kWarpTilePts + 2 * ((j0 + j) * 32 + lane) + h);
                key[2 * j + h] = out ? ((d2 >> 17) << 32) | idx : 0ull;
                bin[2 * j + h] = star_bin(dx, dy);
                nout += out ? 1u : 0u;
            }
        }
        unsigned long long cur[2 * kHalf];
#pragma unroll
        for (int i = 0; i < 2 * kHalf; ++i) cur[i] = key[i] ? __ldcg(bins + bin[i]) : ~0ull;
#pragma unroll
        for (int i = 0; i < 2 * kHalf; ++i)
            if (key[i] > cur[i]) atomicMax(&bins[bin[i]], key[i]);
    }
}

__global__ void __launch_bounds__(kStarThreads, 8) star_kernel(const float* __restrict__ pts, long long n, int head,
                                                               long long ntiles, Ctl* ctl, unsigned long long* bins) {
    __shared__ int s_in[8];
    __shared__ float s_edge[24];
    __shared__ int s_go, s_cx, s_cy, s_last;
    __shared__ unsigned s_pts, s_out;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = kStarThreads / 32;
    CH_TL(ctl, 7, 0);
    if (threadIdx.x == 0) {
        s_go = *(volatile int*)&ctl->samp_ok;
        s_pts = 0u;
        s_out = 0u;
    }
    __syncthreads();
    const Octagon& o = ctl->oct_s;
    if (s_go) {
        if (threadIdx.x < 4) {
            s_in[threadIdx.x] = o.in_lo[threadIdx.x];
            s_in[4 + threadIdx.x] = o.in_hi[threadIdx.x];
        }
        if (threadIdx.x < 8) {
            s_edge[3 * threadIdx.x] = o.oct[threadIdx.x].A;
            s_edge[3 * threadIdx.x + 1] = o.oct[threadIdx.x].B;
            s_edge[3 * threadIdx.x + 2] = o.oct[threadIdx.x].C;
        }
        if (threadIdx.x == 0) {
            s_cx = (o.vx[W] + o.vx[E]) / 2;
            s_cy = (o.vy[S] + o.vy[N]) / 2;
        }
    }
    __syncthreads();
    const long long nsamp = s_go ? sample_tiles(ntiles) : 0;
    const long long nextra = s_go ? (ntiles < kStarExtraTiles ? ntiles : kStarExtraTiles) : 0;
    const float4* p4 = reinterpret_cast<const float4*>(pts + 2 * head);
    const unsigned long long pol = l2_evict_first();
    unsigned nout = 0u, npts = 0u;
    // tile k of a phase belongs to block k % grid, warp (k / grid) % kWarps
    const long long stride = (long long)gridDim.x * kWarps;
    for (long long k = blockIdx.x + (long long)gridDim.x * warp; k < nsamp; k += stride) {
        star_tile_pass(p4, star_tile(k, nsamp, nextra, ntiles), head, s_in, s_edge, s_cx, s_cy, bins, nout, pol);
        npts += 2 * kLoadsPerLane;
    }
    nout = __reduce_add_sync(0xFFFFFFFFu, nout);
    npts = __reduce_add_sync(0xFFFFFFFFu, npts);
    if (lane == 0 && npts) { atomicAdd(&s_pts, npts); atomicAdd(&s_out, nout); }
    __syncthreads();
    const bool dense = s_out * 32u > s_pts;   // this block's sample tiles
    __syncthreads();
    if (dense) {
        nout = 0u;
        npts = 0u;
        for (long long k = blockIdx.x + (long long)gridDim.x * warp; k < nextra; k += stride) {
            star_tile_pass(p4, star_tile(nsamp + k, nsamp, nextra, ntiles), head, s_in, s_edge, s_cx, s_cy, bins,
                           nout, pol);
            npts += 2 * kLoadsPerLane;
        }
        nout = __reduce_add_sync(0xFFFFFFFFu, nout);
        npts = __reduce_add_sync(0xFFFFFFFFu, npts);
        if (lane == 0 && npts) { atomicAdd(&s_pts, npts); atomicAdd(&s_out, nout); }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_pts) {
        atomicAdd(&ctl->star_pts, s_pts);
        atomicAdd(&ctl->star_out, s_out);
    }
    CH_TL(ctl, 7, 1);
    if (!last_block(&ctl->star_done, &s_last)) return;
    const unsigned tot_pts = *(volatile unsigned*)&ctl->star_pts;
    const unsigned tot_out = *(volatile unsigned*)&ctl->star_out;
    if (tot_out * 32ull > (unsigned long long)tot_pts && tot_out >= 1024u) {
        if (threadIdx.x == 0) {   // dense: the post pass builds the polygon (and clears the bins)
            ctl->star_cx = s_cx;
            ctl->star_cy = s_cy;
            __threadfence();
            ctl->star_ok = 1;
        }
    } else if (tot_out > 0u) {   // a few points were binned: clear the bins for the next call
        for (int b = threadIdx.x; b < kStarBins; b += kStarThreads) bins[b] = 0ull;
    }
    CH_TL(ctl, 7, 1);
}

void launch_star(const float* pts, long long n, int head, long long ntiles, Ctl* ctl, void* bins, int grid,
                 cudaStream_t s) {
    star_kernel<<<grid, kStarThreads, 0, s>>>(pts, n, head, ntiles, ctl, (unsigned long long*)bins);
}

// The star pass shares SMs with the main pass: an SM that takes a star block
// first must keep its shared memory at the maximum split, or the main pass's
// blocks (91 KB each) cannot join it until the star block has left.
cudaError_t configure_star_kernel() {
    return cudaFuncSetAttribute(star_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

size_t star_bins_bytes() { return sizeof(unsigned long long) * kStarBins; }

}  // namespace ch
