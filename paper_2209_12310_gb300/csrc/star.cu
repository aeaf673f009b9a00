// star.cu -- the star pass: the filter polygon of dense data (star.cuh).
//
// star_kernel runs on a branch of its own beside the main pass (it needs only
// the sample octagon).  Each warp reads warp tiles of the input: first the
// sample pass's tiles (still in L2), then, in blocks whose first tiles showed
// dense data (more than 1/32 of the points outside the sample octagon),
// kStarExtraTiles more tiles spread over the input.  Every point outside the
// sample octagon goes to its angular bin around the sample octagon's centre
// c, where a 64-bit atomicMax keeps the point farthest from c (its squared
// distance, truncated, above its index).
//
// The block that finishes last decides: when the points it saw outside the
// sample octagon are more than 1/32 of those read (the main pass's own
// threshold for dense data), it builds the polygon:
//   1. each non-empty bin's point is re-read from the input by its index (so
//      every vertex is an input point of this call, whatever the bins held)
//      and kept if it is a valid coordinate and falls in that bin again;
//   2. the kept points, in bin order, are the vertices; kStarRounds rounds
//      each drop, first at even then at odd positions, the vertices that are
//      reflex or flat (orient(V_j-1, V_j, V_j+1) <= 0) when their neighbours
//      still turn by less than pi around c, which only enlarges the polygon;
//   3. it is accepted only if every wedge turns counter-clockwise by less
//      than pi (orient(c, V_j, V_j+1) > 0) and the wedges wind once around c
//      (exactly one edge crosses the ray from c along +x), so c is strictly
//      inside and the polygon is star-shaped around it;
//   4. the bin table and the repeated first two vertices complete StarPoly.
// The bins are left at zero for the next call.  Nothing here waits for
// another block.
#include "ch_internal.cuh"
#include "launch.h"
#include "octagon.cuh"
#include "star.cuh"
#include "tma.cuh"

namespace ch {

constexpr int kStarThreads = 128;
constexpr int kStarRounds = 4;
constexpr int kStarPer = kStarBins / kStarThreads;   // bins per thread of the building block
constexpr int kStarBatch = 8;                        // independent loads in flight per thread

struct StarWork {
    int2 va[kStarBins], vb[kStarBins];               // vertex lists (relative to c), ping-pong
    unsigned short ba[kStarBins], bb[kStarBins];     // their bins
};
constexpr size_t kStarWorkBytes = sizeof(StarWork);

// Warp tile of the star pass's k-th read: the sample pass's tiles first, then
// the extra tiles, half a stride away from an even spread.
__device__ __forceinline__ long long star_tile(long long k, long long nsamp, long long nextra, long long ntiles) {
    if (k < nsamp) return k * ntiles / nsamp;
    const long long e = k - nsamp;
    return ((2 * e + 1) * ntiles) / (2 * nextra);
}

// One warp tile: counts the points read and those outside the sample octagon
// (per lane), and bins the latter.
__device__ __forceinline__ void star_tile_pass(const float4* __restrict__ p4, long long t, int head, const int* s_in,
                                               const float* s_edge, int cx, int cy, unsigned long long* bins,
                                               unsigned& nout, unsigned long long pol) {
    const int lane = threadIdx.x & 31;
    const float4* base = p4 + t * kWarpTileF4 + lane;
    float4 v[kLoadsPerLane];
#pragma unroll
    for (int j = 0; j < kLoadsPerLane; ++j) v[j] = ld_stream_f4(base + j * 32, pol);
#pragma unroll
    for (int j = 0; j < kLoadsPerLane; ++j) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float x = h ? v[j].z : v[j].x, y = h ? v[j].w : v[j].y;
            const int X = __float2int_rn(x), Y = __float2int_rn(y);
            if (pt_in_inner(X, Y, s_in) || pt_in_sample(x, y, s_edge)) continue;
            const int dx = X - cx, dy = Y - cy;
            const unsigned long long d2 = (unsigned long long)((long long)dx * dx + (long long)dy * dy);
            const unsigned idx = (unsigned)(head + t * kWarpTilePts + 2 * (j * 32 + lane) + h);
            atomicMax(&bins[star_bin(dx, dy)], ((d2 >> 17) << 32) | idx);
            ++nout;
        }
    }
}

// Block-wide exclusive scan of one count per thread (warp shuffles, then the
// warp totals); returns the thread's offset and leaves the total in *total.
// s holds one word per warp.
__device__ __forceinline__ int star_scan(int c, unsigned* s, int* total) {
    constexpr int kWarps = kStarThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned incl = (unsigned)c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s[warp] = incl;
    __syncthreads();
    unsigned before = 0u, all = 0u;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const unsigned x = s[w];
        before += w < warp ? x : 0u;
        all += x;
    }
    if (threadIdx.x == 0) *total = (int)all;
    __syncthreads();
    return (int)(before + incl - (unsigned)c);
}

// The building block (the last to finish).  c = (cx, cy).
__device__ void star_build(const float* __restrict__ pts, long long n, Ctl* ctl, unsigned long long* bins,
                           StarPoly* poly, StarWork* w, int cx, int cy) {
    __shared__ unsigned s_scan[kStarThreads / 32];
    __shared__ int s_K, s_bad, s_cross;
    const int t = threadIdx.x;
    if (t == 0) { s_bad = 0; s_cross = 0; }
    // 1. re-read each non-empty bin's point; park (dx, dy) in vb by bin
    unsigned long long kept = 0ull;   // bit i: bin t * kStarPer + i holds a vertex
    for (int i0 = 0; i0 < kStarPer; i0 += kStarBatch) {
        unsigned long long key[kStarBatch];
#pragma unroll
        for (int i = 0; i < kStarBatch; ++i) key[i] = __ldcg(bins + t * kStarPer + i0 + i);
        float2 p[kStarBatch];
#pragma unroll
        for (int i = 0; i < kStarBatch; ++i) {
            const long long idx = (long long)(unsigned)key[i];
            p[i] = (key[i] != 0ull && idx < n) ? __ldcg(reinterpret_cast<const float2*>(pts) + idx)
                                               : make_float2(-1.0f, -1.0f);
        }
#pragma unroll
        for (int i = 0; i < kStarBatch; ++i) {
            const int b = t * kStarPer + i0 + i;
            if (key[i] != 0ull) bins[b] = 0ull;
            const int X = __float2int_rn(p[i].x), Y = __float2int_rn(p[i].y);
            const bool valid = __int2float_rn(X) == p[i].x && __int2float_rn(Y) == p[i].y &&
                               ((unsigned)(X | Y) >> kCoordBits) == 0u;
            if (key[i] != 0ull && valid && star_bin(X - cx, Y - cy) == b) {
                kept |= 1ull << (i0 + i);
                w->vb[b] = make_int2(X - cx, Y - cy);
            }
        }
    }
    int off = star_scan(__popcll(kept), s_scan, &s_K);
    for (int i = 0; i < kStarPer; ++i) {
        if ((kept >> i) & 1ull) {
            const int b = t * kStarPer + i;
            w->va[off] = w->vb[b];
            w->ba[off] = (unsigned short)b;
            ++off;
        }
    }
    __syncthreads();
    // 2. reflex-removal rounds, va/ba -> vb/bb -> va/ba ...
    int2* src = w->va;
    int2* dst = w->vb;
    unsigned short* bsrc = w->ba;
    unsigned short* bdst = w->bb;
    int idle = 0;   // consecutive sweeps that removed nothing
    for (int sweep = 0; sweep < 2 * kStarRounds && idle < 2; ++sweep) {
        const int K = s_K;
        if (K <= 3) break;
        const int par = sweep & 1;
        const int chunk = (K + kStarThreads - 1) / kStarThreads;   // <= kStarPer
        const int lo = t * chunk, hi = min(K, lo + chunk);
        unsigned long long keep = 0ull;
        for (int j0 = lo; j0 < hi; j0 += kStarBatch) {
            int2 a[kStarBatch], m[kStarBatch], z[kStarBatch];
#pragma unroll
            for (int i = 0; i < kStarBatch; ++i) {
                const int j = min(j0 + i, hi - 1);
                a[i] = src[j == 0 ? K - 1 : j - 1];
                m[i] = src[j];
                z[i] = src[j + 1 == K ? 0 : j + 1];
            }
#pragma unroll
            for (int i = 0; i < kStarBatch; ++i) {
                const int j = j0 + i;
                if (j >= hi) break;
                bool drop = (j & 1) == par && !((K & 1) && j == K - 1);
                if (drop) {
                    const long long turn = (long long)(m[i].x - a[i].x) * (z[i].y - a[i].y) -
                                           (long long)(m[i].y - a[i].y) * (z[i].x - a[i].x);
                    drop = turn <= 0 && star_orient_c(a[i], z[i].x, z[i].y) > 0;
                }
                if (!drop) keep |= 1ull << (j - lo);
            }
        }
        const int nk = __popcll(keep);
        __syncthreads();   // every read of K and src of this sweep is done
        int o = star_scan(nk, s_scan, &s_K);
        idle = s_K == K ? idle + 1 : 0;
        for (int j = lo; j < hi; ++j) {
            if ((keep >> (j - lo)) & 1ull) {
                dst[o] = src[j];
                bdst[o] = bsrc[j];
                ++o;
            }
        }
        __syncthreads();
        int2* tv = src; src = dst; dst = tv;
        unsigned short* tb = bsrc; bsrc = bdst; bdst = tb;
    }
    // 3. validation, 4. the table and the final vertex list
    const int K = s_K;
    const int chunk = (K + kStarThreads - 1) / kStarThreads;
    const int lo = t * chunk, hi = min(K, lo + chunk);
    int bad = 0, cross = 0;
    for (int j = lo; j < hi; ++j) {
        const int2 a = src[j], b = src[j + 1 == K ? 0 : j + 1];
        bad |= star_orient_c(a, b.x, b.y) <= 0;
        cross += (a.y < 0 && b.y >= 0) ? 1 : 0;
        poly->v[j] = a;
        const int b0 = bsrc[j];
        const int b1 = j + 1 < K ? (int)bsrc[j + 1] : (int)bsrc[0] + kStarBins;
        for (int b = b0 + 1; b <= b1; ++b) poly->tbl[b & (kStarBins - 1)] = (unsigned short)j;
    }
    if (bad) atomicOr(&s_bad, 1);
    if (cross) atomicAdd(&s_cross, cross);
    if (t == 0 && K >= 3) {
        poly->v[K] = src[0];
        poly->v[K + 1] = src[1];
    }
    __syncthreads();
    if (t == 0) {
        const bool ok = K >= 3 && !s_bad && s_cross == 1;
        ctl->star_k = K;
        ctl->star_cx = cx;
        ctl->star_cy = cy;
        __threadfence();
        ctl->star_ok = ok ? 1 : 0;
    }
}

__global__ void __launch_bounds__(kStarThreads, 5) star_kernel(const float* __restrict__ pts, long long n, int head,
                                                               long long ntiles, Ctl* ctl, unsigned long long* bins,
                                                               StarPoly* poly, StarWork* work) {
    __shared__ int s_in[8];
    __shared__ float s_edge[24];
    __shared__ int s_go, s_cx, s_cy, s_last;
    __shared__ unsigned s_pts, s_out;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = kStarThreads / 32;
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
    if (!last_block(&ctl->star_done, &s_last)) return;
    const unsigned tot_pts = *(volatile unsigned*)&ctl->star_pts;
    const unsigned tot_out = *(volatile unsigned*)&ctl->star_out;
    if (tot_out * 32ull > (unsigned long long)tot_pts && tot_out >= 1024u) {
        star_build(pts, n, ctl, bins, poly, work, s_cx, s_cy);
    } else if (tot_out > 0u) {   // a few points were binned: clear the bins for the next call
        for (int b = threadIdx.x; b < kStarBins; b += kStarThreads) bins[b] = 0ull;
    }
}

void launch_star(const float* pts, long long n, int head, long long ntiles, Ctl* ctl, void* bins, void* poly,
                 void* work, int grid, cudaStream_t s) {
    star_kernel<<<grid, kStarThreads, 0, s>>>(pts, n, head, ntiles, ctl, (unsigned long long*)bins, (StarPoly*)poly,
                                             (StarWork*)work);
}

size_t star_bins_bytes() { return sizeof(unsigned long long) * kStarBins; }
size_t star_poly_bytes() { return kStarPolyBytes; }
size_t star_work_bytes() { return kStarWorkBytes; }

}  // namespace ch
