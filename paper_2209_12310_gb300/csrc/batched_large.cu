// batched_large.cu -- the sets of a batch whose survivors exceed one block,
// all at once (the bucketed large-survivor path of bucket.cu and hull.cu,
// segmented by set).  A segment is one (set, queue) pair.
//   btl_prep     per segment: bucket count from its record count, bucket and
//                chain-tile offsets (prefix over all segments), the bucket
//                map (u range, scale); record tiles per set;
//   btl_hist     record tiles: records per bucket;
//   btl_alloc    bucket ranges in the scatter buffer;
//   btl_scatter  record tiles: records into their bucket's range;
//   btl_bucket_hull  one warp per bucket: its lower chain;
//   btl_chain    chain tiles: bucket chains merged up each segment's tree;
//                the block completing a set's fourth root joins its chains.
// A set whose bucket chains overflow is left to the single-hull path (the
// host reads the per-set flags after the launches).
#include "batched_large.h"
#include "bkwarp.cuh"
#include "ch_internal.cuh"
#include "host.h"
#include "hullcore.cuh"
#include "launch.h"
#include "merge.cuh"

#include <algorithm>

namespace ch {

constexpr int kBLWarps = 8;

// Exclusive prefix in place over n entries by one block of 1024 threads
// (contiguous chunks per thread); returns the total in every thread.
__device__ unsigned block_prefix_inplace(unsigned* a, int n, unsigned* s_part, int* map = nullptr,
                                        unsigned map_cap = 0u) {
    const int tid = threadIdx.x;
    const int per = (n + 1023) / 1024;
    const int lo = tid * per, hi = min(n, lo + per);
    unsigned sum = 0u;
    for (int j = lo; j < hi; ++j) sum += a[j];
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
        const unsigned c = a[j];
        a[j] = run;
        if (map)   // the entry owning each unit (never past the map's capacity)
            for (unsigned t = 0; t < c && run + t < map_cap; ++t) map[run + t] = j;
        run += c;
    }
    const unsigned total = s_part[1023];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(1024) btl_prep(BLArgs a) {
    __shared__ unsigned s_part[1024];
    const int tid = threadIdx.x;
    const int nseg = 4 * a.k;
    for (int sg = tid; sg < nseg; sg += 1024) {
        const int i = sg >> 2, q = sg & 3;
        unsigned nb = 0u;
        if (a.big[i]) {
            const Ctl* c = a.ctl + i;
            nb = bk_buckets_for(c->counts4[q]);
            // Records that a star polygon left are mostly near the hull, a
            // large share of them hull vertices: 16 of them per bucket, or
            // 32 or kBkNearHull (64) when the smaller size does not fit the
            // set's share of the workspace (n / kBkAvg + 4 kBkMinQ + 4
            // buckets): 16 fits with at most n / 16 records left, 32 with
            // n / 8, 64 with n / 4.
            const long long ni = a.offsets[i + 1] - a.offsets[i];
            const long long m = c->count;
            if (c->star_k > 0 && 4 * m <= ni) {
                unsigned per = kBkNearHull / 4;
                while (per < (unsigned)kBkNearHull && (long long)(kBkAvg / per) * m > ni) per *= 2;
                const unsigned nh = (c->counts4[q] + per - 1) / per;
                nb = nb > nh ? nb : nh;
            }
            const int va = 2 * q, vb = (2 * q + 2) & 7;
            uint32_t ulo, uhi, v;
            queue_frame(q, c->oct.vx[va], c->oct.vy[va], ulo, v);
            queue_frame(q, c->oct.vx[vb], c->oct.vy[vb], uhi, v);
            const long long span = (long long)uhi - (long long)ulo + 1;
            a.seg_lo[sg] = (int)ulo;
            a.seg_scale[sg] = span > 0 ? (float)nb / (float)span : 0.0f;
        }
        a.seg_nb[sg] = nb;
        a.seg_bbase[sg] = nb;
        a.seg_tbase[sg] = (nb + kBkGroup - 1) / kBkGroup;
    }
    for (int i = tid; i < a.k; i += 1024) {
        Ctl* c = a.ctl + i;
        a.rt_base[i] = a.big[i] ? (c->count + kBLTile - 1) / kBLTile : 0u;
        if (a.big[i]) {
            c->bk_state = 1;
            c->blocks_done[3] = 0u;
        }
    }
    __syncthreads();
    const unsigned nb_total = block_prefix_inplace(a.seg_bbase, nseg, s_part);
    const unsigned nt_total = block_prefix_inplace(a.seg_tbase, nseg, s_part, a.ct_map, a.tcap);
    const unsigned rt_total = block_prefix_inplace(a.rt_base, a.k, s_part, a.rt_map, a.rtcap);
    if (tid == 0) {
        a.totals[4] = 0u;
        a.totals[5] = 0u;   // next bucket for a btl_bucket warp
        const bool fits = nb_total <= a.bcap && nt_total <= a.tcap;   // always, by the workspace bounds
        a.seg_bbase[nseg] = fits ? nb_total : 0u;
        a.seg_tbase[nseg] = fits ? nt_total : 0u;
        a.rt_base[a.k] = fits ? rt_total : 0u;
        a.totals[0] = fits ? nb_total : 0u;
        a.totals[1] = fits ? nt_total : 0u;
        a.totals[2] = fits ? rt_total : 0u;
        a.totals[3] = fits ? 1u : 0u;
    }
}

struct BLTileCtx {
    int set;
    long long rb;   // region base of the set's records
    unsigned r0, r1;
    unsigned bbase[4], nb[4];
    int lo[4];
    float scale[4];
};

__device__ __forceinline__ void btl_tile_ctx(const BLArgs& a, unsigned t, BLTileCtx& x) {
    const int i = a.rt_map[t];
    x.set = i;
    x.rb = a.offsets[i] + 16ll * i;
    const unsigned cnt = a.ctl[i].count;
    x.r0 = (t - a.rt_base[i]) * (unsigned)kBLTile;
    x.r1 = min(cnt, x.r0 + (unsigned)kBLTile);
    for (int q = 0; q < 4; ++q) {
        x.bbase[q] = a.seg_bbase[4 * i + q];
        x.nb[q] = a.seg_nb[4 * i + q];
        x.lo[q] = a.seg_lo[4 * i + q];
        x.scale[q] = a.seg_scale[4 * i + q];
    }
}

__device__ __forceinline__ unsigned btl_bucket(const BLTileCtx& x, uint32_t key) {
    const int q = (int)(key >> kKeyBits);
    const int u = (int)(key & kKeyMask);
    int b = (int)((float)(u - x.lo[q]) * x.scale[q]);
    b = b < 0 ? 0 : b;
    b = b >= (int)x.nb[q] ? (int)x.nb[q] - 1 : b;
    return x.bbase[q] + (unsigned)b;
}

__global__ void __launch_bounds__(256) btl_hist(BLArgs a) {
    __shared__ BLTileCtx s_x;
    const unsigned nt = a.totals[2];
    for (unsigned t = blockIdx.x; t < nt; t += gridDim.x) {
        if (threadIdx.x == 0) btl_tile_ctx(a, t, s_x);
        __syncthreads();
        for (unsigned j = s_x.r0 + threadIdx.x; j < s_x.r1; j += blockDim.x)
            atomicAdd(&a.bcount[btl_bucket(s_x, __ldcs(a.keys + s_x.rb + j))], 1u);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) btl_alloc(BLArgs a) {
    __shared__ int s_tmp[33];
    __shared__ unsigned s_base;
    const unsigned nb = a.totals[0];
    const int tid = threadIdx.x;
    for (unsigned b0 = blockIdx.x * 1024u; b0 < nb; b0 += gridDim.x * 1024u) {
        const unsigned b = b0 + tid;
        const int c = b < nb ? (int)a.bcount[b] : 0;
        int tot;
        const int ex = block_excl_scan(c, s_tmp, &tot);
        if (tid == 0) s_base = tot ? atomicAdd(&a.totals[4], (unsigned)tot) : 0u;
        __syncthreads();
        if (b < nb) a.bstart[b] = s_base + (unsigned)ex;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) btl_scatter(BLArgs a) {
    __shared__ BLTileCtx s_x;
    const unsigned nt = a.totals[2];
    for (unsigned t = blockIdx.x; t < nt; t += gridDim.x) {
        if (threadIdx.x == 0) btl_tile_ctx(a, t, s_x);
        __syncthreads();
        for (unsigned j = s_x.r0 + threadIdx.x; j < s_x.r1; j += blockDim.x) {
            const uint32_t k = __ldcs(a.keys + s_x.rb + j);
            const uint64_t w = __ldcs(a.vals + s_x.rb + j);
            const unsigned b = btl_bucket(s_x, k);
            const unsigned pos = a.bstart[b] + atomicAdd(&a.bcur[b], 1u);
            a.kP[pos] = k;
            a.vP[pos] = w;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBLWarps * 32, 4) btl_bucket_hull(BLArgs a) {
    __shared__ BkWarp s_w[kBLWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BkWarp& w = s_w[warp];
    const unsigned nb = a.totals[0];
    for (;;) {   // buckets taken one at a time: sizes differ
        unsigned b = 0u;
        if (lane == 0) b = atomicAdd(&a.totals[5], 1u);
        b = __shfl_sync(0xFFFFFFFFu, b, 0);
        if (b >= nb) break;
        const int len = bk_bucket_chain(w, a.kP, a.vP, a.bstart[b], a.bcount[b]);
        const size_t o = (size_t)b * kBkChain;
        for (int j = lane; j < len; j += 32) {
            a.bu[o + j] = w.cu[j];
            a.bv[o + j] = w.cv[j];
            a.bi[o + j] = w.ci[j];
        }
        if (lane == 0) a.blen[b] = len;   // -1: overflow, the set takes the single-hull path
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kChainThreads) btl_chain(BLArgs a) {
    extern __shared__ int smem[];
    int* su = smem;
    int* sv = su + kMergeSmemCap;
    int* si = sv + kMergeSmemCap;
    __shared__ int s_len[kChainThreads];
    __shared__ int s_red[4];
    __shared__ int s_old, s_seg, s_fail;
    __shared__ int s_mv[kChainThreads / 2][3];
    const int tid = threadIdx.x;
    const unsigned ntiles = a.totals[1];
    const TreeBufs tb{a.cu, a.cv, a.ci, a.clen, a.counters, (int)a.tcap};
    for (unsigned c = blockIdx.x; c < ntiles; c += gridDim.x) {
        if (tid == 0) {
            s_seg = a.ct_map[c];
            s_fail = 0;
        }
        __syncthreads();
        const int sg = s_seg, i = sg >> 2;
        const unsigned rb = a.seg_tbase[sg], ct = a.seg_tbase[sg + 1] - rb, t_local = c - rb;
        const unsigned b0 = a.seg_bbase[sg] + t_local * kBkGroup, b1 = a.seg_bbase[sg + 1];
        int len = 0;
        if (tid < kBkGroup && b0 + tid < b1) {
            len = __ldcg(a.blen + b0 + tid);
            if (len < 0) {
                s_fail = 1;
                len = 0;
            }
        }
        s_len[tid] = len;
        {   // the tile's bucket chain slots are contiguous: coalesced block copy
            const unsigned nb_t = b1 > b0 ? min(b1 - b0, (unsigned)kBkGroup) : 0u;
            const size_t o0 = (size_t)b0 * kBkChain;
            for (unsigned e = tid; e < nb_t * kBkChain; e += blockDim.x) {
                su[e] = __ldcg(a.bu + o0 + e);
                sv[e] = __ldcg(a.bv + o0 + e);
                si[e] = __ldcg(a.bi + o0 + e);
            }
        }
        __syncthreads();
        if (s_fail && tid == 0) atomicExch(&a.ctl[i].bk_state, 2);
        const bool root = tile_merge_climb(su, sv, si, s_len, s_mv, kBkChain, kBkGroup, tb, c, rb, ct, t_local,
                                           s_red, &s_old);
        __syncthreads();
        if (!root) continue;
        // the block completing the set's fourth queue root joins its chains
        __threadfence();
        __syncthreads();
        if (tid == 0) s_old = (int)atomicAdd(&a.ctl[i].blocks_done[3], 1u);
        __syncthreads();
        if (s_old != 3) continue;
        CH_MG_DECL
        __threadfence();
        if (tid == 0) s_fail = *(volatile int*)&a.ctl[i].bk_state == 2;
        __syncthreads();
        if (s_fail) continue;   // the host redoes this set
        const unsigned t0 = a.seg_tbase[4 * i];
        int off[5];
        off[0] = 0;
        for (int q = 0; q < 4; ++q) off[q + 1] = off[q] + __ldcg(a.clen + a.seg_tbase[4 * i + q]) - 1;
        const int m = off[4];
        const long long base = a.offsets[i], ni = a.offsets[i + 1] - base;
        const long long rbase = base + 16ll * i;
        const unsigned cnt = a.ctl[i].count;
        if (m < 0 || m > (int)cnt) {   // inconsistent state: report, never read out of range
            if (tid == 0) { set_status(a.ctl + i, CH_ECUDA); a.out_n[i] = CH_ECUDA; }
            continue;
        }
        // the cycle (index, x, y) into the set's record region, free by now
        int* V = reinterpret_cast<int*>(a.keys + rbase);
        int* X = reinterpret_cast<int*>(a.vals + rbase);
        int* Y = X + m;
        for (int q = 0; q < 4; ++q) {
            const size_t o = (size_t)a.seg_tbase[4 * i + q] * kChainTile;
            for (int j = tid; j < off[q + 1] - off[q]; j += blockDim.x) {
                int x, y;
                frame_to_xy(q, __ldcg(a.cu + o + j), __ldcg(a.cv + o + j), x, y);
                V[off[q] + j] = __ldcg(a.ci + o + j);
                X[off[q] + j] = x;
                Y[off[q] + j] = y;
            }
        }
        __syncthreads();
        // flag / comp scratch: the set's chain storage (its roots are copied out)
        int* flag = a.cu + (size_t)t0 * kChainTile;
        int* comp = a.cv + (size_t)t0 * kChainTile;
        stitch_core(V, m, flag, comp,
                    [&](int p, long long& x, long long& y) { x = __ldcg(X + p); y = __ldcg(Y + p); }, ni,
                    a.ctl + i, a.out_idx + base, a.out_n + i);
        __syncthreads();
        CH_MG(7);   // debug builds: the set's join and stitch
    }
}

// Sets flagged large whose bucket chains overflowed: 1 (redo on the host).
__global__ void btl_flags(BLArgs a, unsigned char* redo) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.k) return;
    redo[i] = (a.big[i] && (*(volatile int*)&a.ctl[i].bk_state == 2 || a.totals[3] == 0u)) ? 1 : 0;
}

static int g_occ_bucket_hull = 1;   // resident btl_bucket_hull blocks per SM (set by configure_batched_large)

void launch_batched_large(const BLArgs& a, unsigned char* redo, int sms, cudaStream_t s) {
    { ProfScope p("bl_prep", s); btl_prep<<<1, 1024, 0, s>>>(a); }
    { ProfScope p("bl_hist", s); btl_hist<<<sms * 8, 256, 0, s>>>(a); }
    { ProfScope p("bl_alloc", s); btl_alloc<<<sms, 1024, 0, s>>>(a); }
    { ProfScope p("bl_scatter", s); btl_scatter<<<sms * 8, 256, 0, s>>>(a); }
    {
        ProfScope p("bl_bucket", s);
        // one wave of resident warps that take buckets from a counter
        btl_bucket_hull<<<sms * g_occ_bucket_hull, kBLWarps * 32, 0, s>>>(a);
    }
    { ProfScope p("bl_chain", s); btl_chain<<<sms * 2, kChainThreads, chain_smem_bytes(), s>>>(a); }
    btl_flags<<<(a.k + 255) / 256, 256, 0, s>>>(a, redo);
}

cudaError_t configure_batched_large() {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, btl_bucket_hull, kBLWarps * 32, 0);
    if (e != cudaSuccess) return e;
    g_occ_bucket_hull = occ > 0 ? occ : 1;
    return cudaFuncSetAttribute(btl_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chain_smem_bytes());
}

}  // namespace ch

#ifdef CH_PHASEPROF
// Debug builds: the merge tree's phase cycles of the batched path (this
// translation unit's copy of the counters).
extern "C" int ch_phase_read_batched_merge(unsigned long long* out16) {
    return cudaMemcpyFromSymbol(out16, ch::g_mg_phase, sizeof(unsigned long long) * 16) == cudaSuccess ? 0 : -4;
}
extern "C" int ch_phase_reset_batched_merge(void) {
    unsigned long long z[16] = {};
    return cudaMemcpyToSymbol(ch::g_mg_phase, z, sizeof(z)) == cudaSuccess ? 0 : -4;
}
#endif
