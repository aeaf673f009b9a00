// bucket.cu -- hull of many survivors without a full sort.
//
// The queue chains need the survivors in u order only up to the chain: the
// lower chain of a set of points equals the lower chain of the chains of any
// partition of it into u-ranges, joined in u order.  So instead of sorting
// every record (three radix passes), each queue's u-range is cut into
// buckets of about kBkAvg records (equal width in u; the queue frames make
// the density along u nearly flat for points near the hull), the records are
// scattered by bucket (one counting pass, one scatter pass), and one warp per
// bucket computes the bucket's lower chain in shared memory by quickhull
// rounds.  The bucket chains, a few vertices each, then enter the merge tree
// of chain_kernel as its leaves.
//   bk_prep     buckets per queue from the records' queue counts; counters
//               cleared;
//   bk_hist     records per bucket;
//   bk_bsum, bk_bstart  each bucket's range, in bucket order (block sums,
//               then per-block scans offset by the sums before them);
//   bk_part1    records to the scratch buffer grouped by coarse group (2^shift
//               consecutive buckets): ranks from shared-memory atomics, one
//               global atomic per group and chunk of 8192 records;
//   bk_part2    one block per coarse group moves its records back into their
//               buckets' ranges (shared-memory cursors only), so the record
//               buffer still holds every record for the sort-based path;
//   bk_hull     one warp per bucket: its lower chain (at most kBkChain
//               vertices; more sends the call to the sort-based path).
#include "ch_internal.cuh"
#include "hullcore.cuh"
#include "host.h"
#include "launch.h"
#include "bkwarp.cuh"
#include "partition.cuh"

#include <climits>

namespace ch {

constexpr int kBkWarps = 8;             // warps per bk_hull block
constexpr int kBkAllocThreads = 1024;
constexpr int kBkShiftMax = 11;         // at most 2048 buckets per coarse group
static_assert(kBkCoarseMax <= kPtGroups && (1 << kBkShiftMax) <= kPtGroups, "partition groups");
static_assert(kBkCoarseMax % kPtThreads == 0, "bk_items scan");
constexpr int kBkUnroll = 8;            // records per thread and step (bk_hist)

// Bucket of a record in queue r (monotone in u; the same float arithmetic in
// every kernel, so every kernel agrees).
struct BkParams {
    unsigned base[5], nb[4];
    int lo[4];
    float scale[4];
};

__device__ __forceinline__ void bk_load_params(const Ctl* ctl, BkParams& p) {
    for (int r = 0; r < 4; ++r) {
        p.base[r] = ctl->bk_base[r];
        p.nb[r] = ctl->bk_nb[r];
        p.lo[r] = ctl->bk_lo[r];
        p.scale[r] = ctl->bk_scale[r];
    }
    p.base[4] = ctl->bk_base[4];
}

__device__ __forceinline__ unsigned bk_bucket(const BkParams& p, uint32_t key) {
    const int r = (int)(key >> kKeyBits);
    const int u = (int)(key & kKeyMask);
    int b = (int)((float)(u - p.lo[r]) * p.scale[r]);
    b = b < 0 ? 0 : b;
    b = b >= (int)p.nb[r] ? (int)p.nb[r] - 1 : b;
    return p.base[r] + (unsigned)b;
}

__global__ void bk_prep(Ctl* ctl, unsigned* bcount, unsigned bmax) {
    __shared__ unsigned s_q[4], s_base[5];
    __shared__ int s_go;
    const int tid = threadIdx.x;
    if (tid == 0) s_go = !*(volatile int*)&ctl->done && read_status(ctl) == CH_OK;
    if (tid < 4) s_q[tid] = 0u;
    __syncthreads();
    if (!s_go) return;
    if (tid < 4) s_q[tid] = ctl->rec_q[tid];
    __syncthreads();
    if (tid == 0) {
        // Records that a star polygon left are mostly near the hull, so a
        // bucket of kBkAvg of them would hold too many chain vertices: then
        // at most kBkNearHull records per bucket, when that fits the
        // workspace's bucket capacity.
        const bool near_hull = *(volatile int*)&ctl->star_final != 0;
        unsigned tot_near = 0u;
        for (int r = 0; r < 4; ++r) {
            const unsigned nb = bk_buckets_for(s_q[r]);
            const unsigned nh = (s_q[r] + kBkNearHull - 1) / kBkNearHull;
            tot_near += nb > nh ? nb : nh;
        }
        const bool use_near = near_hull && tot_near <= bmax;
        s_base[0] = 0u;
        for (int r = 0; r < 4; ++r) {
            unsigned nb = bk_buckets_for(s_q[r]);
            const unsigned nh = (s_q[r] + kBkNearHull - 1) / kBkNearHull;
            if (use_near && nh > nb) nb = nh;
            s_base[r + 1] = s_base[r] + nb;
        }
    }
    __syncthreads();
    const unsigned nbk = s_base[4];
    if (nbk > bmax) {   // cannot happen with the workspace's bucket capacity
        if (blockIdx.x == 0 && tid == 0) ctl->bk_state = 2;
        return;
    }
    for (unsigned b = blockIdx.x * blockDim.x + tid; b < nbk; b += gridDim.x * blockDim.x) bcount[b] = 0u;
    if (blockIdx.x == 0 && tid < 4) {
        const int r = tid, a = 2 * r, b = (2 * r + 2) & 7;
        uint32_t ulo, uhi, v;
        queue_frame(r, ctl->oct.vx[a], ctl->oct.vy[a], ulo, v);
        queue_frame(r, ctl->oct.vx[b], ctl->oct.vy[b], uhi, v);
        const unsigned nb = s_base[r + 1] - s_base[r];
        ctl->bk_nb[r] = nb;
        ctl->bk_base[r] = s_base[r];
        ctl->bk_lo[r] = (int)ulo;
        const long long span = (long long)uhi - (long long)ulo + 1;
        ctl->bk_scale[r] = span > 0 ? (float)nb / (float)span : 0.0f;
        if (r == 0) {
            // about as many coarse groups as buckets per group: the runs of
            // both partition levels are then about equally long
            int shift = 0;
            while (((nbk + (1u << shift) - 1) >> shift) > (2u << shift)) ++shift;
            ctl->bk_shift = shift;
            ctl->bk_base[4] = nbk;
            ctl->bk_cursor = 0u;
            ctl->bk_next = 0u;
            ctl->bk_state = shift <= kBkShiftMax && ((nbk + (1u << shift) - 1) >> shift) <= (unsigned)kBkCoarseMax ? 1 : 2;
        }
    }
}

__global__ void __launch_bounds__(256) bk_hist(Ctl* ctl, const uint32_t* keys, unsigned* bcount) {
    __shared__ BkParams s_p;
    __shared__ int s_go;
    __shared__ unsigned s_n;
    if (threadIdx.x == 0) {
        s_go = *(volatile int*)&ctl->bk_state == 1 && !*(volatile int*)&ctl->done;
        s_n = ctl->count;
        bk_load_params(ctl, s_p);
    }
    __syncthreads();
    if (!s_go) return;
    const unsigned n = s_n;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * kBkUnroll) {
        uint32_t k[kBkUnroll];
#pragma unroll
        for (int j = 0; j < kBkUnroll; ++j) {
            const unsigned i = i0 + j * stride;
            if (i < n) k[j] = __ldcs(keys + i);
        }
#pragma unroll
        for (int j = 0; j < kBkUnroll; ++j)
            if (i0 + j * stride < n) atomicAdd(&bcount[bk_bucket(s_p, k[j])], 1u);
    }
}

// Bucket ranges in bucket order: per block of kBkAllocThreads buckets its sum
// (bk_bsum), then each block adds the sums before it to its own exclusive
// scan (bk_bstart); coarse-group cursors start at their first bucket.
__global__ void __launch_bounds__(kBkAllocThreads) bk_bsum(Ctl* ctl, const unsigned* bcount, unsigned* bsum) {
    __shared__ int s_go, s_tmp[33];
    __shared__ unsigned s_nb;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_go = *(volatile int*)&ctl->bk_state == 1 && !*(volatile int*)&ctl->done;
        s_nb = ctl->bk_base[4];
    }
    __syncthreads();
    if (!s_go) return;
    for (unsigned b0 = blockIdx.x * kBkAllocThreads; b0 < s_nb; b0 += gridDim.x * kBkAllocThreads) {
        const unsigned b = b0 + tid;
        int tot;
        block_excl_scan(b < s_nb ? (int)bcount[b] : 0, s_tmp, &tot);
        if (tid == 0) bsum[b0 / kBkAllocThreads] = (unsigned)tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBkAllocThreads) bk_bstart(Ctl* ctl, const unsigned* bcount, const unsigned* bsum,
                                                            unsigned* bstart, unsigned* bcur, unsigned* gcur) {
    __shared__ int s_go, s_tmp[33];
    __shared__ unsigned s_nb, s_pre[32];
    __shared__ int s_shift;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_go = *(volatile int*)&ctl->bk_state == 1 && !*(volatile int*)&ctl->done;
        s_nb = ctl->bk_base[4];
        s_shift = ctl->bk_shift;
    }
    __syncthreads();
    if (!s_go) return;
    for (unsigned b0 = blockIdx.x * kBkAllocThreads; b0 < s_nb; b0 += gridDim.x * kBkAllocThreads) {
        const unsigned blk = b0 / kBkAllocThreads;
        unsigned pre = 0u;   // sum of the block sums before this block
        for (unsigned j = tid; j < blk; j += kBkAllocThreads) pre += bsum[j];
#pragma unroll
        for (int o = 16; o; o >>= 1) pre += __shfl_xor_sync(0xFFFFFFFFu, pre, o);
        if (lane == 0) s_pre[warp] = pre;
        __syncthreads();
        pre = 0u;
        for (int w = 0; w < kBkAllocThreads / 32; ++w) pre += s_pre[w];
        const unsigned b = b0 + tid;
        int tot;
        const int ex = block_excl_scan(b < s_nb ? (int)bcount[b] : 0, s_tmp, &tot);
        if (b < s_nb) {
            bstart[b] = pre + (unsigned)ex;
            bcur[b] = pre + (unsigned)ex;
            if ((b & ((1u << s_shift) - 1u)) == 0u) gcur[b >> s_shift] = pre + (unsigned)ex;
        }
        __syncthreads();
    }
}

// Tiles of the second level: items (group c, tile t), item_start[c] the
// first item of group c.
__global__ void __launch_bounds__(kPtThreads) bk_items(Ctl* ctl, const unsigned* bcount, const unsigned* bstart,
                                                     unsigned* item_start) {
    __shared__ int s_go, s_shift, s_tmp[33];
    __shared__ unsigned s_nb;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_go = *(volatile int*)&ctl->bk_state == 1 && !*(volatile int*)&ctl->done;
        s_nb = ctl->bk_base[4];
        s_shift = ctl->bk_shift;
    }
    __syncthreads();
    if (!s_go) return;
    const unsigned nb = s_nb, nc = (nb + (1u << s_shift) - 1u) >> s_shift;
    constexpr int kE = kBkCoarseMax / kPtThreads;
    unsigned t[kE], part = 0u;
#pragma unroll
    for (int e = 0; e < kE; ++e) {
        const unsigned c = tid * kE + e;
        t[e] = 0u;
        if (c < nc) {
            const unsigned b0 = c << s_shift, b1 = min(nb, b0 + (1u << s_shift));
            const unsigned len = bstart[b1 - 1] + bcount[b1 - 1] - bstart[b0];
            t[e] = (len + kPtTile - 1) / kPtTile;
        }
        part += t[e];
    }
    int tot;
    unsigned run = (unsigned)block_excl_scan((int)part, s_tmp, &tot);
#pragma unroll
    for (int e = 0; e < kE; ++e) {
        const unsigned c = tid * kE + e;
        if (c < nc) item_start[c] = run;
        run += t[e];
    }
    if (tid == 0) {
        item_start[nc] = (unsigned)tot;
        ctl->bk_cursor = (unsigned)tot;
    }
}

// First level: tiles of the record buffer by coarse group (bucket >> shift);
// each nonempty group of a tile reserves its run on the group's cursor.
__global__ void __launch_bounds__(kPtThreads, 1) bk_part1(Ctl* ctl, const uint32_t* kin, const uint64_t* vin,
                                                         unsigned* gcur, uint32_t* kout, uint64_t* vout) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    PartSmem& sm = *reinterpret_cast<PartSmem*>(s_dyn);
    __shared__ BkParams s_p;
    __shared__ int s_go, s_shift;
    __shared__ unsigned s_n, s_nc;
    if (threadIdx.x == 0) {
        s_go = *(volatile int*)&ctl->bk_state == 1 && !*(volatile int*)&ctl->done;
        s_n = ctl->count;
        s_shift = ctl->bk_shift;
        bk_load_params(ctl, s_p);
        s_nc = (s_p.base[4] + (1u << s_shift) - 1u) >> s_shift;
    }
    __syncthreads();
    if (!s_go) return;
    const unsigned n = s_n;
    const int shift = s_shift;
    for (unsigned i0 = blockIdx.x * kPtTile; i0 < n; i0 += gridDim.x * kPtTile)
        partition_tile(
            sm, kin, vin, i0, min((unsigned)kPtTile, n - i0), s_nc,
            [&](uint32_t key) { return bk_bucket(s_p, key) >> shift; },
            [&](unsigned g, unsigned c) { return atomicAdd(&gcur[g], c); }, kout, vout);
}

// Second level: each tile of one coarse group's range by bucket; each
// nonempty bucket of a tile reserves its run on the bucket's cursor.
__global__ void __launch_bounds__(kPtThreads, 1) bk_part2(Ctl* ctl, const uint32_t* kin, const uint64_t* vin,
                                                         const unsigned* bstart, const unsigned* bcount,
                                                         const unsigned* item_start, unsigned* bcur, uint32_t* kout,
                                                         uint64_t* vout) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    PartSmem& sm = *reinterpret_cast<PartSmem*>(s_dyn);
    __shared__ BkParams s_p;
    __shared__ int s_go, s_shift;
    __shared__ unsigned s_nc, s_items, s_c;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_go = *(volatile int*)&ctl->bk_state == 1 && !*(volatile int*)&ctl->done;
        s_shift = ctl->bk_shift;
        bk_load_params(ctl, s_p);
        s_nc = (s_p.base[4] + (1u << s_shift) - 1u) >> s_shift;
        s_items = ctl->bk_cursor;
    }
    __syncthreads();
    if (!s_go) return;
    const int shift = s_shift;
    const unsigned nb = s_p.base[4];
    for (unsigned it = blockIdx.x; it < s_items; it += gridDim.x) {
        if (tid == 0) {   // the item's group: last c with item_start[c] <= it
            unsigned lo = 0u, hi = s_nc;
            while (hi - lo > 1u) {
                const unsigned mid = (lo + hi) >> 1;
                if (item_start[mid] <= it) lo = mid; else hi = mid;
            }
            s_c = lo;
        }
        __syncthreads();
        const unsigned c = s_c;
        const unsigned b0 = c << shift, b1 = min(nb, b0 + (1u << shift));
        const unsigned gend = bstart[b1 - 1] + bcount[b1 - 1];
        const unsigned i0 = bstart[b0] + (it - item_start[c]) * kPtTile;
        partition_tile(
            sm, kin, vin, i0, min((unsigned)kPtTile, gend - i0), b1 - b0,
            [&](uint32_t key) { return bk_bucket(s_p, key) - b0; },
            [&](unsigned g, unsigned cnt) { return atomicAdd(&bcur[b0 + g], cnt); }, kout, vout);
    }
}

__global__ void __launch_bounds__(kBkWarps * 32, 4) bk_hull(Ctl* ctl, const uint32_t* keys, const uint64_t* vals,
                                                        const unsigned* bstart, const unsigned* bcount,
                                                        int* bu, int* bv, int* bi, int* blen) {
    __shared__ BkWarp s_w[kBkWarps];
    __shared__ int s_go;
    __shared__ unsigned s_nb;
    if (threadIdx.x == 0) {
        s_go = *(volatile int*)&ctl->bk_state == 1 && !*(volatile int*)&ctl->done;
        s_nb = ctl->bk_base[4];
    }
    __syncthreads();
    if (!s_go) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BkWarp& w = s_w[warp];
    for (;;) {   // buckets taken one at a time: sizes differ
        unsigned b = 0u;
        if (lane == 0) b = atomicAdd(&ctl->bk_next, 1u);
        b = __shfl_sync(0xFFFFFFFFu, b, 0);
        if (b >= s_nb) break;
        int len = bk_bucket_chain(w, keys, vals, bstart[b], bcount[b]);
        if (len < 0) {
            if (lane == 0) ctl->bk_state = 2;   // the sort-based path takes over
            len = 0;
        }
        const size_t o = (size_t)b * kBkChain;
        for (int j = lane; j < len; j += 32) {
            bu[o + j] = w.cu[j];
            bv[o + j] = w.cv[j];
            bi[o + j] = w.ci[j];
        }
        if (lane == 0) blen[b] = len;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
static int g_occ_bk_hull = 1;   // resident bk_hull blocks per SM (set by configure_bucket_kernels)

void launch_bucket_pass(Ctl* ctl, uint32_t* kA, uint64_t* vA, uint32_t* kB, uint64_t* vB, unsigned* bcount,
                        unsigned* bcur, unsigned* bstart, unsigned* bsum, int* bu, int* bv, int* bi, int* blen,
                        unsigned bmax, int sms, cudaStream_t s) {
    unsigned* gcur = bsum + bmax / kBkAllocThreads + 2;
    unsigned* item_start = gcur + kBkCoarseMax;
    { ProfScope p("bk_prep", s); bk_prep<<<sms, 256, 0, s>>>(ctl, bcount, bmax); }
    { ProfScope p("bk_hist", s); bk_hist<<<sms * 8, 256, 0, s>>>(ctl, kA, bcount); }
    {
        ProfScope p("bk_scan", s);
        bk_bsum<<<sms, kBkAllocThreads, 0, s>>>(ctl, bcount, bsum);
        bk_bstart<<<sms, kBkAllocThreads, 0, s>>>(ctl, bcount, bsum, bstart, bcur, gcur);
        bk_items<<<1, kPtThreads, 0, s>>>(ctl, bcount, bstart, item_start);
    }
    // records A -> B by coarse group, then B -> A by bucket
    {
        ProfScope p("bk_part1", s);
        bk_part1<<<sms, kPtThreads, sizeof(PartSmem), s>>>(ctl, kA, vA, gcur, kB, vB);
    }
    {
        ProfScope p("bk_part2", s);
        bk_part2<<<sms, kPtThreads, sizeof(PartSmem), s>>>(ctl, kB, vB, bstart, bcount, item_start, bcur, kA, vA);
    }
    {
        ProfScope p("bk_hull", s);
        // one wave of resident warps that take buckets from a counter
        bk_hull<<<sms * g_occ_bk_hull, kBkWarps * 32, 0, s>>>(ctl, kA, vA, bstart, bcount, bu, bv, bi, blen);
    }
}

#ifdef CH_PHASEPROF
}  // namespace ch
extern "C" int ch_phase_read(unsigned long long* out16) {
    return cudaMemcpyFromSymbol(out16, ch::g_bk_phase, sizeof(unsigned long long) * 16) == cudaSuccess ? 0 : -4;
}
extern "C" int ch_phase_reset(void) {
    unsigned long long z[16] = {};
    return cudaMemcpyToSymbol(ch::g_bk_phase, z, sizeof(z)) == cudaSuccess ? 0 : -4;
}
namespace ch {
#endif

cudaError_t configure_bucket_kernels() {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bk_hull, kBkWarps * 32, 0);
    if (e != cudaSuccess) return e;
    g_occ_bk_hull = occ > 0 ? occ : 1;
    e = cudaFuncSetAttribute(bk_part1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PartSmem));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(bk_part2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PartSmem));
}

}  // namespace ch
