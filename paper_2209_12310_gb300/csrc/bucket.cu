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
//   bk_alloc    each bucket's range in the scatter buffer (block scans, one
//               atomic per block: bucket ranges need not be in bucket order);
//   bk_scatter  records into their bucket's range;
//   bk_hull     one warp per bucket: its lower chain (at most kBkChain
//               vertices; more sends the call to the sort-based path).
#include "ch_internal.cuh"
#include "hullcore.cuh"
#include "host.h"
#include "launch.h"
#include "bkwarp.cuh"

#include <climits>

namespace ch {

constexpr int kBkWarps = 8;             // warps per bk_hull block
constexpr int kBkAllocThreads = 1024;
constexpr int kBkUnroll = 8;            // records per thread and step (hist, scatter)

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

__global__ void bk_prep(Ctl* ctl, unsigned* bcount, unsigned* bcur, unsigned bmax) {
    __shared__ unsigned s_q[4], s_base[5];
    __shared__ int s_go;
    const int tid = threadIdx.x;
    if (tid == 0) s_go = !*(volatile int*)&ctl->done && read_status(ctl) == CH_OK;
    if (tid < 4) s_q[tid] = 0u;
    __syncthreads();
    if (!s_go) return;
    for (int d = tid; d < kDigits; d += blockDim.x) {
        const unsigned c = ctl->digit_hist[kSortPasses - 1][d];
        if (c) atomicAdd(&s_q[d >> (kDigitBits - 2)], c);
    }
    __syncthreads();
    if (tid == 0) {
        s_base[0] = 0u;
        for (int r = 0; r < 4; ++r) {
            s_base[r + 1] = s_base[r] + bk_buckets_for(s_q[r]);
        }
    }
    __syncthreads();
    const unsigned nbk = s_base[4];
    if (nbk > bmax) {   // cannot happen with the workspace's bucket capacity
        if (blockIdx.x == 0 && tid == 0) ctl->bk_state = 2;
        return;
    }
    for (unsigned b = blockIdx.x * blockDim.x + tid; b < nbk; b += gridDim.x * blockDim.x) {
        bcount[b] = 0u;
        bcur[b] = 0u;
    }
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
            ctl->bk_base[4] = nbk;
            ctl->bk_cursor = 0u;
            ctl->bk_state = 1;
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

__global__ void __launch_bounds__(kBkAllocThreads) bk_alloc(Ctl* ctl, const unsigned* bcount, unsigned* bstart) {
    __shared__ int s_go, s_tmp[33];
    __shared__ unsigned s_nb, s_base;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_go = *(volatile int*)&ctl->bk_state == 1 && !*(volatile int*)&ctl->done;
        s_nb = ctl->bk_base[4];
    }
    __syncthreads();
    if (!s_go) return;
    for (unsigned b0 = blockIdx.x * kBkAllocThreads; b0 < s_nb; b0 += gridDim.x * kBkAllocThreads) {
        const unsigned b = b0 + tid;
        const int c = b < s_nb ? (int)bcount[b] : 0;
        int tot;
        const int ex = block_excl_scan(c, s_tmp, &tot);
        if (tid == 0) s_base = tot ? atomicAdd(&ctl->bk_cursor, (unsigned)tot) : 0u;
        __syncthreads();
        if (b < s_nb) bstart[b] = s_base + (unsigned)ex;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) bk_scatter(Ctl* ctl, const uint32_t* kin, const uint64_t* vin,
                                                  const unsigned* bstart, unsigned* bcur, uint32_t* kout,
                                                  uint64_t* vout) {
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
    // kBkUnroll records per thread and step, their atomics in flight together
    // (each returns the record's slot; a lone atomic per step leaves the
    // pass waiting on one round trip at a time).
    const unsigned n = s_n;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * kBkUnroll) {
        uint32_t k[kBkUnroll];
        uint64_t w[kBkUnroll];
        unsigned pos[kBkUnroll];
#pragma unroll
        for (int j = 0; j < kBkUnroll; ++j) {
            const unsigned i = i0 + j * stride;
            if (i < n) {
                k[j] = __ldcs(kin + i);
                w[j] = __ldcs(vin + i);
            }
        }
#pragma unroll
        for (int j = 0; j < kBkUnroll; ++j) {
            const unsigned i = i0 + j * stride;
            if (i < n) {
                const unsigned b = bk_bucket(s_p, k[j]);
                pos[j] = bstart[b] + atomicAdd(&bcur[b], 1u);
            }
        }
#pragma unroll
        for (int j = 0; j < kBkUnroll; ++j) {
            const unsigned i = i0 + j * stride;
            if (i < n) {
                kout[pos[j]] = k[j];
                vout[pos[j]] = w[j];
            }
        }
    }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBkWarps * 32) bk_hull(Ctl* ctl, const uint32_t* keys, const uint64_t* vals,
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
    const unsigned nwarps = gridDim.x * kBkWarps;
    for (unsigned b = blockIdx.x * kBkWarps + warp; b < s_nb; b += nwarps) {
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
void launch_bucket_pass(Ctl* ctl, const uint32_t* kA, const uint64_t* vA, uint32_t* kB, uint64_t* vB,
                        unsigned* bcount, unsigned* bcur, unsigned* bstart, int* bu, int* bv, int* bi, int* blen,
                        unsigned bmax, int sms, cudaStream_t s) {
    { ProfScope p("bk_prep", s); bk_prep<<<sms, 256, 0, s>>>(ctl, bcount, bcur, bmax); }
    { ProfScope p("bk_hist", s); bk_hist<<<sms * 8, 256, 0, s>>>(ctl, kA, bcount); }
    { ProfScope p("bk_alloc", s); bk_alloc<<<sms, kBkAllocThreads, 0, s>>>(ctl, bcount, bstart); }
    { ProfScope p("bk_scatter", s); bk_scatter<<<sms * 8, 256, 0, s>>>(ctl, kA, vA, bstart, bcur, kB, vB); }
    {
        ProfScope p("bk_hull", s);
        bk_hull<<<sms * 4, kBkWarps * 32, 0, s>>>(ctl, kB, vB, bstart, bcount, bu, bv, bi, blen);
    }
}

cudaError_t configure_bucket_kernels() { return cudaSuccess; }

}  // namespace ch
