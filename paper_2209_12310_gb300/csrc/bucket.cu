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

#include <climits>

namespace ch {

constexpr int kBkPer = 9;               // records per lane
constexpr int kBkWCap = 32 * kBkPer;    // records a warp holds at once
constexpr int kBkV = kBkChain + 2;      // quickhull vertices of one bucket
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
            const unsigned nb = (s_q[r] + kBkAvg - 1) / kBkAvg;
            s_base[r + 1] = s_base[r] + (nb > 0u ? nb : 1u);
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
// One warp's quickhull over m <= kBkWCap records of one queue frame: the
// lower chain from S (minimum u, v, index) to E (maximum u, then minimum v,
// index); the same rounds and tie rules as qh_chains, synchronised within the
// warp only.  The records live in registers (slot k of lane l is record
// 32 k + l), so a round's loads are only of the few chain vertices.
struct BkWarp {   // shared memory of one warp: the chain under construction
    unsigned long long segmax[kBkV], segarg[kBkV];
    int vu[kBkV], vv[kBkV], vi[kBkV], vnext[kBkV], splitu[kBkV], child[kBkV];
    int cu[kBkV], cv[kBkV], ci[kBkV];   // the finished chain in order
};

struct BkRecs {
    int u[kBkPer], v[kBkPer], i[kBkPer], s[kBkPer];
};

__device__ __forceinline__ long long bk_depth(const BkWarp& w, int a, int b, int u, int v) {
    return (long long)(w.vv[b] - w.vv[a]) * (u - w.vu[a]) - (long long)(w.vu[b] - w.vu[a]) * (v - w.vv[a]);
}

// Returns the chain length, its vertices in order in w.cu / cv / ci; -1 when
// the chain would exceed kBkV vertices.
__device__ int bk_warp_chain(BkWarp& w, BkRecs& R, int m) {
    const int lane = threadIdx.x & 31;
    constexpr unsigned long long kVMask = (1ull << kKeyBits) - 1ull;
    unsigned long long ks = ~0ull, ke = 0ull;
#pragma unroll
    for (int k = 0; k < kBkPer; ++k) {
        if (k * 32 + lane < m) {
            const unsigned long long a = ((unsigned long long)R.u[k] << kKeyBits) | (unsigned)R.v[k];
            const unsigned long long b = ((unsigned long long)R.u[k] << kKeyBits) | (kVMask - (unsigned)R.v[k]);
            ks = a < ks ? a : ks;
            ke = b > ke ? b : ke;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xFFFFFFFFu, ks, o), b = __shfl_xor_sync(0xFFFFFFFFu, ke, o);
        ks = a < ks ? a : ks;
        ke = b > ke ? b : ke;
    }
    unsigned is = 0xFFFFFFFFu, ie = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < kBkPer; ++k) {
        if (k * 32 + lane < m) {
            const unsigned long long a = ((unsigned long long)R.u[k] << kKeyBits) | (unsigned)R.v[k];
            const unsigned long long b = ((unsigned long long)R.u[k] << kKeyBits) | (kVMask - (unsigned)R.v[k]);
            if (a == ks) is = min(is, (unsigned)R.i[k]);
            if (b == ke) ie = min(ie, (unsigned)R.i[k]);
        }
    }
    is = __reduce_min_sync(0xFFFFFFFFu, is);
    ie = __reduce_min_sync(0xFFFFFFFFu, ie);
    const int su = (int)(ks >> kKeyBits), eu = (int)(ke >> kKeyBits);
    for (int a = lane; a < kBkV; a += 32) {
        w.segmax[a] = 0ull;
        w.segarg[a] = ~0ull;
        w.splitu[a] = -1;
    }
    if (lane == 0) {
        w.vu[0] = su;
        w.vv[0] = (int)(ks & kVMask);
        w.vi[0] = (int)is;
        w.vu[1] = eu;
        w.vv[1] = (int)(kVMask - (ke & kVMask));
        w.vi[1] = (int)ie;
        w.vnext[0] = su < eu ? 1 : -1;
        w.vnext[1] = -1;
    }
#pragma unroll
    for (int k = 0; k < kBkPer; ++k)
        R.s[k] = (k * 32 + lane < m && su < R.u[k] && R.u[k] < eu) ? 0 : -1;
    __syncwarp();
    int nv = 2;
    for (int round = 0;; ++round) {
        // depths; each segment's maximum
#pragma unroll
        for (int k = 0; k < kBkPer; ++k) {
            int a = R.s[k];
            if (a >= 0) {
                const int sp = w.splitu[a];
                if (sp >= 0) {
                    if (R.u[k] > sp) a = w.child[a];
                    else if (R.u[k] == sp) a = -1;
                }
                const int b = a >= 0 ? w.vnext[a] : -1;
                if (b < 0) {
                    a = -1;
                } else {
                    const long long d = bk_depth(w, a, b, R.u[k], R.v[k]);
                    if (d <= 0) a = -1;
                    else if ((unsigned long long)d > *(volatile unsigned long long*)&w.segmax[a])
                        atomicMax(&w.segmax[a], (unsigned long long)d);
                }
                R.s[k] = a;
            }
        }
        __syncwarp();
        // the deepest record per segment: smallest u, then index
#pragma unroll
        for (int k = 0; k < kBkPer; ++k) {
            const int a = R.s[k];
            if (a >= 0 && (unsigned long long)bk_depth(w, a, w.vnext[a], R.u[k], R.v[k]) == w.segmax[a])
                atomicMin(&w.segarg[a], ((unsigned long long)R.u[k] << 31) | (unsigned)R.i[k]);
        }
        __syncwarp();
        int added = 0;
        bool over = false;
        for (int a0 = 0; a0 < nv; a0 += 32) {
            const int a = a0 + lane;
            const unsigned long long dm = a < nv ? w.segmax[a] : 0ull;
            const bool split = dm != 0ull;
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, split);
            if (a < nv) w.splitu[a] = -1;
            if (split) {
                const int f = nv + added + __popc(bal & lanemask_lt());
                if (f < kBkV) {
                    const int b = w.vnext[a];
                    const unsigned long long key = w.segarg[a];
                    const int fu = (int)(key >> 31), fi = (int)(key & 0x7FFFFFFFull);
                    const long long num = (long long)(w.vv[b] - w.vv[a]) * (fu - w.vu[a]) - (long long)dm;
                    w.vu[f] = fu;
                    w.vv[f] = w.vv[a] + (int)(num / (long long)(w.vu[b] - w.vu[a]));
                    w.vi[f] = fi;
                    w.vnext[f] = b;
                    w.vnext[a] = f;
                    w.child[a] = f;
                    w.splitu[a] = fu;
                } else {
                    over = true;
                }
                w.segmax[a] = 0ull;
                w.segarg[a] = ~0ull;
            }
            added += __popc(bal);
        }
        if (__any_sync(0xFFFFFFFFu, over)) return -1;
        __syncwarp();
        if (added == 0) break;
        nv += added;
        if (round + 1 >= kBkV) return -1;
    }
    int len = 0;
    if (lane == 0)
        for (int a = 0; a >= 0 && len < kBkV; a = w.vnext[a], ++len) {
            w.cu[len] = w.vu[a];
            w.cv[len] = w.vv[a];
            w.ci[len] = w.vi[a];
        }
    len = __shfl_sync(0xFFFFFFFFu, len, 0);
    __syncwarp();
    return len;
}

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
        const unsigned start = bstart[b], cnt = bcount[b];
        int len = 0;   // chain vertices carried into the next chunk (w.cu / cv / ci)
        bool fail = false;
        for (unsigned c0 = 0; c0 < cnt;) {
            const unsigned take = min(cnt - c0, (unsigned)(kBkWCap - len));
            const int m = len + (int)take;
            BkRecs R;
#pragma unroll
            for (int k = 0; k < kBkPer; ++k) {
                const int j = k * 32 + lane;
                R.u[k] = 0;
                R.v[k] = 0;
                R.i[k] = 0;
                if (j < len) {
                    R.u[k] = w.cu[j];
                    R.v[k] = w.cv[j];
                    R.i[k] = w.ci[j];
                } else if (j < m) {
                    const unsigned g = start + c0 + (unsigned)(j - len);
                    const uint32_t kk = __ldcs(keys + g);
                    const uint64_t vv = __ldcs(vals + g);
                    R.u[k] = (int)(kk & kKeyMask);
                    R.v[k] = (int)(vv >> 31);
                    R.i[k] = (int)(vv & 0x7FFFFFFFull);
                }
            }
            __syncwarp();
            const int l2 = bk_warp_chain(w, R, m);
            if (l2 < 0 || l2 > kBkChain) { fail = true; break; }
            len = l2;
            c0 += take;
        }
        if (fail) {
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
