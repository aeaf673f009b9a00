// hull.cu -- hull of the sorted survivors on the device.
//
// The paper ends with "for i = 1..4: CH <- CH U hull(Q_i, n_i)" (Alg. 1): one
// hull per queue, joined.  Here every queue r is a chain from quad vertex r
// to quad vertex r+1 that is strictly monotone in the queue-frame coordinate u
// (see queue_frame), and its hull chain is Andrew's lower chain (Table I) in
// the (u, v) frame:
//   chain_kernel   queue boundaries from the top-digit histogram; per tile
//                  of 4096 records: keep the minimum-(v, index)
//                  record of every run of equal u (only it can be a vertex),
//                  build per-thread chains, merge them pairwise in shared
//                  memory, then merge tiles pairwise up a binary tree: the
//                  block that completes a pair (second arrival on an atomic
//                  counter) performs that merge, so no block ever waits;
//                  the block completing the fourth queue root joins the
//                  chains (stitch_core: collinear junction vertices dropped,
//                  degenerate cases, rotation to the lex-smallest vertex).
//
// Merging two chains A, B (all u of A below all u of B): a_k (k > 0) stays iff
// every b in B is strictly left of a_{k-1} -> a_k; b_l (l < |B|-1) stays iff
// every a in A is strictly left of b_l -> b_{l+1}.  Both predicates hold on a
// prefix of A / a suffix of B, and "every b" reduces to the minimum of a
// linear function over the convex chain B, found by binary search.
#include "ch_internal.cuh"
#include "hullcore.cuh"
#include "launch.h"

#include <climits>

namespace ch {

// Block-cooperative bridge: repeated 256-way probing of the monotone keep
// predicates (each probe is a sequential binary search over the other chain).
template <bool kGlobal>
__device__ void bridge_block(const ChainPtr& A, int la, const ChainPtr& B, int lb, int& is, int& js,
                             int* s_red) {
    const int T = blockDim.x;
    // A: largest k with keep_a(k); predicate true on [0, is]
    int lo = 0, hi = la - 1;
    while (lo < hi) {
        const long long span = (long long)hi - lo;
        const int k = lo + 1 + (int)(span * threadIdx.x / T);   // probes in (lo, hi]
        const bool ok = (k <= hi) && keep_a<kGlobal>(A, k, B, lb);
        if (threadIdx.x == 0) { s_red[0] = lo; s_red[1] = hi; }
        __syncthreads();
        if (k <= hi) {
            if (ok) atomicMax(&s_red[0], k);
            else atomicMin(&s_red[1], k - 1);
        }
        __syncthreads();
        const int nlo = s_red[0], nhi = s_red[1];
        __syncthreads();
        lo = nlo; hi = max(nhi, nlo);
    }
    is = lo;
    lo = 0; hi = lb - 1;   // smallest l with keep_b(l); true on [js, lb-1]
    while (lo < hi) {
        const long long span = (long long)hi - lo;
        const int l = lo + (int)(span * threadIdx.x / T);       // probes in [lo, hi)
        const bool ok = (l < hi) && keep_b<kGlobal>(A, la, B, l, lb);
        if (threadIdx.x == 0) { s_red[0] = lo; s_red[1] = hi; }
        __syncthreads();
        if (l < hi) {
            if (ok) atomicMin(&s_red[1], l);
            else atomicMax(&s_red[0], l + 1);
        }
        __syncthreads();
        const int nlo = s_red[0], nhi = s_red[1];
        __syncthreads();
        hi = nhi; lo = min(nlo, nhi);
    }
    js = lo;
}

// ---------------------------------------------------------------------------
struct HullBufs {
    const uint32_t* keys;   // sorted records (sort-based path)
    const uint64_t* vals;
    const int* bu;          // bucket chains (bucketed path): bucket b at [b*kBkChain, ...)
    const int* bv;
    const int* bi;
    const int* blen;
    int* cu;                // chain storage: tile c at [c*kChainTile, ...)
    int* cv;
    int* ci;
    int* clen;
    int* counters;          // merge-tree arrival counters (zero at rest)
    int ctcap;
    int* vbuf;              // stitch scratch (2 * records ints)
    int* kbuf;              // stitch scratch (records ints)
    int* xbuf;              // stitch coordinates (records ints each)
    int* ybuf;
    const float* pts;
    long long n;
    int32_t* out_idx;
    int64_t* out_n;
};

// Block-wide forward copy of n entries, dst <= src (possibly overlapping),
// in chunks fully loaded before they are stored.
__device__ void copy_down(int* du, int* dv, int* di, const int* su, const int* sv, const int* si, int n) {
    for (int base = 0; base < n; base += blockDim.x) {
        const int j = base + threadIdx.x;
        int a = 0, b = 0, c = 0;
        if (j < n) { a = __ldcg(su + j); b = __ldcg(sv + j); c = __ldcg(si + j); }
        __syncthreads();
        if (j < n) { du[j] = a; dv[j] = b; di[j] = c; }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kChainThreads) chain_kernel(Ctl* ctl, HullBufs hb) {
    extern __shared__ int smem[];
    int* su = smem;
    int* sv = su + kMergeSmemCap;
    int* si = sv + kMergeSmemCap;
    __shared__ int s_len[kChainThreads];
    __shared__ int s_red[4];
    __shared__ int s_old;
    __shared__ unsigned s_qn[4], s_q0[5], s_tb[5];
    __shared__ int s_mv[kChainThreads / 2][3];   // per pair: destination, source, count

    if (*(volatile int*)&ctl->done) return;
    const int st0 = read_status(ctl);
    if (st0 != CH_OK) {   // a sort pass gave up (timed-out wait): report it
        if (blockIdx.x == 0 && threadIdx.x == 0) *hb.out_n = st0;
        return;
    }
    const int tid = threadIdx.x;
    // Bucketed input: the leaves are bucket chains, kBkGroup per tile; queue
    // r owns buckets [bk_base[r], bk_base[r+1]).  Sorted input: queue r holds
    // the top-pass digits [128 r, 128 (r + 1)), so its size is a sum of that
    // histogram.
    const bool bk = *(volatile int*)&ctl->bk_state == 1;
    if (tid < 4) s_qn[tid] = 0u;
    __syncthreads();
    if (bk) {
        if (tid < 4) s_qn[tid] = ctl->bk_base[tid + 1] - ctl->bk_base[tid];
    } else {
        for (int d = tid; d < kDigits; d += blockDim.x) {
            const unsigned c = ctl->digit_hist[kSortPasses - 1][d];
            if (c) atomicAdd(&s_qn[d >> (kDigitBits - 2)], c);
        }
    }
    __syncthreads();
    if (tid == 0) {
        const unsigned per = bk ? (unsigned)kBkGroup : (unsigned)kChainTile;
        unsigned q = 0, tb = 0;
        for (int r = 0; r < 4; ++r) {
            s_q0[r] = q;
            s_tb[r] = tb;
            q += s_qn[r];
            tb += (s_qn[r] + per - 1) / per;
        }
        s_q0[4] = q;
        s_tb[4] = tb;
    }
    __syncthreads();
    const unsigned total_tiles = s_tb[4];
    const unsigned nrec = ctl->count;
    const int seg = bk ? kBkChain : kChainItems;           // shared-memory slot per leaf chain
    const int nseg = bk ? kBkGroup : kChainThreads;        // leaf chains per tile

    for (unsigned c = blockIdx.x; c < total_tiles; c += gridDim.x) {
        int r = 0;
        while (r < 3 && c >= s_tb[r + 1]) ++r;
        const unsigned rb = s_tb[r];
        const unsigned ct = s_tb[r + 1] - rb;
        const unsigned t_local = c - rb;
        const unsigned q0 = s_q0[r], q1 = s_q0[r + 1];
        const unsigned ts = q0 + t_local * (bk ? (unsigned)kBkGroup : (unsigned)kChainTile);
        const unsigned te = min(q1, ts + (bk ? (unsigned)kBkGroup : (unsigned)kChainTile));

        if (bk) {
            // 1') the tile's bucket chains (buckets q0 + t_local * kBkGroup + tid)
            int len = 0;
            if (tid < kBkGroup) {
                const unsigned b = ts + tid;
                if (b < te) {
                    len = __ldcg(hb.blen + b);
                    const size_t o = (size_t)b * kBkChain;
                    for (int j = 0; j < len; ++j) {
                        su[tid * kBkChain + j] = __ldcg(hb.bu + o + j);
                        sv[tid * kBkChain + j] = __ldcg(hb.bv + o + j);
                        si[tid * kBkChain + j] = __ldcg(hb.bi + o + j);
                    }
                }
            }
            s_len[tid] = len;
        } else {
        // 1) run reduction + per-thread chain (records [ts + 16 tid, +16)).
        {
            const int sbase = tid * kChainItems;
            int sp = 0;
            const unsigned p0 = ts + tid * kChainItems;
            for (int m = 0; m < kChainItems; ++m) {
                const unsigned p = p0 + m;
                if (p >= te) break;
                const uint32_t key = hb.keys[p];
                if (p != q0 && hb.keys[p - 1] == key) continue;   // not a run start
                uint64_t best = hb.vals[p];
                for (unsigned q = p + 1; q < q1; ++q) {
                    if (hb.keys[q] != key) break;
                    const uint64_t w = hb.vals[q];
                    best = w < best ? w : best;
                }
                const int pu = (int)(key & kKeyMask);
                const int pv = (int)(best >> 31);
                const int pi = (int)(best & 0x7FFFFFFFull);
                while (sp >= 2 && cross_uv(su[sbase + sp - 2], sv[sbase + sp - 2], su[sbase + sp - 1],
                                           sv[sbase + sp - 1], pu, pv) <= 0)
                    --sp;
                su[sbase + sp] = pu; sv[sbase + sp] = pv; si[sbase + sp] = pi;
                ++sp;
            }
            s_len[tid] = sp;
        }
        }
        __syncthreads();
        // 2) pairwise merge of the tile's leaf chains: the bridge of each pair
        //    by its leader thread, then the kept part of the right chain moved
        //    down by one warp per pair (a left shift, copied forward in chunks
        //    of 32, never overwrites entries still to be read).
        for (int l = 0; (1 << l) < nseg; ++l) {
            const int g = 1 << l;
            const int npairs = nseg >> (l + 1);
            if (tid < nseg && (tid & (2 * g - 1)) == 0) {
                const int b = tid + g, la = s_len[tid], lb = s_len[b];
                int dst = tid * seg, src = b * seg, cnt = 0, len = la;
                if (lb > 0) {
                    if (la == 0) {
                        cnt = lb;
                        len = lb;
                    } else {
                        ChainPtr A{su + tid * seg, sv + tid * seg, si + tid * seg};
                        ChainPtr B{su + b * seg, sv + b * seg, si + b * seg};
                        int is, js;
                        bridge_seq<false>(A, la, B, lb, is, js);
                        dst += is + 1;
                        src += js;
                        cnt = lb - js;
                        len = is + 1 + cnt;
                    }
                }
                const int p = tid / (2 * g);
                s_mv[p][0] = dst;
                s_mv[p][1] = src;
                s_mv[p][2] = cnt;
                s_len[tid] = len;
            }
            __syncthreads();
            const int lane = tid & 31;
            for (int p = tid >> 5; p < npairs; p += kChainThreads / 32) {
                const int dst = s_mv[p][0], src = s_mv[p][1], cnt = s_mv[p][2];
                if (dst == src) continue;
                for (int c = 0; c < cnt; c += 32) {
                    const int j = c + lane;
                    int a = 0, b2 = 0, d = 0;
                    if (j < cnt) { a = su[src + j]; b2 = sv[src + j]; d = si[src + j]; }
                    __syncwarp();
                    if (j < cnt) { su[dst + j] = a; sv[dst + j] = b2; si[dst + j] = d; }
                    __syncwarp();
                }
            }
            __syncthreads();
        }
        // 3) write the tile chain.
        const int len = s_len[0];
        {
            const size_t o = (size_t)c * kChainTile;
            for (int j = tid; j < len; j += blockDim.x) {
                hb.cu[o + j] = su[j]; hb.cv[o + j] = sv[j]; hb.ci[o + j] = si[j];
            }
            if (tid == 0) hb.clen[c] = len;
        }
        // 4) climb the merge tree of queue r.
        unsigned L = 0, k = t_local;
        bool root = false;
        for (;;) {
            if (k == 0 && (1u << L) >= ct) { root = true; break; }   // root of queue r
            const unsigned sib = k ^ 1u;
            if ((sib << L) >= ct) { ++L; k >>= 1; continue; }  // no sibling: pass through
            __threadfence();
            __syncthreads();
            if (tid == 0)
                s_old = atomicAdd(&hb.counters[(size_t)L * hb.ctcap + rb + ((k >> 1) << (L + 1))], 1);
            __syncthreads();
            if (s_old == 0) break;                              // sibling merges later
            __threadfence();
            const unsigned left = rb + ((k & ~1u) << L), right = rb + ((k | 1u) << L);
            const int la = __ldcg(hb.clen + left), lb = __ldcg(hb.clen + right);
            const size_t oa = (size_t)left * kChainTile, ob = (size_t)right * kChainTile;
            int is, js;
            if (lb == 0) {
                // nothing to add
            } else if (la == 0) {
                copy_down(hb.cu + oa, hb.cv + oa, hb.ci + oa, hb.cu + ob, hb.cv + ob, hb.ci + ob, lb);
                if (tid == 0) hb.clen[left] = lb;
            } else if (la + lb <= kMergeSmemCap) {
                for (int j = tid; j < la; j += blockDim.x) {
                    su[j] = __ldcg(hb.cu + oa + j); sv[j] = __ldcg(hb.cv + oa + j); si[j] = __ldcg(hb.ci + oa + j);
                }
                for (int j = tid; j < lb; j += blockDim.x) {
                    su[la + j] = __ldcg(hb.cu + ob + j); sv[la + j] = __ldcg(hb.cv + ob + j);
                    si[la + j] = __ldcg(hb.ci + ob + j);
                }
                __syncthreads();
                ChainPtr A{su, sv, si}, B{su + la, sv + la, si + la};
                bridge_block<false>(A, la, B, lb, is, js, s_red);
                const int n = lb - js;
                for (int j = tid; j < n; j += blockDim.x) {
                    hb.cu[oa + is + 1 + j] = su[la + js + j];
                    hb.cv[oa + is + 1 + j] = sv[la + js + j];
                    hb.ci[oa + is + 1 + j] = si[la + js + j];
                }
                if (tid == 0) hb.clen[left] = is + 1 + n;
            } else {
                ChainPtr A{hb.cu + oa, hb.cv + oa, hb.ci + oa}, B{hb.cu + ob, hb.cv + ob, hb.ci + ob};
                bridge_block<true>(A, la, B, lb, is, js, s_red);
                const int n = lb - js;
                copy_down(hb.cu + oa + is + 1, hb.cv + oa + is + 1, hb.ci + oa + is + 1,
                          hb.cu + ob + js, hb.cv + ob + js, hb.ci + ob + js, n);
                if (tid == 0) hb.clen[left] = is + 1 + n;
            }
            if (tid == 0) hb.counters[(size_t)L * hb.ctcap + rb + ((k >> 1) << (L + 1))] = 0;
            __syncthreads();
            ++L;
            k >>= 1;
        }
        __syncthreads();
        if (!root) continue;
        // 5) the block completing the fourth queue root joins the chains.
        __threadfence();
        __syncthreads();
        if (tid == 0) s_old = (int)atomicAdd(&ctl->blocks_done[3], 1u);
        __syncthreads();
        if (s_old != 3) continue;
        __threadfence();
        if (tid == 0) ctl->blocks_done[3] = 0u;
        int off[5];
        off[0] = 0;
        for (int q = 0; q < 4; ++q) off[q + 1] = off[q] + __ldcg(hb.clen + s_tb[q]) - 1;
        const int m = off[4];
        if (m < 0 || m > (int)nrec) {   // inconsistent state: report, never read out of range
            if (tid == 0) { set_status(ctl, CH_ECUDA); *hb.out_n = CH_ECUDA; }
            return;
        }
        // the cycle's coordinates from the chains' frames (no reads of the
        // points), into the sort/scatter buffers, free by now
        for (int q = 0; q < 4; ++q) {
            const size_t o = (size_t)s_tb[q] * kChainTile;
            for (int j = tid; j < off[q + 1] - off[q]; j += blockDim.x) {
                int x, y;
                frame_to_xy(q, __ldcg(hb.cu + o + j), __ldcg(hb.cv + o + j), x, y);
                hb.vbuf[off[q] + j] = __ldcg(hb.ci + o + j);
                hb.xbuf[off[q] + j] = x;
                hb.ybuf[off[q] + j] = y;
            }
        }
        __syncthreads();
        const int* X = hb.xbuf;
        const int* Y = hb.ybuf;
        stitch_core(hb.vbuf, m, hb.kbuf, hb.vbuf + m,
                    [&](int p, long long& x, long long& y) { x = __ldcg(X + p); y = __ldcg(Y + p); }, hb.n, ctl,
                    hb.out_idx, hb.out_n);
        return;
    }
}

// ---------------------------------------------------------------------------
size_t chain_smem_bytes() { return (size_t)3 * kMergeSmemCap * sizeof(int); }

void launch_chain(Ctl* ctl, const uint32_t* keys, const uint64_t* vals, const int* bu, const int* bv,
                  const int* bi, const int* blen, int* cu, int* cv, int* ci, int* clen, int* counters, int ctcap,
                  int* vbuf, int* kbuf, int* xbuf, int* ybuf, const float* pts, long long n, int32_t* out_idx,
                  int64_t* out_n, int grid, cudaStream_t s) {
    HullBufs hb{keys, vals, bu, bv, bi, blen, cu, cv, ci, clen, counters, ctcap, vbuf, kbuf, xbuf, ybuf, pts, n,
                out_idx, out_n};
    chain_kernel<<<grid, kChainThreads, chain_smem_bytes(), s>>>(ctl, hb);
}

cudaError_t configure_hull_kernels() {
    return cudaFuncSetAttribute(chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)chain_smem_bytes());
}


cudaError_t occupancy_chain(int* b) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, chain_kernel, kChainThreads, chain_smem_bytes());
}

}  // namespace ch
