// merge.cuh -- the merge tree of queue chains: block-level bridges between
// two lower chains and the per-tile merge-and-climb step, shared by the
// single-hull chain kernel and the batched large-survivor path.
//
// Merging two chains A, B (all u of A below all u of B): a_k (k > 0) stays iff
// every b in B is strictly left of a_{k-1} -> a_k; b_l (l < |B|-1) stays iff
// every a in A is strictly left of b_l -> b_{l+1}.  Both predicates hold on a
// prefix of A / a suffix of B (see hullcore.cuh).
#pragma once

#include "ch_internal.cuh"
#include "hullcore.cuh"

namespace ch {

// Debug builds (-DCH_PHASEPROF): cycles per phase of the merge tree, summed
// over blocks (thread 0 adds each phase's clock delta).
#ifdef CH_PHASEPROF
static __device__ unsigned long long g_mg_phase[16];
#define CH_MG_DECL unsigned long long _mg_t = clock64();
#define CH_MG(k) do { const unsigned long long _t = clock64(); \
    if (threadIdx.x == 0) atomicAdd(&g_mg_phase[k], _t - _mg_t); _mg_t = _t; } while (0)
#else
#define CH_MG_DECL
#define CH_MG(k) do { } while (0)
#endif

// Block-cooperative bridge: repeated 256-way probing of the monotone keep
// predicates (each probe is a sequential binary search over the other chain).
template <bool kGlobal>
static __device__ void bridge_block(const ChainPtr& A, int la, const ChainPtr& B, int lb, int& is, int& js,
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

// Warp-cooperative bridge (all 32 lanes, the same arguments): each round
// probes 32 evenly spread candidates of the monotone keep predicate, one per
// lane, and narrows the range to the gap where it turns, so a bridge between
// chains of a few hundred vertices takes two or three rounds of one
// sequential inner search instead of a sequential outer one.
template <bool kGlobal>
static __device__ void bridge_warp(const ChainPtr& A, int la, const ChainPtr& B, int lb, int& is, int& js) {
    const int lane = threadIdx.x & 31;
    // A: largest k with keep_a(k); the predicate holds on [0, is]
    int lo = 0, hi = la - 1;
    while (lo < hi) {
        const long long span = (long long)hi - lo;
        const int k = lo + 1 + (int)(span * lane / 32);   // in (lo, hi], non-decreasing in lane
        const unsigned ok = __ballot_sync(0xFFFFFFFFu, keep_a<kGlobal>(A, k, B, lb));
        if (ok == 0u) {
            hi = __shfl_sync(0xFFFFFFFFu, k, 0) - 1;
        } else {
            const int last = 31 - __clz((int)ok);             // the true probes are a prefix
            const int klast = __shfl_sync(0xFFFFFFFFu, k, last);
            const int knext = __shfl_sync(0xFFFFFFFFu, k, last < 31 ? last + 1 : 31);
            lo = klast;
            if (last < 31 && knext > klast) hi = knext - 1;
        }
    }
    is = lo;
    // B: smallest l with keep_b(l); the predicate holds on [js, lb - 1]
    lo = 0;
    hi = lb - 1;
    while (lo < hi) {
        const long long span = (long long)hi - lo;
        const int l = lo + (int)(span * lane / 32);       // in [lo, hi), non-decreasing in lane
        const unsigned ok = __ballot_sync(0xFFFFFFFFu, keep_b<kGlobal>(A, la, B, l, lb));
        if (ok == 0u) {
            lo = __shfl_sync(0xFFFFFFFFu, l, 31) + 1;
        } else {
            const int first = __ffs((int)ok) - 1;             // the true probes are a suffix
            const int lfirst = __shfl_sync(0xFFFFFFFFu, l, first);
            const int lprev = __shfl_sync(0xFFFFFFFFu, l, first > 0 ? first - 1 : 0);
            hi = lfirst;
            if (first > 0 && lprev < lfirst) lo = lprev + 1;
        }
    }
    js = lo;
}

// Block-wide forward copy of n entries, dst <= src (possibly overlapping),
// in chunks fully loaded before they are stored.
static __device__ void copy_down(int* du, int* dv, int* di, const int* su, const int* sv, const int* si, int n) {
    for (int base = 0; base < n; base += blockDim.x) {
        const int j = base + threadIdx.x;
        int a = 0, b = 0, c = 0;
        if (j < n) { a = __ldcg(su + j); b = __ldcg(sv + j); c = __ldcg(si + j); }
        __syncthreads();
        if (j < n) { du[j] = a; dv[j] = b; di[j] = c; }
        __syncthreads();
    }
}

// Chain storage of the merge tree: tile c's chain at [c * kChainTile, ...);
// a merged chain of 2^L tiles stays at its leftmost tile's offset and may
// extend over the tiles it replaced.
struct TreeBufs {
    int* cu;
    int* cv;
    int* ci;
    int* clen;
    int* counters;   // arrival counters per level and pair (zero at rest)
    int ctcap;       // tiles of the storage (counter row length)
};

// One tile of a segment (tiles [rb, rb + ct), this is tile rb + t_local =
// c): its leaf chains are in shared memory (slot tid * seg, length
// s_len[tid], tid < nseg).  Merges them pairwise, writes the tile chain, and
// climbs the segment's binary merge tree: the block that completes a pair
// (second arrival on its counter) merges it, so no block waits.  Returns true
// in the block that completed the segment's root (its chain at tile rb).
static __device__ bool tile_merge_climb(int* su, int* sv, int* si, int* s_len, int (*s_mv)[3], int seg, int nseg,
                                        const TreeBufs& hb, unsigned c, unsigned rb, unsigned ct, unsigned t_local,
                                        int* s_red, int* s_old_p) {
    const int tid = threadIdx.x;
    int& s_old = *s_old_p;
    CH_MG_DECL
        // 2) pairwise merge of the tile's leaf chains: the bridge of each pair
        //    by its leader thread, then the kept part of the right chain moved
        //    down by one warp per pair (a left shift, copied forward in chunks
        //    of 32, never overwrites entries still to be read).
        for (int l = 0; (1 << l) < nseg; ++l) {
            const int g = 1 << l;
            const int npairs = nseg >> (l + 1);
            if (npairs <= 4 * (int)(blockDim.x >> 5)) {
                // few, longer pairs: one warp per pair
                const int lane = tid & 31;
                for (int p = tid >> 5; p < npairs; p += (int)(blockDim.x >> 5)) {
                    const int a0 = p * 2 * g, b = a0 + g, la = s_len[a0], lb = s_len[b];
                    int dst = a0 * seg, src = b * seg, cnt = 0, len = la;
                    if (lb > 0) {
                        if (la == 0) {
                            cnt = lb;
                            len = lb;
                        } else {
                            ChainPtr A{su + a0 * seg, sv + a0 * seg, si + a0 * seg};
                            ChainPtr B{su + b * seg, sv + b * seg, si + b * seg};
                            int is, js;
                            bridge_warp<false>(A, la, B, lb, is, js);
                            dst += is + 1;
                            src += js;
                            cnt = lb - js;
                            len = is + 1 + cnt;
                        }
                    }
                    if (lane == 0) {
                        s_mv[p][0] = dst;
                        s_mv[p][1] = src;
                        s_mv[p][2] = cnt;
                        s_len[a0] = len;
                    }
                }
            } else if (tid < nseg && (tid & (2 * g - 1)) == 0) {
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
        CH_MG(1);
        // 3) write the tile chain.
        const int len = s_len[0];
        {
            const size_t o = (size_t)c * kChainTile;
            for (int j = tid; j < len; j += blockDim.x) {
                hb.cu[o + j] = su[j]; hb.cv[o + j] = sv[j]; hb.ci[o + j] = si[j];
            }
            if (tid == 0) hb.clen[c] = len;
        }
        CH_MG(2);
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
            CH_MG(L < 4 ? 3 : (L < 8 ? 4 : 5));
            ++L;
            k >>= 1;
        }
        CH_MG(6);
    return root;
}

}  // namespace ch
