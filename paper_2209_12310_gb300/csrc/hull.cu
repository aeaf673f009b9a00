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
#include "merge.cuh"

#include <climits>

namespace ch {

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
        CH_MG_DECL
        int r = 0;
        while (r < 3 && c >= s_tb[r + 1]) ++r;
        const unsigned rb = s_tb[r];
        const unsigned ct = s_tb[r + 1] - rb;
        const unsigned t_local = c - rb;
        const unsigned q0 = s_q0[r], q1 = s_q0[r + 1];
        const unsigned ts = q0 + t_local * (bk ? (unsigned)kBkGroup : (unsigned)kChainTile);
        const unsigned te = min(q1, ts + (bk ? (unsigned)kBkGroup : (unsigned)kChainTile));

        if (bk) {
            // 1') the tile's bucket chains (buckets ts .. te): their slots are
            // contiguous, so the whole block copies them with coalesced loads
            s_len[tid] = (tid < kBkGroup && ts + tid < te) ? __ldcg(hb.blen + ts + tid) : 0;
            const size_t o0 = (size_t)ts * kBkChain;
            for (unsigned e = tid; e < (te - ts) * kBkChain; e += blockDim.x) {
                su[e] = __ldcg(hb.bu + o0 + e);
                sv[e] = __ldcg(hb.bv + o0 + e);
                si[e] = __ldcg(hb.bi + o0 + e);
            }
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
        CH_MG(0);
        const TreeBufs tb{hb.cu, hb.cv, hb.ci, hb.clen, hb.counters, hb.ctcap};
        const bool root = tile_merge_climb(su, sv, si, s_len, s_mv, seg, nseg, tb, c, rb, ct, t_local, s_red, &s_old);
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
        CH_MG(7);
        stitch_core(hb.vbuf, m, hb.kbuf, hb.vbuf + m,
                    [&](int p, long long& x, long long& y) { x = __ldcg(X + p); y = __ldcg(Y + p); }, hb.n, ctl,
                    hb.out_idx, hb.out_n);
        CH_MG(8);
        return;
    }
}

// ---------------------------------------------------------------------------
#ifdef CH_PHASEPROF
}  // namespace ch
extern "C" int ch_phase_read_merge(unsigned long long* out16) {
    return cudaMemcpyFromSymbol(out16, ch::g_mg_phase, sizeof(unsigned long long) * 16) == cudaSuccess ? 0 : -4;
}
extern "C" int ch_phase_reset_merge(void) {
    unsigned long long z[16] = {};
    return cudaMemcpyToSymbol(ch::g_mg_phase, z, sizeof(z)) == cudaSuccess ? 0 : -4;
}
namespace ch {
#endif

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
