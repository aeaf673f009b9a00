// post.cu -- the loop of Alg. 1/2 after findExtremes, on the survivors.
//
// post_kernel classifies, against the octagon of the true extremes (hull
// rule, findQueue by the quadrilateral rule), either the raw survivors of the
// fused main pass or, in two-pass mode, every point; kept points become sort
// records (queue | u, v | index).  The block that finishes last adds the
// records of the support-line end points and, when the records are few,
// computes the hull itself (quickhull rounds over the queues), so the
// sort-based path that follows finds ctl->done set and exits at once.
#include "ch_internal.cuh"
#include "hullcore.cuh"
#include "launch.h"
#include "octagon.cuh"
#include "records.cuh"
#include "star.cuh"

#include <climits>

namespace ch {

constexpr int kPostThreads = 512;
static_assert(kPostThreads % 128 == 0, "mid_hull splits the block in four");

// Records are staged per warp in shared memory; a full buffer goes out with
// one atomic on the record counter, and at the end the block's remainders go
// out together with one atomic (a single counter hit once per warp batch
// serialises at L2).
constexpr int kRecBuf = 256;
struct RecBuf {
    unsigned long long val[kRecBuf];
    unsigned key[kRecBuf];
};

__device__ __forceinline__ void rec_flush_warp(RecBuf& b, unsigned& cnt, Ctl* ctl, uint32_t* keys, uint64_t* vals) {
    const int lane = threadIdx.x & 31;
    unsigned base = 0u;
    if (lane == 0) base = atomicAdd(&ctl->count, cnt);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (unsigned i = lane; i < cnt; i += 32) {
        keys[base + i] = b.key[i];
        vals[base + i] = b.val[i];
    }
    __syncwarp();
    cnt = 0u;
}

// Warp-collective: stages one classified point per lane (r = -1 for none).
// Records per queue are counted per lane in `tally`.
__device__ __forceinline__ void post_stage(int r, int X, int Y, unsigned idx, const Octagon& o, RecBuf& b,
                                           unsigned& cnt, Ctl* ctl, uint32_t* keys, uint64_t* vals,
                                           QueueTally& tally) {
    bool keep = r >= 0;
    if (!__any_sync(0xFFFFFFFFu, keep)) return;
    if (reduce_on_line(o, keep, X, Y, idx, ctl)) keep = false;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
    if (!bal) return;
    if (cnt + (unsigned)__popc(bal) > (unsigned)kRecBuf) rec_flush_warp(b, cnt, ctl, keys, vals);
    tally.add(keep, r);
    if (keep) {
        uint32_t u, v;
        queue_frame(r, X, Y, u, v);
        const unsigned pos = cnt + __popc(bal & lanemask_lt());
        b.key[pos] = make_key(r, u);
        b.val[pos] = make_val(v, idx);
    }
    cnt += __popc(bal);
    __syncwarp();
}

// The star polygon in shared memory (null when this call has none) and its
// centre; points strictly inside it are dropped before the octagon test.
struct StarView {
    const StarPoly* P;
    int cx, cy;
    __device__ __forceinline__ bool inside(int X, int Y) const {
        return P != nullptr && star_inside(X - cx, Y - cy, *P);
    }
};

// Warp-collective: classifies one point per lane (valid = false for none) and
// stages it; folds the tally (one add per lane and call).
__device__ __forceinline__ void post_point(bool valid, float x, float y, unsigned idx, const Octagon& o,
                                           const StarView& sv, RecBuf& b, unsigned& cnt, Ctl* ctl, uint32_t* keys,
                                           uint64_t* vals, QueueTally& tally) {
    int r = -1, X = 0, Y = 0;
    if (valid) {
        X = __float2int_rn(x);
        Y = __float2int_rn(y);
        if (!sv.inside(X, Y)) r = classify_hull(x, y, o);
    }
    post_stage(r, X, Y, idx, o, b, cnt, ctl, keys, vals, tally);
    tally.fold();
}

// Whole block: the warps' staged records go out with one atomic.
__device__ void rec_flush_block(RecBuf& b, unsigned cnt, Ctl* ctl, uint32_t* keys, uint64_t* vals) {
    __shared__ unsigned s_off[kPostThreads / 32];
    __shared__ unsigned s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_off[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0u;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const unsigned c = s_off[w];
            s_off[w] = tot;
            tot += c;
        }
        s_base = tot ? atomicAdd(&ctl->count, tot) : 0u;
    }
    __syncthreads();
    const unsigned base = s_base + s_off[warp];
    for (unsigned i = lane; i < cnt; i += 32) {
        keys[base + i] = b.key[i];
        vals[base + i] = b.val[i];
    }
}

// The block's records per queue (lane tallies) into ctl->rec_q.
__device__ __forceinline__ void flush_queue_counts(QueueTally& tally, Ctl* ctl) {
    __shared__ unsigned s_q[4];
    if (threadIdx.x < 4) s_q[threadIdx.x] = 0u;
    __syncthreads();
    tally.fold();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned w = tally.warp_total(q);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&s_q[q], w);
    }
    __syncthreads();
    if (threadIdx.x < 4 && s_q[threadIdx.x]) atomicAdd(&ctl->rec_q[threadIdx.x], s_q[threadIdx.x]);
}

// The block that finished last: support-line records, then with at most
// kMidCap records the hull (quickhull rounds, else the sort-based mid_hull).
// Every other record is already in keys/vals and in the per-queue counts.
__device__ void post_last_block(const float* __restrict__ pts, long long n, Ctl* ctl, const Octagon& o,
                                uint32_t* keys, uint64_t* vals, int32_t* out_idx, int64_t* out_n, char* dyn,
                                unsigned long long cond) {
    __shared__ unsigned long long s_lep[8];
    __shared__ uint64_t s_lval[8];
    __shared__ unsigned s_lkey[8];
    __shared__ int s_lpos[8];
    __shared__ unsigned s_m, s_total;
    __shared__ int s_mv;
    const int tid = threadIdx.x;
    CH_TRACE_DECL
    CH_TRACE_MARK();
    // one round of loads: line end points and the record count
    if (tid < 8) s_lep[tid] = *(volatile unsigned long long*)&ctl->line_ep[tid];
    if (tid == 8) s_m = *(volatile unsigned*)&ctl->count;
    __syncthreads();
    if (tid < 8) s_lpos[tid] = line_record(o, tid, s_lep[tid], s_lkey[tid], s_lval[tid]) ? 1 : -1;
    __syncthreads();
    if (tid == 0) {
        unsigned m = s_m;
        for (int t = 0; t < 8; ++t)
            if (s_lpos[t] > 0) s_lpos[t] = (int)m++;
        s_total = m;
        ctl->count = m;
    }
    __syncthreads();
    const unsigned total = s_total;
    const bool small = total <= (unsigned)kMidCap;
    if (tid < 8 && s_lpos[tid] >= 0) {
        keys[s_lpos[tid]] = s_lkey[tid];
        vals[s_lpos[tid]] = s_lval[tid];
        if (!small) atomicAdd(&ctl->rec_q[s_lkey[tid] >> kKeyBits], 1u);
    }
    if (!small) {   // the large-survivor path follows
        if (cond && tid == 0) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 1u);
        return;
    }
    __syncthreads();      // also makes this block's line records visible to it
    QhSmem& q = *reinterpret_cast<QhSmem*>(dyn);
    for (unsigned i = tid; i < total; i += blockDim.x) {
        const uint32_t k = __ldcg(keys + i);
        const uint64_t w = __ldcg(vals + i);
        q.ru[i] = (int)(k & kKeyMask);
        q.rv[i] = (int)(w >> 31);
        q.ri[i] = (int)(w & 0x7FFFFFFFull);
        q.rs[i] = (int)(k >> kKeyBits);
    }
    __syncthreads();
    CH_TRACE_MARK();
    const bool ok = qh_chains(q, (int)total, &s_mv);
    CH_TRACE_MARK();
    if (ok) {
        stitch_cycle(q.ru, q.rv, q.ri, s_mv, q.rs, ctl, n, out_idx, out_n);
    } else {
        __syncthreads();
        mid_hull(keys, vals, (int)total, pts, n, ctl, out_idx, out_n, dyn);
    }
    if (tid == 0) ctl->done = 1;
    CH_TRACE_MARK();
#ifdef CH_TRACE
    if (tid == 0) printf("[post] records %u raw %u mv %d ok %d\n", total, ctl->count_raw, s_mv, (int)ok);
#endif
    CH_TRACE_PRINT("post-last");
}

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

// Points of dense data that the star polygon's radius test leaves undecided,
// queued per warp and taken 32 at a time through the exact tests, so that a
// few such points do not hold a whole warp in the slow path.
constexpr int kQueueCap = 96;   // < 32 waiting + 64 added per step
struct WarpQueue {
    int x[kQueueCap], y[kQueueCap];
    unsigned idx[kQueueCap];
};

// Dynamic shared memory while points are classified: the star polygon, the
// warps' record buffers, the warps' queues.  The polygon is finished first,
// with the region from the record buffers on as its work area A; afterwards
// the last block's hull reuses all of it.
constexpr size_t kRecBufOff = (sizeof(StarPoly) + 15) / 16 * 16;
constexpr size_t kQueueOff = kRecBufOff + (size_t)(kPostThreads / 32) * sizeof(RecBuf);
constexpr size_t kClassifyBytes = kQueueOff + (size_t)(kPostThreads / 32) * sizeof(WarpQueue);
constexpr size_t kWorkABytes = (sizeof(int2) + sizeof(unsigned short)) * kStarBins;
constexpr size_t kPostSmemBytes =
    cmax(cmax(kMidSmemBytes, sizeof(QhSmem)), cmax(kClassifyBytes, kRecBufOff + kWorkABytes));

// Warp-collective: the exact star test and the octagon classification of one
// queued point per lane (valid = false for none), then staging.
__device__ __forceinline__ void post_queued(bool valid, int X, int Y, unsigned idx, const Octagon& o,
                                            const StarView& sv, RecBuf& b, unsigned& cnt, Ctl* ctl, uint32_t* keys,
                                            uint64_t* vals, QueueTally& tally) {
    int r = -1;
    if (valid) {
        const int px = X - sv.cx, py = Y - sv.cy;
        if (!star_inside_exact(px, py, star_bin(px, py), *sv.P)) r = classify_hull((float)X, (float)Y, o);
    }
    post_stage(r, X, Y, idx, o, b, cnt, ctl, keys, vals, tally);
}

__global__ void __launch_bounds__(kPostThreads, 1) post_kernel(const float* __restrict__ pts, long long n, int head,
                                                               long long ntiles, Ctl* ctl, const uint64_t* raw_xy,
                                                               const uint32_t* raw_idx, uint32_t* keys,
                                                               uint64_t* vals, int32_t* out_idx, int64_t* out_n,
                                                               unsigned long long* star_bins,
                                                               unsigned long long cond) {
    extern __shared__ __align__(16) char dyn[];
    __shared__ Octagon s_o;
    __shared__ int s_flag, s_mode, s_star, s_scx, s_scy;
    __shared__ unsigned s_nraw;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    CH_TL(ctl, 5, 0);
    if (tid == 0) {
        s_flag = read_status(ctl);
        s_mode = *(volatile int*)&ctl->mode;
        s_nraw = *(volatile unsigned*)&ctl->count_raw;
        s_star = star_bins != nullptr && *(volatile int*)&ctl->star_ok;
        s_scx = ctl->star_cx;
        s_scy = ctl->star_cy;
    }
    copy_octagon(&s_o, &ctl->oct);
    __syncthreads();
    if (s_flag != CH_OK) {   // data error or timeout of an earlier stage
        if (blockIdx.x == 0 && tid == 0) { *out_n = s_flag; ctl->done = 1; }
        if (blockIdx.x == 0 && s_star)   // leave the star bins clear for the next call
            for (int b = tid; b < kStarBins; b += blockDim.x) star_bins[b] = 0ull;
        return;
    }
    StarView sv{nullptr, s_scx, s_scy};
    if (s_star) {   // the star pass gathered a vertex list: finish the polygon here
        StarPoly* P = reinterpret_cast<StarPoly*>(dyn);
        int2* va = reinterpret_cast<int2*>(dyn + kRecBufOff);
        unsigned short* ba = reinterpret_cast<unsigned short*>(dyn + kRecBufOff + sizeof(int2) * kStarBins);
        CH_TL(ctl, 8, 0);
        const int k = star_finish<kPostThreads>(star_bins, pts, n, s_scx, s_scy, va, ba, *P, ctl);
        if (k) sv.P = P;
        CH_TL(ctl, 8, 1);
        if (blockIdx.x == 0 && tid == 0) {
            ctl->star_final = k ? 1 : 0;
            ctl->star_k = k;
        }
        __syncthreads();
    }
    RecBuf& rb = reinterpret_cast<RecBuf*>(dyn + kRecBufOff)[warp];
    unsigned rc = 0u;
    QueueTally tally;
    if (s_mode == 1) {   // two-pass mode: every point
        // n < 2^31, so step and point numbers fit in 32 bits
        const unsigned gwarp = (blockIdx.x * blockDim.x + tid) >> 5;
        const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
        const float4* p4 = reinterpret_cast<const float4*>(pts + 2 * head);
        const unsigned long long pol = l2_evict_first();
        // one float4 (two points, classified together) per step with the
        // loads of the next kAhead steps in flight: a rolled loop keeps the
        // classification code small.  Steps run over this warp's tiles,
        // kLoadsPerLane float4 per tile.
        constexpr int kAhead = 8;
        const unsigned total = (unsigned)ntiles * kLoadsPerLane;
        const unsigned sstep = nwarps * kLoadsPerLane;
        auto next_step = [&](unsigned st) {
            return (st % kLoadsPerLane == kLoadsPerLane - 1) ? st + sstep - (kLoadsPerLane - 1) : st + 1;
        };
        unsigned s = gwarp * kLoadsPerLane, sl = s;   // sl: the step of the newest load
        WarpQueue& wq = reinterpret_cast<WarpQueue*>(dyn + kQueueOff)[warp];
        unsigned qn = 0u;   // points waiting in wq (warp-uniform)
        float4 q[kAhead];
#pragma unroll
        for (int a = 0; a < kAhead; ++a) {
            q[a] = sl < total ? ld_stream_f4(p4 + sl * 32 + lane, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
            sl = next_step(sl);
        }
#pragma unroll 1
        while (s < total) {
            const float4 v = q[0];
#pragma unroll
            for (int a = 0; a + 1 < kAhead; ++a) q[a] = q[a + 1];
            q[kAhead - 1] = sl < total ? ld_stream_f4(p4 + sl * 32 + lane, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
            sl = next_step(sl);
            const unsigned i0 = (unsigned)head + (s / kLoadsPerLane) * kWarpTilePts + 64u * (s % kLoadsPerLane) +
                                2u * lane;
            const int X0 = __float2int_rn(v.x), Y0 = __float2int_rn(v.y);
            const int X1 = __float2int_rn(v.z), Y1 = __float2int_rn(v.w);
            if (sv.P) {
                // most points of dense data are inside the star polygon's
                // radius bound of their bin; the rest wait in the queue
                const int px0 = X0 - sv.cx, py0 = Y0 - sv.cy, px1 = X1 - sv.cx, py1 = Y1 - sv.cy;
                const bool d0 = star_inside_fast(px0, py0, star_bin(px0, py0), *sv.P);
                const bool d1 = star_inside_fast(px1, py1, star_bin(px1, py1), *sv.P);
                const unsigned m0 = __ballot_sync(0xFFFFFFFFu, !d0), m1 = __ballot_sync(0xFFFFFFFFu, !d1);
                if (m0 | m1) {
                    const unsigned lt = lanemask_lt();
                    if (!d0) {
                        const unsigned pos = qn + __popc(m0 & lt);
                        wq.x[pos] = X0; wq.y[pos] = Y0; wq.idx[pos] = i0;
                    }
                    if (!d1) {
                        const unsigned pos = qn + __popc(m0) + __popc(m1 & lt);
                        wq.x[pos] = X1; wq.y[pos] = Y1; wq.idx[pos] = i0 + 1u;
                    }
                    qn += __popc(m0) + __popc(m1);
                    __syncwarp();
                    while (qn >= 32u) {
                        qn -= 32u;
                        const int X = wq.x[qn + lane], Y = wq.y[qn + lane];
                        const unsigned id = wq.idx[qn + lane];
                        __syncwarp();
                        post_queued(true, X, Y, id, s_o, sv, rb, rc, ctl, keys, vals, tally);
                    }
                }
            } else {
                int r0 = classify_hull_fast(v.x, v.y, X0, Y0, s_o);
                int r1 = classify_hull_fast(v.z, v.w, X1, Y1, s_o);
                if (r0 == kUndecided) r0 = classify_hull_slow(v.x, v.y, &s_o);
                if (r1 == kUndecided) r1 = classify_hull_slow(v.z, v.w, &s_o);
                post_stage(r0, X0, Y0, i0, s_o, rb, rc, ctl, keys, vals, tally);
                post_stage(r1, X1, Y1, i0 + 1u, s_o, rb, rc, ctl, keys, vals, tally);
            }
            if (s % kLoadsPerLane == kLoadsPerLane - 1) tally.fold();   // at most 2 kLoadsPerLane adds
            s = next_step(s);
        }
        if (qn) {   // the queue's remainder
            const bool valid = (unsigned)lane < qn;
            const int X = valid ? wq.x[lane] : 0, Y = valid ? wq.y[lane] : 0;
            const unsigned id = valid ? wq.idx[lane] : 0u;
            __syncwarp();
            post_queued(valid, X, Y, id, s_o, sv, rb, rc, ctl, keys, vals, tally);
            tally.fold();
        }
        if (gwarp == 0) {   // the unaligned head point and the ragged tail
            const long long ranges[2][2] = {{0, head}, {head + ntiles * kWarpTilePts, n}};
            for (int rg = 0; rg < 2; ++rg)
                for (long long b = ranges[rg][0]; b < ranges[rg][1]; b += 32) {
                    const long long i = b + lane;
                    const bool valid = i < ranges[rg][1];
                    float x = 0.0f, y = 0.0f;
                    if (valid) { x = pts[2 * i]; y = pts[2 * i + 1]; }
                    post_point(valid, x, y, (unsigned)i, s_o, sv, rb, rc, ctl, keys, vals, tally);
                }
        }
    } else {   // fused mode: the raw survivors of the main pass
        const unsigned nraw = s_nraw;
        const unsigned stride = gridDim.x * blockDim.x;
        for (unsigned b = blockIdx.x * blockDim.x + warp * 32; b < nraw; b += stride) {
            const unsigned i = b + lane;
            const bool valid = i < nraw;
            float x = 0.0f, y = 0.0f;
            unsigned idx = 0u;
            if (valid) {
                const unsigned long long xy = raw_xy[i];
                x = (float)(unsigned)(xy >> 32);
                y = (float)(unsigned)(xy & 0xFFFFFFFFull);
                idx = raw_idx[i];
            }
            post_point(valid, x, y, idx, s_o, sv, rb, rc, ctl, keys, vals, tally);
        }
    }
    rec_flush_block(rb, rc, ctl, keys, vals);
    flush_queue_counts(tally, ctl);
    CH_TL(ctl, 5, 1);
    if (!last_block(&ctl->blocks_done[2], &s_flag)) return;
    CH_TL(ctl, 6, 0);
    if (s_star)   // every block has built its polygon: clear the bins for the next call
        for (int b = tid; b < kStarBins; b += blockDim.x) star_bins[b] = 0ull;
    post_last_block(pts, n, ctl, s_o, keys, vals, out_idx, out_n, dyn, cond);
    CH_TL(ctl, 6, 1);
}

// ---------------------------------------------------------------------------
void launch_post(const float* pts, long long n, int head, long long ntiles, Ctl* ctl, const uint64_t* raw_xy,
                 const uint32_t* raw_idx, uint32_t* keys, uint64_t* vals, int32_t* out_idx, int64_t* out_n,
                 void* star_bins, unsigned long long cond, int grid, cudaStream_t s) {
    post_kernel<<<grid, kPostThreads, kPostSmemBytes, s>>>(pts, n, head, ntiles, ctl, raw_xy, raw_idx, keys, vals,
                                                          out_idx, out_n, (unsigned long long*)star_bins, cond);
}

cudaError_t configure_post_kernel() {
    return cudaFuncSetAttribute(post_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPostSmemBytes);
}

cudaError_t occupancy_post(int* blocks) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, post_kernel, kPostThreads, kPostSmemBytes);
}

}  // namespace ch
