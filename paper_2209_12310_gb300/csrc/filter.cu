// filter.cu -- the filtering stage of GPU heaphull (Alg. 2, GPUfilter) on sm_103a.
//
// Kernels (in launch order):
//   init_kernel     reset the per-call control block.
//   sample_kernel   extremes of an evenly spaced sample of warp tiles; its last
//                   block builds the sample octagon (vertices are input points).
//   main_kernel     findExtremes (Alg. 2; Sec. 3) over every point: all 8
//                   directional extremes in one pass (the paper's second
//                   kernel finds the corner points by Manhattan distance to the
//                   bounding-box corners; that distance is x+y or x-y up to a
//                   constant, so one pass suffices), with the lowest index on
//                   ties.  In fused mode (ch_hull) the same pass also drops the
//                   points in the closed sample octagon and compacts the rest
//                   ("raw" survivors): one streaming read of the input instead
//                   of two.  When the raw survivors grow past a threshold
//                   (adversarial data such as points on a circle), the pass
//                   stops filtering and the second pass does it (two-pass mode).
//                   Its last block builds the octagon of the true extremes
//                   and the records of the chain end points.
//   (post.cu)       the classification of the survivors and the hull.
//   labels_kernel   ch_filter: the label array Q of Alg. 2 (paper rule).
#include "ch_internal.cuh"
#include "hullcore.cuh"
#include "launch.h"
#include "extremes.cuh"
#include "octagon.cuh"
#include "tma.cuh"

#include <climits>

namespace ch {

// ---------------------------------------------------------------------------
__global__ void init_kernel(Ctl* ctl, int mode) {
    const int t = threadIdx.x;
    if (t < 8) {
        ctl->ext_packed[t] = 0ull;
        ctl->samp_packed[t] = 0ull;
        ctl->line_ep[t] = (t & 1) ? 0ull : ~0ull;   // even: minimum slot, odd: maximum slot
    }
    if (t < 4) { ctl->tile_ctr[t] = 0u; ctl->counts4[t] = 0u; ctl->blocks_done[t] = 0u; ctl->rec_q[t] = 0u; }
    if (t == 0) {
        ctl->status = CH_OK;
        ctl->abort = 0;
        ctl->count = 8u;
        ctl->count_raw = 0u;
        ctl->epoch += 1u;
        ctl->mode = mode;
        ctl->done = 0;
        ctl->records_ready = 0;
        ctl->bk_state = 0;
        ctl->bk_cursor = 0u;
        ctl->samp_ok = 0;
        ctl->star_ok = 0;
        ctl->star_k = 0;
        ctl->star_final = 0;
        ctl->star_pts = 0u;
        ctl->star_out = 0u;
        ctl->star_done = 0u;
    }
    unsigned* h = &ctl->digit_hist[0][0];
    for (int i = t; i < kSortPasses * kDigits; i += blockDim.x) h[i] = 0u;
#if defined(CH_TRACE) || defined(CH_TIMELINE)
    if (t < 14) { ctl->tl[t][0] = ~0ull; ctl->tl[t][1] = 0ull; }
    __syncthreads();
    CH_TL(ctl, 0, 0);
    CH_TL(ctl, 0, 1);
#endif
}


// ---------------------------------------------------------------------------
// Sample pass: packed (key, other coordinate) maxima per direction; the other
// coordinate recovers the point (no index needed: the sample octagon only
// filters, and its vertices are input points).
__device__ __forceinline__ unsigned long long samp_pack(int d, int X, int Y) {
    const unsigned k = (unsigned)dir_key(d, X, Y);
    const unsigned aux = (d == W || d == E) ? (unsigned)Y : (unsigned)X;
    const unsigned hk = dir_is_max(d) ? k : 0xFFFFFFFFu - k;
    return ((unsigned long long)hk << 32) | aux;
}

__global__ void __launch_bounds__(256) sample_kernel(const float* __restrict__ pts, long long n, int head,
                                                     long long ntiles, Ctl* ctl) {
    __shared__ unsigned long long s_red[8][8];
    __shared__ Octagon s_o;
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    CH_TL(ctl, 1, 0);
    unsigned long long best[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) best[d] = 0ull;
    const long long nsamp = sample_tiles(ntiles);
    const float4* p4 = reinterpret_cast<const float4*>(pts + 2 * head);
    const unsigned long long pol = l2_evict_first();
    for (long long k = gwarp; k < nsamp; k += nwarps) {
        const long long t = k * ntiles / nsamp;
        const float4* base = p4 + t * kWarpTileF4 + lane;
        float4 v[kLoadsPerLane];
#pragma unroll
        for (int j = 0; j < kLoadsPerLane; ++j) v[j] = ld_stream_f4(base + j * 32, pol);
#pragma unroll
        for (int j = 0; j < kLoadsPerLane; ++j) {
            const int X0 = __float2int_rn(v[j].x), Y0 = __float2int_rn(v[j].y);
            const int X1 = __float2int_rn(v[j].z), Y1 = __float2int_rn(v[j].w);
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                const unsigned long long a = samp_pack(d, X0, Y0), b = samp_pack(d, X1, Y1);
                const unsigned long long m = a > b ? a : b;
                best[d] = m > best[d] ? m : best[d];
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        unsigned long long p = best[d];
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long q = __shfl_xor_sync(0xFFFFFFFFu, p, o);
            p = q > p ? q : p;
        }
        if (lane == 0) s_red[warp][d] = p;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        unsigned long long m = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = s_red[w][threadIdx.x] > m ? s_red[w][threadIdx.x] : m;
        if (m) atomicMax(&ctl->samp_packed[threadIdx.x], m);
    }
    CH_TL(ctl, 1, 1);
    if (!last_block(&ctl->blocks_done[0], &s_last)) return;
    CH_TL(ctl, 2, 0);
    CH_TRACE_DECL
    CH_TRACE_MARK();
    __shared__ int s_v[2][8];
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = nsamp > 0;
    __syncthreads();
    if (threadIdx.x < 8) {
        const int d = threadIdx.x;
        const unsigned long long p = *(volatile unsigned long long*)&ctl->samp_packed[d];
        if (p == 0ull) atomicAnd(&s_ok, 0);
        const unsigned hk = (unsigned)(p >> 32), aux = (unsigned)p;
        const int key = dir_is_max(d) ? (int)hk : (int)(0xFFFFFFFFu - hk);
        int x, y;
        switch (d) {
            case W: case E: x = key; y = (int)aux; break;
            case S: case N: y = key; x = (int)aux; break;
            case SW: case NE: x = (int)aux; y = key - x; break;
            default: x = (int)aux; y = x - (key - kCoordLimit); break;
        }
        s_v[0][d] = x;
        s_v[1][d] = y;
    }
    __syncthreads();
    CH_TRACE_MARK();
    if (!s_ok) {   // too few points to sample: run the two-pass path
        if (threadIdx.x == 0) ctl->mode = 1;
        return;
    }
    const int ext[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    setup_octagon_block(s_o, s_v[0], s_v[1], ext, true);
    CH_TRACE_MARK();

    if (s_o.discard_none) {
        if (threadIdx.x == 0) ctl->mode = 1;
        return;
    }
    copy_octagon(&ctl->oct_s, &s_o);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        ctl->samp_ok = 1;
    }
    CH_TRACE_MARK();
    CH_TL(ctl, 2, 1);
    CH_TRACE_PRINT("sample-last");
}

// Strictly inside the inner region of the sample octagon: the tile's key
// extremes (or one point's keys) against the bounds, strict comparisons.
// Bounds are read from shared memory (lo = in[0..3], hi = in[4..7]) to keep
// them out of the streaming loop's registers.
__device__ __forceinline__ bool tile_in_inner(const int (&tk)[8], const int* in) {
    return tk[W] > in[0] && tk[E] < in[4] && tk[S] > in[1] && tk[N] < in[5] &&
           tk[SW] > in[2] && tk[NE] < in[6] && tk[NW] > in[3] && tk[SE] < in[7];
}


// Raw survivors are staged per warp in shared memory and written out in
// batches: one global atomic per batch instead of one per warp tile (a single
// contended counter otherwise serialises at L2).
constexpr int kWarpBuf = 256;
struct RawBuf {
    unsigned long long xy[kWarpBuf];
    unsigned idx[kWarpBuf];
};

// Warp-collective; returns the global raw count after this batch.
__device__ __forceinline__ unsigned flush_raw(RawBuf& b, unsigned& cnt, Ctl* ctl, uint64_t* raw_xy,
                                              uint32_t* raw_idx) {
    const int lane = threadIdx.x & 31;
    if (cnt == 0u) return 0u;
    unsigned base = 0u;
    if (lane == 0) base = atomicAdd(&ctl->count_raw, cnt);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    __syncwarp();
    for (unsigned i = lane; i < cnt; i += 32) {
        raw_xy[base + i] = b.xy[i];
        raw_idx[base + i] = b.idx[i];
    }
    __syncwarp();
    const unsigned after = base + cnt;
    cnt = 0u;
    return after;
}

// Warp-collective compaction of a lane's kept slots into the warp's buffer.
// get(s, idx, x, y) reads slot s; slots are unrolled so get indexes registers.
// Returns the global raw count when a batch was written out, else 0.
template <int kSlots, typename Get>
__device__ __forceinline__ unsigned emit_raw(unsigned keep, Get get, RawBuf& b, unsigned& cnt, Ctl* ctl,
                                             uint64_t* raw_xy, uint32_t* raw_idx) {
    const int lane = threadIdx.x & 31;
    const unsigned c = __popc(keep);
    unsigned incl, total;
    if constexpr (kSlots == 1) {
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep != 0u);
        incl = __popc(bal & lanemask_lt()) + c;
        total = __popc(bal);
    } else {
        incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    if (total == 0u) return 0u;
    unsigned after = 0u;
    if (cnt + total > (unsigned)kWarpBuf) after = flush_raw(b, cnt, ctl, raw_xy, raw_idx);
    const bool direct = total > (unsigned)kWarpBuf;   // a dense tile: straight to global memory
    unsigned base = cnt;
    if (direct) {
        if (lane == 31) base = atomicAdd(&ctl->count_raw, total);
        base = __shfl_sync(0xFFFFFFFFu, base, 31);
        after = base + total;
    }
    unsigned pos = base + incl - c;
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        if ((keep >> s) & 1u) {
            long long idx;
            float x, y;
            get(s, idx, x, y);
            const unsigned long long xy =
                ((unsigned long long)(unsigned)__float2int_rn(x) << 32) | (unsigned)__float2int_rn(y);
            if (direct) { raw_xy[pos] = xy; raw_idx[pos] = (uint32_t)idx; }
            else { b.xy[pos] = xy; b.idx[pos] = (unsigned)idx; }
            ++pos;
        }
    }
    __syncwarp();
    if (!direct) cnt += total;
    return after;
}

// Finalize of the main pass (whole block, the main pass's last block):
// lowest-index tie-break, octagon of the true extremes (-> s_o and ctl->oct),
// the chain end-point records.  The inner region of the true octagon is only
// searched in two-pass mode, where it settles most points of the second pass;
// raw survivors of the fused pass lie outside the sample octagon's inner
// region, so for them it would almost never apply.
__device__ __noinline__ void finalize_block(const float* __restrict__ pts, long long n, int head, Ctl* ctl,
                                            Octagon& s_o, uint32_t* keys, uint64_t* vals) {
    __shared__ unsigned long long s_ext[8];
    __shared__ int s_G[8];
    __shared__ long long s_lo[8], s_hi[8];
    if (threadIdx.x < 8) {
        const int d = threadIdx.x;
        const unsigned long long pk = *(volatile unsigned long long*)&ctl->ext_packed[d];
        const unsigned code = 0xFFFFFFFFu - (unsigned)(pk & 0xFFFFFFFFull);
        const unsigned hi32 = (unsigned)(pk >> 32);
        s_G[d] = dir_is_max(d) ? (int)hi32 : (int)(0xFFFFFFFFu - hi32);
        long long lo, hi;
        if (code == 0u) { lo = 0; hi = head; }
        else { lo = head + (long long)(code - 1u) * kWarpTilePts; hi = min(n, lo + kWarpTilePts); }
        s_lo[d] = lo;
        s_hi[d] = hi;
        s_ext[d] = ~0ull;
    }
    __syncthreads();
    CH_TRACE_MARK();
    // One round of independent loads for all 8 directions (a tile has at
    // most kWarpTilePts points; blockDim.x >= kWarpTilePts / 2).
    {
        float2 p[8][2];
        bool valid[8][2];
#pragma unroll
        for (int d = 0; d < 8; ++d) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long i = s_lo[d] + threadIdx.x + (long long)h * blockDim.x;
                valid[d][h] = i < s_hi[d];
                p[d][h] = valid[d][h] ? reinterpret_cast<const float2*>(pts)[i] : make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int d = 0; d < 8; ++d) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long i = s_lo[d] + threadIdx.x + (long long)h * blockDim.x;
                if (valid[d][h] && dir_key(d, __float2int_rn(p[d][h].x), __float2int_rn(p[d][h].y)) == s_G[d])
                    atomicMin(&s_ext[d], (unsigned long long)i);
            }
        }
    }
    __syncthreads();
    bool bad = false;
    for (int d = 0; d < 8; ++d) bad |= s_ext[d] >= (unsigned long long)n;
    if (bad) {   // cannot happen for valid input; fail safe
        if (threadIdx.x == 0) set_status(ctl, CH_ECUDA);
        return;
    }
    __shared__ int s_vx[8], s_vy[8], s_id[8];
    if (threadIdx.x < 8) {
        const long long i = (long long)s_ext[threadIdx.x];
        s_id[threadIdx.x] = (int)i;
        s_vx[threadIdx.x] = __float2int_rn(pts[2 * i]);
        s_vy[threadIdx.x] = __float2int_rn(pts[2 * i + 1]);
    }
    __syncthreads();
    CH_TRACE_MARK();
    setup_octagon_block(s_o, s_vx, s_vy, s_id, *(volatile int*)&ctl->mode != 0);
    CH_TRACE_MARK();
    if (threadIdx.x < 12) {
        // Threads 0..7: chain end points (queue r runs from quad vertex r to
        // r+1).  Threads 8..11: the diagonal extreme of queue r, when it lies
        // strictly right of the quad edge (the hull rule drops every point of
        // the closed octagon, vertices included, so the vertices that can be
        // hull vertices get their own record; on the edge it cannot be one).
        const int lane = threadIdx.x;
        int r, d;
        bool emit = true;
        if (lane < 8) {
            r = lane >> 1;
            d = (lane & 1) ? ((2 * r + 2) & 7) : 2 * r;
        } else {
            r = lane - 8;
            d = 2 * r + 1;
            const int a = 2 * r, b = (2 * r + 2) & 7;
            emit = orient64(s_vx[a], s_vy[a], s_vx[b], s_vy[b], s_vx[d], s_vy[d]) < 0;
        }
        if (emit) {
            uint32_t u, v;
            queue_frame(r, s_vx[d], s_vy[d], u, v);
            const uint32_t key = make_key(r, u);
            const unsigned pos = lane < 8 ? (unsigned)lane : atomicAdd(&ctl->count, 1u);
            keys[pos] = key;
            vals[pos] = make_val(v, (uint32_t)s_id[d]);
            atomicAdd(&ctl->rec_q[r], 1u);
        }
    }
    __syncthreads();
    copy_octagon(&ctl->oct, &s_o);
    __syncthreads();
}

constexpr size_t kMainSmemBytes = (size_t)8 * kStages * kWarpTileF4 * sizeof(float4);

__global__ void __launch_bounds__(256, 2) main_kernel(const float* __restrict__ pts, long long n, int head,
                                                      long long ntiles, Ctl* ctl, uint64_t* raw_xy,
                                                      uint32_t* raw_idx, unsigned switch_at, uint32_t* keys,
                                                      uint64_t* vals) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ int s_inner[8];
    __shared__ float s_edge[24];
    __shared__ unsigned long long s_red[8][8];
    __shared__ int s_mode;
    __shared__ RawBuf s_buf[8];
    __shared__ unsigned long long s_bar[8][kStages];
    __shared__ unsigned char s_q[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    CH_TL(ctl, 3, 0);
    if (threadIdx.x == 0) s_mode = *(volatile int*)&ctl->mode;   // one read: uniform per block
    if (threadIdx.x < 4) {
        s_inner[threadIdx.x] = ctl->oct_s.in_lo[threadIdx.x];
        s_inner[4 + threadIdx.x] = ctl->oct_s.in_hi[threadIdx.x];
    }
    if (threadIdx.x < 8) {
        s_edge[3 * threadIdx.x] = ctl->oct_s.oct[threadIdx.x].A;
        s_edge[3 * threadIdx.x + 1] = ctl->oct_s.oct[threadIdx.x].B;
        s_edge[3 * threadIdx.x + 2] = ctl->oct_s.oct[threadIdx.x].C;
    }
    __syncthreads();
    bool filt = s_mode == 0;
    RawBuf& wbuf = s_buf[warp];
    unsigned wcnt = 0u;
    Track tr;
    track_init(tr);
    // Scalar ranges (warp 0): the unaligned head point first and the ragged
    // tail last, so every lane visits tile codes in increasing order.
    auto scalar_range = [&](long long lo_i, long long hi_i, unsigned code) {
        int tk[8];
        bool any = false;
        for (long long b = lo_i; b < hi_i; b += 32) {
            const long long i = b + lane;
            unsigned keep = 0u;
            float x = 0.0f, y = 0.0f;
            if (i < hi_i) {
                x = pts[2 * i]; y = pts[2 * i + 1];
                int X, Y;
                convert_pt(x, y, X, Y, tr);
                tile_keys2(tk, X, Y, X, Y, !any);
                any = true;
                if (filt && !pt_in_inner(X, Y, s_inner) && !pt_in_sample(x, y, s_edge)) keep = 1u;
            }
            auto get = [&](int, long long& idx, float& px, float& py) { idx = i; px = x; py = y; };
            if (filt) emit_raw<1>(keep, get, wbuf, wcnt, ctl, raw_xy, raw_idx);
        }
        if (any) track_tile(tr, tk, code);
    };
    if (gwarp == 0 && head) scalar_range(0, head, 0u);

    // Warp tiles t = gwarp + k * nwarps stream through a double-buffered
    // shared-memory ring filled by bulk asynchronous copies (TMA).
    WarpStream ws{reinterpret_cast<float4*>(dsm) + warp * kStages * kWarpTileF4, s_bar[warp],
                  reinterpret_cast<const float4*>(pts + 2 * head), gwarp, nwarps, ntiles, lane};
    ws.start();
    for (long long k = 0;; ++k) {
        const long long t = gwarp + k * nwarps;
        if (t >= ntiles) break;
        const float4* cur = ws.acquire(k, ctl);
        if (!cur) {   // a copy never completed: status is CH_ETIMEOUT
            ws.drain(k);
            break;
        }
        int tk[8];
#pragma unroll
        for (int j = 0; j < kLoadsPerLane; ++j) {
            const float4 v = cur[j * 32 + lane];
            int X0, Y0, X1, Y1;
            convert_pt(v.x, v.y, X0, Y0, tr);
            convert_pt(v.z, v.w, X1, Y1, tr);
            tile_keys2(tk, X0, Y0, X1, Y1, j == 0);
        }
        track_tile(tr, tk, (unsigned)(t + 1));
        if (filt) {
            // Points strictly inside the inner region of the sample octagon
            // are strictly inside the hull; every other point is a raw
            // survivor, classified against the true octagon once its extremes
            // are known.  The 16 points of each lane whose tile test failed
            // are spread over the warp (two lane tiles per round) and tested
            // one per lane from the ring slot, so an outlier costs the warp
            // one round instead of a 16-point slow path on one lane.
            const bool inside = tile_in_inner(tk, s_inner);
            const unsigned fail = __ballot_sync(0xFFFFFFFFu, !inside);
            if (fail) {
                if (!inside) s_q[warp][__popc(fail & lanemask_lt())] = (unsigned char)lane;
                __syncwarp();
                const unsigned slots = 16u * (unsigned)__popc(fail);
                const float2* cur2 = reinterpret_cast<const float2*>(cur);
                unsigned upto = 0u;
                for (unsigned s0 = 0; s0 < slots; s0 += 32u) {
                    const unsigned s = s0 + (unsigned)lane;
                    unsigned keep = 0u;
                    float x = 0.0f, y = 0.0f;
                    long long idx = 0;
                    if (s < slots) {
                        // slot s: lane tile of rank s / 16, float4 (s / 2) % 8, half s % 2
                        const int ln = s_q[warp][s >> 4];
                        const int f2 = 2 * ((int)((s >> 1) & 7u) * 32 + ln) + (int)(s & 1u);
                        const float2 v = cur2[f2];
                        x = v.x;
                        y = v.y;
                        keep = (pt_in_inner(__float2int_rn(x), __float2int_rn(y), s_inner) ||
                                pt_in_sample(x, y, s_edge)) ? 0u : 1u;
                        idx = head + t * kWarpTilePts + f2;
                    }
                    auto get = [&](int, long long& id, float& px, float& py) { id = idx; px = x; py = y; };
                    const unsigned a = emit_raw<1>(keep, get, wbuf, wcnt, ctl, raw_xy, raw_idx);
                    upto = a > upto ? a : upto;
                }
                __syncwarp();
                if (upto > switch_at) {   // dense data: leave filtering to the second pass
                    if (lane == 0) atomicExch(&ctl->mode, 1);
                    filt = false;
                }
            }
            if ((k & 7) == 7) {
                int m = 0;
                if (lane == 0) m = *(volatile int*)&ctl->mode;
                filt = filt && __shfl_sync(0xFFFFFFFFu, m, 0) == 0;
            }
        }
        ws.release(k);
    }
    if (gwarp == 0 && head + ntiles * kWarpTilePts < n)
        scalar_range(head + ntiles * kWarpTilePts, n, (unsigned)(ntiles + 1));
    flush_raw(wbuf, wcnt, ctl, raw_xy, raw_idx);

    const bool err = tr.bad || (tr.orv >> kCoordBits) != 0u;
    if (__any_sync(0xFFFFFFFFu, err) && lane == 0) set_status(ctl, CH_ERANGE);
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        unsigned long long p = pack_best(d, tr.best[d], tr.code[d]);
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long q = __shfl_xor_sync(0xFFFFFFFFu, p, o);
            p = q > p ? q : p;
        }
        if (lane == 0) s_red[warp][d] = p;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        unsigned long long m = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = s_red[w][threadIdx.x] > m ? s_red[w][threadIdx.x] : m;
        if (m) atomicMax(&ctl->ext_packed[threadIdx.x], m);
    }
    // The block that finishes last builds the octagon of the true extremes.
    // Every bulk copy of this block has completed (or was drained), so the
    // ring's shared memory is free for it.
    CH_TL(ctl, 3, 1);
    if (!last_block(&ctl->blocks_done[1], &s_mode)) return;
    CH_TL(ctl, 4, 0);
    CH_TRACE_DECL
    CH_TRACE_MARK();
    if (__syncthreads_or(read_status(ctl) != CH_OK)) return;
    finalize_block(pts, n, head, ctl, *reinterpret_cast<Octagon*>(dsm), keys, vals);
    CH_TRACE_PRINT("finalize");
    CH_TL(ctl, 4, 1);
}

// ---------------------------------------------------------------------------
// ch_filter: the label array Q of Alg. 2 and the queue sizes (paper rule).
__global__ void __launch_bounds__(256) labels_kernel(const float* __restrict__ pts, long long n,
                                                     Ctl* ctl, uint8_t* labels) {
    __shared__ Octagon s_o;
    __shared__ unsigned s_cnt[4];
    if (read_status(ctl) != CH_OK) return;
    copy_octagon(&s_o, &ctl->oct);
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    unsigned c[4] = {0u, 0u, 0u, 0u};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float2 p = reinterpret_cast<const float2*>(pts)[i];
        const int X = __float2int_rn(p.x), Y = __float2int_rn(p.y);
        const int r = in_inner_strict(s_o, X, Y) ? -1 : classify_paper_slow(p.x, p.y, &s_o);
        if (labels) labels[i] = (uint8_t)(r + 1);
        if (r >= 0) c[r]++;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        unsigned v = c[r];
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_cnt[r], v);
    }
    __syncthreads();
    if (threadIdx.x < 4 && s_cnt[threadIdx.x]) atomicAdd(&ctl->counts4[threadIdx.x], s_cnt[threadIdx.x]);
}

// The label of one point by the paper rule: -1 inside the octagon's inner
// region or the octagon, else its queue.
__device__ __forceinline__ int label_of(float x, float y, const Octagon& o) {
    const int X = __float2int_rn(x), Y = __float2int_rn(y);
    return in_inner_strict(o, X, Y) ? -1 : classify_paper_slow(x, y, &o);
}

// The label pass fed by bulk copies, for 16-byte aligned points and a 4-byte
// aligned label array: each warp streams its warp tiles (512 points) through
// a double-buffered shared-memory ring, as the main pass does, and labels 4
// consecutive points per lane and round (one 32-bit store of 4 labels; a
// tile is 4 rounds).  The ragged tail (fewer than 512 points) is labelled
// point by point by the first warp.
constexpr size_t kLabStreamSmemBytes = (size_t)8 * kStages * kWarpTileF4 * sizeof(float4);

__global__ void __launch_bounds__(256) labels_stream_kernel(const float4* __restrict__ p4, long long n,
                                                            long long ntiles, Ctl* ctl, uint32_t* labels4) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ Octagon s_o;
    __shared__ unsigned s_cnt[4];
    __shared__ unsigned long long s_bar[8][kStages];
    if (read_status(ctl) != CH_OK) return;
    copy_octagon(&s_o, &ctl->oct);
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned c[4] = {0u, 0u, 0u, 0u};
    WarpStream ws{reinterpret_cast<float4*>(dsm) + warp * kStages * kWarpTileF4, s_bar[warp], p4, gwarp, nwarps,
                  ntiles, lane};
    ws.start();
    for (long long k = 0;; ++k) {
        const long long t = gwarp + k * nwarps;
        if (t >= ntiles) break;
        const float4* cur = ws.acquire(k, ctl);
        if (!cur) {   // a copy never completed: status is CH_ETIMEOUT
            ws.drain(k);
            break;
        }
#pragma unroll
        for (int r = 0; r < kWarpTilePts / 128; ++r) {
            const int q = r * 32 + lane;   // 4 points: float4 2q and 2q + 1 of the tile
            const float4 a = cur[2 * q], b = cur[2 * q + 1];
            const float xs[4] = {a.x, a.z, b.x, b.z}, ys[4] = {a.y, a.w, b.y, b.w};
            uint32_t word = 0u;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int X = __float2int_rn(xs[m]), Y = __float2int_rn(ys[m]);
                int lab = -1;
                if (!in_inner_strict(s_o, X, Y)) lab = classify_paper_slow(xs[m], ys[m], &s_o);
                word |= (uint32_t)(lab + 1) << (8 * m);
                c[0] += lab == 0; c[1] += lab == 1; c[2] += lab == 2; c[3] += lab == 3;
            }
            if (labels4) labels4[t * (kWarpTilePts / 4) + q] = word;
        }
        ws.release(k);
    }
    if (gwarp == 0) {   // the ragged tail
        for (long long i = ntiles * kWarpTilePts + lane; i < n; i += 32) {
            const float2 p = reinterpret_cast<const float2*>(p4)[i];
            const int lab = label_of(p.x, p.y, s_o);
            if (labels4) reinterpret_cast<uint8_t*>(labels4)[i] = (uint8_t)(lab + 1);
            if (lab >= 0) c[lab]++;
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        unsigned v = c[r];
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if (lane == 0 && v) atomicAdd(&s_cnt[r], v);
    }
    __syncthreads();
    if (threadIdx.x < 4 && s_cnt[threadIdx.x]) atomicAdd(&ctl->counts4[threadIdx.x], s_cnt[threadIdx.x]);
}

__global__ void filter_output_kernel(const Ctl* ctl, long long n, int32_t* out_ext8, int64_t* out_counts4) {
    const int t = threadIdx.x;
    const int st = read_status(ctl);
    if (t < 8 && out_ext8) out_ext8[t] = (n == 0 || st != CH_OK) ? -1 : ctl->oct.ext[t];
    if (t < 4 && out_counts4) out_counts4[t] = (st != CH_OK) ? (int64_t)st : (int64_t)ctl->counts4[t];
}

// ---------------------------------------------------------------------------
// Host launchers
void launch_init(Ctl* ctl, int mode, cudaStream_t s) { init_kernel<<<1, 256, 0, s>>>(ctl, mode); }

void launch_sample(const float* pts, long long n, int head, long long ntiles, Ctl* ctl, int grid, cudaStream_t s) {
    sample_kernel<<<grid, 256, 0, s>>>(pts, n, head, ntiles, ctl);
}

void launch_main(const float* pts, long long n, int head, long long ntiles, Ctl* ctl, uint64_t* raw_xy,
                 uint32_t* raw_idx, unsigned switch_at, uint32_t* keys, uint64_t* vals, int grid, cudaStream_t s) {
    main_kernel<<<grid, 256, kMainSmemBytes, s>>>(pts, n, head, ntiles, ctl, raw_xy, raw_idx, switch_at, keys, vals);
}

void launch_labels(const float* pts, long long n, Ctl* ctl, uint8_t* labels, int grid, cudaStream_t s) {
    if (((uintptr_t)pts & 15u) == 0u && ((uintptr_t)labels & 3u) == 0u) {
        const long long ntiles = n / kWarpTilePts;
        labels_stream_kernel<<<grid, 256, kLabStreamSmemBytes, s>>>(reinterpret_cast<const float4*>(pts), n, ntiles,
                                                                    ctl, reinterpret_cast<uint32_t*>(labels));
    } else {
        labels_kernel<<<grid, 256, 0, s>>>(pts, n, ctl, labels);
    }
}

void launch_filter_output(const Ctl* ctl, long long n, int32_t* out_ext8, int64_t* out_counts4, cudaStream_t s) {
    filter_output_kernel<<<1, 32, 0, s>>>(ctl, n, out_ext8, out_counts4);
}

long long sample_tiles_host(long long ntiles) { return sample_tiles(ntiles); }

cudaError_t configure_filter_kernels() {
    cudaError_t e = cudaFuncSetAttribute(main_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMainSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(labels_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kLabStreamSmemBytes);
    return e;
}

cudaError_t occupancy_filter(int* main_k, int* labels) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(main_k, main_kernel, 256, kMainSmemBytes);
    int a = 0, b = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, labels_kernel, 256, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, labels_stream_kernel, 256, kLabStreamSmemBytes);
    *labels = a < b ? a : b;   // one grid size for both label kernels
    return e;
}

}  // namespace ch
