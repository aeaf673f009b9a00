// bkwarp.cuh -- one warp's lower chain of a bucket of sort records (quickhull
// rounds with the records in registers), shared by the single-hull bucket
// pass and the batched large-survivor path.
#pragma once

#include "ch_internal.cuh"

namespace ch {

// Debug builds (-DCH_PHASEPROF): cycles per phase of the warp chain, summed
// over all warps (lane 0 adds each phase's clock delta).
#ifdef CH_PHASEPROF
static __device__ unsigned long long g_bk_phase[16];
#define CH_PH_DECL unsigned long long _ph_t = clock64();
#define CH_PH(k) do { const unsigned long long _t = clock64(); \
    if ((threadIdx.x & 31) == 0) atomicAdd(&g_bk_phase[k], _t - _ph_t); _ph_t = _t; } while (0)
#define CH_PH_COUNT(k) do { if ((threadIdx.x & 31) == 0) atomicAdd(&g_bk_phase[k], 1ull); } while (0)
#else
#define CH_PH_DECL
#define CH_PH(k) do { } while (0)
#define CH_PH_COUNT(k) do { } while (0)
#endif

constexpr int kBkPer = 9;               // records per lane
constexpr int kBkWCap = 32 * kBkPer;    // records a warp holds at once
constexpr int kBkV = kBkChain + 2;      // quickhull vertices of one bucket

// One warp's quickhull over m <= kBkWCap records of one queue frame: the
// lower chain from S (minimum u, v, index) to E (maximum u, then minimum v,
// index); the same rounds and tie rules as qh_chains, synchronised within the
// warp only.  The records live in registers (slot k of lane l is record
// 32 k + l), so a round's loads are only of the few chain vertices.
struct BkWarp {   // shared memory of one warp: the chain under construction
    int4 seg[kBkV];    // segment from vertex a to its successor: u_a, v_a, du, dv
    int2 sc[kBkV];     // split of segment a in the last round: u of the new vertex (-1: none), new segment
    unsigned long long segmax[kBkV], segarg[kBkV];
    int vu[kBkV], vv[kBkV], vi[kBkV], vnext[kBkV];
    int cu[kBkV], cv[kBkV], ci[kBkV];   // the finished chain in order
    int tu[kBkWCap], tv[kBkWCap], ti[kBkWCap];   // live records between rounds (u | segment << 25)
};

struct BkRecs {
    int u[kBkPer], v[kBkPer], i[kBkPer], s[kBkPer];
};

// Depth of (u, v) below segment g (positive: strictly below).
__device__ __forceinline__ long long bk_depth(const int4 g, int u, int v) {
    return (long long)g.w * (u - g.x) - (long long)g.z * (v - g.y);
}

// Returns the chain length, its vertices in order in w.cu / cv / ci; -1 when
// the chain would exceed kBkV vertices.
static __device__ int bk_warp_chain(BkWarp& w, BkRecs& R, int m) {
    const int lane = threadIdx.x & 31;
    CH_PH_DECL
    CH_PH_COUNT(15);
    constexpr unsigned long long kVMask = (1ull << kKeyBits) - 1ull;
    unsigned long long ks = ~0ull, ke = 0ull;
#pragma unroll
    for (int k = 0; k < kBkPer; ++k) {
        if (k * 32 >= m) break;   // warp-uniform: slots past the records
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
        if (k * 32 >= m) break;
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
    const int vs = (int)(ks & kVMask), ve = (int)(kVMask - (ke & kVMask));
    CH_PH(1);
    for (int a = lane; a < kBkV; a += 32) {
        w.segmax[a] = 0ull;
        w.segarg[a] = ~0ull;
        w.sc[a] = make_int2(-1, -1);
    }
#pragma unroll
    for (int k = 0; k < kBkPer; ++k)
        R.s[k] = (k * 32 + lane < m && su < R.u[k] && R.u[k] < eu) ? 0 : -1;
    // First round, on the chord S -> E with every record in registers: the
    // deepest record below it (smallest u, then index, on ties) becomes F.
    const long long cdu = (long long)(eu - su), cdv = (long long)(ve - vs);
    unsigned long long dmax = 0ull;
#pragma unroll
    for (int k = 0; k < kBkPer; ++k) {
        if (k * 32 >= m) break;
        if (R.s[k] == 0) {
            const long long d = cdv * (R.u[k] - su) - cdu * (R.v[k] - vs);
            if (d <= 0) R.s[k] = -1;
            else dmax = (unsigned long long)d > dmax ? (unsigned long long)d : dmax;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xFFFFFFFFu, dmax, o);
        dmax = t > dmax ? t : dmax;
    }
    if (dmax == 0ull) {   // S, E (one vertex when every record has the same u)
        if (lane == 0) {
            w.cu[0] = su;
            w.cv[0] = vs;
            w.ci[0] = (int)is;
            w.cu[1] = eu;
            w.cv[1] = ve;
            w.ci[1] = (int)ie;
        }
        __syncwarp();
        return su < eu ? 2 : 1;
    }
    unsigned long long best = ~0ull;
#pragma unroll
    for (int k = 0; k < kBkPer; ++k) {
        if (k * 32 >= m) break;
        if (R.s[k] == 0 && (unsigned long long)(cdv * (R.u[k] - su) - cdu * (R.v[k] - vs)) == dmax) {
            const unsigned long long key = ((unsigned long long)R.u[k] << 31) | (unsigned)R.i[k];
            best = key < best ? key : best;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xFFFFFFFFu, best, o);
        best = t < best ? t : best;
    }
    const int fu = (int)(best >> 31), fi = (int)(best & 0x7FFFFFFFull);
    int fv = 0;
    bool own = false;
#pragma unroll
    for (int k = 0; k < kBkPer; ++k) {
        if (k * 32 >= m) break;
        if (R.s[k] == 0 && R.u[k] == fu && R.i[k] == fi) {
            own = true;
            fv = R.v[k];
        }
    }
    fv = __shfl_sync(0xFFFFFFFFu, fv, __ffs(__ballot_sync(0xFFFFFFFFu, own)) - 1);
    if (lane == 0) {   // chain S -> F -> E; vertex 2 = F
        w.vu[0] = su;
        w.vv[0] = vs;
        w.vi[0] = (int)is;
        w.vu[1] = eu;
        w.vv[1] = ve;
        w.vi[1] = (int)ie;
        w.vu[2] = fu;
        w.vv[2] = fv;
        w.vi[2] = fi;
        w.vnext[0] = 2;
        w.vnext[2] = 1;
        w.vnext[1] = -1;
        w.seg[0] = make_int4(su, vs, fu - su, fv - vs);
        w.seg[2] = make_int4(fu, fv, eu - fu, ve - fv);
    }
#pragma unroll
    for (int k = 0; k < kBkPer; ++k)
        if (R.s[k] == 0) R.s[k] = R.u[k] < fu ? 0 : (R.u[k] > fu ? 2 : -1);
    __syncwarp();
    CH_PH(2);
    int nv = 3;
    for (int round = 1;; ++round) {
        CH_PH_COUNT(14);
        // depths; each segment's maximum
        int live = 0;
#pragma unroll
        for (int k = 0; k < kBkPer; ++k) {
            if (k * 32 >= m) break;
            int a = R.s[k];
            if (a >= 0) {   // every live record's segment has a successor
                const int2 sc = w.sc[a];
                if (sc.x >= 0) {
                    if (R.u[k] > sc.x) a = sc.y;
                    else if (R.u[k] == sc.x) a = -1;
                }
                if (a >= 0) {
                    const long long d = bk_depth(w.seg[a], R.u[k], R.v[k]);
                    if (d <= 0) a = -1;
                    else if ((unsigned long long)d > *(volatile unsigned long long*)&w.segmax[a])
                        atomicMax(&w.segmax[a], (unsigned long long)d);
                }
                R.s[k] = a;
            }
            live += __popc(__ballot_sync(0xFFFFFFFFu, R.s[k] >= 0));
        }
        CH_PH(3);
        // records below the chain only: packed to the first slots when that
        // saves slots (each round keeps a small part of the records)
        if (live + 31 < ((m + 31) & ~31)) {
            int pos = 0;
#pragma unroll
            for (int k = 0; k < kBkPer; ++k) {
                if (k * 32 >= m) break;
                const bool keep = R.s[k] >= 0;
                const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
                if (keep) {
                    const int p = pos + __popc(bal & lanemask_lt());
                    w.tu[p] = R.u[k] | (R.s[k] << 25);
                    w.tv[p] = R.v[k];
                    w.ti[p] = R.i[k];
                }
                pos += __popc(bal);
            }
            __syncwarp();
            m = live;
#pragma unroll
            for (int k = 0; k < kBkPer; ++k) {
                if (k * 32 >= m) break;
                const int j = k * 32 + lane;
                R.s[k] = -1;
                if (j < m) {
                    const int t = w.tu[j];
                    R.u[k] = t & 0x1FFFFFF;
                    R.s[k] = t >> 25;
                    R.v[k] = w.tv[j];
                    R.i[k] = w.ti[j];
                }
            }
            __syncwarp();
        }
        __syncwarp();
        CH_PH(4);
        // the deepest record per segment: smallest u, then index
#pragma unroll
        for (int k = 0; k < kBkPer; ++k) {
            if (k * 32 >= m) break;
            const int a = R.s[k];
            if (a >= 0 && (unsigned long long)bk_depth(w.seg[a], R.u[k], R.v[k]) == w.segmax[a])
                atomicMin(&w.segarg[a], ((unsigned long long)R.u[k] << 31) | (unsigned)R.i[k]);
        }
        __syncwarp();
        CH_PH(5);
        int added = 0;
        bool over = false;
        for (int a0 = 0; a0 < nv; a0 += 32) {
            const int a = a0 + lane;
            const unsigned long long dm = a < nv ? w.segmax[a] : 0ull;
            const bool split = dm != 0ull;
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, split);
            if (a < nv) w.sc[a] = make_int2(-1, -1);
            if (split) {
                const int f = nv + added + __popc(bal & lanemask_lt());
                if (f < kBkV) {
                    const int b = w.vnext[a];
                    const int4 g = w.seg[a];
                    const unsigned long long key = w.segarg[a];
                    const int fu = (int)(key >> 31), fi = (int)(key & 0x7FFFFFFFull);
                    // v of the new vertex from its depth (an exact quotient)
                    const long long num = (long long)g.w * (fu - g.x) - (long long)dm;
                    const int fv = g.y + (int)(num / (long long)g.z);
                    w.vu[f] = fu;
                    w.vv[f] = fv;
                    w.vi[f] = fi;
                    w.vnext[f] = b;
                    w.vnext[a] = f;
                    w.seg[a] = make_int4(g.x, g.y, fu - g.x, fv - g.y);
                    w.seg[f] = make_int4(fu, fv, g.x + g.z - fu, g.y + g.w - fv);
                    w.sc[a] = make_int2(fu, f);
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
        CH_PH(6);
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
    CH_PH(7);
    return len;
}


// The lower chain of a stream of cnt records (one queue frame) by one warp,
// kBkWCap records at a time: each chunk's chain is carried into the next
// chunk as records.  load(j, u, v, i) reads record j of the stream.  Returns
// the chain's length (<= kBkChain, the chain in w.cu / cv / ci), or -1 when
// it has more than kBkChain vertices.
template <typename Load>
__device__ __forceinline__ int bk_stream_chain(BkWarp& w, unsigned cnt, Load load) {
    const int lane = threadIdx.x & 31;
    int len = 0;
    for (unsigned c0 = 0; c0 < cnt;) {
        CH_PH_DECL
        const unsigned take = min(cnt - c0, (unsigned)(kBkWCap - len));
        const int m = len + (int)take;
        BkRecs R;
        // every slot loads (an index clamped into this chunk, take >= 1), so
        // the loads of all slots are in flight together; then the carried
        // chain and the empty slots override
#pragma unroll
        for (int k = 0; k < kBkPer; ++k) {
            const int j = k * 32 + lane;
            const int g = min(max(j - len, 0), (int)take - 1);
            load(c0 + (unsigned)g, R.u[k], R.v[k], R.i[k]);
        }
#pragma unroll
        for (int k = 0; k < kBkPer; ++k) {
            const int j = k * 32 + lane;
            if (j < len) {
                R.u[k] = w.cu[j];
                R.v[k] = w.cv[j];
                R.i[k] = w.ci[j];
            } else if (j >= m) {
                R.u[k] = 0;
                R.v[k] = 0;
                R.i[k] = 0;
            }
        }
        __syncwarp();
        CH_PH(0);
        const int l2 = bk_warp_chain(w, R, m);
        if (l2 < 0 || l2 > kBkChain) return -1;
        len = l2;
        c0 += take;
    }
    return len;
}

// The lower chain of bucket records [start, start + cnt) of keys / vals.
__device__ __forceinline__ int bk_bucket_chain(BkWarp& w, const uint32_t* keys, const uint64_t* vals,
                                               unsigned start, unsigned cnt) {
    return bk_stream_chain(w, cnt, [&](unsigned j, int& u, int& v, int& i) {
        const uint32_t kk = __ldcs(keys + start + j);
        const uint64_t vv = __ldcs(vals + start + j);
        u = (int)(kk & kKeyMask);
        v = (int)(vv >> 31);
        i = (int)(vv & 0x7FFFFFFFull);
    });
}

}  // namespace ch
