// hullcore.cuh -- block-level pieces of the hull stage shared by the kernels:
//   stitch_core  joins the four queue chains into the output list;
//   tiny_hull    the whole hull stage for a few hundred records in one block
//                (no sort): used when the filter leaves few survivors.
#pragma once

#include <climits>

#include "ch_internal.cuh"

namespace ch {

// ---------------------------------------------------------------------------
// Lower convex chains in a queue frame (u strictly increasing).  Merging two
// chains A, B with every u of A below every u of B: a_k (k > 0) stays iff every
// b in B is strictly left of a_{k-1} -> a_k; b_l (l < |B| - 1) stays iff every
// a in A is strictly left of b_l -> b_{l+1}.  Both predicates hold on a prefix
// of A / a suffix of B, and "every b" reduces to the minimum of a linear
// function over the convex chain B, found by binary search.
struct ChainPtr {   // structure-of-arrays view of a chain (u, v, index)
    int* u;
    int* v;
    int* i;
};

__device__ __forceinline__ long long cross_uv(int ou, int ov, int au, int av, int bu, int bv) {
    return (long long)(au - ou) * (long long)(bv - ov) - (long long)(av - ov) * (long long)(bu - ou);
}

template <bool kGlobal>
__device__ __forceinline__ int ldi(const int* p) {
    if (kGlobal) return __ldcg(p);
    return *p;
}

// Minimum over chain C[0..lc) of f(c) = cross(p, q, c), q.u > p.u.  Along a
// lower convex chain the increments cross(q - p, c_{l+1} - c_l) change sign
// once (negative, then >= 0), so f is minimal at the first l whose next edge
// does not decrease it.
template <bool kGlobal>
__device__ long long min_cross_over(const int* cu, const int* cv, int lc, int pu, int pv, int qu,
                                    int qv) {
    int lo = 0, hi = lc - 1;   // answer in [lo, hi]
    const long long du = qu - pu, dv = qv - pv;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const long long eu = (long long)ldi<kGlobal>(cu + mid + 1) - ldi<kGlobal>(cu + mid);
        const long long ev = (long long)ldi<kGlobal>(cv + mid + 1) - ldi<kGlobal>(cv + mid);
        if (du * ev - dv * eu >= 0) hi = mid; else lo = mid + 1;
    }
    return cross_uv(pu, pv, qu, qv, ldi<kGlobal>(cu + lo), ldi<kGlobal>(cv + lo));
}

template <bool kGlobal>
__device__ __forceinline__ bool keep_a(const ChainPtr& A, int k, const ChainPtr& B, int lb) {
    if (k == 0) return true;
    return min_cross_over<kGlobal>(B.u, B.v, lb, ldi<kGlobal>(A.u + k - 1), ldi<kGlobal>(A.v + k - 1),
                                   ldi<kGlobal>(A.u + k), ldi<kGlobal>(A.v + k)) > 0;
}

template <bool kGlobal>
__device__ __forceinline__ bool keep_b(const ChainPtr& A, int la, const ChainPtr& B, int l, int lb) {
    if (l == lb - 1) return true;
    return min_cross_over<kGlobal>(A.u, A.v, la, ldi<kGlobal>(B.u + l), ldi<kGlobal>(B.v + l),
                                   ldi<kGlobal>(B.u + l + 1), ldi<kGlobal>(B.v + l + 1)) > 0;
}

// Sequential bridge (one thread): last kept index of A, first kept of B.
template <bool kGlobal>
__device__ void bridge_seq(const ChainPtr& A, int la, const ChainPtr& B, int lb, int& is, int& js) {
    int lo = 0, hi = la - 1;               // keep_a(lo) true
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (keep_a<kGlobal>(A, mid, B, lb)) lo = mid; else hi = mid - 1;
    }
    is = lo;
    lo = 0; hi = lb - 1;                   // keep_b(hi) true
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (keep_b<kGlobal>(A, la, B, mid, lb)) hi = mid; else lo = mid + 1;
    }
    js = lo;
}

// Merge chain B (at sb, length lb) into chain A (at sa, length la) in shared
// memory, one thread.  Returns the new length of A.
static __device__ int merge_smem_seq(int* su, int* sv, int* si, int sa, int la, int sb, int lb) {
    if (lb == 0) return la;
    if (la == 0) {
        for (int j = 0; j < lb; ++j) { su[sa + j] = su[sb + j]; sv[sa + j] = sv[sb + j]; si[sa + j] = si[sb + j]; }
        return lb;
    }
    ChainPtr A{su + sa, sv + sa, si + sa}, B{su + sb, sv + sb, si + sb};
    int is, js;
    bridge_seq<false>(A, la, B, lb, is, js);
    const int n = lb - js;
    for (int j = 0; j < n; ++j) {
        su[sa + is + 1 + j] = su[sb + js + j];
        sv[sa + is + 1 + j] = sv[sb + js + j];
        si[sa + is + 1 + j] = si[sb + js + j];
    }
    return is + 1 + n;
}

template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T* s_tmp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v = op(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    __syncthreads();
    if (lane == 0) s_tmp[warp] = v;
    __syncthreads();
    T r = s_tmp[0];
    for (int w = 1; w < nw; ++w) r = op(r, s_tmp[w]);
    __syncthreads();
    return r;
}

// Exclusive block scan of one int per thread; *total receives the sum.
__device__ __forceinline__ int block_excl_scan(int x, int* s_tmp, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();
    if (lane == 31) s_tmp[warp] = incl;
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < warp) off += s_tmp[w];
        tot += s_tmp[w];
    }
    __syncthreads();
    *total = tot;
    return off + incl - x;
}

__device__ __forceinline__ void pt_xy(const float* pts, int i, long long& x, long long& y) {
    const float2 p = reinterpret_cast<const float2*>(pts)[i];
    x = (long long)p.x;
    y = (long long)p.y;
}

__device__ __forceinline__ unsigned long long xy_key(long long x, long long y) {
    return ((unsigned long long)x << 24) | (unsigned long long)y;
}

// V[0..m): point indices of the concatenated queue chains W..S, S..E, E..N,
// N..W (each without its last point), a weakly convex cyclic polygon; xy(p,
// x, y) gives the coordinates of cycle position p.  Writes the strictly
// convex vertices counter-clockwise from the lexicographically smallest one;
// all-collinear input gives [lex-min, lex-max], one distinct point gives
// [it].  flag and comp are scratch arrays of m ints.
template <typename XY>
__device__ void stitch_core(const int* V, int m, int* flag, int* comp, XY xy, long long n, Ctl* ctl,
                            int32_t* out_idx, int64_t* out_n) {
    __shared__ long long s_ll[32];
    __shared__ unsigned long long s_ull[32];
    __shared__ int s_int[33];
    __shared__ int s_a, s_b;
    const int tid = threadIdx.x, T = blockDim.x;
    if (m == 0) {   // all four quadrilateral vertices coincide
        if (tid == 0) { out_idx[0] = ctl->oct.ext[W]; *out_n = 1; }
        return;
    }
    long long npos = 0, nneg = 0;
    for (int i = tid; i < m; i += T) {
        long long ax, ay, bx, by, cx, cy;
        xy(i == 0 ? m - 1 : i - 1, ax, ay);
        xy(i, bx, by);
        xy(i + 1 == m ? 0 : i + 1, cx, cy);
        const long long tr = orient64(ax, ay, bx, by, cx, cy);
        flag[i] = tr > 0;
        npos += tr > 0;
        nneg += tr < 0;
    }
    auto add = [](long long a, long long b) { return a + b; };
    auto mn = [](unsigned long long a, unsigned long long b) { return a < b ? a : b; };
    auto mx = [](unsigned long long a, unsigned long long b) { return a > b ? a : b; };
    npos = block_reduce<long long>(npos, add, s_ll);
    nneg = block_reduce<long long>(nneg, add, s_ll);
    if (npos == 0) {   // degenerate: a segment or a single point
        unsigned long long lo = ~0ull, hi = 0ull;
        for (int i = tid; i < m; i += T) {
            long long x, y;
            xy(i, x, y);
            const unsigned long long k = xy_key(x, y);
            lo = k < lo ? k : lo;
            hi = k > hi ? k : hi;
        }
        lo = block_reduce<unsigned long long>(lo, mn, s_ull);
        hi = block_reduce<unsigned long long>(hi, mx, s_ull);
        if (tid == 0) { s_a = INT_MAX; s_b = INT_MAX; }
        __syncthreads();
        for (int i = tid; i < m; i += T) {
            long long x, y;
            xy(i, x, y);
            const unsigned long long k = xy_key(x, y);
            if (k == lo) atomicMin(&s_a, V[i]);
            if (k == hi) atomicMin(&s_b, V[i]);
        }
        __syncthreads();
        if (tid == 0) {
            out_idx[0] = s_a;
            if (lo == hi) *out_n = 1;
            else { out_idx[1] = s_b; *out_n = 2; }
        }
        return;
    }
    if (nneg != 0 && tid == 0) set_status(ctl, CH_ECUDA);   // internal consistency check
    // Compact the strictly convex vertices; lexicographic minimum among them.
    int written = 0;
    unsigned long long best = ~0ull;
    for (int base = 0; base < m; base += T) {
        const int i = base + tid;
        const int f = (i < m) ? flag[i] : 0;
        int tot;
        const int ex = block_excl_scan(f, s_int, &tot);
        if (f) {
            long long x, y;
            xy(i, x, y);
            const unsigned long long k = xy_key(x, y);
            best = k < best ? k : best;
            comp[written + ex] = V[i];
        }
        if (i < m) flag[i] = f ? written + ex : -1;   // compacted position
        written += tot;
    }
    best = block_reduce<unsigned long long>(best, mn, s_ull);
    const int h = written;
    if (h > n) {   // cannot happen for a correct hull; never write past out_idx
        if (tid == 0) { set_status(ctl, CH_ECUDA); *out_n = CH_ECUDA; }
        return;
    }
    if (tid == 0) s_a = 0;
    __syncthreads();
    for (int i = tid; i < m; i += T) {
        if (flag[i] < 0) continue;
        long long x, y;
        xy(i, x, y);
        if (xy_key(x, y) == best) s_a = flag[i];
    }
    __syncthreads();
    const int start = s_a;
    for (int j = tid; j < h; j += T) {
        const int k = start + j;
        out_idx[j] = comp[k < h ? k : k - h];
    }
    __syncthreads();
    if (tid == 0) {
        const int st = read_status(ctl);
        *out_n = (st == CH_OK) ? h : st;
    }
}

// Dynamic shared memory of mid_hull: sort keys (kMidCap u64) followed by the
// chain arrays u | queue, v, index (kMidCap ints each).
constexpr size_t kMidSmemBytes = (size_t)kMidCap * 8 + (size_t)3 * kMidCap * 4;

// The whole hull stage for m <= kMidCap sort records (queue | u, v | index) in
// one block: bitonic sort of (key, position) in shared memory, run reduction
// (minimum (v, index) per key), the four queue chains built concurrently by a
// quarter of the block each (per-thread chains, then pairwise merges), and the
// stitch.  blockDim.x must be a multiple of 128.
static __device__ void mid_hull(const uint32_t* keys, const uint64_t* vals, int m, const float* __restrict__ pts,
                                long long n, Ctl* ctl, int32_t* out_idx, int64_t* out_n, char* smem) {
    __shared__ int s_rs[5];
    __shared__ int s_int[33];
    __shared__ int s_clen[1024];
    unsigned long long* sk = reinterpret_cast<unsigned long long*>(smem);
    int* cu = reinterpret_cast<int*>(sk + kMidCap);
    int* cv = cu + kMidCap;
    int* ci = cv + kMidCap;
    CH_TRACE_DECL
    CH_TRACE_MARK();
    const int tid = threadIdx.x, T = blockDim.x;
    int P = 1;
    while (P < m) P <<= 1;
    for (int i = tid; i < P; i += T)
        sk[i] = i < m ? (((unsigned long long)keys[i] << 13) | (unsigned long long)i) : ~0ull;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {          // bitonic sort, ascending
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += T) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long a = sk[i], b = sk[l];
                    if ((a > b) == ((i & k) == 0)) { sk[i] = b; sk[l] = a; }
                }
            }
            __syncthreads();
        }
    }
    CH_TRACE_MARK();
    // run reduction: one point per (queue, u), the minimum (v, index)
    int written = 0;
    for (int base = 0; base < m; base += T) {
        const int p = base + tid;
        int f = 0;
        unsigned key = 0u;
        unsigned long long best = 0ull;
        if (p < m) {
            key = (unsigned)(sk[p] >> 13);
            f = (p == 0) || (unsigned)(sk[p - 1] >> 13) != key;
            if (f) {
                best = vals[sk[p] & 8191ull];
                for (int q = p + 1; q < m && (unsigned)(sk[q] >> 13) == key; ++q) {
                    const unsigned long long w = vals[sk[q] & 8191ull];
                    best = w < best ? w : best;
                }
            }
        }
        int tot;
        const int ex = block_excl_scan(f, s_int, &tot);
        if (f) {
            cu[written + ex] = (int)key;                 // queue in bits 25..26, u below
            cv[written + ex] = (int)(best >> 31);
            ci[written + ex] = (int)(best & 0x7FFFFFFFull);
        }
        written += tot;
    }
    __syncthreads();
    const int m2 = written;
    for (int p = tid; p <= m2; p += T) {         // queue boundaries
        const int prev = p == 0 ? -1 : (cu[p - 1] >> kKeyBits);
        const int cur = p == m2 ? 4 : (cu[p] >> kKeyBits);
        for (int r = prev + 1; r <= cur; ++r) s_rs[r] = p;
    }
    __syncthreads();
    CH_TRACE_MARK();
    // four queues at once, a quarter of the block each; queue bits are equal
    // within a queue, so cross products of cu differences are those of u
    const int G = T / 4, g = tid / G, lt = tid % G;
    const int qa = s_rs[g], qb = s_rs[g + 1];
    const int chunk = (qb - qa + G - 1) / G;
    const int my0 = qa + lt * chunk, my1 = min(qb, my0 + chunk);
    {
        int sp = 0;
        for (int p = my0; p < my1; ++p) {
            const int pu = cu[p], pv = cv[p], pi = ci[p];
            while (sp >= 2 && cross_uv(cu[my0 + sp - 2], cv[my0 + sp - 2], cu[my0 + sp - 1], cv[my0 + sp - 1], pu, pv) <= 0)
                --sp;
            cu[my0 + sp] = pu; cv[my0 + sp] = pv; ci[my0 + sp] = pi;
            ++sp;
        }
        s_clen[tid] = my1 > my0 ? sp : 0;
    }
    __syncthreads();
    for (int l = 0; (1 << l) < G; ++l) {
        const int gsz = 1 << l;
        if ((lt & (2 * gsz - 1)) == 0 && lt + gsz < G) {
            const int b0 = qa + (lt + gsz) * chunk;
            if (b0 < qb)
                s_clen[tid] = merge_smem_seq(cu, cv, ci, my0, s_clen[tid], b0, s_clen[tid + gsz]);
        }
        __syncthreads();
    }
    CH_TRACE_MARK();
    // stitch: V (in the sort buffer) = the queue chains without their last point
    int* V = reinterpret_cast<int*>(sk);
    int* flag = V + kMidCap;
    int off[5];
    off[0] = 0;
    for (int r = 0; r < 4; ++r) off[r + 1] = off[r] + max(s_clen[r * G] - 1, 0);
    for (int r = 0; r < 4; ++r)
        for (int j = tid; j < off[r + 1] - off[r]; j += T) V[off[r] + j] = ci[s_rs[r] + j];
    __syncthreads();
    CH_TRACE_MARK();
    stitch_core(V, off[4], flag, cu, [&](int p, long long& x, long long& y) { pt_xy(pts, V[p], x, y); }, n, ctl,
                out_idx, out_n);
    CH_TRACE_MARK();
    CH_TRACE_PRINT("mid_hull");
}

// ---------------------------------------------------------------------------
// Quickhull rounds over the four queue chains at once (quickhull is among the
// sequential algorithms of Table I; here every segment of every queue is
// refined in the same round, so the rounds grow with the logarithm of the
// chain length rather than with the vertex count).
//
// In queue r's frame the chain is the lower convex chain from S (minimum u,
// then v, then index) to E (maximum u, then minimum v, then index).  A segment
// a -> b of consecutive chain vertices owns the records with a.u < u < b.u.
// Each round every segment takes the record farthest below it,
// d = (b.v - a.v)(u - a.u) - (b.u - a.u)(v - a.v) > 0 largest, as a new vertex
// between a and b; among records at that distance (a line parallel to a -> b)
// the smallest u, then the lowest index: an end point of that line, hence a
// vertex.  Records on or above their segment are dropped: they are no strict
// vertices.  The round ends the process when no segment owns a record.
constexpr int kQhCap = 1024;     // chain vertices of all four queues
constexpr int kQhRounds = 64;

// Inverse of queue_frame.
__device__ __forceinline__ void frame_to_xy(int r, int u, int v, int& x, int& y) {
    const int off = kCoordLimit, top = 2 * kCoordLimit - 2;
    switch (r) {
        case 0: x = (u + v - off) / 2; y = (v - u + off) / 2; break;
        case 1: x = (u - v + off) / 2; y = (u + v - off) / 2; break;
        case 2: x = (top - v - u + off) / 2; y = (top - v + u - off) / 2; break;
        default: x = (top - u + v - off) / 2; y = (top - u - v + off) / 2; break;
    }
}

// Shared memory of the small hull (dynamic, placed by the caller).  After the
// rounds the record arrays hold the joined cycle (x, y, index) and the output.
// RCAP records, VCAP chain vertices of all four queues.
template <int RCAP, int VCAP>
struct QhSmemT {
    static constexpr int kRecords = RCAP, kVertices = VCAP;
    int ru[RCAP], rv[RCAP], ri[RCAP];            // records: u, v, index
    int rs[RCAP];                                // queue (on entry), then segment (left vertex), -1 dropped
    unsigned long long segmax[VCAP], segarg[VCAP];
    int vu[VCAP], vv[VCAP], vi[VCAP], vnext[VCAP];
    int splitu[VCAP], child[VCAP];
};
using QhSmem = QhSmemT<kMidCap, kQhCap>;

template <class Q>
__device__ __forceinline__ long long qh_depth(const Q& q, int a, int b, int u, int v) {
    return (long long)(q.vv[b] - q.vv[a]) * (u - q.vu[a]) - (long long)(q.vu[b] - q.vu[a]) * (v - q.vv[a]);
}

// The four chains; on success the joined cycle (every chain without its end
// vertex, which starts the next chain) is in q.ru / q.rv / q.ri as x, y,
// index, and its length in *mv.  False when a limit is exceeded (the caller
// falls back to the sort-based path).  Whole block; m records in q.
template <class Q>
static __device__ bool qh_chains(Q& q, int m, int* mv) {
    constexpr int kQhCap = Q::kVertices;
    __shared__ unsigned long long s_s[4], s_e[4];
    __shared__ int s_si[4], s_ei[4], s_len[4], s_nvert, s_changed, s_fail;
    const int tid = threadIdx.x, T = blockDim.x;
    constexpr int kVBits = kKeyBits;   // v < 2^25 in every frame
    constexpr unsigned long long kVMask = (1ull << kVBits) - 1ull;
    if (tid < 4) { s_s[tid] = ~0ull; s_e[tid] = 0ull; s_si[tid] = INT_MAX; s_ei[tid] = INT_MAX; }
    if (tid == 0) { s_nvert = 8; s_fail = 0; s_changed = 0; }
    for (int a = tid; a < kQhCap; a += T) { q.segmax[a] = 0ull; q.segarg[a] = ~0ull; q.splitu[a] = -1; }
    __syncthreads();
    // S = minimum (u, v); E = maximum u, then minimum v; then lowest indices
    for (int i = tid; i < m; i += T) {
        const int r = q.rs[i];
        const unsigned long long ks = ((unsigned long long)q.ru[i] << kVBits) | (unsigned)q.rv[i];
        const unsigned long long ke = ((unsigned long long)q.ru[i] << kVBits) | (kVMask - (unsigned)q.rv[i]);
        if (ks < *(volatile unsigned long long*)&s_s[r]) atomicMin(&s_s[r], ks);
        if (ke > *(volatile unsigned long long*)&s_e[r]) atomicMax(&s_e[r], ke);
    }
    __syncthreads();
    for (int i = tid; i < m; i += T) {
        const int r = q.rs[i];
        const unsigned long long ks = ((unsigned long long)q.ru[i] << kVBits) | (unsigned)q.rv[i];
        const unsigned long long ke = ((unsigned long long)q.ru[i] << kVBits) | (kVMask - (unsigned)q.rv[i]);
        if (ks == s_s[r]) atomicMin(&s_si[r], q.ri[i]);
        if (ke == s_e[r]) atomicMin(&s_ei[r], q.ri[i]);
    }
    __syncthreads();
    if (tid < 4) {
        const int r = tid;
        if (s_si[r] == INT_MAX || s_ei[r] == INT_MAX) s_fail = 1;   // empty queue: cannot happen
        q.vu[2 * r] = (int)(s_s[r] >> kVBits);
        q.vv[2 * r] = (int)(s_s[r] & kVMask);
        q.vi[2 * r] = s_si[r];
        q.vu[2 * r + 1] = (int)(s_e[r] >> kVBits);
        q.vv[2 * r + 1] = (int)(kVMask - (s_e[r] & kVMask));
        q.vi[2 * r + 1] = s_ei[r];
        q.vnext[2 * r] = q.vu[2 * r] < q.vu[2 * r + 1] ? 2 * r + 1 : -1;   // S == E: a one-point chain
        q.vnext[2 * r + 1] = -1;
    }
    __syncthreads();
    if (s_fail) return false;
    for (int i = tid; i < m; i += T) {
        const int r = q.rs[i], u = q.ru[i];
        q.rs[i] = (q.vu[2 * r] < u && u < q.vu[2 * r + 1]) ? 2 * r : -1;
    }
    CH_TRACE_MARK();
    for (int round = 0;; ++round) {
        const int nv = s_nvert;
        // depths; each segment's maximum
        for (int i = tid; i < m; i += T) {
            int a = q.rs[i];
            if (a < 0) continue;
            const int u = q.ru[i], v = q.rv[i];
            const int su = q.splitu[a];
            if (su >= 0) {   // split last round: stay left of the new vertex, or move right of it
                if (u > su) a = q.child[a];
                else if (u == su) a = -1;
            }
            const int b = a >= 0 ? q.vnext[a] : -1;
            if (b < 0) {
                a = -1;   // (a segment always has a right end; defensive)
            } else {
                const long long d = qh_depth(q, a, b, u, v);
                if (d <= 0) a = -1;
                else if ((unsigned long long)d > *(volatile unsigned long long*)&q.segmax[a])
                    atomicMax(&q.segmax[a], (unsigned long long)d);
            }
            q.rs[i] = a;
        }
        __syncthreads();
        CH_TRACE_MARK();
        if (tid == 0) s_changed = 0;
        // the deepest record per segment: smallest u, then index
        for (int i = tid; i < m; i += T) {
            const int a = q.rs[i];
            if (a < 0) continue;
            const int u = q.ru[i];
            const long long d = qh_depth(q, a, q.vnext[a], u, q.rv[i]);
            if ((unsigned long long)d == q.segmax[a])
                atomicMin(&q.segarg[a], ((unsigned long long)u << 31) | (unsigned)q.ri[i]);
        }
        __syncthreads();
        CH_TRACE_MARK();
        // insert the new vertices
        for (int a = tid; a < nv; a += T) {
            q.splitu[a] = -1;
            const unsigned long long dm = q.segmax[a];
            if (dm == 0ull) continue;
            const int b = q.vnext[a];
            const unsigned long long key = q.segarg[a];
            const int fu = (int)(key >> 31), fi = (int)(key & 0x7FFFFFFFull);
            // v from the depth: exact (the quotient of an exact integer identity)
            const long long num = (long long)(q.vv[b] - q.vv[a]) * (fu - q.vu[a]) - (long long)dm;
            const int fv = q.vv[a] + (int)(num / (long long)(q.vu[b] - q.vu[a]));
            const int f = atomicAdd(&s_nvert, 1);
            if (f < kQhCap) {
                q.vu[f] = fu;
                q.vv[f] = fv;
                q.vi[f] = fi;
                q.vnext[f] = b;
                q.vnext[a] = f;
                q.child[a] = f;
                q.splitu[a] = fu;
            } else {
                s_fail = 1;
            }
            q.segmax[a] = 0ull;
            q.segarg[a] = ~0ull;
            s_changed = 1;
        }
        __syncthreads();
        CH_TRACE_MARK();
        if (s_fail || (s_changed && round + 1 >= kQhRounds)) return false;
        if (!s_changed) break;
    }
    // chain lengths, then the joined cycle (chain r without its end vertex)
    if (tid < 4) {
        int len = 0;
        for (int a = 2 * tid; a >= 0 && len <= kQhCap; a = q.vnext[a]) ++len;
        s_len[tid] = len;
    }
    __syncthreads();
    int off[5];
    off[0] = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) off[r + 1] = off[r] + max(s_len[r] - 1, 0);
    if (tid < 4) {
        const int r = tid;
        int pos = off[r];
        for (int a = 2 * r; a >= 0 && pos < off[r + 1]; a = q.vnext[a], ++pos) {
            int x, y;
            frame_to_xy(r, q.vu[a], q.vv[a], x, y);
            q.ru[pos] = x;
            q.rv[pos] = y;
            q.ri[pos] = q.vi[a];
        }
    }
    __syncthreads();
    *mv = off[4];
    return true;
}

// Joins the cycle (x, y, index in X, Y, V; mv points) into the output: the
// strictly convex vertices, counter-clockwise from the lexicographically
// smallest; a degenerate cycle gives [lex-min, lex-max] (or one point).  One
// warp (warp 0) works; tmp holds mv ints.
static __device__ void stitch_cycle(const int* X, const int* Y, const int* V, int mv, int* tmp, Ctl* ctl,
                                    long long n, int32_t* out_idx, int64_t* out_n) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp != 0) return;
    if (mv == 0) {   // all four quadrilateral vertices coincide
        if (lane == 0) { out_idx[0] = ctl->oct.ext[W]; *out_n = 1; }
        return;
    }
    int npos = 0, nneg = 0;
    for (int i = lane; i < mv; i += 32) {
        const int p = i == 0 ? mv - 1 : i - 1, q = i + 1 == mv ? 0 : i + 1;
        const long long tr = orient64(X[p], Y[p], X[i], Y[i], X[q], Y[q]);
        npos += tr > 0;
        nneg += tr < 0;
        tmp[i] = tr > 0;
    }
    npos = __reduce_add_sync(0xFFFFFFFFu, (unsigned)npos);
    nneg = __reduce_add_sync(0xFFFFFFFFu, (unsigned)nneg);
    if (npos == 0) {   // degenerate: [lex-min, lex-max], lowest index per coordinate
        unsigned long long lo = ~0ull, hi = 0ull;
        for (int i = lane; i < mv; i += 32) {
            const unsigned long long kxy = xy_key(X[i], Y[i]);
            lo = kxy < lo ? kxy : lo;
            hi = kxy > hi ? kxy : hi;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long a2 = __shfl_xor_sync(0xFFFFFFFFu, lo, o), b2 = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
            lo = a2 < lo ? a2 : lo;
            hi = b2 > hi ? b2 : hi;
        }
        unsigned ilo = 0xFFFFFFFFu, ihi = 0xFFFFFFFFu;
        for (int i = lane; i < mv; i += 32) {
            const unsigned long long kxy = xy_key(X[i], Y[i]);
            if (kxy == lo) ilo = min(ilo, (unsigned)V[i]);
            if (kxy == hi) ihi = min(ihi, (unsigned)V[i]);
        }
        ilo = __reduce_min_sync(0xFFFFFFFFu, ilo);
        ihi = __reduce_min_sync(0xFFFFFFFFu, ihi);
        if (lane == 0) {
            out_idx[0] = (int)ilo;
            if (lo == hi) *out_n = 1;
            else { out_idx[1] = (int)ihi; *out_n = 2; }
        }
        return;
    }
    if (nneg != 0 && lane == 0) set_status(ctl, CH_ECUDA);   // internal consistency check
    // strictly convex vertices in order, the lexicographically smallest first
    int h = 0;
    unsigned long long best = ~0ull;
    for (int base = 0; base < mv; base += 32) {
        const int i = base + lane;
        const bool f = i < mv && tmp[i] != 0;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, f);
        __syncwarp();
        if (f) {
            const int pos = h + __popc(bal & lanemask_lt());
            const unsigned long long kxy = (xy_key(X[i], Y[i]) << 16) | (unsigned)pos;
            best = kxy < best ? kxy : best;
            tmp[pos] = V[i];   // pos <= i: entries still to be read are not overwritten
        }
        h += __popc(bal);
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long a2 = __shfl_xor_sync(0xFFFFFFFFu, best, o);
        best = a2 < best ? a2 : best;
    }
    if (h > n) {
        if (lane == 0) { set_status(ctl, CH_ECUDA); *out_n = CH_ECUDA; }
        return;
    }
    const int start = (int)(best & 0xFFFFull);
    for (int j = lane; j < h; j += 32) {
        const int k = start + j;
        out_idx[j] = tmp[k < h ? k : k - h];
    }
    if (lane == 0) *out_n = nneg != 0 ? (int64_t)CH_ECUDA : (int64_t)h;
}

}  // namespace ch
