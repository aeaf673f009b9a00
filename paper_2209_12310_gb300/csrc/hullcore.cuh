// hullcore.cuh -- block-level pieces of the hull stage shared by the kernels:
//   stitch_core  joins the four queue chains into the output list;
//   tiny_hull    the whole hull stage for a few hundred records in one block
//                (no sort): used when the filter leaves few survivors.
#pragma once

#include <climits>

#include "ch_internal.cuh"

namespace ch {

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
// N..W (each without its last point), a weakly convex cyclic polygon.  Writes
// the strictly convex vertices counter-clockwise from the lexicographically
// smallest one; all-collinear input gives [lex-min, lex-max], one distinct
// point gives [it].  flag and comp are scratch arrays of m ints.
static __device__ void stitch_core(const int* V, int m, int* flag, int* comp, const float* __restrict__ pts,
                            long long n, Ctl* ctl, int32_t* out_idx, int64_t* out_n) {
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
        pt_xy(pts, V[(i + m - 1) % m], ax, ay);
        pt_xy(pts, V[i], bx, by);
        pt_xy(pts, V[(i + 1) % m], cx, cy);
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
            pt_xy(pts, V[i], x, y);
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
            pt_xy(pts, V[i], x, y);
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
            pt_xy(pts, V[i], x, y);
            const unsigned long long k = xy_key(x, y);
            best = k < best ? k : best;
            comp[written + ex] = V[i];
        }
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
    for (int j = tid; j < h; j += T) {
        long long x, y;
        pt_xy(pts, comp[j], x, y);
        if (xy_key(x, y) == best) s_a = j;
    }
    __syncthreads();
    const int start = s_a;
    for (int j = tid; j < h; j += T) out_idx[j] = comp[(start + j) % h];
    __syncthreads();
    if (tid == 0) {
        const int st = read_status(ctl);
        *out_n = (st == CH_OK) ? h : st;
    }
}

// Shared memory of tiny_hull (kTinyCap records).
struct TinySmem {
    uint32_t key[kTinyCap];
    uint64_t val[kTinyCap];
    int vert[kTinyCap];      // 1 = chain vertex
    int rank[kTinyCap];
    int V[kTinyCap];
    int flag[kTinyCap];
    int comp[kTinyCap];
    int len[4];
};

__device__ __forceinline__ int rec_u(uint32_t k) { return (int)(k & kKeyMask); }
__device__ __forceinline__ int rec_v(uint64_t v) { return (int)(v >> 31); }

// The hull stage for m <= kTinyCap sort records (queue | u, v | index) in one
// block, without sorting: a record survives its queue's run reduction when no
// record of equal (queue, u) has a smaller (v, index); a survivor is a chain
// vertex when it is an end of its queue or strictly below the line through its
// steepest left neighbour and its flattest right neighbour (Andrew's lower
// chain in the queue frame); its position is its rank by u.
static __device__ void tiny_hull(const uint32_t* keys, const uint64_t* vals, int m, const float* __restrict__ pts,
                          long long n, Ctl* ctl, int32_t* out_idx, int64_t* out_n, TinySmem& sm) {
    const int tid = threadIdx.x, T = blockDim.x;
    for (int i = tid; i < m; i += T) { sm.key[i] = keys[i]; sm.val[i] = vals[i]; }
    if (tid < 4) sm.len[tid] = 0;
    __syncthreads();
    // run reduction: keep the smallest (v, index) per (queue, u); first position on exact ties
    for (int i = tid; i < m; i += T) {
        const uint32_t ki = sm.key[i];
        const uint64_t vi = sm.val[i];
        int alive = 1;
        for (int j = 0; j < m; ++j) {
            if (sm.key[j] == ki && (sm.val[j] < vi || (sm.val[j] == vi && j < i))) { alive = 0; break; }
        }
        sm.vert[i] = alive;
    }
    __syncthreads();
    int vflag[(kTinyCap + 31) / 32];
    int c = 0;
    for (int i = tid; i < m; i += T, ++c) {
        vflag[c] = 0;
        if (!sm.vert[i]) continue;
        const uint32_t qi = sm.key[i] >> kKeyBits;
        const long long ui = rec_u(sm.key[i]), vi = rec_v(sm.val[i]);
        bool has_l = false, has_r = false;
        long long au = 0, av = 0, bu = 0, bv = 0;
        for (int j = 0; j < m; ++j) {
            if (!sm.vert[j] || (sm.key[j] >> kKeyBits) != qi) continue;
            const long long uj = rec_u(sm.key[j]), vj = rec_v(sm.val[j]);
            if (uj < ui) {   // steepest slope (a -> i)
                if (!has_l || (vi - vj) * (ui - au) > (vi - av) * (ui - uj)) { au = uj; av = vj; }
                has_l = true;
            } else if (uj > ui) {   // flattest slope (i -> b)
                if (!has_r || (vj - vi) * (bu - ui) < (bv - vi) * (uj - ui)) { bu = uj; bv = vj; }
                has_r = true;
            }
        }
        const bool is_v = !has_l || !has_r ||
                          (ui - au) * (bv - av) - (vi - av) * (bu - au) > 0;
        vflag[c] = is_v ? 1 : 0;
    }
    __syncthreads();
    c = 0;
    for (int i = tid; i < m; i += T, ++c) sm.vert[i] = vflag[c];
    __syncthreads();
    for (int i = tid; i < m; i += T) {
        if (!sm.vert[i]) continue;
        const uint32_t ki = sm.key[i];
        int rk = 0;
        for (int j = 0; j < m; ++j)
            if (sm.vert[j] && (sm.key[j] >> kKeyBits) == (ki >> kKeyBits) && sm.key[j] < ki) ++rk;
        sm.rank[i] = rk;
        atomicAdd(&sm.len[ki >> kKeyBits], 1);
    }
    __syncthreads();
    int off[5];
    off[0] = 0;
    for (int r = 0; r < 4; ++r) off[r + 1] = off[r] + max(sm.len[r] - 1, 0);
    const int mv = off[4];
    for (int i = tid; i < m; i += T) {
        if (!sm.vert[i]) continue;
        const int r = (int)(sm.key[i] >> kKeyBits);
        if (sm.rank[i] < sm.len[r] - 1) sm.V[off[r] + sm.rank[i]] = (int)(sm.val[i] & 0x7FFFFFFFull);
    }
    __syncthreads();
    stitch_core(sm.V, mv, sm.flag, sm.comp, pts, n, ctl, out_idx, out_n);
}

}  // namespace ch
