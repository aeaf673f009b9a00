// noalloc.cu -- ch_hull_noalloc: the hull of a small point set with no
// device allocation at call time.
//
// Some callers cannot let the library allocate: code that runs under a fixed
// device-memory budget decided up front, or a latency-critical loop that must
// not pay cudaMalloc's implicit device-wide synchronisation (ch_hull grows a
// workspace on first use of a size).  For them, this entry point runs the
// whole hull of up to kNoAllocMaxPoints points in one block whose global
// scratch (a control block and the sort records) is a fixed array in this
// module's static device memory; everything else lives in shared memory.
//
// The kernel is a single-block variant of the post pass's last block: it
// finds the 8 extremes itself (lowest index on ties), builds the octagon,
// classifies every point by the hull rule, and joins the quickhull chains
// (with the sort-based mid_hull as the fallback), exactly like ch_hull.
//
// Scratch contract: nothing in the scratch has to start at zero; the kernel
// writes every field it reads (status, record count, octagon) before reading
// it.  Two calls that overlap in time (different streams, or different host
// threads) share the one scratch array and race: the caller must order them.
#include "ch_internal.cuh"
#include "hullcore.cuh"
#include "octagon.cuh"

#include <climits>
#include <mutex>

namespace ch {
namespace {

constexpr int kNoAllocMaxPoints = 8000;     // records <= n + 12 <= kMidCap
constexpr int kNoAllocThreads = 512;
constexpr int kNoAllocRecCap = kNoAllocMaxPoints + 16;
static_assert(kNoAllocRecCap <= kMidCap, "records must fit the one-block hull");

struct NoAllocScratch {
    Ctl ctl;
    uint32_t keys[kNoAllocRecCap];
    uint64_t vals[kNoAllocRecCap];
};

// The scratch: about 100 KB of static device memory, set aside when the
// module loads (not by a call).
static __device__ __align__(256) unsigned char g_scratch[sizeof(NoAllocScratch)];

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kNoAllocSmemBytes = cmax(kMidSmemBytes, sizeof(QhSmem));

__device__ __forceinline__ bool na_dir_is_max(int d) { return d >= SE && d <= N; }

__device__ __forceinline__ int na_dir_key(int d, int X, int Y) {
    switch (d) {
        case W: case E: return X;
        case S: case N: return Y;
        case SW: case NE: return X + Y;
        default: return X - Y + kCoordLimit;
    }
}

// (key, lowest index) packed so that the maximum is the winner: maxima keep
// the key, minima its complement; the index is complemented (lowest wins).
__device__ __forceinline__ unsigned long long na_pack(int d, int X, int Y, unsigned idx) {
    const unsigned k = (unsigned)na_dir_key(d, X, Y);
    const unsigned hk = na_dir_is_max(d) ? k : 0xFFFFFFFFu - k;
    return ((unsigned long long)hk << 32) | (unsigned long long)(0xFFFFFFFFu - idx);
}

__global__ void __launch_bounds__(kNoAllocThreads, 1)
    noalloc_kernel(const float* __restrict__ pts, int n, int32_t* out_idx, int64_t* out_n, NoAllocScratch* sc) {
    extern __shared__ __align__(16) char dyn[];
    __shared__ Octagon s_o;
    __shared__ unsigned long long s_best[8];
    __shared__ int s_vx[8], s_vy[8], s_id[8];
    __shared__ int s_bad, s_m, s_mv;
    const int tid = threadIdx.x, lane = tid & 31;
    Ctl* ctl = &sc->ctl;
    if (tid < 8) s_best[tid] = 0ull;
    if (tid == 0) {
        s_bad = 0;
        s_m = 0;
        ctl->status = CH_OK;
        ctl->abort = 0;
        ctl->done = 0;
    }
    __syncthreads();
    if (n == 0) {
        if (tid == 0) *out_n = 0;
        return;
    }
    // extremes with the lowest index on ties; validity of every coordinate
    unsigned long long best[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) best[d] = 0ull;
    bool bad = false;
    for (int i = tid; i < n; i += blockDim.x) {
        const float x = pts[2 * i], y = pts[2 * i + 1];
        const int X = __float2int_rn(x), Y = __float2int_rn(y);
        bad |= (__int2float_rn(X) != x) | (__int2float_rn(Y) != y) | (((unsigned)X | (unsigned)Y) >> kCoordBits) != 0u;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const unsigned long long p = na_pack(d, X, Y, (unsigned)i);
            best[d] = p > best[d] ? p : best[d];
        }
    }
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) s_bad = 1;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        unsigned long long p = best[d];
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long q = __shfl_xor_sync(0xFFFFFFFFu, p, o);
            p = q > p ? q : p;
        }
        if (lane == 0) atomicMax(&s_best[d], p);
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) *out_n = CH_ERANGE;
        return;
    }
    if (tid < 8) {
        const int i = (int)(0xFFFFFFFFu - (unsigned)(s_best[tid] & 0xFFFFFFFFull));
        s_id[tid] = i;
        s_vx[tid] = __float2int_rn(pts[2 * i]);
        s_vy[tid] = __float2int_rn(pts[2 * i + 1]);
    }
    __syncthreads();
    setup_octagon_block(s_o, s_vx, s_vy, s_id, false);
    copy_octagon(&ctl->oct, &s_o);
    // records: the 8 chain end points, the diagonal extremes strictly right of
    // their quad edge, then every point outside the closed octagon
    QhSmem& q = *reinterpret_cast<QhSmem*>(dyn);
    auto put = [&](int r, int X, int Y, unsigned idx) {
        uint32_t u, v;
        queue_frame(r, X, Y, u, v);
        const int pos = atomicAdd(&s_m, 1);
        const uint32_t key = make_key(r, u);
        const uint64_t val = make_val(v, idx);
        sc->keys[pos] = key;
        sc->vals[pos] = val;
        q.ru[pos] = (int)u;
        q.rv[pos] = (int)v;
        q.ri[pos] = (int)idx;
        q.rs[pos] = r;
    };
    if (tid < 12) {
        int r, d;
        bool emit = true;
        if (tid < 8) {
            r = tid >> 1;
            d = (tid & 1) ? ((2 * r + 2) & 7) : 2 * r;
        } else {
            r = tid - 8;
            d = 2 * r + 1;
            const int a = 2 * r, b = (2 * r + 2) & 7;
            emit = orient64(s_vx[a], s_vy[a], s_vx[b], s_vy[b], s_vx[d], s_vy[d]) < 0;
        }
        if (emit) put(r, s_vx[d], s_vy[d], (unsigned)s_id[d]);
    }
    for (int i = tid; i < n; i += blockDim.x) {
        const float x = pts[2 * i], y = pts[2 * i + 1];
        const int r = classify_hull_slow(x, y, &s_o);
        if (r >= 0) put(r, __float2int_rn(x), __float2int_rn(y), (unsigned)i);
    }
    __syncthreads();
    const int m = s_m;
    if (tid == 0) ctl->count = (unsigned)m;
    if (qh_chains(q, m, &s_mv)) {
        stitch_cycle(q.ru, q.rv, q.ri, s_mv, q.rs, ctl, n, out_idx, out_n);
    } else {
        __syncthreads();
        mid_hull(sc->keys, sc->vals, m, pts, n, ctl, out_idx, out_n, dyn);
    }
}

std::mutex g_mu;
void* g_ptr[64];                   // scratch address per device
unsigned long long g_ctx[64];      // id of the context that address belongs to

// Id of the calling thread's current CUDA context (unique for the life of
// the process), 0 when there is none yet or the driver cannot say.  A new id
// for a device means its context was destroyed and re-created (for example
// by cudaDeviceReset): the static array then has a new address and the
// kernel attribute must be set again.  The driver calls are looked up
// through the runtime, so the library needs no link to the driver library.
unsigned long long current_context_id() {
    typedef int (*GetCurrentFn)(void**);
    typedef int (*GetIdFn)(void*, unsigned long long*);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_current, 12000, cudaEnableDefault,
                                             &q1) != cudaSuccess || q1 != cudaDriverEntryPointSuccess)
            get_current = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess || q2 != cudaDriverEntryPointSuccess)
            get_id = nullptr;
        cudaGetLastError();
    }
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
    return 0;
}

}  // namespace
}  // namespace ch

extern "C" int ch_hull_noalloc(const float* pts, int64_t n, int32_t* out_idx, int64_t* out_n, void* stream) {
    using namespace ch;
    if (!out_n || n < 0 || (n > 0 && (!pts || !out_idx))) return CH_EINVAL;
    if (n > kNoAllocMaxPoints) return CH_EINVAL;   // beyond the fixed scratch
    if (((uintptr_t)pts & 7u) != 0u || ((uintptr_t)out_n & 7u) != 0u || ((uintptr_t)out_idx & 3u) != 0u)
        return CH_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CH_ECUDA;
    void* sc = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        const unsigned long long ctx = current_context_id();
        if (!g_ptr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
            // set-up, once per device and context (that device current); a
            // thread whose context is not current yet redoes the lookup once
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return CH_ECUDA;
            }
            if (cudaFuncSetAttribute(noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kNoAllocSmemBytes) != cudaSuccess) {
                cudaGetLastError();
                return CH_ECUDA;
            }
            g_ptr[dev] = p;
            g_ctx[dev] = current_context_id();
        }
        sc = g_ptr[dev];
    }
    noalloc_kernel<<<1, kNoAllocThreads, kNoAllocSmemBytes, (cudaStream_t)stream>>>(
        pts, (int)n, out_idx, out_n, reinterpret_cast<NoAllocScratch*>(sc));
    return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ECUDA;
}
