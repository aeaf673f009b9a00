// tma.cuh -- bulk asynchronous copies (TMA, cp.async.bulk) into shared memory
// with mbarrier completion, for the streaming passes.  Every wait is bounded:
// a wait that gives up raises CH_ETIMEOUT and the abort flag instead of
// spinning forever.
#pragma once

#include "ch_internal.cuh"

namespace ch {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the async proxy.
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses before later async-proxy
// (TMA) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar,
                                         unsigned long long pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Bounded wait for phase `parity` of `bar`; false when it gave up (the copy
// never completed) or another wait already gave up (ctl->abort).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, Ctl* ctl) {
    for (unsigned i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 1023u) == 1023u && *(volatile int*)&ctl->abort) return false;
    }
    set_status(ctl, CH_ETIMEOUT);
    atomicExch(&ctl->abort, 1);
    return false;
}

// A warp's double-buffered stream of its warp tiles t = first + k * stride
// (k = 0, 1, ...) below ntiles, each kF4 float4 copied by one bulk copy
// issued by lane 0.  Usage: for (k...) { cur = acquire(k); ...read cur...;
// release(k); }
constexpr int kStages = 2;

template <int kF4>
struct WarpStreamT {
    float4* ring;                 // kStages * kF4 float4 of shared memory
    unsigned long long* bar;      // kStages barriers
    const float4* src;            // 16-byte aligned body of the point array
    long long first, stride, ntiles;
    int lane;

    __device__ __forceinline__ void issue(long long k) {
        const long long t = first + k * stride;
        if (t < ntiles && lane == 0) {
            const int s = (int)(k % kStages);
            fence_proxy_async();
            mbar_expect_tx(&bar[s], kF4 * 16);
            tma_load(ring + s * kF4, src + t * kF4, kF4 * 16, &bar[s], l2_evict_first());
        }
    }
    __device__ __forceinline__ void start() {
        if (lane == 0) {
            for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
            fence_barrier_init();
        }
        __syncwarp();
        for (int s = 0; s < kStages; ++s) issue(s);
    }
    // Waits for tile k; nullptr when the wait gave up.
    __device__ __forceinline__ const float4* acquire(long long k, Ctl* ctl) {
        const int s = (int)(k % kStages);
        const unsigned parity = (unsigned)((k / kStages) & 1);
        if (!mbar_wait(&bar[s], parity, ctl)) return nullptr;
        return ring + s * kF4;
    }
    // Every lane is done reading tile k: refill its stage with tile k + kStages.
    __device__ __forceinline__ void release(long long k) {
        __syncwarp();
        issue(k + kStages);
    }
    // After an abandoned wait at tile k: wait (bounded) for the copies still in
    // flight so no copy lands after the block has exited.
    __device__ __forceinline__ void drain(long long k) {
        for (long long j = k; j < k + kStages; ++j) {
            const long long t = first + j * stride;
            if (t >= ntiles) break;
            const int s = (int)(j % kStages);
            const unsigned parity = (unsigned)((j / kStages) & 1);
            for (unsigned i = 0; i < kSpinLimit; ++i)
                if (mbar_try_wait(&bar[s], parity)) break;
        }
        __syncwarp();
    }
};

using WarpStream = WarpStreamT<kWarpTileF4>;

}  // namespace ch
