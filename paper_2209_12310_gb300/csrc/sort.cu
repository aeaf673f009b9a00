// sort.cu -- stable LSD radix sort of the survivor records by (queue, u).
//
// The paper keeps the survivors of each queue semi-ordered in a priority
// queue (a heap, Sec. 1.2, "partial ordering") and builds each queue's hull
// sequentially on the CPU.  On the GPU the four queues are ordered at once by
// a 27-bit key (queue in the top 2 bits, queue-frame coordinate u below),
// three 9-bit digit passes of a single-pass ("onesweep") radix sort: each
// pass ranks a 4096-record tile in shared memory, publishes its per-digit
// counts, resolves its global offsets by decoupled look-back over the
// preceding tiles, and scatters.  The digit histograms of all three passes
// come from one counting pass over the records (sort_hist_kernel) before the
// first scatter; the post pass keeps only per-queue counts.
//
// Look-back waits are bounded (kSpinLimit polls with back-off); a wait that
// gives up raises CH_ETIMEOUT and the abort flag, after which every other
// wait gives up too.  Tiles are claimed in order through an atomic counter, so
// a tile only ever waits for tiles whose blocks are already running.
#include "ch_internal.cuh"
#include "launch.h"

namespace ch {

constexpr unsigned long long kFlagPrefix = 1ull << 31;

__device__ __forceinline__ unsigned long long pack_status(unsigned epoch, bool prefix, unsigned cnt) {
    return ((unsigned long long)epoch << 32) | (prefix ? kFlagPrefix : 0ull) | (unsigned long long)cnt;
}

__device__ __forceinline__ void st_volatile(unsigned long long* p, unsigned long long v) {
    *(volatile unsigned long long*)p = v;
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
    return *(volatile const unsigned long long*)p;
}

// Exclusive scan of 2 values per thread over a 256-thread block.
__device__ __forceinline__ unsigned block_excl_scan(unsigned x, unsigned* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    unsigned off = 0;
    for (int w = 0; w < warp; ++w) off += s_warp[w];
    __syncthreads();
    return off + incl - x;
}

__global__ void __launch_bounds__(kSortThreads) onesweep_kernel(
    const uint32_t* __restrict__ kin, const uint64_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint64_t* __restrict__ vout, Ctl* ctl, unsigned long long* status, int pass) {
    __shared__ unsigned s_base[kDigits];
    __shared__ unsigned s_excl[kDigits];
    __shared__ unsigned short s_wcnt[kSortThreads / 32][kDigits];
    __shared__ unsigned s_warp[kSortThreads / 32];
    __shared__ unsigned s_tile;

    if (*(volatile int*)&ctl->done || read_status(ctl) != CH_OK || *(volatile int*)&ctl->bk_state == 1) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned count = ctl->count;
    const unsigned ntiles = (count + kSortTile - 1) / kSortTile;
    const unsigned epoch = ctl->epoch * 4u + (unsigned)pass;
    const int shift = pass * kDigitBits;

    bool have_base = false;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&ctl->tile_ctr[pass], 1u);
        for (int i = threadIdx.x; i < (kSortThreads / 32) * kDigits; i += kSortThreads)
            (&s_wcnt[0][0])[i] = 0;
        __syncthreads();
        const unsigned tile = s_tile;
        if (tile >= ntiles) break;
        if (!have_base) {   // global digit offsets of this pass (once per block)
            const unsigned a = ctl->digit_hist[pass][2 * threadIdx.x];
            const unsigned b = ctl->digit_hist[pass][2 * threadIdx.x + 1];
            const unsigned ex = block_excl_scan(a + b, s_warp);
            s_base[2 * threadIdx.x] = ex;
            s_base[2 * threadIdx.x + 1] = ex + a;
            have_base = true;
        }

        const unsigned tbase = tile * kSortTile + warp * (32 * kSortItems);
        uint32_t k[kSortItems];
        unsigned short rk[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const unsigned pos = tbase + j * 32 + lane;
            k[j] = pos < count ? kin[pos] : 0xFFFFFFFFu;
        }
        const unsigned lt = lanemask_lt();
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const unsigned pos = tbase + j * 32 + lane;
            const bool valid = pos < count;
            const unsigned vmask = __ballot_sync(0xFFFFFFFFu, valid);
            rk[j] = 0;
            if (valid) {
                const unsigned dg = (k[j] >> shift) & (kDigits - 1);
                const unsigned peers = __match_any_sync(vmask, dg);
                const unsigned old = s_wcnt[warp][dg];
                rk[j] = (unsigned short)(old + __popc(peers & lt));
                __syncwarp(vmask);
                if ((peers & lt) == 0u) s_wcnt[warp][dg] = (unsigned short)(old + __popc(peers));
                __syncwarp(vmask);
            }
        }
        __syncthreads();

        // Per digit: exclusive offsets of the warps inside the tile, tile total.
        unsigned tot[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int d = threadIdx.x + h * kSortThreads;
            unsigned run = 0;
#pragma unroll
            for (int w = 0; w < kSortThreads / 32; ++w) {
                const unsigned c = s_wcnt[w][d];
                s_wcnt[w][d] = (unsigned short)run;
                run += c;
            }
            tot[h] = run;
        }
        // Decoupled look-back, two digits per thread.
        unsigned long long* my = status + (size_t)tile * kDigits;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int d = threadIdx.x + h * kSortThreads;
            st_volatile(my + d, pack_status(epoch, tile == 0, tot[h]));
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int d = threadIdx.x + h * kSortThreads;
            unsigned excl = 0;
            if (tile > 0) {
                long long tp = (long long)tile - 1;
                unsigned spins = 0;
                while (tp >= 0) {
                    const unsigned long long w = ld_volatile(status + (size_t)tp * kDigits + d);
                    if ((unsigned)(w >> 32) == epoch) {
                        excl += (unsigned)(w & 0x7FFFFFFFull);
                        if (w & kFlagPrefix) break;
                        --tp;
                        continue;
                    }
                    if (spin_give_up(spins, ctl)) break;
                }
                st_volatile(my + d, pack_status(epoch, true, excl + tot[h]));
            }
            s_excl[d] = excl;
        }
        __syncthreads();

#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const unsigned pos = tbase + j * 32 + lane;
            if (pos < count) {
                const unsigned dg = (k[j] >> shift) & (kDigits - 1);
                const unsigned dst = s_base[dg] + s_excl[dg] + s_wcnt[warp][dg] + rk[j];
                if (dst < count) {
                    kout[dst] = k[j];
                    vout[dst] = vin[pos];
                }
            }
        }
        __syncthreads();
    }
}

// Digit histograms of the records for the three passes (the sort-based
// fallback only: the bucketed path needs none and leaves bk_state == 1).
__global__ void __launch_bounds__(kSortThreads) sort_hist_kernel(const uint32_t* __restrict__ keys, Ctl* ctl) {
    __shared__ unsigned s_h[kSortPasses][kDigits];
    if (*(volatile int*)&ctl->done || read_status(ctl) != CH_OK || *(volatile int*)&ctl->bk_state == 1) return;
    for (int i = threadIdx.x; i < kSortPasses * kDigits; i += blockDim.x) (&s_h[0][0])[i] = 0u;
    __syncthreads();
    const unsigned count = ctl->count;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
#pragma unroll
        for (int p = 0; p < kSortPasses; ++p) atomicAdd(&s_h[p][(k >> (p * kDigitBits)) & (kDigits - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSortPasses * kDigits; i += blockDim.x) {
        const unsigned c = (&s_h[0][0])[i];
        if (c) atomicAdd(&(&ctl->digit_hist[0][0])[i], c);
    }
}

void launch_sort_hist(const uint32_t* keys, Ctl* ctl, int grid, cudaStream_t s) {
    sort_hist_kernel<<<grid, kSortThreads, 0, s>>>(keys, ctl);
}

void launch_sort_pass(const uint32_t* kin, const uint64_t* vin, uint32_t* kout, uint64_t* vout,
                      Ctl* ctl, unsigned long long* status, int pass, int grid, cudaStream_t s) {
    onesweep_kernel<<<grid, kSortThreads, 0, s>>>(kin, vin, kout, vout, ctl, status, pass);
}


cudaError_t occupancy_sort(int* b) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, onesweep_kernel, kSortThreads, 0);
}

}  // namespace ch
