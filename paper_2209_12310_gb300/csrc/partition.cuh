// partition.cuh -- one block moves a tile of (key, value) records to their
// groups' ranges with coalesced writes.
//
// A scatter of single records to random ranges writes one 32-byte sector per
// record and lane; the tile is instead ordered by group in shared memory
// first, so that consecutive threads write consecutive positions of a run
// (the records of one group in the tile).  Ranks within the tile come from
// shared-memory atomics; each nonempty group reserves its run with one call
// of the caller's reserve(g, count), which returns the run's first position.
#pragma once
#include "ch_internal.cuh"
#include "hullcore.cuh"

namespace ch {

constexpr int kPtThreads = 1024;                  // threads of a partition block
constexpr int kPtPer = 8;                         // records per thread and tile
constexpr int kPtTile = kPtThreads * kPtPer;      // records per tile
constexpr int kPtGroups = 4096;                   // groups per tile at most

struct PartSmem {
    uint64_t val[kPtTile];
    uint32_t key[kPtTile];
    unsigned off[kPtGroups];                      // count, then first local position
    unsigned dst[kPtGroups];                      // run start minus first local position
    unsigned short grp[kPtTile];
    int tmp[33];
};

// Records [i0, i0 + cnt) of (kin, vin), cnt <= kPtTile, into (kout, vout);
// bin(key) < ngroups <= kPtGroups.  Whole block; ends with a barrier.
template <class Bin, class Reserve>
__device__ __forceinline__ void partition_tile(PartSmem& sm, const uint32_t* kin, const uint64_t* vin, unsigned i0,
                                               unsigned cnt, unsigned ngroups, Bin bin, Reserve reserve,
                                               uint32_t* kout, uint64_t* vout) {
    const int tid = threadIdx.x;
    for (unsigned g = tid; g < ngroups; g += kPtThreads) sm.off[g] = 0u;
    __syncthreads();
    uint32_t k[kPtPer];
    unsigned gg[kPtPer], rk[kPtPer];
#pragma unroll
    for (int j = 0; j < kPtPer; ++j) {
        const unsigned i = j * kPtThreads + tid;
        if (i < cnt) {
            k[j] = __ldcs(kin + i0 + i);
            gg[j] = bin(k[j]);
            rk[j] = atomicAdd(&sm.off[gg[j]], 1u);
        }
    }
    __syncthreads();
    // local offsets (exclusive scan over the groups, a few per thread) and runs
    constexpr int kE = kPtGroups / kPtThreads;
    unsigned c[kE], part = 0u;
    const unsigned g0 = tid * kE;
#pragma unroll
    for (int e = 0; e < kE; ++e) {
        c[e] = g0 + e < ngroups ? sm.off[g0 + e] : 0u;
        part += c[e];
    }
    int tot;
    unsigned run = (unsigned)block_excl_scan((int)part, sm.tmp, &tot);
#pragma unroll
    for (int e = 0; e < kE; ++e) {
        if (g0 + e < ngroups) {
            sm.off[g0 + e] = run;
            if (c[e]) sm.dst[g0 + e] = reserve(g0 + e, c[e]) - run;
            run += c[e];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPtPer; ++j) {
        const unsigned i = j * kPtThreads + tid;
        if (i < cnt) {
            const unsigned p = sm.off[gg[j]] + rk[j];
            sm.key[p] = k[j];
            sm.grp[p] = (unsigned short)gg[j];
            sm.val[p] = __ldcs(vin + i0 + i);
        }
    }
    __syncthreads();
    for (unsigned p = tid; p < cnt; p += kPtThreads) {
        const unsigned d = sm.dst[sm.grp[p]] + p;
        kout[d] = sm.key[p];
        vout[d] = sm.val[p];
    }
    __syncthreads();
}

}  // namespace ch
