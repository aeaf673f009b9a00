// batched_large.h -- arguments of the batched large-survivor path (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ch {

struct Ctl;

constexpr int kBLTile = 4096;   // records per record tile of the large-survivor path

struct BLArgs {
    const float* pts;
    const int64_t* offsets;        // device, k + 1
    int k;
    Ctl* ctl;                      // k control blocks (batched)
    uint32_t* keys;                // batched records: set i at offsets[i] + 16 i
    uint64_t* vals;
    const unsigned char* big;      // k: the set's records exceed one block
    int32_t* out_idx;
    int64_t* out_n;
    // per segment (set, queue): 4k (+1 for the prefixes)
    unsigned* seg_nb;
    unsigned* seg_bbase;
    int* seg_lo;
    float* seg_scale;
    unsigned* seg_tbase;
    int* ct_map;                   // segment of every chain tile
    unsigned* rt_base;             // k + 1: record tiles per set (prefix)
    int* rt_map;                   // set of every record tile
    unsigned* totals;              // buckets, chain tiles, record tiles, fits, allocation cursor
    // buckets
    unsigned* bcount;
    unsigned* bcur;
    unsigned* bstart;
    int* blen;
    int* bu;
    int* bv;
    int* bi;
    uint32_t* kP;                  // records scattered by bucket
    uint64_t* vP;
    // chain merge tree
    int* cu;
    int* cv;
    int* ci;
    int* clen;
    int* counters;
    unsigned bcap, tcap, rtcap;
};

void launch_batched_large(const BLArgs& a, unsigned char* redo, int sms, cudaStream_t s);
cudaError_t configure_batched_large();

}  // namespace ch
