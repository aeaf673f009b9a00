// host.h -- host-side internals shared by api.cu, batched.cu and server.cu.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace ch {

// Workspace layout of one hull of up to n points (byte offsets from the base).
struct Layout {
    size_t off_ctl, off_kA, off_kB, off_vA, off_vB, off_status, zero_bytes;
    size_t off_cu, off_cv, off_ci, off_clen, off_counters;
    size_t off_bcount, off_bcur, off_bstart, off_bsum, off_blen, off_bu, off_bv, off_bi, total;
    size_t off_star_bins;
    long long cap, sort_tiles, ctcap, bmax;
};

Layout make_layout(long long n);
int get_workspace(int dev, cudaStream_t s, long long n, char** base, Layout* L);
int enqueue_hull(const float* pts, long long n, int32_t* out_idx, int64_t* out_n, cudaStream_t s, int dev);
// The same launches without the CUDA-graph cache (callers with many distinct
// argument sets, where capturing each would only thrash the cache).
int enqueue_hull_nograph(const float* pts, long long n, int32_t* out_idx, int64_t* out_n, cudaStream_t s,
                         int dev);
int check_points_args(const float* pts, long long n);

int reserve_batched(int dev, cudaStream_t s, long long n, int k);
void drop_batched_graphs(int dev, cudaStream_t s);
// ch_hull_batched; allow_tune = false takes the nearest tuned size class
// instead of tuning a new one (for callers that must not block).  With
// redo_host (pinned, k bytes) nothing synchronises: the per-set flags of sets
// left to the single-hull path are copied there asynchronously, and the
// caller runs hull_batched_redo on them once they have arrived (host_offsets
// is then required).
int hull_batched_impl(const float* pts, const int64_t* offsets, int32_t k, int32_t* out_idx, int64_t* out_n,
                      const int64_t* host_offsets, cudaStream_t s, bool allow_tune, unsigned char* redo_host);
int hull_batched_redo(const float* pts, const int64_t* host_offsets, int32_t k, int32_t* out_idx, int64_t* out_n,
                      const unsigned char* flags, cudaStream_t s);
bool prof_enabled();
void release_stream_workspace(int dev, cudaStream_t s);
void release_batched();
// The batched workspace of one stream (freed with the stream's other workspace).
void release_batched_stream(int dev, cudaStream_t s);

// Records a CUDA event pair around a scope when profiling is enabled.
class ProfScope {
  public:
    ProfScope(const char* name, cudaStream_t s);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

  private:
    const char* name_;
    cudaStream_t s_;
    void* a_;
};

}  // namespace ch
