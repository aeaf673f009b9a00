// launch.h -- host-side launchers of the device kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace ch {

struct Ctl;

void launch_init(Ctl* ctl, int mode, cudaStream_t s);
void launch_sample(const float* pts, long long n, int head, long long ntiles, Ctl* ctl, int grid, cudaStream_t s);
void launch_main(const float* pts, long long n, int head, long long ntiles, Ctl* ctl, uint64_t* raw_xy,
                 uint32_t* raw_idx, unsigned switch_at, uint32_t* keys, uint64_t* vals, int grid, cudaStream_t s);
void launch_post(const float* pts, long long n, int head, long long ntiles, Ctl* ctl, const uint64_t* raw_xy,
                 const uint32_t* raw_idx, uint32_t* keys, uint64_t* vals, int32_t* out_idx, int64_t* out_n,
                 void* star_bins, unsigned long long cond, int grid, cudaStream_t s);
void launch_labels(const float* pts, long long n, Ctl* ctl, uint8_t* labels, int grid, cudaStream_t s);
// The star pass (star.cu): its angular bins live in the workspace.
void launch_star(const float* pts, long long n, int head, long long ntiles, Ctl* ctl, void* bins, int grid,
                 cudaStream_t s);
cudaError_t configure_star_kernel();
size_t star_bins_bytes();
void launch_filter_output(const Ctl* ctl, long long n, int32_t* out_ext8, int64_t* out_counts4, cudaStream_t s);

void launch_sort_hist(const uint32_t* keys, Ctl* ctl, int grid, cudaStream_t s);
void launch_sort_pass(const uint32_t* kin, const uint64_t* vin, uint32_t* kout, uint64_t* vout,
                      Ctl* ctl, unsigned long long* status, int pass, int grid, cudaStream_t s);

void launch_chain(Ctl* ctl, const uint32_t* keys, const uint64_t* vals, const int* bu, const int* bv,
                  const int* bi, const int* blen, int* cu, int* cv, int* ci, int* clen, int* counters, int ctcap,
                  int* vbuf, int* kbuf, int* xbuf, int* ybuf, const float* pts, long long n, int32_t* out_idx,
                  int64_t* out_n, int grid, cudaStream_t s);
void launch_bucket_pass(Ctl* ctl, uint32_t* kA, uint64_t* vA, uint32_t* kB, uint64_t* vB, unsigned* bcount,
                        unsigned* bcur, unsigned* bstart, unsigned* bsum, int* bu, int* bv, int* bi, int* blen,
                        unsigned bmax, int sms, cudaStream_t s);
cudaError_t configure_bucket_kernels();
size_t chain_smem_bytes();
cudaError_t configure_hull_kernels();
cudaError_t configure_filter_kernels();
cudaError_t configure_post_kernel();
long long sample_tiles_host(long long ntiles);

// Occupancy (resident blocks per SM at each kernel's launch shape).
cudaError_t occupancy_filter(int* main_k, int* labels);
cudaError_t occupancy_post(int* post);
cudaError_t occupancy_sort(int* sort);
cudaError_t occupancy_chain(int* chain);

}  // namespace ch
