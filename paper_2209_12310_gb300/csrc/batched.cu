// batched.cu -- k independent hulls packed back to back (ch_hull_batched).
//
// Every set runs the full single-hull launch sequence on the caller's stream,
// in stream order, sharing that stream's workspace; each result is therefore
// identical to ch_hull on the set alone.
#include "ch_internal.cuh"
#include "host.h"
#include "launch.h"

#include <vector>

namespace ch {

int reserve_batched(int dev, cudaStream_t s, long long n, int k) {
    (void)dev; (void)s; (void)n; (void)k;
    return CH_OK;
}

void release_batched() {}

}  // namespace ch

using namespace ch;

extern "C" int ch_hull_batched(const float* pts, const int64_t* offsets, int32_t k, int32_t* out_idx,
                               int64_t* out_n, const int64_t* host_offsets, void* stream) {
    if (k < 0 || k > (1 << 20)) return CH_EINVAL;
    if (k == 0) return CH_OK;
    if (!offsets || !out_n) return CH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> off((size_t)k + 1);
    if (host_offsets) {
        for (int i = 0; i <= k; ++i) off[i] = host_offsets[i];
    } else {
        if (cudaMemcpyAsync(off.data(), offsets, sizeof(int64_t) * ((size_t)k + 1), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
            return CH_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return CH_ECUDA;
    }
    if (off[0] != 0) return CH_EINVAL;
    for (int i = 0; i < k; ++i)
        if (off[i + 1] < off[i] || off[i + 1] - off[i] > CH_MAX_POINTS) return CH_EINVAL;
    const int64_t total = off[k];
    int st = check_points_args(pts, total);
    if (st != CH_OK) return st;
    if (total > 0 && !out_idx) return CH_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CH_ECUDA;
    for (int i = 0; i < k; ++i) {
        const int64_t ni = off[i + 1] - off[i];
        if (ni == 0) {
            if (cudaMemsetAsync(out_n + i, 0, sizeof(int64_t), s) != cudaSuccess) return CH_ECUDA;
            continue;
        }
        st = enqueue_hull(pts + 2 * off[i], ni, out_idx + off[i], out_n + i, s, dev);
        if (st != CH_OK) return st;
    }
    return CH_OK;
}
