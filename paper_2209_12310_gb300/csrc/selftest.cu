// selftest.cu -- the library's bounded device waits, made to run out on
// purpose: a wait on a flag that nothing sets (the look-back poll of the
// radix-sort passes) and a wait on a bulk-copy barrier whose copy is never
// issued (the streaming passes).  Each gives up after its limit, sets
// CH_ETIMEOUT and returns; nothing faults, traps or hangs, and the context
// stays usable.  Test support for the failure-detection path.
#include "ch_internal.cuh"
#include "tma.cuh"

namespace ch {

__global__ void selftest_kernel(Ctl* ctl, const unsigned long long* flag, int which) {
    __shared__ __align__(8) unsigned long long s_bar;
    if (threadIdx.x != 0) return;
    if (which == 0) {   // poll a status word that stays 0, as the look-back does
        unsigned spins = 0;
        while (*(volatile const unsigned long long*)flag == 0ull)
            if (spin_give_up(spins, ctl)) break;
    } else {            // wait on a barrier that expects bytes no copy delivers
        mbar_init(&s_bar, 1);
        fence_barrier_init();
        mbar_expect_tx(&s_bar, 16);
        if (mbar_wait(&s_bar, 0, ctl)) set_status(ctl, CH_ECUDA);   // cannot complete
    }
}

}  // namespace ch

using namespace ch;

// which = 0: look-back poll; 1: bulk-copy barrier.  Returns the status the
// device wrote (CH_ETIMEOUT when the wait gave up as designed), or a
// negative status for a launch or copy failure.  Synchronises the stream.
extern "C" int ch_selftest_timeout(int which, void* stream) {
    if (which != 0 && which != 1) return CH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    char* mem = nullptr;
    const size_t bytes = sizeof(Ctl) + 256;
    if (cudaMalloc(&mem, bytes) != cudaSuccess) return CH_ENOMEM;
    int st = CH_ECUDA;
    Ctl* ctl = (Ctl*)mem;
    const size_t flag_off = (sizeof(Ctl) + 7) / 8 * 8 + 64;   // a zeroed word after the control block
    const unsigned long long* flag = (const unsigned long long*)(mem + flag_off);
    if (cudaMemsetAsync(mem, 0, bytes, s) == cudaSuccess) {
        selftest_kernel<<<1, 32, 0, s>>>(ctl, flag, which);
        int dev_status = CH_ECUDA;
        if (cudaGetLastError() == cudaSuccess &&
            cudaMemcpyAsync(&dev_status, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaStreamSynchronize(s) == cudaSuccess)
            st = dev_status;
    }
    cudaFree(mem);
    return st;
}
