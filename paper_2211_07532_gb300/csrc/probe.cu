// Failure detection without a fault: a probe that makes the library's bounded device waits
// run out.  One block of 64 threads; thread 0 waits on phase 0 of an mbarrier that nothing
// arrives on, through the same bounded wait the operator kernels use, with a caller-chosen
// poll limit; when it gives up it records AEXP_ERR_DEVICE_TIMEOUT in the workspace status word
// and raises the CTA's abort flag.  Thread 32 waits on a second such barrier through the
// tensor-core kernels' wait, which polls the abort flag and must give up as soon as thread 0
// has.  Nothing is copied or issued asynchronously, so nothing is in flight when the block
// exits, and every wait ends after a bounded number of polls.
#include "tc_common.cuh"

namespace aexp {
namespace {

__global__ void bounded_wait_probe_kernel(int polls, int *status, int *result) {
    __shared__ uint64_t bar[2];
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool ok = mbar_wait_bounded(&bar[0], 0, status, polls);
        if (!ok) *(volatile int *)&abort_flag = 1;
        result[0] = ok ? 0 : 1;
    } else if (threadIdx.x == 32) {
        const bool ok = wait_or_abort(&bar[1], 0, &abort_flag, status);
        result[1] = ok ? 0 : 1;
    }
}

}  // namespace

cudaError_t bounded_wait_probe(int polls, int *status, int *result, cudaStream_t st) {
    bounded_wait_probe_kernel<<<1, 64, 0, st>>>(polls, status, result);
    return cudaGetLastError();
}

}  // namespace aexp
