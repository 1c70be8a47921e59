// Self-test of the bounded device wait: one thread waits on an mbarrier that
// nothing ever arrives on; the wait gives up after limit_ns, records
// TOK_ETIMEOUT in the status word and the kernel returns normally.
#include "common.cuh"

namespace tok {

namespace {
__global__ void timeout_selftest_kernel(int* status, unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0, status, limit_ns);
}
}  // namespace

int launch_timeout_selftest(int* status, unsigned long long limit_ns, cudaStream_t s) {
    timeout_selftest_kernel<<<1, 32, 0, s>>>(status, limit_ns);
    return (int)cudaGetLastError();
}

}  // namespace tok
