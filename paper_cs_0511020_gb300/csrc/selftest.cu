// selftest.cu -- the bounded device wait, exercised without a fault.
//
// Every wait of the library's kernels (the MSD pass waiting for its tile
// copies) polls an mbarrier a bounded number of times and for at most 2 s,
// then records PBIT_ETIMEOUT in the call's status word and returns, so a
// copy that never lands ends the call with an error instead of a hung GPU.
// This kernel makes that wait run out on purpose: its mbarrier expects one
// arrival that never comes, and nothing is copied, so nothing is in flight
// when it gives up.
#include "engine.h"

namespace pbit {

__global__ void k_wait_selftest(int32_t *status, long long iterations) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival expected; none is ever made
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u, iterations))
        set_status(status, PBIT_ETIMEOUT);
}

}  // namespace pbit

extern "C" pbit_status pbit_selftest_bounded_wait(int64_t iterations, void *stream) {
    if (iterations < 1 || iterations > (1ll << 24))
        return PBIT_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t *d = nullptr;
    if (cudaMalloc(&d, sizeof(int32_t)) != cudaSuccess)
        return PBIT_ECUDA;
    int32_t h = 0;
    pbit_status st = PBIT_ECUDA;
    if (cudaMemsetAsync(d, 0, sizeof(int32_t), s) == cudaSuccess) {
        pbit::k_wait_selftest<<<1, 32, 0, s>>>(d, (long long)iterations);
        if (cudaGetLastError() == cudaSuccess &&
            cudaMemcpyAsync(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaStreamSynchronize(s) == cudaSuccess)
            st = pbit::map_status(h);
    }
    cudaFree(d);
    return st;
}
