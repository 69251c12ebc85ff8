// k_selftest.cu -- a check of the failure path the pipelined kernels rely on:
// a bounded wait on an mbarrier that nothing completes gives up after its
// polls, records an error code, and the kernel returns, leaving the context
// usable (the wait a time-out of the update's pipeline goes through).
#include <cuda_runtime.h>

#include "clbm.h"
#include "clbm_internal.cuh"
#include "clbm_sync.cuh"

namespace clbm {
namespace {

__global__ void k_selftest_wait(int* err, int polls, long long* cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival expected; none comes
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        const bool done = mbar_wait_n(&bar, 0, polls);
        *cycles = clock64() - t0;
        *err = done ? 0 : 1;
    }
}

}  // namespace
}  // namespace clbm

extern "C" clbm_status clbm_selftest_bounded_wait(int device, int polls, double* ms) {
    if (polls < 1 || polls > (1 << 22)) {
        clbm::set_last_error("polls must be in [1, 2^22]");
        return CLBM_EINVAL;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        clbm::set_last_error("cudaSetDevice failed");
        return CLBM_ECUDA;
    }
    void* buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&buf, 16) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(buf);
        clbm::set_last_error("self-test set-up failed");
        return CLBM_ECUDA;
    }
    int* err = (int*)buf;
    long long* cyc = (long long*)((char*)buf + 8);
    cudaEventRecord(e0, 0);
    clbm::k_selftest_wait<<<1, 32>>>(err, polls, cyc);
    cudaEventRecord(e1, 0);
    cudaError_t ce = cudaEventSynchronize(e1);
    int h = -1;
    float t = 0.f;
    if (ce == cudaSuccess) ce = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (ce != cudaSuccess) {
        clbm::set_last_error(cudaGetErrorString(ce));
        return CLBM_ECUDA;
    }
    if (ms) *ms = t;
    if (h != 0) {
        clbm::set_last_error("the bounded wait gave up, as it must on a barrier nothing completes");
        return CLBM_ETIMEOUT;
    }
    clbm::set_last_error("a barrier nothing arrives on completed: the bounded wait is defective");
    return CLBM_OK;
}
