// Self-test of the bounded device-side wait used by the exchange-variant
// agent sweep (agent_xpose.cuh): one CTA waits on an mbarrier that nothing
// completes; the wait must give up after its poll limit, set the error
// word and return, so the host sees PMACE_ERR_TIMEOUT and the context stays
// usable.  Nothing else is involved, so giving up cannot leave a copy in
// flight.
#include "agent_xpose.cuh"
#include "pmace.h"

namespace pmace {
namespace {

__global__ void bounded_wait_kernel(int* err) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);   // one arrival expected, none ever made
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait_bounded(b, 0, err);
}

}  // namespace
}  // namespace pmace

extern "C" pmace_status pmace_selftest_bounded_wait(void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* err = nullptr;
    int h = 0;
    cudaError_t e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        pmace::bounded_wait_kernel<<<1, 32, 0, s>>>(err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (err) cudaFree(err);
    if (e != cudaSuccess) {
        pmace::set_unbound_error(cudaGetErrorString(e));
        return PMACE_ERR_CUDA;
    }
    if (h & 2) {
        pmace::set_unbound_error("the bounded wait gave up as designed");
        return PMACE_ERR_TIMEOUT;
    }
    return PMACE_OK;
}
