// Self-test of the kernels' bounded waits: one CTA waits on an mbarrier that
// nothing arrives on, with a short limit, through the same wait routine the
// de-dispersion kernel uses.  The wait must give up, record a timeout in the
// status word and return -- no fault, no hang -- and the host reads the
// status back.
#include <cuda_runtime.h>

#include <string>

#include "dd_kernel.cuh"

namespace dd {
namespace {

__global__ void wait_timeout_kernel(uint64_t limit_ns, int *status) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t mb = smem_addr(&bar);
    if (threadIdx.x == 0)
        mbar_init(mb, 1);  // expects one arrival that never comes
    __syncthreads();
    if (!mbar_wait(mb, 0, limit_ns))
        record(status, kDevTimeout);
}

}  // namespace
}  // namespace dd

extern "C" dd_status dd_selftest_wait_timeout(int64_t limit_ns, void *stream) {
    using dd::fail;
    if (limit_ns < 1000 || limit_ns > 2000000000LL)
        return fail(DD_ERR_INVALID, "limit must be between 1 us and 2 s");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *status = nullptr;
    if (cudaMalloc((void **)&status, sizeof(int)) != cudaSuccess)
        return fail(DD_ERR_NOMEM, "status allocation failed");
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        dd::wait_timeout_kernel<<<1, 32, 0, s>>>((uint64_t)limit_ns, status);
        e = cudaGetLastError();
    }
    int word = -1;
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        e = cudaMemcpy(&word, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(status);
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("self-test: ") + cudaGetErrorString(e));
    dd::count_launch();
    if (word == dd::kDevTimeout)
        return fail(DD_ERR_TIMEOUT, "the bounded wait ran out and reported it (expected)");
    return word == dd::kDevOk ? DD_OK : fail(DD_ERR_DEVICE, "unexpected status word");
}

// The same bounded wait, recording into the status word of the fixed array
// of dd_execute_noalloc instead of a word of its own, so that a test can check
// that dd_sync_noalloc reports such a timeout.  Allocates nothing; returns
// once the kernel is queued on stream.
extern "C" dd_status dd_selftest_noalloc_timeout(int64_t limit_ns, void *stream) {
    using dd::fail;
    if (limit_ns < 1000 || limit_ns > 2000000000LL)
        return fail(DD_ERR_INVALID, "limit must be between 1 us and 2 s");
    int *status = nullptr;
    dd_status st = dd::noalloc_status_word(&status);
    if (st != DD_OK)
        return st;
    dd::wait_timeout_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>((uint64_t)limit_ns,
                                                                           status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("self-test launch: ") + cudaGetErrorString(e));
    dd::count_launch();
    return DD_OK;
}
