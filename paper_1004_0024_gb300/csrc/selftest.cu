// Failure detection without a GPU fault: kernels whose bounded waits are made
// to run out (a grid-barrier count and an mbarrier phase that nothing
// completes).  Each raises the error flag and returns, so the host reads
// ISING_ERR_TIMEOUT and the context stays usable.
#include <cuda_runtime.h>

#include "fast_impl.cuh"
#include "handle.h"

namespace isg {
namespace {

// grid_sync towards a target one more than the blocks that will ever arrive
__global__ void barrier_timeout_kernel(unsigned* ctr, int* err)
{
    __shared__ int s_flag;
    fast_detail::grid_sync(ctr, gridDim.x + 1u, err, &s_flag);
}

// an mbarrier phase that no thread arrives on
__global__ void mbarrier_timeout_kernel(int* err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0)
        mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0, kWaitPolls))
        set_err(err, kErrTimeout);
}

}  // namespace
}  // namespace isg

extern "C" int32_t ising_selftest_wait(int32_t kind, void* stream)
{
    int32_t rc = isg_device_setup();
    if (rc)
        return rc;
    if (kind != 0 && kind != 1)
        return isg_fail(ISING_ERR_INVALID_ARG, "kind must be 0 (grid barrier) or 1 (mbarrier)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 16);
    if (e != cudaSuccess)
        return isg_fail(ISING_ERR_OOM, cudaGetErrorString(e));
    unsigned* ctr = static_cast<unsigned*>(buf);
    int* err = reinterpret_cast<int*>(static_cast<char*>(buf) + 8);
    e = cudaMemsetAsync(buf, 0, 16, st);
    if (e == cudaSuccess) {
        if (kind == 0)
            isg::barrier_timeout_kernel<<<2, 32, 0, st>>>(ctr, err);
        else
            isg::mbarrier_timeout_kernel<<<1, 32, 0, st>>>(err);
        e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess)
        return isg_fail(ISING_ERR_CUDA, cudaGetErrorString(e));
    if (h == isg::kErrTimeout)
        return isg_fail(ISING_ERR_TIMEOUT, "a bounded device wait gave up (as the self-test intends)");
    return ISING_OK;
}
