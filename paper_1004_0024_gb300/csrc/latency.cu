// Dependent-chain latencies of the operations on a sweep level's critical
// path, measured on the current GPU: ising_measure_latencies.  One block of
// 256 threads (the packed kernel's resident block); each chain is 4096
// operations that depend on one another, timed with clock64.
#include <cuda_runtime.h>

#include "handle.h"
#include "ising_gb300.h"

namespace isg {
namespace {

constexpr int kChain = 4096;

__global__ void __launch_bounds__(256) latency_kernel(long long* out, unsigned* sink)
{
    __shared__ unsigned sh[1024];
    const int tid = threadIdx.x;
    for (int i = tid; i < 1024; i += blockDim.x)
        sh[i] = unsigned(i * 7 + 1) & 1023u;  // a permutation of 0..1023
    __syncthreads();
    unsigned x = unsigned(tid) & 1023u;
    const long long t0 = clock64();
    for (int i = 0; i < kChain; ++i)
        x = sh[x];  // shared-memory load whose address is the previous result
    const long long t1 = clock64();
    unsigned y = x + 3u;
    for (int i = 0; i < kChain; ++i)
        y = y * 2654435761u + x;  // integer multiply-add
    const long long t2 = clock64();
    unsigned z = y;
    for (int i = 0; i < kChain; ++i)
        z = __shfl_sync(0xFFFFFFFFu, z, (z + unsigned(i)) & 31u);  // warp shuffle
    const long long t3 = clock64();
    for (int i = 0; i < kChain; ++i)
        __syncthreads();  // barrier of the block's 8 warps
    const long long t4 = clock64();
    if (tid == 0) {
        out[0] = t1 - t0;
        out[1] = t2 - t1;
        out[2] = t3 - t2;
        out[3] = t4 - t3;
    }
    sink[tid] = z;  // keeps the chains alive
}

}  // namespace
}  // namespace isg

extern "C" int32_t ising_measure_latencies(double* cycles)
{
    if (!cycles)
        return isg_fail(ISING_ERR_INVALID_ARG, "NULL output");
    int32_t rc = isg_device_setup();
    if (rc)
        return rc;
    void* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 4 * sizeof(long long) + 256 * sizeof(unsigned));
    if (e != cudaSuccess)
        return isg_fail(ISING_ERR_OOM, cudaGetErrorString(e));
    long long* out = static_cast<long long*>(buf);
    unsigned* sink = reinterpret_cast<unsigned*>(out + 4);
    long long h[4] = {0, 0, 0, 0};
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the second run is timed warm
        isg::latency_kernel<<<1, 256>>>(out, sink);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpy(h, out, sizeof h, cudaMemcpyDeviceToHost);
    }
    cudaFree(buf);
    if (e != cudaSuccess)
        return isg_fail(ISING_ERR_CUDA, cudaGetErrorString(e));
    for (int k = 0; k < 4; ++k)
        cycles[k] = double(h[k]) / double(isg::kChain);
    return ISING_OK;
}
