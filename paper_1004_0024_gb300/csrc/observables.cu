// Per-temperature observables of a handle: energy E and magnetisation
// m = sum_i s_i of the replica that currently holds each temperature index
// (replicas exchange temperature labels under parallel tempering, section
// 3.1).  One block per replica slot sums its int8 spins.
#include <cuda_runtime.h>

#include <vector>

#include "handle.h"
#include "ising_internal.cuh"

namespace isg {
namespace {

__global__ void __launch_bounds__(256) magnetisation_kernel(const int8_t* __restrict__ spins, int N,
                                                            long long* __restrict__ out)
{
    __shared__ int red[256];
    const int8_t* s = spins + size_t(blockIdx.x) * N;
    int acc = 0;
    const int n16 = (reinterpret_cast<uintptr_t>(s) & 15) == 0 ? N / 16 : 0;
    for (int c = threadIdx.x; c < n16; c += blockDim.x) {
        const int4 w = reinterpret_cast<const int4*>(s)[c];
        const int v[4] = {w.x, w.y, w.z, w.w};
        for (int k = 0; k < 4; ++k)  // four signed bytes per word
            acc += int(int8_t(v[k])) + int(int8_t(v[k] >> 8)) + int(int8_t(v[k] >> 16)) + int(int8_t(v[k] >> 24));
    }
    for (int i = n16 * 16 + threadIdx.x; i < N; i += blockDim.x)
        acc += s[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        out[blockIdx.x] = red[0];
}

}  // namespace
}  // namespace isg

extern "C" int32_t ising_read_observables(ising_t h, int64_t* energy_by_temp, int64_t* magnetisation_by_temp)
{
    if (!h)
        return isg_fail(ISING_ERR_INVALID_ARG, "handle is NULL");
    if (!h->inited)
        return isg_fail(ISING_ERR_NOT_INITIALISED, "call ising_replicas_init first");
    const int R = h->R;
    cudaError_t e = cudaSuccess;
    if (!h->d_obs) {
        e = cudaMalloc(reinterpret_cast<void**>(&h->d_obs), sizeof(long long) * size_t(R));
        if (e != cudaSuccess) {
            h->d_obs = nullptr;
            return isg_fail(e == cudaErrorMemoryAllocation ? ISING_ERR_OOM : ISING_ERR_CUDA, cudaGetErrorString(e));
        }
    }
    isg::magnetisation_kernel<<<R, 256, 0, h->stream>>>(h->d_spins, h->n, h->d_obs);
    std::vector<long long> m(R);
    std::vector<int> E(R), temp(R);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m.data(), h->d_obs, sizeof(long long) * R, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E.data(), h->d_E, sizeof(int) * R, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(temp.data(), h->d_temp, sizeof(int) * R, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess)
        return isg_fail(ISING_ERR_CUDA, cudaGetErrorString(e));
    for (int r = 0; r < R; ++r) {
        const int k = temp[r];
        if (k < 0 || k >= R)
            return isg_fail(ISING_ERR_CUDA, "temperature labels are not a permutation");
        if (energy_by_temp)
            energy_by_temp[k] = E[r];
        if (magnetisation_by_temp)
            magnetisation_by_temp[k] = m[r];
    }
    return ISING_OK;
}
