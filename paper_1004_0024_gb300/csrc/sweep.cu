// Launch helpers of the wavefront sweep (kernels are instantiated per field
// width in sweep_i16.cu / sweep_i32.cu).
#include <algorithm>

#include "sweep_impl.cuh"

namespace isg {
namespace {

void* pick_kernel(int field_bits, int rng, int cmax)
{
    return field_bits == 16 ? sweep_kernel_i16(rng, cmax) : sweep_kernel_i32(rng, cmax);
}

}  // namespace

int sweep_cmax_for(int c)
{
    for (int m : {1, 2, 4, 8, 16, 32})
        if (c <= m)
            return m;
    return 0;
}

size_t sweep_smem_bytes(const SweepArgs& a, int field_bits)
{
    return sweep_detail::smem_layout(a, field_bits == 16 ? 2 : 4).total;
}

size_t g_max_dyn_smem = 0;

cudaError_t sweep_set_smem_limits()
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess)
        return e;
    size_t lim = size_t(optin);
    for (int fb : {16, 32})
        for (int rng : {0, 1})
            for (int cm : {1, 2, 4, 8, 16, 32}) {
                cudaFuncAttributes fa;
                e = cudaFuncGetAttributes(&fa, pick_kernel(fb, rng, cm));
                if (e != cudaSuccess)
                    return e;
                const size_t dyn = size_t(optin) - fa.sharedSizeBytes;
                e = cudaFuncSetAttribute(pick_kernel(fb, rng, cm),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn));
                if (e != cudaSuccess)
                    return e;
                lim = std::min(lim, dyn);
            }
    g_max_dyn_smem = lim;
    return cudaSuccess;
}

size_t sweep_max_dynamic_smem() { return g_max_dyn_smem; }

cudaError_t sweep_max_blocks_per_sm(int field_bits, int cmax, int rng, int threads, size_t smem,
                                    int* out)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, pick_kernel(field_bits, rng, cmax),
                                                         threads, smem);
}

cudaError_t launch_sweep(const SweepArgs& a, int field_bits, int cmax, int threads, int blocks,
                         size_t smem, cudaStream_t st)
{
    void* fn = pick_kernel(field_bits, a.rng, cmax);
    if (!fn)
        return cudaErrorInvalidValue;
    SweepArgs copy = a;
    void* args[] = {&copy};
    return cudaLaunchKernel(fn, dim3(blocks), dim3(threads), args, smem, st);
}

}  // namespace isg
