// Launch helpers of the register-resident sweep kernel (fast_impl.cuh).
#include <algorithm>

#include "lean_impl.cuh"
#include "packed_impl.cuh"
#include "track_impl.cuh"

namespace isg {
namespace {

void* pick(int field_bits, int rng, int cmax, int variant = 0, bool batch = false, bool split = false)
{
    if (variant == 5)  // packed: plain couplings; cmax = slot rounds per thread
        return split ? nullptr : packed_kernel_ptr(rng, cmax, batch);
    if (split)  // lean variants only, single-instance launches only
        return (batch || !(variant == 1 || variant == 3 || variant == 4))
                   ? nullptr
                   : (field_bits == 16 ? lean_split_kernel_i16(rng, cmax, variant == 3, variant == 4)
                                       : lean_split_kernel_i32(rng, cmax, variant == 3, variant == 4));
    if (variant == 2)
        return field_bits == 16 ? track_kernel_i16(rng, batch) : track_kernel_i32(rng, batch);
    if (variant == 1 || variant == 3 || variant == 4)  // 3: small blocks, 4: long columns
        return field_bits == 16 ? lean_kernel_i16(rng, cmax, batch, variant == 3, variant == 4)
                                : lean_kernel_i32(rng, cmax, batch, variant == 3, variant == 4);
    return field_bits == 16 ? fast_kernel_i16(rng, cmax, batch) : fast_kernel_i32(rng, cmax, batch);
}

size_t g_fast_max_dyn = 0;

}  // namespace

size_t fast_smem_bytes(const SweepArgs& a, int field_bits, int variant, int threads)
{
    const int fb = field_bits == 16 ? 2 : 4;
    const size_t b = variant == 5   ? packed_smem_bytes(a, threads)
                     : variant == 2 ? track_detail::track_layout(a, fb, threads).total
                                    : fast_detail::fast_layout(a, fb).total;
    return (g_fast_max_dyn && b > g_fast_max_dyn) ? size_t(-1) : b;
}

cudaError_t fast_set_smem_limits()
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess)
        return e;
    size_t lim = size_t(optin);
    for (int batch : {0, 1, 2})  // 2: the split-coupling instantiations
    for (int variant : {0, 1, 2, 3, 4, 5})
        for (int fb : {16, 32})
            for (int rng : {0, 1})
                for (int cm : {1, 2, 3, 4, 5, 8, 101, 102}) {
                    if ((variant == 2 && cm != 1) || (variant == 5 && (batch == 2 || fb != 16)) ||
                        (variant != 5 && (cm == 3 || cm == 5 || cm > 100)) || (cm > 100 && batch != 0))
                        continue;
                    void* fn = pick(fb, rng, cm, variant, batch == 1, batch == 2);
                    if (!fn)
                        continue;
                    cudaFuncAttributes fa;
                    e = cudaFuncGetAttributes(&fa, fn);
                    if (e != cudaSuccess)
                        return e;
                    const size_t dyn = size_t(optin) - fa.sharedSizeBytes;
                    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn));
                    if (e != cudaSuccess)
                        return e;
                    lim = std::min(lim, dyn);
                }
    g_fast_max_dyn = lim;
    return cudaSuccess;
}

cudaError_t fast_max_blocks_per_sm(int field_bits, int cmax, int rng, int threads, size_t smem,
                                   int* out, int variant, bool split)
{
    void* fn = pick(field_bits, rng, cmax, variant, false, split);
    if (!fn)
        return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fn, threads, smem);
}

cudaError_t launch_fast(const SweepArgs& a, int field_bits, int cmax, int threads, int blocks,
                        size_t smem, bool cooperative, cudaStream_t st, int variant)
{
    void* fn = pick(field_bits, a.rng, cmax, variant, false, a.split != 0);
    if (!fn)
        return cudaErrorInvalidValue;
    if (variant == 5)  // the packed kernel's blocks: its sweep threads and the generator warps
        threads = a.sweep_threads + 32 * a.gen;
    SweepArgs copy = a;
    void* args[] = {&copy};
    if (cooperative)
        return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(threads), args, smem, st);
    return cudaLaunchKernel(fn, dim3(blocks), dim3(threads), args, smem, st);
}

cudaError_t fast_max_blocks_per_sm_batch(int rng, int cmax, int threads, size_t smem, int* out)
{
    void* fn = pick(16, rng, cmax, 5, true, false);
    if (!fn)
        return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fn, threads, smem);
}

cudaError_t launch_packed_batch(const SweepArgs* args, const BatchItem* items, int n_items, int rng, int rmax,
                                int threads, size_t smem, cudaStream_t st)
{
    void* fn = pick(16, rng, rmax, 5, true, false);
    if (!fn)
        return cudaErrorInvalidValue;
    void* params[] = {&args, &items};
    return cudaLaunchCooperativeKernel(fn, dim3(n_items), dim3(threads), params, smem, st);
}

cudaError_t launch_fast_batch(const SweepArgs* args, const BatchItem* items, int n_items,
                              int field_bits, int rng, int cmax, int threads, size_t smem, int variant,
                              cudaStream_t st)
{
    void* fn = pick(field_bits, rng, cmax, variant, true);
    if (!fn)
        return cudaErrorInvalidValue;
    void* params[] = {&args, &items};
    return cudaLaunchKernel(fn, dim3(n_items), dim3(threads), params, smem, st);
}

}  // namespace isg
