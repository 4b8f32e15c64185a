// MT19937 instantiations of the packed sweep kernel, and its layout size.
#include "packed_impl.cuh"

namespace isg {
void* packed_kernel_mt(int rmax, bool batch)
{
    return batch ? packed_detail::pick_packed_batch<0>(rmax) : packed_detail::pick_packed<0>(rmax);
}

size_t packed_smem_bytes(const SweepArgs& a, int threads)
{
    return packed_detail::packed_layout(a, threads).total;
}
}  // namespace isg
