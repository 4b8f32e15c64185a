// Philox4x32-10 instantiations of the packed sweep kernel.
#include "packed_impl.cuh"

namespace isg {
void* packed_kernel_philox(int rmax, bool batch)
{
    return batch ? packed_detail::pick_packed_batch<1>(rmax) : packed_detail::pick_packed<1>(rmax);
}
}  // namespace isg
