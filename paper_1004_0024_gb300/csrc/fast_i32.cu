// int32-field instantiations of the register-resident sweep kernel.
#include "fast_impl.cuh"

namespace isg {
void* fast_kernel_i32(int rng, int cmax, bool batch)
{
    return rng == 0 ? fast_detail::pick_fast<int32_t, 0>(cmax, batch) : fast_detail::pick_fast<int32_t, 1>(cmax, batch);
}
}  // namespace isg
