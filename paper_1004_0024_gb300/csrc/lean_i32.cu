// int32-field instantiations of the lean sweep kernel.
#include "lean_impl.cuh"

namespace isg {
void* lean_kernel_i32(int rng, int cmax, bool batch)
{
    return rng == 0 ? lean_detail::pick_lean<int32_t, 0>(cmax, batch) : lean_detail::pick_lean<int32_t, 1>(cmax, batch);
}
}  // namespace isg
