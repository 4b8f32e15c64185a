// int32-field instantiations of the wavefront sweep kernel.
#include "sweep_impl.cuh"

namespace isg {
void* sweep_kernel_i32(int rng, int cmax)
{
    return rng == 0 ? sweep_detail::pick_cmax<int32_t, 0>(cmax)
                    : sweep_detail::pick_cmax<int32_t, 1>(cmax);
}
}  // namespace isg
