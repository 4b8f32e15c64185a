// int16-field instantiations of the wavefront sweep kernel.
#include "sweep_impl.cuh"

namespace isg {
void* sweep_kernel_i16(int rng, int cmax)
{
    return rng == 0 ? sweep_detail::pick_cmax<int16_t, 0>(cmax)
                    : sweep_detail::pick_cmax<int16_t, 1>(cmax);
}
}  // namespace isg
