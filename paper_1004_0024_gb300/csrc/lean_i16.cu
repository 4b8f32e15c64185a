// int16-field instantiations of the lean sweep kernel.
#include "lean_impl.cuh"

namespace isg {
void* lean_kernel_i16(int rng, int cmax, bool batch, bool small, bool longc)
{
    return rng == 0 ? lean_detail::pick_lean<int16_t, 0>(cmax, batch, small, longc)
                    : lean_detail::pick_lean<int16_t, 1>(cmax, batch, small, longc);
}
}  // namespace isg
