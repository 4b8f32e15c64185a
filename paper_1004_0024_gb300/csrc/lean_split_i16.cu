// int16-field instantiations of the lean sweep kernel with split couplings.
#include "lean_impl.cuh"

namespace isg {
void* lean_split_kernel_i16(int rng, int cmax, bool small, bool longc)
{
    return rng == 0 ? lean_detail::pick_lean_split<int16_t, 0>(cmax, small, longc)
                    : lean_detail::pick_lean_split<int16_t, 1>(cmax, small, longc);
}
}  // namespace isg
