// int16-field instantiations of the register-resident sweep kernel.
#include "fast_impl.cuh"

namespace isg {
void* fast_kernel_i16(int rng, int cmax, bool batch)
{
    return rng == 0 ? fast_detail::pick_fast<int16_t, 0>(cmax, batch) : fast_detail::pick_fast<int16_t, 1>(cmax, batch);
}
}  // namespace isg
