// int32-field instantiations of the track-scheduled sweep kernel.
#include "track_impl.cuh"

namespace isg {
void* track_kernel_i32(int rng, bool batch)
{
    return rng == 0 ? track_detail::pick_track<int32_t, 0>(batch) : track_detail::pick_track<int32_t, 1>(batch);
}
}  // namespace isg
