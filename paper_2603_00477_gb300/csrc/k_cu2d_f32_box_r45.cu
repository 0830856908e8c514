// k_cu2d_f32_box_r45.cu -- instantiations of the CUDA-core sweep launchers: 2-D FP32 box, r = 4..5.
#include "k_cuda_core_impl.cuh"

namespace gbs {

stencil_status launch_cu2d_f32_box_r45(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st)
{
    return cuimpl::launch2d_range<float, 0, 4, 5>(p, in, out, t, band, st);
}

}  // namespace gbs
