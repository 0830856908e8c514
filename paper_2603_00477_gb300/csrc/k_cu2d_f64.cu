// k_cu2d_f64.cu -- instantiations of the CUDA-core sweep launchers: 2-D FP64 box and star, r = 1..7.
#include "k_cuda_core_impl.cuh"

namespace gbs {

stencil_status launch_cu2d_f64(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st)
{
    if (p.pat.shape == STENCIL_BOX) return cuimpl::launch2d_range<double, 0, 1, 7>(p, in, out, t, band, st);
    return cuimpl::launch2d_range<double, 1, 1, 7>(p, in, out, t, band, st);
}

}  // namespace gbs
