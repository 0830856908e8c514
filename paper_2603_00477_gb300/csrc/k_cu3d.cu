// k_cu3d.cu -- instantiations of the CUDA-core sweep launchers: 3-D FP64 and FP32, box r = 1..2, star r = 1..4.
#include "k_cuda_core_impl.cuh"

namespace gbs {

namespace {

template <typename T>
stencil_status launch3d_typed(const Plan &p, const void *in, void *out, int t, cudaStream_t st)
{
    const int r = p.pat.r;
    if (p.pat.shape == STENCIL_BOX) {
        switch (r) {
        case 1: return cuimpl::launch3d<T, 0, 1>(p, in, out, t, st);
        case 2: return cuimpl::launch3d<T, 0, 2>(p, in, out, t, st);
        }
    } else {
        switch (r) {
        case 1: return cuimpl::launch3d<T, 1, 1>(p, in, out, t, st);
        case 2: return cuimpl::launch3d<T, 1, 2>(p, in, out, t, st);
        case 3: return cuimpl::launch3d<T, 1, 3>(p, in, out, t, st);
        case 4: return cuimpl::launch3d<T, 1, 4>(p, in, out, t, st);
        }
    }
    return fail(STENCIL_ERR_UNSUPPORTED, "no CUDA-core kernel for this (shape, d, r)");
}

}  // namespace

stencil_status launch_cu3d(const Plan &p, const void *in, void *out, int t, cudaStream_t st)
{
    if (p.dtype == STENCIL_F64) return launch3d_typed<double>(p, in, out, t, st);
    return launch3d_typed<float>(p, in, out, t, st);
}

}  // namespace gbs
