// lf_step3d.cu -- D3Q19 step (three dimensions, walls normal to z).
#include "lf_internal.cuh"

namespace lf {

template <typename R>
cudaError_t launch_step3d(const Geom&, const Phys<R>&, const StepIO<R>&, bool, cudaStream_t)
{
    return cudaErrorNotSupported;
}

template cudaError_t launch_step3d<float>(const Geom&, const Phys<float>&, const StepIO<float>&, bool, cudaStream_t);
template cudaError_t launch_step3d<double>(const Geom&, const Phys<double>&, const StepIO<double>&, bool, cudaStream_t);

}  // namespace lf
