// lf_step3d_passes.cu -- the three-pass D3Q19 step (LF_VARIANT_SPLIT3) of
// arXiv:1102.3094, Sec. 2: pass A (mu and F = -d_a P_ab, Eqs. chem, ff), pass B
// (collision and push streaming, Eqs. moment, evoleqn, latticeforceterm) and
// pass C (phi(t+1), Eq. massdiff, and the first temperature sub-step), from
// lf_step3d_split.cu with the compact stencils and lf_step3d_iso.cu (passes A
// and C) with the isotropic ones, launched in order on one stream.  With pass
// timing on (lf_set_pass_timing), a CUDA event is recorded before pass A and
// after each pass.
#include "lf_internal.cuh"

namespace lf {

constexpr int kZC = 16;   // planes per segment of the phi pass unless the variant's param sets them

template <typename R>
cudaError_t launch_split3d(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s, cudaEvent_t* ev)
{
    const bool iso = g.stencil == LF_STENCIL_ISOTROPIC;
    cudaError_t e;
    if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
    e = iso ? launch_force3d_iso<R>(g, p, io, s) : launch_force3d_compact<R>(g, p, io, s);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return e;
    if (p.hydro && (e = launch_lb3d<R>(g, p, io, s)) != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[2], s)) != cudaSuccess) return e;
    // planes per segment of the phi pass: (param >> 20) & 255, 0 = kZC
    int zc = (g.tune >> 20) & 255;
    if (zc <= 0) zc = kZC;
    e = iso ? launch_phi3d_iso<R>(g, p, io, zc, s) : launch_phi3d_compact<R>(g, p, io, zc, s);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[3], s)) != cudaSuccess) return e;
    return cudaSuccess;
}

template cudaError_t launch_split3d<float>(const Geom&, const Phys<float>&, const StepIO<float>&, cudaStream_t,
                                           cudaEvent_t*);
template cudaError_t launch_split3d<double>(const Geom&, const Phys<double>&, const StepIO<double>&, cudaStream_t,
                                            cudaEvent_t*);

}  // namespace lf
