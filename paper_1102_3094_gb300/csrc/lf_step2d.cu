// lf_step2d.cu -- one fused pass per time step of the hybrid LB/FD method of
// arXiv:1102.3094, Sec. 2, on the D2Q9 lattice: the kernels and launchers of
// the tile form (its body, described here, is in lf_tile2d.cuh, shared with
// the ensembles) and of the row-marching forms (lf_march2d.cuh,
// lf_march2d_x2.cuh).
//
// A CTA owns a TX x TY tile of sites.  From HBM it reads phi with a halo of 4,
// T with a halo of 2 and the populations of its tile plus a one-site ring; it
// writes phi(t+1), T(t+1) of the tile and pushes the post-collision
// populations to their destinations.  Everything in between lives in shared
// memory, each stage on a region one site smaller than the one before:
//
//   r=4  phi, r=2 T                       (loaded; halo mapped by the walls)
//   r=3  psi = nabla^2 phi                 (5-point)
//   r=2  lam = nabla^2 psi = nabla^4 phi;  P_ab (pressure tensor, Sec. 2)
//   r=1  mu (Eq. chem);  F_b = -d_a P_ab   (Eq. ff, central differences)
//   r=1  n, u = (sum f e + F/2)/n (Eq. moment); g = phi u;
//        interior sites: BGK + Guo collision (Eqs. evoleqn, latticeforceterm)
//        and push streaming with halfway bounce-back at the walls
//   r=0  phi += -div(g) + Gamma nabla^2 mu (Eq. massdiff); T += dxi nabla^2 T
//
// Halo sites are read through the boundary map: x wraps; along y the lattice
// is either periodic or reflected evenly about the planes half a spacing
// outside rows 0 and ny-1 (the walls).  Every derived field at a halo site is
// then computed from the reflected state, which is the wall rule itself.  The
// one odd quantity, the wall-normal flux g_y, is reflected with a sign flip
// in the last stage.  Populations are stored as deviations f_i - w_i n0.
//
// With the isotropic stencils the march variants run the row march of
// lf_march2d_iso.cuh (sliding row sums); the tile kernel below serves
// LF_VARIANT_TILE and the derived fields.
//
// With ISO set, every derivative takes the isotropic 9-point form instead:
// lap A = [4 (nearest) + (diagonal) - 20 A]/6 and d_x A = [4 (E - W) + (NE - NW)
// + (SE - SW)]/12 (the D2Q9 weights: d_a = 3 sum w_i e_ia A(r + e_i), lap = 6
// sum w_i [A(r + e_i) - A(r)]).  The regions are the same; the flux g is then
// also needed on the corners of the r = 1 ring, and the wall images of g and
// of the halfway temperature ghost are applied to whole rows.
#include "lf_internal.cuh"
#include "lf_march2d.cuh"
#include "lf_march2d_iso.cuh"
#include "lf_march2d_x2.cuh"
#include "lf_tile2d.cuh"

namespace lf {

namespace {

// The tile kernel: one CTA per tile (lf_tile2d.cuh).
template <typename R, int TX, int TY, int NT, bool AUX, bool ISO>
__global__ void __launch_bounds__(NT) k_step2d(Geom g, Phys<R> p, StepIO<R> io)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile::step2d_tile<R, TX, TY, NT, AUX, ISO>(g, p, io, blockIdx.x, blockIdx.y, smem_raw);
}

// Row-marching variant (the default for lf_step): see lf_march2d.cuh.
template <typename R, int NT, int D>
__global__ void __launch_bounds__(NT) k_march2d(Geom g, Phys<R> p, StepIO<R> io, int H)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    march::march2d_segment<R, NT, D>(g, p, io, blockIdx.x, blockIdx.y, H, smem_raw);
}

// The row march with the isotropic 9-point stencils: see lf_march2d_iso.cuh.
template <typename R, int NT, int D>
__global__ void __launch_bounds__(NT) k_march2d_iso(Geom g, Phys<R> p, StepIO<R> io, int H)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    march::march2d_segment_iso<R, NT, D>(g, p, io, blockIdx.x, blockIdx.y, H, smem_raw);
}

// The isotropic row march on two segments per CTA (packed FP32x2 lanes).
template <int NT, int D, bool HYDRO, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_march2d_iso_x2(Geom g, Phys<float> p, StepIO<float> io, int npairs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    march::march2d_pair_iso<NT, D, HYDRO>(g, p, io, blockIdx.x, blockIdx.y, npairs, smem_raw);
}

// Two segments per CTA in the lanes of float2 (packed FP32x2 arithmetic).
template <int NT, int D, bool HYDRO, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_march2d_x2(Geom g, Phys<float> p, StepIO<float> io, int npairs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    march::march2d_pair<NT, D, HYDRO>(g, p, io, blockIdx.x, blockIdx.y, npairs, smem_raw);
}

template <int NT, int D, bool HYDRO, int MINB>
cudaError_t launch_march_x2(const Geom& g, const Phys<float>& p, const StepIO<float>& io, cudaStream_t s)
{
    using M = march::March2<NT, D>;
    auto kern = k_march2d_x2<NT, D, HYDRO, MINB>;
    static unsigned long long attr_done = 0;
    cudaError_t e = raise_smem_limit(kern, (int)M::BYTES, &attr_done);
    if (e != cudaSuccess) return e;
    int sms = 0;
    if ((e = device_sms(&sms)) != cudaSuccess) return e;
    const int H = march::march2_rows_for(g.nx, g.ny, M::U, g.tune & 0xFFFF, sms);
    int npairs = (g.ny + 2 * H - 1) / (2 * H);
    if (npairs > g.ny / 2) npairs = g.ny / 2;       // every lane keeps at least one row
    dim3 grid((g.nx + M::U - 1) / M::U, npairs);
    kern<<<grid, NT, M::BYTES, s>>>(g, p, io, npairs);
    return cudaGetLastError();
}

template <typename R, int NT, int D>
cudaError_t launch_march(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s)
{
    using M = march::March<R, NT, D>;
    auto kern = k_march2d<R, NT, D>;
    static unsigned long long attr_done = 0;
    cudaError_t e = raise_smem_limit(kern, (int)M::BYTES, &attr_done);
    if (e != cudaSuccess) return e;
    int sms = 0;
    if ((e = device_sms(&sms)) != cudaSuccess) return e;
    const int H = march::march2_rows_for(g.nx, g.ny, M::U, g.tune & 0xFFFF, sms);
    dim3 grid((g.nx + M::U - 1) / M::U, (g.ny + H - 1) / H);
    kern<<<grid, NT, M::BYTES, s>>>(g, p, io, H);
    return cudaGetLastError();
}

template <int NT, int D, bool HYDRO, int MINB>
cudaError_t launch_march_iso_x2(const Geom& g, const Phys<float>& p, const StepIO<float>& io, cudaStream_t s)
{
    using M = march::MarchIso2<NT, D>;
    auto kern = k_march2d_iso_x2<NT, D, HYDRO, MINB>;
    static unsigned long long attr_done = 0;
    cudaError_t e = raise_smem_limit(kern, (int)M::BYTES, &attr_done);
    if (e != cudaSuccess) return e;
    int sms = 0;
    if ((e = device_sms(&sms)) != cudaSuccess) return e;
    const int H = march::march2_rows_for(g.nx, g.ny, M::U, g.tune & 0xFFFF, sms);
    int npairs = (g.ny + 2 * H - 1) / (2 * H);
    if (npairs > g.ny / 2) npairs = g.ny / 2;       // every lane keeps at least one row
    dim3 grid((g.nx + M::U - 1) / M::U, npairs);
    kern<<<grid, NT, M::BYTES, s>>>(g, p, io, npairs);
    return cudaGetLastError();
}

template <typename R, int NT, int D>
cudaError_t launch_march_iso(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s)
{
    using M = march::MarchIso<R, NT, D>;
    auto kern = k_march2d_iso<R, NT, D>;
    static unsigned long long attr_done = 0;
    cudaError_t e = raise_smem_limit(kern, (int)M::BYTES, &attr_done);
    if (e != cudaSuccess) return e;
    int sms = 0;
    if ((e = device_sms(&sms)) != cudaSuccess) return e;
    const int H = march::march2_rows_for(g.nx, g.ny, M::U, g.tune & 0xFFFF, sms);
    dim3 grid((g.nx + M::U - 1) / M::U, (g.ny + H - 1) / H);
    kern<<<grid, NT, M::BYTES, s>>>(g, p, io, H);
    return cudaGetLastError();
}

template <typename R, int TX, int TY, int NT, bool AUX, bool ISO>
cudaError_t launch_cfg(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s)
{
    constexpr size_t bytes = tile::Tile<R, TX, TY>::BYTES;
    auto kern = k_step2d<R, TX, TY, NT, AUX, ISO>;
    static unsigned long long attr_done = 0;      // per instantiation and device
    const cudaError_t e = raise_smem_limit(kern, (int)bytes, &attr_done);
    if (e != cudaSuccess) return e;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);
    kern<<<grid, NT, bytes, s>>>(g, p, io);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Extra temperature sub-steps (xi/nsub each) when nsub > 1.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_tsub2d(Geom g, Phys<R> p, const R* __restrict__ Tin, R* __restrict__ Tout)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    march::tsub2d_site(g, p, Tin, Tout, x, y);
}

// The same sub-step with the isotropic 9-point Laplacian (lf_tile2d.cuh).
template <typename R>
__global__ void k_tsub2d_iso(Geom g, Phys<R> p, const R* __restrict__ Tin, R* __restrict__ Tout)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    tile::tsub2d_site_iso(g, p, Tin, Tout, x, y);
}

}  // namespace

template <typename R>
cudaError_t launch_step2d(const Geom& g, const Phys<R>& p, const StepIO<R>& io, bool aux, cudaStream_t s)
{
    if (g.stencil == LF_STENCIL_ISOTROPIC) {           // the row marches or the tile kernel
        if constexpr (sizeof(R) == 4) {
            if (!aux && g.variant == LF_VARIANT_MARCH2 && g.ny >= 2) {
                if ((g.tune >> 16) == 1)
                    return p.hydro ? launch_march_iso_x2<64, 3, true, 6>(g, p, io, s)
                                   : launch_march_iso_x2<64, 3, false, 6>(g, p, io, s);
                return p.hydro ? launch_march_iso_x2<128, 3, true, 3>(g, p, io, s)
                               : launch_march_iso_x2<128, 3, false, 3>(g, p, io, s);
            }
        }
        if (!aux && (g.variant == LF_VARIANT_MARCH || g.variant == LF_VARIANT_MARCH2) && g.ny >= 2)
            return (g.tune >> 16) == 1 ? launch_march_iso<R, 64, 3>(g, p, io, s) : launch_march_iso<R, 128, 3>(g, p, io, s);
        if constexpr (sizeof(R) == 4)
            return aux ? launch_cfg<R, 64, 16, 256, true, true>(g, p, io, s)
                       : launch_cfg<R, 64, 16, 256, false, true>(g, p, io, s);
        else
            return aux ? launch_cfg<R, 32, 16, 256, true, true>(g, p, io, s)
                       : launch_cfg<R, 32, 16, 256, false, true>(g, p, io, s);
    }
    if constexpr (sizeof(R) == 4) {
        if (!aux && g.variant == LF_VARIANT_MARCH2 && g.ny >= 2)
        {
            if ((g.tune >> 16) == 1)
                return p.hydro ? launch_march_x2<64, 3, true, 6>(g, p, io, s)
                               : launch_march_x2<64, 3, false, 6>(g, p, io, s);
            return p.hydro ? launch_march_x2<128, 3, true, 3>(g, p, io, s) : launch_march_x2<128, 3, false, 3>(g, p, io, s);
        }
    }
    if (!aux && (g.variant == LF_VARIANT_MARCH || g.variant == LF_VARIANT_MARCH2))
        return (g.tune >> 16) == 1 ? launch_march<R, 64, 3>(g, p, io, s) : launch_march<R, 128, 3>(g, p, io, s);
    if constexpr (sizeof(R) == 4) {
        return aux ? launch_cfg<R, 64, 16, 256, true, false>(g, p, io, s)
                   : launch_cfg<R, 64, 16, 256, false, false>(g, p, io, s);
    } else {
        return aux ? launch_cfg<R, 32, 16, 256, true, false>(g, p, io, s)
                   : launch_cfg<R, 32, 16, 256, false, false>(g, p, io, s);
    }
}

template <typename R>
cudaError_t launch_tsub(const Geom& g, const Phys<R>& p, const R* Tin, R* Tout, cudaStream_t s)
{
    if (g.d == 3) return launch_tsub3d<R>(g, p, Tin, Tout, s);
    dim3 blk(32, 8), grd((g.nx + 31) / 32, (g.ny + 7) / 8);
    if (g.stencil == LF_STENCIL_ISOTROPIC)
        k_tsub2d_iso<R><<<grd, blk, 0, s>>>(g, p, Tin, Tout);
    else
        k_tsub2d<R><<<grd, blk, 0, s>>>(g, p, Tin, Tout);
    return cudaGetLastError();
}

template cudaError_t launch_step2d<float>(const Geom&, const Phys<float>&, const StepIO<float>&, bool, cudaStream_t);
template cudaError_t launch_step2d<double>(const Geom&, const Phys<double>&, const StepIO<double>&, bool, cudaStream_t);
template cudaError_t launch_tsub<float>(const Geom&, const Phys<float>&, const float*, float*, cudaStream_t);
template cudaError_t launch_tsub<double>(const Geom&, const Phys<double>&, const double*, double*, cudaStream_t);

}  // namespace lf
