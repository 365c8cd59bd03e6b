// lf_util.cu -- initial state and layout conversion kernels.
#include "lf_internal.cuh"

namespace lf {

namespace {

// SplitMix64 (Steele, Lea & Flood 2014): the k-th output of the generator
// whose state starts at `seed`.  Counter-based, so every site draws its own
// value independently of the launch shape.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Initial state (arXiv:1102.3094 Sec. 3: disordered phi around zero, T above
// Tc with the walls at T_w).  phi = amp (2u - 1), u the top 53 bits of the
// generator output; the products are rounded explicitly so the FP64 value is
// the same on every compiler and machine.
template <typename R>
__global__ void k_init(Geom g, uint64_t seed, double amp, double T0, double T_w, int quench,
                       R* __restrict__ phi, R* __restrict__ T)
{
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    const int wall_len = (g.d == 2) ? g.ny : g.nz;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % g.nx);
        const int64_t row = k / g.nx;                   // y + ny z
        const int y = (int)(row % g.ny);
        const int z = (int)(row / g.ny);
        const int h = (g.d == 2) ? y : z;               // position along the wall axis
        const uint64_t r = splitmix64_at(seed, (uint64_t)k);
        const double u = (double)(r >> 11) * 0x1.0p-53;
        const double v = __dadd_rn(__dmul_rn(2.0, u), -1.0);
        const int64_t site = row * g.pitch + x;
        phi[site] = (R)__dmul_rn(amp, v);
        double t = T0;
        if (quench) t = T_w;
        else if (g.walls && g.t_mode == LF_TWALL_LAYERS && (h == 0 || h == wall_len - 1)) t = T_w;
        T[site] = (R)t;
    }
}

template <typename R, typename D>
__global__ void k_pack(Geom g, const R* __restrict__ src, D* __restrict__ dst, double add)
{
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = k / g.nx;
        const int x = (int)(k - row * g.nx);
        dst[k] = (D)((double)src[row * g.pitch + x] + add);
    }
}

template <typename R, typename D>
__global__ void k_unpack(Geom g, const D* __restrict__ src, R* __restrict__ dst, double sub)
{
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = k / g.nx;
        const int x = (int)(k - row * g.nx);
        dst[row * g.pitch + x] = (R)((double)src[k] - sub);
    }
}

inline unsigned grid_for(const Geom& g)
{
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    int64_t b = (N + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

template <typename R>
cudaError_t launch_init(const Geom& g, uint64_t seed, double amp, double T0, double T_w, int quench,
                        R* phi, R* T, cudaStream_t s)
{
    k_init<R><<<grid_for(g), 256, 0, s>>>(g, seed, amp, T0, T_w, quench, phi, T);
    return cudaGetLastError();
}

template <typename R, typename D>
cudaError_t launch_pack(const Geom& g, const R* src, D* dst, double add, cudaStream_t s)
{
    k_pack<R, D><<<grid_for(g), 256, 0, s>>>(g, src, dst, add);
    return cudaGetLastError();
}

template <typename R, typename D>
cudaError_t launch_unpack(const Geom& g, const D* src, R* dst, double sub, cudaStream_t s)
{
    k_unpack<R, D><<<grid_for(g), 256, 0, s>>>(g, src, dst, sub);
    return cudaGetLastError();
}

template cudaError_t launch_init<float>(const Geom&, uint64_t, double, double, double, int, float*, float*, cudaStream_t);
template cudaError_t launch_init<double>(const Geom&, uint64_t, double, double, double, int, double*, double*, cudaStream_t);
template cudaError_t launch_pack<float, float>(const Geom&, const float*, float*, double, cudaStream_t);
template cudaError_t launch_pack<float, double>(const Geom&, const float*, double*, double, cudaStream_t);
template cudaError_t launch_pack<double, float>(const Geom&, const double*, float*, double, cudaStream_t);
template cudaError_t launch_pack<double, double>(const Geom&, const double*, double*, double, cudaStream_t);
template cudaError_t launch_unpack<float, float>(const Geom&, const float*, float*, double, cudaStream_t);
template cudaError_t launch_unpack<float, double>(const Geom&, const double*, float*, double, cudaStream_t);
template cudaError_t launch_unpack<double, float>(const Geom&, const float*, double*, double, cudaStream_t);
template cudaError_t launch_unpack<double, double>(const Geom&, const double*, double*, double, cudaStream_t);

}  // namespace lf
