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

// Layout conversion between the padded state ([rows][pitch], deviations for
// the populations) and a packed caller array ([rows][nx]).  Work comes in
// chunks of 1024 elements of one row, four consecutive elements per thread;
// when every row of both arrays starts on a 16-byte boundary the four move
// as one vector access (fewer requests when the caller array is host memory
// reached through the device mapping), else as four scalar accesses issued
// before any store.
constexpr int kChunk = 1024;

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = double4_16a;
};

template <typename T>
__device__ __forceinline__ void load4(const T* p, int x, int nx, bool vec, T v[4])
{
    if (vec && x + 3 < nx) {
        const typename Vec4<T>::type w = *reinterpret_cast<const typename Vec4<T>::type*>(p + x);
        v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = x + u < nx ? p[x + u] : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void store4(T* p, int x, int nx, bool vec, const T v[4])
{
    if (vec && x + 3 < nx) {
        typename Vec4<T>::type w;
        w.x = v[0]; w.y = v[1]; w.z = v[2]; w.w = v[3];
        *reinterpret_cast<typename Vec4<T>::type*>(p + x) = w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (x + u < nx) p[x + u] = v[u];
    }
}

template <typename R, typename D>
__global__ void __launch_bounds__(256) k_pack(Geom g, const R* __restrict__ src, D* __restrict__ dst, int nplanes,
                                              PlaneAdd add, int vec)
{
    const int nx = g.nx;
    const int xch = (nx + kChunk - 1) / kChunk;
    const int64_t rows = (int64_t)g.ny * g.nz, per_plane = rows * xch;
    const int64_t N = rows * nx;
    for (int64_t c = blockIdx.x; c < per_plane * nplanes; c += gridDim.x) {
        const int q = (int)(c / per_plane);
        const int64_t cr = c - q * per_plane;
        const int64_t row = cr / xch;
        const int x = (int)(cr - row * xch) * kChunk + 4 * threadIdx.x;
        if (x >= nx) continue;
        R v[4];
        D o[4];
        load4(src + q * g.plane + row * g.pitch, x, nx, vec != 0, v);
        const double a = add.v[q];
#pragma unroll
        for (int u = 0; u < 4; ++u) o[u] = (D)((double)v[u] + a);
        store4(dst + q * N + row * nx, x, nx, vec != 0, o);
    }
}

template <typename R, typename D>
__global__ void __launch_bounds__(256) k_unpack(Geom g, const D* __restrict__ src, R* __restrict__ dst, int nplanes,
                                                PlaneAdd sub, int vec)
{
    const int nx = g.nx;
    const int xch = (nx + kChunk - 1) / kChunk;
    const int64_t rows = (int64_t)g.ny * g.nz, per_plane = rows * xch;
    const int64_t N = rows * nx;
    for (int64_t c = blockIdx.x; c < per_plane * nplanes; c += gridDim.x) {
        const int q = (int)(c / per_plane);
        const int64_t cr = c - q * per_plane;
        const int64_t row = cr / xch;
        const int x = (int)(cr - row * xch) * kChunk + 4 * threadIdx.x;
        if (x >= nx) continue;
        D v[4];
        R o[4];
        load4(src + q * N + row * nx, x, nx, vec != 0, v);
        const double b = sub.v[q];
#pragma unroll
        for (int u = 0; u < 4; ++u) o[u] = (R)((double)v[u] - b);
        store4(dst + q * g.plane + row * g.pitch, x, nx, vec != 0, o);
    }
}

// Vector accesses need every row and plane start of both arrays 16-byte
// aligned (a: the padded state in R, b: the packed array in D).
template <typename R, typename D>
int vec_ok(const Geom& g, const void* a, const void* b)
{
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    const bool rows = ((size_t)g.nx * sizeof(D)) % 16 == 0 && ((size_t)g.pitch * sizeof(R)) % 16 == 0 &&
                      ((size_t)N * sizeof(D)) % 16 == 0 && ((size_t)g.plane * sizeof(R)) % 16 == 0;
    return rows && ((uintptr_t)a % 16 == 0) && ((uintptr_t)b % 16 == 0);
}

inline unsigned grid_for(const Geom& g)
{
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    int64_t b = (N + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

inline unsigned grid_chunks(const Geom& g, int nplanes)
{
    const int64_t n = (int64_t)nplanes * g.ny * g.nz * ((g.nx + kChunk - 1) / kChunk);
    const int64_t cap = 152 * 8;
    return (unsigned)(n < 1 ? 1 : (n > cap ? cap : n));
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
cudaError_t launch_pack(const Geom& g, const R* src, D* dst, int nplanes, const PlaneAdd& add, cudaStream_t s)
{
    k_pack<R, D><<<grid_chunks(g, nplanes), 256, 0, s>>>(g, src, dst, nplanes, add, vec_ok<R, D>(g, src, dst));
    return cudaGetLastError();
}

template <typename R, typename D>
cudaError_t launch_unpack(const Geom& g, const D* src, R* dst, int nplanes, const PlaneAdd& sub, cudaStream_t s)
{
    k_unpack<R, D><<<grid_chunks(g, nplanes), 256, 0, s>>>(g, src, dst, nplanes, sub, vec_ok<R, D>(g, dst, src));
    return cudaGetLastError();
}

template cudaError_t launch_init<float>(const Geom&, uint64_t, double, double, double, int, float*, float*, cudaStream_t);
template cudaError_t launch_init<double>(const Geom&, uint64_t, double, double, double, int, double*, double*, cudaStream_t);
template cudaError_t launch_pack<float, float>(const Geom&, const float*, float*, int, const PlaneAdd&, cudaStream_t);
template cudaError_t launch_pack<float, double>(const Geom&, const float*, double*, int, const PlaneAdd&, cudaStream_t);
template cudaError_t launch_pack<double, float>(const Geom&, const double*, float*, int, const PlaneAdd&, cudaStream_t);
template cudaError_t launch_pack<double, double>(const Geom&, const double*, double*, int, const PlaneAdd&, cudaStream_t);
template cudaError_t launch_unpack<float, float>(const Geom&, const float*, float*, int, const PlaneAdd&, cudaStream_t);
template cudaError_t launch_unpack<float, double>(const Geom&, const double*, float*, int, const PlaneAdd&, cudaStream_t);
template cudaError_t launch_unpack<double, float>(const Geom&, const float*, double*, int, const PlaneAdd&, cudaStream_t);
template cudaError_t launch_unpack<double, double>(const Geom&, const double*, double*, int, const PlaneAdd&, cudaStream_t);

}  // namespace lf
