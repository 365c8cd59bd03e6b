// lf_step3d_common.cuh -- index maps and copy helpers shared by the passes of
// the three-pass D3Q19 step (lf_step3d_split.cu, lf_step3d_iso.cu).
#pragma once

#include "lf_internal.cuh"

namespace lf {
namespace {

__device__ __forceinline__ int wrap_s(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Storage plane of an unwrapped z (periodic, or mirrored about the half-way
// walls with period 2n); the division only for v outside [-n, 2n).
__device__ __forceinline__ int map_z(int v, int n, int walls)
{
    if (v >= 0 && v < n) return v;
    const int d = walls ? (v < 0 ? -1 - v : 2 * n - 1 - v) : (v < 0 ? v + n : v - n);
    if (d >= 0 && d < n) return d;
    if (!walls) return wrap_s(v, n);
    const int m = wrap_s(v, 2 * n);
    return m < n ? m : 2 * n - 1 - m;
}

template <typename R>
__device__ __forceinline__ R rcp_s(R x) { return R(1) / x; }
template <>
__device__ __forceinline__ float rcp_s<float>(float x) { return __frcp_rn(x); }

template <int B>
__device__ __forceinline__ void cp_async_s(void* dst, const void* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (B == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

}  // namespace
}  // namespace lf
