// lf_iso3.cuh -- the isotropic 19-point operators (D3Q19 weights) on three
// shared-memory planes, used by the fused plane march (lf_step3d.cu) and the
// three-pass step (lf_step3d_split.cu) when the context's stencil is
// LF_STENCIL_ISOTROPIC:
//   d_a A = 3 sum_i w_i e_ia A(r + e_i) = [2 (nearest difference) + (edge differences)] / 12,
//   lap A = 6 sum_i w_i [A(r + e_i) - A(r)] = [2 (6 nearest) + (12 edges) - 24 A] / 6.
#pragma once

namespace lf {
namespace {

// Isotropic 19-point operators on three planes (below, at, above) of a
// row-major region of row length W, centre c.
template <typename R, int W>
__device__ __forceinline__ R lap19(const R* dn, const R* md, const R* up, int c)
{
    const R nn = md[c - 1] + md[c + 1] + md[c - W] + md[c + W] + dn[c] + up[c];
    const R ed = (md[c - W - 1] + md[c - W + 1] + md[c + W - 1] + md[c + W + 1])
               + (dn[c - 1] + dn[c + 1] + dn[c - W] + dn[c + W])
               + (up[c - 1] + up[c + 1] + up[c - W] + up[c + W]);
    return (R(2) * nn + ed - R(24) * md[c]) * R(1.0 / 6.0);
}

template <typename R, int W>
__device__ __forceinline__ R grad19(const R* dn, const R* md, const R* up, int c, int axis)
{
    R v;
    if (axis == 0)
        v = R(2) * (md[c + 1] - md[c - 1]) + (md[c + W + 1] - md[c + W - 1]) + (md[c - W + 1] - md[c - W - 1])
          + (up[c + 1] - up[c - 1]) + (dn[c + 1] - dn[c - 1]);
    else if (axis == 1)
        v = R(2) * (md[c + W] - md[c - W]) + (md[c + W + 1] - md[c - W + 1]) + (md[c + W - 1] - md[c - W - 1])
          + (up[c + W] - up[c - W]) + (dn[c + W] - dn[c - W]);
    else
        v = R(2) * (up[c] - dn[c]) + (up[c + 1] - dn[c + 1]) + (up[c - 1] - dn[c - 1])
          + (up[c + W] - dn[c + W]) + (up[c - W] - dn[c - W]);
    return v * R(1.0 / 12.0);
}

}  // namespace
}  // namespace lf
