// lf_iso3.cuh -- the isotropic 19-point operators (D3Q19 weights) on three
// shared-memory planes, used by the fused plane march (lf_step3d.cu), and the
// same operators split by plane for the column marches of the three-pass step
// (lf_step3d_iso.cu), when the context's stencil is LF_STENCIL_ISOTROPIC:
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

namespace lf {
namespace {

// The same operators split by plane, for a column march along z that loads
// each plane's in-plane neighbours once.  For one plane of A around centre c
// (row length W):
//   s  = 2 A_c + (A_e + A_w + A_n + A_s)             its part in lap and d_z of the planes beside it,
//   l  = 2 (A_e + A_w + A_n + A_s) + (corners) - 24 A_c   its part in its own lap,
//   gx = 2 (A_e - A_w) + (A_ne - A_nw) + (A_se - A_sw),   ax = A_e - A_w,
//   gy = 2 (A_n - A_s) + (A_ne - A_se) + (A_nw - A_sw),   ay = A_n - A_s;
// then with the planes m - 1, m, m + 1:
//   lap A(m) = [l(m) + s(m - 1) + s(m + 1)] / 6,
//   d_x A(m) = [gx(m) + ax(m - 1) + ax(m + 1)] / 12   (d_y alike),
//   d_z A(m) = [s(m + 1) - s(m - 1)] / 12.
template <typename R>
struct Plane19 {
    R s, l, gx, gy, ax, ay;
};

template <typename R, int W>
__device__ __forceinline__ Plane19<R> plane19(const R* a, int c, R ac)
{
    const R e = a[c + 1], w = a[c - 1], n = a[c + W], so = a[c - W];
    const R ne = a[c + W + 1], nw = a[c + W - 1], se = a[c - W + 1], sw = a[c - W - 1];
    const R cross = (e + w) + (n + so);
    Plane19<R> r;
    r.s = R(2) * ac + cross;
    r.l = R(2) * cross + ((ne + nw) + (se + sw)) - R(24) * ac;
    r.ax = e - w;
    r.ay = n - so;
    r.gx = R(2) * r.ax + (ne - nw) + (se - sw);
    r.gy = R(2) * r.ay + (ne - se) + (nw - sw);
    return r;
}

// Sliding state of one field along the march: the sums of centre m that
// still lack plane m + 1, and the parts of plane m that the centre m + 1
// takes.  push(plane m + 1) completes centre m and moves on.
template <typename R>
struct Slide19 {
    R l = 0, gx = 0, gy = 0, s_prev = 0, s = 0, ax = 0, ay = 0;   // l/gx/gy of centre m, s(m - 1), s(m), ax(m), ay(m)
    __device__ __forceinline__ void push(const Plane19<R>& q, R& lap, R& dx, R& dy, R& dz)
    {
        lap = (l + q.s) * R(1.0 / 6.0);
        dx = (gx + q.ax) * R(1.0 / 12.0);
        dy = (gy + q.ay) * R(1.0 / 12.0);
        dz = (q.s - s_prev) * R(1.0 / 12.0);
        l = q.l + s;
        gx = q.gx + ax;
        gy = q.gy + ay;
        s_prev = s;
        s = q.s;
        ax = q.ax;
        ay = q.ay;
    }
};

}  // namespace
}  // namespace lf
