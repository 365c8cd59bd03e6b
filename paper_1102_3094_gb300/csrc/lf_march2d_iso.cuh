// lf_march2d_iso.cuh -- the row-marching D2Q9 step of lf_march2d.cuh with the
// isotropic 9-point stencils (LF_STENCIL_ISOTROPIC) for every derivative.
//
// Every 9-point operator is a sum over the rows m - 1, m, m + 1 of in-row
// stencils, and the part of one row can be formed as soon as that row is
// known.  With, for one row of A around column c,
//   s  = 4 A_c + A_e + A_w          (its part in lap and d_y of the rows beside it),
//   l  = 4 (A_e + A_w) - 20 A_c     (its part in its own lap),
//   ax = A_e - A_w,
// the D2Q9-weighted operators (lap = 6 sum w_i [A(r + e_i) - A(r)], d_a =
// 3 sum w_i e_ia A(r + e_i)) are
//   lap A(m) = [l(m) + s(m - 1) + s(m + 1)] / 6,
//   d_x A(m) = [4 ax(m) + ax(m - 1) + ax(m + 1)] / 12,
//   d_y A(m) = [s(m + 1) - s(m - 1)] / 12.
// A thread marching its column therefore loads the two in-row neighbours of
// each new row of a field once and keeps the open sums of its column in
// registers.  Since a row's neighbours are known only after the barrier that
// follows its computation, each stage runs two rows behind the one it reads
// from.  At iteration k (phi and T of row k have arrived, the populations of
// row k - 5 too), after one barrier:
//   phi, T of row k        -> psi, grad phi, lap T at k - 1; T(t+1) of row k - 1
//   psi of row k - 2       -> lam, grad psi at k - 3; mu, P_ab of row k - 3
//   P_ab of row k - 4      -> F at k - 5; n, u, g = phi u; collide and push row k - 5
//   mu of row k - 4        -> lap mu at k - 5 (kept two iterations)
//   g of row k - 6         -> div g at k - 7; phi(t+1) of row k - 7
// Each stage writes the ring slot of its row's parity and reads the other, so
// one barrier per row orders everything; the march runs H + 11 iterations.
//
// Rows beyond a wall: phi and T arrive as the mirror image (even reflection
// about the half-way plane), so psi, lam, mu and P there are computed from it
// as in the compact march.  The flux g is not computed beyond a wall: its
// image row enters the sums as the parts of the wall row transformed (g_x
// even: unchanged; g_y odd: s -> -s), and with halfway temperature ghosts the
// T row beyond a wall enters as 2 T_w minus the wall row (s -> 12 T_w - s).
#pragma once

#include "lf_march2d.cuh"
#include "lf_march2d_x2.cuh"      // packed FP32x2 helpers, pair_rows

namespace lf {
namespace march {

template <typename R, int NT, int D>
struct MarchIso {
    static constexpr int U = NT - 8;          // columns written per CTA
    static constexpr int SIN = D + 1;         // phi / T rows in flight or in use
    static constexpr int SF = D + 1;          // population rows in flight or in use
    static constexpr int PHI = 0;
    static constexpr int TT = PHI + SIN * NT;
    static constexpr int F = TT + SIN * NT;
    static constexpr int PSI = F + SF * 9 * NT;
    static constexpr int MU = PSI + 2 * NT;
    static constexpr int PXX = MU + 2 * NT;
    static constexpr int PXY = PXX + 2 * NT;
    static constexpr int PYY = PXY + 2 * NT;
    static constexpr int GX = PYY + 2 * NT;
    static constexpr int GY = GX + 2 * NT;
    static constexpr int TOTAL = GY + 2 * NT;
    static constexpr size_t BYTES = sizeof(R) * TOTAL;
};

// Parts of one row (see above) and the open sums of one column.
template <typename R>
struct Row9 {
    R s, l, ax;
};

template <typename R>
__device__ __forceinline__ Row9<R> row9(R w, R c, R e)
{
    Row9<R> q;
    q.s = R(4) * c + (e + w);
    q.l = R(4) * (e + w) - R(20) * c;
    q.ax = e - w;
    return q;
}

template <typename R>
struct Slide9 {
    R l = 0, gx = 0, s_prev = 0, s = 0, ax = 0;   // l, 4 ax of centre m with row m - 1's parts; s(m - 1), s(m), ax(m)
    // row m + 1 arrives: the operators at m, then move to centre m + 1
    __device__ __forceinline__ void push(const Row9<R>& q, R& lap, R& dx, R& dy)
    {
        lap = (l + q.s) * R(1.0 / 6.0);
        dx = (gx + q.ax) * R(1.0 / 12.0);
        dy = (q.s - s_prev) * R(1.0 / 12.0);
        l = q.l + s;
        gx = R(4) * q.ax + ax;
        s_prev = s;
        s = q.s;
        ax = q.ax;
    }
    // the row before the next one pushed is an image with parts (s, ax)
    __device__ __forceinline__ void set_last(R s_img, R ax_img)
    {
        s = s_img;
        ax = ax_img;
    }
};

template <typename R, int NT, int D>
__device__ __forceinline__ void march2d_segment_iso(const Geom& g, const Phys<R>& p, const StepIO<R>& io, int strip,
                                                    int seg, int H, unsigned char* smem_raw)
{
    using L = D2Q9;
    using M = MarchIso<R, NT, D>;
    static_assert(M::SF == 4, "population ring indexed with & 3");
    R* sm = reinterpret_cast<R*>(smem_raw);
    R* sphi = sm + M::PHI;
    R* sT = sm + M::TT;
    R* sf = sm + M::F;
    R* spsi = sm + M::PSI;
    R* smu = sm + M::MU;
    R* sPxx = sm + M::PXX;
    R* sPxy = sm + M::PXY;
    R* sPyy = sm + M::PYY;
    R* sgx = sm + M::GX;
    R* sgy = sm + M::GY;

    const int t = threadIdx.x;
    const int nx = g.nx, ny = g.ny, pitch = g.pitch, walls = g.walls;
    const int plane = (int)g.plane;                 // Q * plane < 2^31 (checked at creation)
    const int x0 = strip * M::U;
    const int y0 = seg * H;
    const int y1 = min(y0 + H, ny);
    const int cx = x0 - 4 + t;                      // unwrapped column of this thread
    const int gx = wrap_any(cx, nx);
    const int gxm = wrap_any(cx - 1, nx), gxp = wrap_any(cx + 1, nx);
    const bool own = t >= 4 && t < NT - 4 && cx < nx;
    const bool r3 = t >= 1 && t < NT - 1;           // columns of psi and grad phi
    const bool r2 = t >= 2 && t < NT - 2;           // columns of lam, mu, P
    const bool has_u = t >= 3 && t < NT - 3;        // columns of F, u, g
    const R half = R(0.5);
    const R omega = p.inv_tau, keep = R(1) - p.inv_tau;
    const bool t_half = walls && g.t_mode == LF_TWALL_HALFWAY;
    const bool t_lay = walls && g.t_mode == LF_TWALL_LAYERS;
    const int kbeg = y0 - 4, kphi = y1 + 3, kend = y1 + 6;   // phi / T rows kbeg .. kphi

    Slide9<R> sl_phi, sl_T, sl_psi, sl_mu, sl_gx, sl_gy;
    R ph1 = 0, ph2 = 0, ph3 = 0, ph4 = 0, ph5 = 0, ph6 = 0, ph7 = 0;   // own phi(k-1) .. phi(k-7)
    R T1 = 0, T2 = 0, T3 = 0;                       // own T(k-1) .. T(k-3)
    R ps1 = 0, ps2 = 0;                             // own psi(k-2), psi(k-3)
    R dx1 = 0, dy1 = 0, dx2 = 0, dy2 = 0;           // grad phi(k-2), grad phi(k-3)
    R mu1 = 0;                                      // own mu(k-4)
    R pxy1 = 0, pyy1 = 0;                           // own P_xy, P_yy of row k-4
    R gy1 = 0;                                      // own g_y of row k-6
    R lm1 = 0, lm2 = 0;                             // lap mu(k-6), lap mu(k-7)
    R aFx = 0, aFy = 0, bFx = 0, bFy = 0;           // -12 F: open sums of centre k-5, parts of row k-5
    R probe = 0;              // sum of the outputs: NaN / Inf anywhere make it non-finite

    int s_issue = 0;                                 // slot of the next phi / T row to fetch
    auto issue = [&](int j) {
        const int r = j + D;                         // phi / T row
        if (r <= kphi) {
            const int off = map_row(r, ny, walls) * pitch + gx;
            cp_async<sizeof(R)>(&sphi[s_issue * NT + t], io.phi_in + off);
            cp_async<sizeof(R)>(&sT[s_issue * NT + t], io.T_in + off);
        }
        s_issue = (s_issue + 1 == M::SIN) ? 0 : s_issue + 1;
        const int rf = j + D - 5;                    // population row
        if (p.hydro && has_u && rf >= y0 - 1 && rf <= y1 && !(walls && (rf < 0 || rf >= ny))) {
            const int grf = walls ? rf : map_row(rf, ny, 0);
            const R* src = io.f_in + (grf * pitch + gx);
            R* dst = sf + ((rf - kbeg) & 3) * L::Q * NT + t;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) cp_async<sizeof(R)>(dst + i * NT, src + i * plane);
        }
        cp_commit();
    };

    for (int j = kbeg - D; j < kbeg; ++j) issue(j);

    int sk = 0;
#pragma unroll 1
    for (int k = kbeg; k <= kend; ++k) {
        cp_wait<D - 1>();
        __syncthreads();
        issue(k);
        const int par = (k - kbeg) & 1;              // ring parity of rows k, k - 2, k - 4, k - 6

        // ---- phi, T of row k: psi, grad phi, T(t+1) at k - 1 -----------------------
        R phk = 0, psk = 0, dxk = 0, dyk = 0, Tk = 0;
        if (k <= kphi) {
            phk = sphi[sk * NT + t];
            Tk = sT[sk * NT + t];
            if (r3) {
                sl_phi.push(row9(sphi[sk * NT + t - 1], phk, sphi[sk * NT + t + 1]), psk, dxk, dyk);
                spsi[(par ^ 1) * NT + t] = psk;      // psi(k - 1)
            }
            if (own) {
                Row9<R> qT = row9(sT[sk * NT + t - 1], Tk, sT[sk * NT + t + 1]);
                if (t_half && k == 0) sl_T.set_last(R(12) * p.T_w - qT.s, R(0));
                if (t_half && k == ny) qT.s = R(12) * p.T_w - sl_T.s;
                R lapT, u0, u1;
                sl_T.push(qT, lapT, u0, u1);
                const int m = k - 1;
                if (m >= y0 && m < y1) {
                    R Tn = T1;
                    if (p.t_update) Tn = (t_lay && (m == 0 || m == ny - 1)) ? p.T_w : T1 + p.dxi * lapT;
                    probe += Tn;
                    io.T_out[m * pitch + gx] = Tn;
                }
            }
        }

        // ---- psi of row k - 2: lam, grad psi, mu, P of row k - 3 --------------------
        R muk = 0, pxyk = 0, pyyk = 0;
        if (r2 && k >= y0 - 1 && k <= y1 + 4) {
            R lam, dsx, dsy;
            sl_psi.push(row9(spsi[par * NT + t - 1], ps1, spsi[par * NT + t + 1]), lam, dsx, dsy);
            if (k >= y0 + 1) {
                const R ph = ph3, ps = ps2;
                const R av = (T3 - p.Tc) * p.inv_Tc;
                muk = av * ph + p.b * ph * ph * ph - p.kappa * ps + p.c * lam;
                smu[(par ^ 1) * NT + t] = muk;
                if (p.hydro) {
                    const R dpx = dx2, dpy = dy2;
                    const R ph2 = ph * ph;
                    const R iso = av * ph2 * half + R(0.75) * p.b * ph2 * ph2
                                - p.kappa * (ph * ps + half * (dpx * dpx + dpy * dpy))
                                + p.c * (ph * lam + half * ps * ps + dpx * dsx + dpy * dsy);
                    pxyk = p.kappa * dpx * dpy - p.c * (dpx * dsy + dpy * dsx);
                    pyyk = iso + p.kappa * dpy * dpy - R(2) * p.c * dpy * dsy;
                    sPxx[(par ^ 1) * NT + t] = iso + p.kappa * dpx * dpx - R(2) * p.c * dpx * dsx;
                    sPxy[(par ^ 1) * NT + t] = pxyk;
                    sPyy[(par ^ 1) * NT + t] = pyyk;
                }
            }
        }

        // ---- P of row k - 4: F at k - 5; n, u, g; collide and push row k - 5 ---------
        R gyk = 0;
        if (p.hydro && has_u && k >= y0 + 2 && k <= y1 + 5) {
            const int q = par * NT + t;
            const R axx = sPxx[q + 1] - sPxx[q - 1];
            const R axy = sPxy[q + 1] - sPxy[q - 1];
            const R sxy = R(4) * pxy1 + (sPxy[q + 1] + sPxy[q - 1]);
            const R syy = R(4) * pyy1 + (sPyy[q + 1] + sPyy[q - 1]);
            // -12 F(m) = O(m) + [A(m - 1) - S(m - 1)] + [A(m + 1) + S(m + 1)]:
            // O = 4 ax(P_xa), A = ax(P_xa), S = s(P_ya)
            const R Fx = -(aFx + (axx + sxy)) * R(1.0 / 12.0);
            const R Fy = -(aFy + (axy + syy)) * R(1.0 / 12.0);
            aFx = R(4) * axx + bFx;
            aFy = R(4) * axy + bFy;
            bFx = axx - sxy;
            bFy = axy - syy;
            const int m = k - 5;
            R gxv = 0;
            if (k >= y0 + 4 && !(walls && (m < 0 || m >= ny))) {
                const R* fr = sf + ((m - kbeg) & 3) * L::Q * NT + t;
                R df[L::Q];
#pragma unroll
                for (int i = 0; i < L::Q; ++i) df[i] = fr[i * NT];
                const R dn = ((df[0] + df[1]) + (df[2] + df[3])) + ((df[4] + df[5]) + (df[6] + df[7])) + df[8];
                const R jx = (df[1] - df[3]) + (df[5] - df[6]) + (df[8] - df[7]);
                const R jy = (df[2] - df[4]) + (df[5] - df[8]) + (df[6] - df[7]);
                const R n = p.n0 + dn;
                const R inv_n = recip(n);
                const R vx = (jx + half * Fx) * inv_n, vy = (jy + half * Fy) * inv_n;
                gxv = ph5 * vx;
                gyk = ph5 * vy;
                if (own && m >= y0 && m < y1) {
                    probe += n;
                    const R on = omega * n;
                    const R C0 = omega * dn - R(1.5) * on * (vx * vx + vy * vy) - R(3) * p.guo * (vx * Fx + vy * Fy);
                    const R a3 = R(3) * on, a45 = R(4.5) * on, g3 = R(3) * p.guo, g9 = R(9) * p.guo;
                    const int site = m * pitch + gx;
                    const int up = ((m + 1 == ny) ? 0 : m + 1) * pitch;
                    const int dn_ = ((m == 0) ? ny - 1 : m - 1) * pitch;
                    const int mid = m * pitch;
                    const bool wall_lo = walls && m == 0, wall_hi = walls && m == ny - 1;
                    R* out = io.f_out;
                    out[site] = keep * df[0] + R(L::w(0)) * C0;
                    auto pair = [&](int i, int j, R s, R e, int off_i, int off_j, bool bb_i, bool bb_j) {
                        const R sym = C0 + s * (a45 * s + g9 * e);
                        const R anti = a3 * s + g3 * e;
                        const R wi = R(L::w(i));
                        const R pi = keep * df[i] + wi * (sym + anti);
                        const R pj = keep * df[j] + wi * (sym - anti);
                        // bounce-back: a population leaving through a wall returns reversed
                        if (bb_i) out[j * plane + site] = pi; else out[i * plane + off_i] = pi;
                        if (bb_j) out[i * plane + site] = pj; else out[j * plane + off_j] = pj;
                    };
                    pair(1, 3, vx, Fx, mid + gxp, mid + gxm, false, false);
                    pair(2, 4, vy, Fy, up + gx, dn_ + gx, wall_hi, wall_lo);
                    pair(5, 7, vx + vy, Fx + Fy, up + gxp, dn_ + gxm, wall_hi, wall_lo);
                    pair(6, 8, vy - vx, Fy - Fx, up + gxm, dn_ + gxp, wall_hi, wall_lo);
                }
            }
            sgx[(par ^ 1) * NT + t] = gxv;           // g of row k - 5 (zero beyond a wall)
            sgy[(par ^ 1) * NT + t] = gyk;
        }

        // ---- mu of row k - 4, g of row k - 6: phi(t+1) of row k - 7 -------------------
        R lmk = 0;
        if (own && k >= y0 + 3 && k <= y1 + 6) {
            R u0, u1;
            if (k <= y1 + 4) sl_mu.push(row9(smu[par * NT + t - 1], mu1, smu[par * NT + t + 1]), lmk, u0, u1);
            if (p.hydro && k >= y0 + 5) {
                const int r = k - 6;                 // the g row pushed now
                const int q = par * NT + t;
                Row9<R> qx = row9(sgx[q - 1], R(0), sgx[q + 1]);
                Row9<R> qy = row9(sgy[q - 1], gy1, sgy[q + 1]);
                if (walls && r == 0) {               // the row below is the wall row's image
                    sl_gx.set_last(R(0), qx.ax);
                    sl_gy.set_last(-qy.s, R(0));
                }
                if (walls && r == ny) {              // the row above is the image of row ny - 1
                    qx.ax = sl_gx.ax;
                    qy.s = -sl_gy.s;
                }
                R dgx, dgy;
                sl_gx.push(qx, u0, dgx, u1);
                sl_gy.push(qy, u0, u1, dgy);
                const int m = k - 7;
                if (m >= y0 && m < y1) {
                    const R phn = ph7 - (dgx + dgy) + p.Gamma * lm2;
                    probe += phn;
                    io.phi_out[m * pitch + gx] = phn;
                }
            } else if (!p.hydro && k >= y0 + 7) {
                const int m = k - 7;
                if (m < y1) {
                    const R phn = ph7 + p.Gamma * lm2;
                    probe += phn;
                    io.phi_out[m * pitch + gx] = phn;
                }
            }
        }

        // ---- shift the windows ---------------------------------------------------------
        ph7 = ph6; ph6 = ph5; ph5 = ph4; ph4 = ph3; ph3 = ph2; ph2 = ph1; ph1 = phk;
        T3 = T2; T2 = T1; T1 = Tk;
        ps2 = ps1; ps1 = psk;
        dx2 = dx1; dy2 = dy1; dx1 = dxk; dy1 = dyk;
        mu1 = muk;
        pxy1 = pxyk; pyy1 = pyyk;
        gy1 = gyk;
        lm2 = lm1; lm1 = lmk;
        sk = (sk + 1 == M::SIN) ? 0 : sk + 1;
    }
    cp_wait<0>();
    if (__any_sync(0xffffffffu, !isfinite(probe)) && (t & 31) == 0) *reinterpret_cast<volatile int*>(io.flag) = 1;
}

}  // namespace march
}  // namespace lf

// ===========================================================================
// The same march on two segments of a strip at once (FP32): lane .x covers
// the rows [ya, ya + ha), lane .y the rows [yb, yb + hb) just above them
// (the two halves of a pair of segments, as pair_rows splits them), both
// marching upwards in lockstep with their own halo rows, every field in the
// lanes of float2 values and the arithmetic on packed FP32x2 instructions.
// The wall rules and the output ranges are applied per lane.
// ===========================================================================
namespace lf {
namespace march {

template <int NT, int D>
struct MarchIso2 {
    static constexpr int U = NT - 8;
    static constexpr int SIN = D + 1;
    static constexpr int SF = D + 1;
    static constexpr int PHI = 0;
    static constexpr int TT = PHI + SIN * NT;
    static constexpr int F = TT + SIN * NT;
    static constexpr int PSI = F + SF * 9 * NT;
    static constexpr int MU = PSI + 2 * NT;
    static constexpr int PXX = MU + 2 * NT;
    static constexpr int PXY = PXX + 2 * NT;
    static constexpr int PYY = PXY + 2 * NT;
    static constexpr int GX = PYY + 2 * NT;
    static constexpr int GY = GX + 2 * NT;
    static constexpr int TOTAL = GY + 2 * NT;          // float2 elements
    static constexpr size_t BYTES = sizeof(float2) * TOTAL;
};

struct Row9x2 {
    float2 s, l, ax;
};

__device__ __forceinline__ Row9x2 row9x2(float2 w, float2 c, float2 e)
{
    const float2 ew = add2(e, w);
    Row9x2 q;
    q.s = fma2(v2(4.f), c, ew);
    q.l = fma2(v2(-20.f), c, mul2(v2(4.f), ew));
    q.ax = sub2(e, w);
    return q;
}

struct Slide9x2 {
    float2 l = v2(0.f), gx = v2(0.f), s_prev = v2(0.f), s = v2(0.f), ax = v2(0.f);
    __device__ __forceinline__ void push(const Row9x2& q, float2& lap, float2& dx, float2& dy)
    {
        lap = mul2(add2(l, q.s), v2(1.f / 6.f));
        dx = mul2(add2(gx, q.ax), v2(1.f / 12.f));
        dy = mul2(sub2(q.s, s_prev), v2(1.f / 12.f));
        l = add2(q.l, s);
        gx = fma2(v2(4.f), q.ax, ax);
        s_prev = s;
        s = q.s;
        ax = q.ax;
    }
};

template <int NT, int D, bool HYDRO>
__device__ __forceinline__ void march2d_pair_iso(const Geom& g, const Phys<float>& p, const StepIO<float>& io,
                                                 int strip, int pair, int npairs, unsigned char* smem_raw)
{
    using L = D2Q9;
    using M = MarchIso2<NT, D>;
    static_assert(M::SF == 4, "population ring indexed with & 3");
    float2* sm = reinterpret_cast<float2*>(smem_raw);
    float2* sphi = sm + M::PHI;
    float2* sT = sm + M::TT;
    float2* sf = sm + M::F;
    float2* spsi = sm + M::PSI;
    float2* smu = sm + M::MU;
    float2* sPxx = sm + M::PXX;
    float2* sPxy = sm + M::PXY;
    float2* sPyy = sm + M::PYY;
    float2* sgx = sm + M::GX;
    float2* sgy = sm + M::GY;

    const int t = threadIdx.x;
    const int nx = g.nx, ny = g.ny, pitch = g.pitch, walls = g.walls;
    const int plane = (int)g.plane;
    const int x0 = strip * M::U;
    int mid, ha, hb;
    pair_rows(ny, npairs, pair, mid, ha, hb);      // rows [mid - ha, mid) and [mid, mid + hb)
    const int ya = mid - ha, yb = mid;             // first row of lane .x / .y
    const int hmax = ha > hb ? ha : hb;
    const int cx = x0 - 4 + t;
    const int gx = wrap_any(cx, nx);
    const int gxm = wrap_any(cx - 1, nx), gxp = wrap_any(cx + 1, nx);
    const bool own = t >= 4 && t < NT - 4 && cx < nx;
    const bool r3 = t >= 1 && t < NT - 1;
    const bool r2 = t >= 2 && t < NT - 2;
    const bool has_u = t >= 3 && t < NT - 3;
    const float2 half = v2(0.5f);
    const float omega = p.inv_tau, keep = 1.f - p.inv_tau;
    const bool t_half = walls && g.t_mode == LF_TWALL_HALFWAY;
    const bool t_lay = walls && g.t_mode == LF_TWALL_LAYERS;
    const int jphi = hmax + 3, jend = hmax + 6;   // relative rows j of both lanes: row ya + j / yb + j

    Slide9x2 sl_phi, sl_T, sl_psi, sl_mu, sl_gx, sl_gy;
    float2 ph1 = v2(0.f), ph2 = v2(0.f), ph3 = v2(0.f), ph4 = v2(0.f), ph5 = v2(0.f), ph6 = v2(0.f), ph7 = v2(0.f);
    float2 T1 = v2(0.f), T2 = v2(0.f), T3 = v2(0.f);
    float2 ps1 = v2(0.f), ps2 = v2(0.f);
    float2 dx1 = v2(0.f), dy1 = v2(0.f), dx2 = v2(0.f), dy2 = v2(0.f);
    float2 mu1 = v2(0.f), pxy1 = v2(0.f), pyy1 = v2(0.f), gy1 = v2(0.f);
    float2 lm1 = v2(0.f), lm2 = v2(0.f);
    float2 aFx = v2(0.f), aFy = v2(0.f), bFx = v2(0.f), bFy = v2(0.f);
    float probe = 0.f;

    int s_issue = 0;
    auto issue = [&](int jj) {
        const int q = jj + D;                        // phi / T row
        if (q <= jphi) {
            const int oa = map_row(ya + q, ny, walls) * pitch + gx, ob = map_row(yb + q, ny, walls) * pitch + gx;
            float* d = reinterpret_cast<float*>(&sphi[s_issue * NT + t]);
            float* e = reinterpret_cast<float*>(&sT[s_issue * NT + t]);
            cp_async<4>(d, io.phi_in + oa);
            cp_async<4>(d + 1, io.phi_in + ob);
            cp_async<4>(e, io.T_in + oa);
            cp_async<4>(e + 1, io.T_in + ob);
        }
        s_issue = (s_issue + 1 == M::SIN) ? 0 : s_issue + 1;
        const int qf = jj + D - 5;                   // population row
        if (HYDRO && has_u && qf >= -1 && qf <= hmax) {
            float* dst = reinterpret_cast<float*>(sf + ((qf + 4) & 3) * L::Q * NT + t);
            const int ra = ya + qf, rb = yb + qf;
            if (qf <= ha && !(walls && (ra < 0 || ra >= ny))) {
                const float* src = io.f_in + ((walls ? ra : map_row(ra, ny, 0)) * pitch + gx);
#pragma unroll
                for (int i = 0; i < L::Q; ++i) cp_async<4>(dst + 2 * i * NT, src + i * plane);
            }
            if (qf <= hb && !(walls && (rb < 0 || rb >= ny))) {
                const float* src = io.f_in + ((walls ? rb : map_row(rb, ny, 0)) * pitch + gx);
#pragma unroll
                for (int i = 0; i < L::Q; ++i) cp_async<4>(dst + 2 * i * NT + 1, src + i * plane);
            }
        }
        cp_commit();
    };

    for (int jj = -4 - D; jj < -4; ++jj) issue(jj);

    int sk = 0;
#pragma unroll 1
    for (int j = -4; j <= jend; ++j) {
        cp_wait<D - 1>();
        __syncthreads();
        issue(j);
        const int par = (j + 4) & 1;

        // ---- phi, T of row j: psi, grad phi, T(t+1) at j - 1 -------------------------
        float2 phk = v2(0.f), psk = v2(0.f), dxk = v2(0.f), dyk = v2(0.f), Tk = v2(0.f);
        if (j <= jphi) {
            phk = sphi[sk * NT + t];
            Tk = sT[sk * NT + t];
            if (r3) {
                sl_phi.push(row9x2(sphi[sk * NT + t - 1], phk, sphi[sk * NT + t + 1]), psk, dxk, dyk);
                spsi[(par ^ 1) * NT + t] = psk;
            }
            if (own) {
                Row9x2 qT = row9x2(sT[sk * NT + t - 1], Tk, sT[sk * NT + t + 1]);
                if (t_half) {
                    const float tw12 = 12.f * p.T_w;
                    if (ya + j == 0) sl_T.s.x = tw12 - qT.s.x;      // the row below is the halfway ghost
                    if (yb + j == 0) sl_T.s.y = tw12 - qT.s.y;
                    if (ya + j == ny) qT.s.x = tw12 - sl_T.s.x;     // the row above is the halfway ghost
                    if (yb + j == ny) qT.s.y = tw12 - sl_T.s.y;
                }
                float2 lapT, u0, u1;
                sl_T.push(qT, lapT, u0, u1);
                const int m = j - 1;
                float2 Tn = T1;
                if (p.t_update) {
                    Tn = fma2(v2(p.dxi), lapT, T1);
                    if (t_lay && (ya + m == 0 || ya + m == ny - 1)) Tn.x = p.T_w;
                    if (t_lay && (yb + m == 0 || yb + m == ny - 1)) Tn.y = p.T_w;
                }
                if (m >= 0 && m < ha) { probe += Tn.x; io.T_out[(ya + m) * pitch + gx] = Tn.x; }
                if (m >= 0 && m < hb) { probe += Tn.y; io.T_out[(yb + m) * pitch + gx] = Tn.y; }
            }
        }

        // ---- psi of row j - 2: lam, grad psi, mu, P of row j - 3 ---------------------
        float2 muk = v2(0.f), pxyk = v2(0.f), pyyk = v2(0.f);
        if (r2 && j >= -1 && j <= hmax + 4) {
            float2 lam, dsx, dsy;
            sl_psi.push(row9x2(spsi[par * NT + t - 1], ps1, spsi[par * NT + t + 1]), lam, dsx, dsy);
            if (j >= 1) {
                const float2 ph = ph3, ps = ps2;
                const float2 av = mul2(sub2(T3, v2(p.Tc)), v2(p.inv_Tc));
                const float2 phsq = mul2(ph, ph);
                muk = fma2(v2(p.c), lam, fma2(v2(-p.kappa), ps, mul2(ph, fma2(v2(p.b), phsq, av))));
                smu[(par ^ 1) * NT + t] = muk;
                if constexpr (HYDRO) {
                    const float2 dpx = dx2, dpy = dy2;
                    const float2 gp2 = fma2(dpx, dpx, mul2(dpy, dpy));
                    const float2 gpgs = fma2(dpx, dsx, mul2(dpy, dsy));
                    float2 iso = mul2(phsq, fma2(v2(0.75f * p.b), phsq, mul2(half, av)));
                    iso = fma2(v2(-p.kappa), fma2(half, gp2, mul2(ph, ps)), iso);
                    iso = fma2(v2(p.c), add2(fma2(ph, lam, mul2(half, mul2(ps, ps))), gpgs), iso);
                    const float2 c2 = v2(-2.f * p.c);
                    pxyk = fma2(v2(p.kappa), mul2(dpx, dpy), mul2(v2(-p.c), fma2(dpx, dsy, mul2(dpy, dsx))));
                    pyyk = fma2(v2(p.kappa), mul2(dpy, dpy), fma2(c2, mul2(dpy, dsy), iso));
                    sPxx[(par ^ 1) * NT + t] = fma2(v2(p.kappa), mul2(dpx, dpx), fma2(c2, mul2(dpx, dsx), iso));
                    sPxy[(par ^ 1) * NT + t] = pxyk;
                    sPyy[(par ^ 1) * NT + t] = pyyk;
                }
            }
        }

        // ---- P of row j - 4: F at j - 5; n, u, g; collide and push row j - 5 -----------
        float2 gyk = v2(0.f);
        if (HYDRO && has_u && j >= 2 && j <= hmax + 5) {
            const int q = par * NT + t;
            const float2 axx = sub2(sPxx[q + 1], sPxx[q - 1]);
            const float2 axy = sub2(sPxy[q + 1], sPxy[q - 1]);
            const float2 sxy = fma2(v2(4.f), pxy1, add2(sPxy[q + 1], sPxy[q - 1]));
            const float2 syy = fma2(v2(4.f), pyy1, add2(sPyy[q + 1], sPyy[q - 1]));
            const float2 m12 = v2(-1.f / 12.f);
            const float2 Fx = mul2(add2(aFx, add2(axx, sxy)), m12);
            const float2 Fy = mul2(add2(aFy, add2(axy, syy)), m12);
            aFx = fma2(v2(4.f), axx, bFx);
            aFy = fma2(v2(4.f), axy, bFy);
            bFx = sub2(axx, sxy);
            bFy = sub2(axy, syy);
            const int m = j - 5;
            float2 gxv = v2(0.f);
            if (j >= 4) {
                const int ma = ya + m, mb = yb + m;
                const bool gha = walls && (ma < 0 || ma >= ny), ghb = walls && (mb < 0 || mb >= ny);
                const float2* fr = sf + ((m + 4) & 3) * L::Q * NT + t;
                float2 df[L::Q];
#pragma unroll
                for (int i = 0; i < L::Q; ++i) {
                    df[i] = fr[i * NT];
                    if (gha) df[i].x = 0.f;
                    if (ghb) df[i].y = 0.f;
                }
                const float2 dn = add2(add2(add2(df[0], df[1]), add2(df[2], df[3])),
                                       add2(add2(df[4], df[5]), add2(add2(df[6], df[7]), df[8])));
                const float2 jx = add2(add2(sub2(df[1], df[3]), sub2(df[5], df[6])), sub2(df[8], df[7]));
                const float2 jy = add2(add2(sub2(df[2], df[4]), sub2(df[5], df[8])), sub2(df[6], df[7]));
                const float2 n = add2(v2(p.n0), dn);
                const float2 inv_n = make_float2(__frcp_rn(n.x), __frcp_rn(n.y));
                const float2 vx = mul2(fma2(half, Fx, jx), inv_n), vy = mul2(fma2(half, Fy, jy), inv_n);
                gxv = mul2(ph5, vx);
                gyk = mul2(ph5, vy);
                if (gha) { gxv.x = 0.f; gyk.x = 0.f; }
                if (ghb) { gxv.y = 0.f; gyk.y = 0.f; }
                const bool col_a = own && m >= 0 && m < ha, col_b = own && m >= 0 && m < hb;
                if (col_a || col_b) {
                    const float2 on = mul2(v2(omega), n);
                    const float2 uu = fma2(vx, vx, mul2(vy, vy));
                    const float2 uF = fma2(vx, Fx, mul2(vy, Fy));
                    const float2 C0 = fma2(v2(-3.f * p.guo), uF, fma2(mul2(v2(-1.5f), on), uu, mul2(v2(omega), dn)));
                    const float2 a3 = mul2(v2(3.f), on), a45 = mul2(v2(4.5f), on);
                    const float2 g3 = v2(3.f * p.guo), g9 = v2(9.f * p.guo);
                    const float2 kp = v2(keep);
                    float2 post[L::Q];
                    post[0] = fma2(kp, df[0], mul2(v2((float)L::w(0)), C0));
                    auto pair_ = [&](int i, int jq, float2 sv, float2 ev) {
                        const float2 sym = fma2(sv, fma2(a45, sv, mul2(g9, ev)), C0);
                        const float2 anti = fma2(a3, sv, mul2(g3, ev));
                        const float2 wi = v2((float)L::w(i));
                        post[i] = fma2(kp, df[i], mul2(wi, add2(sym, anti)));
                        post[jq] = fma2(kp, df[jq], mul2(wi, sub2(sym, anti)));
                    };
                    pair_(1, 3, vx, Fx);
                    pair_(2, 4, vy, Fy);
                    pair_(5, 7, add2(vx, vy), add2(Fx, Fy));
                    pair_(6, 8, sub2(vy, vx), sub2(Fy, Fx));
                    float* out = io.f_out;
                    auto push = [&](auto lane_tag, int r) {
                        constexpr int LN = decltype(lane_tag)::value;
                        auto pv = [&](int i) { return LN == 0 ? post[i].x : post[i].y; };
                        probe += LN == 0 ? n.x : n.y;
                        const int site = r * pitch + gx;
                        const int up = ((r + 1 == ny) ? 0 : r + 1) * pitch;
                        const int dn_ = ((r == 0) ? ny - 1 : r - 1) * pitch;
                        const int mid_ = r * pitch;
                        const bool wall_lo = walls && r == 0, wall_hi = walls && r == ny - 1;
                        out[site] = pv(0);
                        auto st = [&](int i, int jq, int off_i, int off_j, bool bb_i, bool bb_j) {
                            if (bb_i) out[jq * plane + site] = pv(i); else out[i * plane + off_i] = pv(i);
                            if (bb_j) out[i * plane + site] = pv(jq); else out[jq * plane + off_j] = pv(jq);
                        };
                        st(1, 3, mid_ + gxp, mid_ + gxm, false, false);
                        st(2, 4, up + gx, dn_ + gx, wall_hi, wall_lo);
                        st(5, 7, up + gxp, dn_ + gxm, wall_hi, wall_lo);
                        st(6, 8, up + gxm, dn_ + gxp, wall_hi, wall_lo);
                    };
                    if (col_a) push(std::integral_constant<int, 0>{}, ma);
                    if (col_b) push(std::integral_constant<int, 1>{}, mb);
                }
            }
            sgx[(par ^ 1) * NT + t] = gxv;
            sgy[(par ^ 1) * NT + t] = gyk;
        }

        // ---- mu of row j - 4, g of row j - 6: phi(t+1) of row j - 7 -------------------
        float2 lmk = v2(0.f);
        if (own && j >= 3 && j <= jend) {
            float2 u0, u1;
            if (j <= hmax + 4) sl_mu.push(row9x2(smu[par * NT + t - 1], mu1, smu[par * NT + t + 1]), lmk, u0, u1);
            float2 div = v2(0.f);
            if (HYDRO && j >= 5) {
                const int r = j - 6;
                const int q = par * NT + t;
                Row9x2 qx = row9x2(sgx[q - 1], v2(0.f), sgx[q + 1]);
                Row9x2 qy = row9x2(sgy[q - 1], gy1, sgy[q + 1]);
                if (walls) {
                    // the row below the wall row is its image (g_x even, g_y odd)
                    if (ya + r == 0) { sl_gx.ax.x = qx.ax.x; sl_gy.s.x = -qy.s.x; }
                    if (yb + r == 0) { sl_gx.ax.y = qx.ax.y; sl_gy.s.y = -qy.s.y; }
                    // the row above row ny - 1 is the image of row ny - 1
                    if (ya + r == ny) { qx.ax.x = sl_gx.ax.x; qy.s.x = -sl_gy.s.x; }
                    if (yb + r == ny) { qx.ax.y = sl_gx.ax.y; qy.s.y = -sl_gy.s.y; }
                }
                float2 dgx, dgy;
                sl_gx.push(qx, u0, dgx, u1);
                sl_gy.push(qy, u0, u1, dgy);
                div = add2(dgx, dgy);
            }
            const int m = j - 7;
            if ((HYDRO ? j >= 5 : true) && m >= 0) {
                const float2 phn = fma2(v2(p.Gamma), lm2, sub2(ph7, div));
                if (m < ha) { probe += phn.x; io.phi_out[(ya + m) * pitch + gx] = phn.x; }
                if (m < hb) { probe += phn.y; io.phi_out[(yb + m) * pitch + gx] = phn.y; }
            }
        }

        ph7 = ph6; ph6 = ph5; ph5 = ph4; ph4 = ph3; ph3 = ph2; ph2 = ph1; ph1 = phk;
        T3 = T2; T2 = T1; T1 = Tk;
        ps2 = ps1; ps1 = psk;
        dx2 = dx1; dy2 = dy1; dx1 = dxk; dy1 = dyk;
        mu1 = muk;
        pxy1 = pxyk; pyy1 = pyyk;
        gy1 = gyk;
        lm2 = lm1; lm1 = lmk;
        sk = (sk + 1 == M::SIN) ? 0 : sk + 1;
    }
    cp_wait<0>();
    if (__any_sync(0xffffffffu, !isfinite(probe)) && (t & 31) == 0) *reinterpret_cast<volatile int*>(io.flag) = 1;
}

}  // namespace march
}  // namespace lf
