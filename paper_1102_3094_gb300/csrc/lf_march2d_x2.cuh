// lf_march2d_x2.cuh -- FP32 row-marching D2Q9 step on two segments at once,
// marching away from their common boundary.
//
// Same stages, lags, rings and barriers as the row-marching kernel of
// lf_march2d.cuh, but every thread carries one column of TWO vertically
// adjacent segments of a strip in the lanes of float2 values, and the
// arithmetic runs on Blackwell's packed FP32x2 instructions (__fadd2_rn /
// __fmul2_rn / __ffma2_rn), so one instruction advances two sites.
//
// The two segments of a CTA share a boundary row B: lane .y covers rows
// [B, B + hb) and marches up; lane .x covers rows [B - ha, B) and marches
// down.  Lane .x works in the lattice mirrored about y (frame row
// yf = ny - 1 - y, populations with their y-component reversed, y-odd fields
// negated), so both lanes run the same code in a frame where they march
// towards larger yf.  The row just across the boundary of one lane is the
// first row of the other lane: its values come from the other lane of the
// same registers (swapped, and negated for y-odd fields), so nothing is
// recomputed at the boundary; only the far end of each segment needs the
// usual 4-row halo.  The D2Q9 stencils and the BGK/Guo update are symmetric
// under y -> -y, so the mirrored lane computes the same step up to the order
// of floating-point additions.
#pragma once

#include <type_traits>

#include "lf_march2d.cuh"

namespace lf {
namespace march {

__device__ __forceinline__ float2 v2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 swp(float2 a) { return make_float2(a.y, a.x); }    // y-even field
__device__ __forceinline__ float2 swn(float2 a) { return make_float2(-a.y, -a.x); }  // y-odd field
__device__ __forceinline__ float2 sel2(bool cx, float2 a_x, bool cy, float2 a_y, float2 b)
{
    return make_float2(cx ? a_x.x : b.x, cy ? a_y.y : b.y);
}

// D2Q9 population index under y -> -y (0..8 = rest, +x, +y, -x, -y, +x+y,
// -x+y, -x-y, +x-y).
__host__ __device__ constexpr int mirror_y(int i)
{
    return i == 2 ? 4 : i == 4 ? 2 : i == 5 ? 8 : i == 8 ? 5 : i == 6 ? 7 : i == 7 ? 6 : i;
}

template <int NT, int D>
struct March2 {
    static constexpr int U = NT - 8;
    static constexpr int SIN = D + 3;
    static constexpr int SF = D + 1;
    static constexpr int PHI = 8;                         // guard before: lane t-1 of thread 0
    static constexpr int TT = PHI + SIN * NT;
    static constexpr int F = TT + SIN * NT;
    static constexpr int PSI = F + SF * 9 * NT;
    static constexpr int PXX = PSI + 2 * NT;
    static constexpr int PXY = PXX + 2 * NT;
    static constexpr int MU = PXY + 2 * NT;
    static constexpr int GX = MU + 3 * NT;
    static constexpr int TOTAL = GX + 2 * NT + 8;        // float2 elements, guard after
    static constexpr size_t BYTES = sizeof(float2) * TOTAL;
};

// Rows of pair `pair` out of `npairs`: [r0, r1) with boundary b, lane .x
// below b (ha rows), lane .y from b (hb rows); ha, hb >= 1 when ny >= 2 npairs.
__host__ __device__ inline void pair_rows(int ny, int npairs, int pair, int& b, int& ha, int& hb)
{
    const int r0 = (int)((long long)pair * ny / npairs);
    const int r1 = (int)((long long)(pair + 1) * ny / npairs);
    b = r0 + (r1 - r0) / 2;
    ha = b - r0;
    hb = r1 - b;
}

template <int NT, int D, bool HYDRO>
__device__ __forceinline__ void march2d_pair(const Geom& g, const Phys<float>& p, const StepIO<float>& io, int strip,
                                             int pair, int npairs, unsigned char* smem_raw)
{
    using L = D2Q9;
    using M = March2<NT, D>;
    float2* sm = reinterpret_cast<float2*>(smem_raw);
    float2* sphi = sm + M::PHI;
    float2* sT = sm + M::TT;
    float2* sf = sm + M::F;
    float2* spsi = sm + M::PSI;
    float2* sPxx = sm + M::PXX;
    float2* sPxy = sm + M::PXY;
    float2* smu = sm + M::MU;
    float2* sgx = sm + M::GX;

    const int t = threadIdx.x;
    const int nx = g.nx, ny = g.ny, pitch = g.pitch, walls = g.walls;
    const int plane = (int)g.plane;
    const int x0 = strip * M::U;
    int bnd, ha, hb;
    pair_rows(ny, npairs, pair, bnd, ha, hb);
    const int fa = ny - bnd, fb = bnd;              // frame row of q = 0 per lane
    const int hmax = ha > hb ? ha : hb, hmin = ha < hb ? ha : hb;
    const int cx = x0 - 4 + t;
    const int gx = wrap_any(cx, nx);
    const int gxm = wrap_any(cx - 1, nx), gxp = wrap_any(cx + 1, nx);
    const bool own = t >= 4 && t < NT - 4 && cx < nx;
    const bool has_u = t >= 3 && t < NT - 3;
    const float2 half = v2(0.5f), four = v2(4.f);
    const float omega = p.inv_tau, keep = 1.f - p.inv_tau;
    const bool t_half = walls && g.t_mode == LF_TWALL_HALFWAY;
    const bool t_lay = walls && g.t_mode == LF_TWALL_LAYERS;
    float* out = io.f_out;

    // storage offset of frame row yf >= 0 of lane .x / .y (rows past the far
    // end map through the wall reflection or the periodic wrap of the frame)
    auto off_a = [&](int yf) { return (ny - 1 - map_row(yf, ny, walls)) * pitch; };
    auto off_b = [&](int yf) { return map_row(yf, ny, walls) * pitch; };

    float2 phi0 = v2(0), phi1 = v2(0), phi2 = v2(0), phi3 = v2(0), phi4 = v2(0);
    float2 T0 = v2(0), T1 = v2(0), T2 = v2(0);
    float2 psiB = v2(0), psiC = v2(0);
    float2 pxyB = v2(0), pxyC = v2(0), pyyB = v2(0), pyyC = v2(0);
    float2 muB = v2(0), muC = v2(0), muD = v2(0);
    float2 gyB = v2(0), gyC = v2(0);
    float probe = 0.f;

    int s_issue = 0;
    auto issue = [&](int jj) {
        const int q = jj + D - 4;                   // phi / T row (>= 0)
        if (q <= hmax + 3) {
            const int oa = off_a(fa + q) + gx, ob = off_b(fb + q) + gx;
            float* d = reinterpret_cast<float*>(&sphi[s_issue * NT + t]);
            float* e = reinterpret_cast<float*>(&sT[s_issue * NT + t]);
            cp_async<4>(d, io.phi_in + oa);
            cp_async<4>(d + 1, io.phi_in + ob);
            cp_async<4>(e, io.T_in + oa);
            cp_async<4>(e + 1, io.T_in + ob);
        }
        s_issue = (s_issue + 1 == M::SIN) ? 0 : s_issue + 1;
        const int qf = jj + D - 7;                  // population row
        if (HYDRO && has_u && qf >= 0) {
            float* dst = reinterpret_cast<float*>(sf + (qf % M::SF) * L::Q * NT + t);
            if (qf <= ha && !(walls && fa + qf >= ny)) {
                const float* src = io.f_in + (off_a(fa + qf) + gx);
#pragma unroll
                for (int i = 0; i < L::Q; ++i) cp_async<4>(dst + 2 * i * NT, src + mirror_y(i) * plane);
            }
            if (qf <= hb && !(walls && fb + qf >= ny)) {
                const float* src = io.f_in + (off_b(fb + qf) + gx);
#pragma unroll
                for (int i = 0; i < L::Q; ++i) cp_async<4>(dst + 2 * i * NT + 1, src + i * plane);
            }
        }
        cp_commit();
    };

    int sk = 0, m3 = 0, j = 4;

    // One iteration.  S (steady): every stage of both lanes is inside its row
    // range, the boundary rows are behind and the far end is not reached, so
    // range checks, ghost rows, wrap and bounce-back drop out.  Shared-memory
    // loads come first and stores last, so the stages schedule as one block.
    auto body = [&](auto steady_tag) {
        constexpr bool S = decltype(steady_tag)::value;
        cp_wait<D - 1>();
        __syncthreads();
        issue(j);
        const int s1 = sk == 0 ? M::SIN - 1 : sk - 1;
        const int s2 = s1 == 0 ? M::SIN - 1 : s1 - 1;
        const int par = j & 1;
        const int qa = par * NT + t, qb = (par ^ 1) * NT + t;
        const int qm = (m3 == 0 ? 2 : m3 - 1) * NT + t;
        phi0 = sphi[sk * NT + t];
        T0 = sT[sk * NT + t];
        const float2 phl1 = sphi[s1 * NT + t - 1], phr1 = sphi[s1 * NT + t + 1];
        const float2 Tl = sT[s1 * NT + t - 1], Tr = sT[s1 * NT + t + 1];
        const float2 psl = spsi[qa - 1], psr = spsi[qa + 1];
        const float2 phl2 = sphi[s2 * NT + t - 1], phr2 = sphi[s2 * NT + t + 1];
        const float2 mul_ = smu[qm - 1], mur = smu[qm + 1];
        float2 pxxl = v2(0), pxxr = v2(0), pxyl = v2(0), pxyr = v2(0), gxl = v2(0), gxr = v2(0);
        float2 df[L::Q];
        if constexpr (HYDRO) {
            pxxl = sPxx[qb - 1]; pxxr = sPxx[qb + 1];
            pxyl = sPxy[qb - 1]; pxyr = sPxy[qb + 1];
            gxl = sgx[qa - 1]; gxr = sgx[qa + 1];
            // slot of population row q3 = j - 7 (rows r live in slot r mod SF;
            // the offset keeps the operand non-negative for j >= 4)
            const float2* fr = sf + ((j - 7 + 4 * M::SF) % M::SF) * L::Q * NT + t;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) df[i] = fr[i * NT];
        }

        const int q1 = j - 5, q2 = j - 6, q3 = j - 7, q4 = j - 8;
        if constexpr (!S) {
            // the row across the boundary is the first row of the other lane
            if (q1 == 0) { phi2 = swp(phi1); T2 = swp(T1); }
            if (q2 == 0) psiC = swp(psiB);
            if (q3 == 0) { pxyC = swn(pxyB); pyyC = swp(pyyB); }
            if (q4 == 0) { muD = swp(muC); gyC = swn(gyB); }
        }

        // row q1: psi, T(t+1)
        const float2 psiA = fma2(four, sub2(v2(0), phi1), add2(add2(phl1, phr1), add2(phi2, phi0)));
        float2 Tn = T1;
        if (S || (q1 >= 0 && q1 < hmax)) {
            const int ya = fa + q1, yb = fb + q1;
            const float2 gw = sub2(v2(2.f * p.T_w), T1);
            const float2 tu = sel2(t_half && ya == ny - 1, gw, t_half && yb == ny - 1, gw, T0);
            const float2 Tu = fma2(v2(p.dxi), fma2(four, sub2(v2(0), T1), add2(add2(Tl, Tr), add2(tu, T2))), T1);
            const float2 tw = v2(p.T_w);
            const float2 Tw = sel2(t_lay && ya == ny - 1, tw, t_lay && yb == ny - 1, tw, Tu);
            Tn = p.t_update ? Tw : T1;
        }

        // row q2: lam, P, mu
        float2 muA = v2(0), pxx = v2(0), pxyA = v2(0), pyyA = v2(0);
        if (S || (q2 >= 0 && q2 <= hmax + 1)) {
            const float2 ps = psiB, ph = phi2;
            const float2 lam = fma2(four, sub2(v2(0), ps), add2(add2(psl, psr), add2(psiA, psiC)));
            const float2 av = mul2(sub2(T2, v2(p.Tc)), v2(p.inv_Tc));
            const float2 ph2 = mul2(ph, ph);
            // mu = a phi + b phi^3 - kappa psi + c lam
            muA = fma2(v2(p.c), lam, fma2(v2(-p.kappa), ps, mul2(ph, fma2(v2(p.b), ph2, av))));
            if constexpr (HYDRO) {
                const float2 dpx = mul2(half, sub2(phr2, phl2));
                const float2 dpy = mul2(half, sub2(phi1, phi3));
                const float2 dsx = mul2(half, sub2(psr, psl));
                const float2 dsy = mul2(half, sub2(psiA, psiC));
                const float2 gp2 = fma2(dpx, dpx, mul2(dpy, dpy));
                const float2 gpgs = fma2(dpx, dsx, mul2(dpy, dsy));
                // iso = a phi^2/2 + 3b phi^4/4 - kappa (phi psi + gp2/2) + c (phi lam + psi^2/2 + gpgs)
                float2 iso = mul2(ph2, fma2(v2(0.75f * p.b), ph2, mul2(half, av)));
                iso = fma2(v2(-p.kappa), fma2(half, gp2, mul2(ph, ps)), iso);
                iso = fma2(v2(p.c), add2(fma2(ph, lam, mul2(half, mul2(ps, ps))), gpgs), iso);
                const float2 c2 = v2(-2.f * p.c);
                pxx = fma2(v2(p.kappa), mul2(dpx, dpx), fma2(c2, mul2(dpx, dsx), iso));
                pyyA = fma2(v2(p.kappa), mul2(dpy, dpy), fma2(c2, mul2(dpy, dsy), iso));
                pxyA = fma2(v2(p.kappa), mul2(dpx, dpy), mul2(v2(-p.c), fma2(dpx, dsy, mul2(dpy, dsx))));
            }
        }

        // row q3: F, u, fluxes; collide
        float2 gxv = v2(0), gyA = v2(0), n = v2(0);
        float2 post[L::Q];
        bool col_a = false, col_b = false;
        if constexpr (HYDRO) {
            if (S || (q3 >= 0 && q3 <= hmax)) {
                bool gha = false, ghb = false;
                if constexpr (!S) {
                    gha = walls && fa + q3 >= ny;
                    ghb = walls && fb + q3 >= ny;
#pragma unroll
                    for (int i = 0; i < L::Q; ++i) {
                        if (gha) df[i].x = 0.f;
                        if (ghb) df[i].y = 0.f;
                    }
                }
                const float2 Fx = sub2(v2(0), mul2(half, add2(sub2(pxxr, pxxl), sub2(pxyA, pxyC))));
                const float2 Fy = sub2(v2(0), mul2(half, add2(sub2(pxyr, pxyl), sub2(pyyA, pyyC))));
                const float2 dn = add2(add2(add2(df[0], df[1]), add2(df[2], df[3])),
                                       add2(add2(df[4], df[5]), add2(add2(df[6], df[7]), df[8])));
                const float2 jx = add2(add2(sub2(df[1], df[3]), sub2(df[5], df[6])), sub2(df[8], df[7]));
                const float2 jy = add2(add2(sub2(df[2], df[4]), sub2(df[5], df[8])), sub2(df[6], df[7]));
                n = add2(v2(p.n0), dn);
                const float2 inv_n = make_float2(__frcp_rn(n.x), __frcp_rn(n.y));
                const float2 vx = mul2(fma2(half, Fx, jx), inv_n), vy = mul2(fma2(half, Fy, jy), inv_n);
                gxv = mul2(phi3, vx);
                gyA = mul2(phi3, vy);
                if constexpr (!S) {
                    if (gha) { gxv.x = 0.f; gyA.x = 0.f; }
                    if (ghb) { gxv.y = 0.f; gyA.y = 0.f; }
                }
                col_a = own && (S || (q3 >= 0 && q3 < ha));
                col_b = own && (S || (q3 >= 0 && q3 < hb));
                if (S || col_a || col_b) {
                    const float2 on = mul2(v2(omega), n);
                    const float2 uu = fma2(vx, vx, mul2(vy, vy));
                    const float2 uF = fma2(vx, Fx, mul2(vy, Fy));
                    const float2 C0 = fma2(v2(-3.f * p.guo), uF, fma2(mul2(v2(-1.5f), on), uu, mul2(v2(omega), dn)));
                    const float2 a3 = mul2(v2(3.f), on), a45 = mul2(v2(4.5f), on);
                    const float2 g3 = v2(3.f * p.guo), g9 = v2(9.f * p.guo);
                    const float2 kp = v2(keep);
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
                }
            }
        }

        // row q4: phi(t+1)
        float2 phn = v2(0);
        if (S || (q4 >= 0 && q4 < hmax)) {
            const float2 lapmu = fma2(four, sub2(v2(0), muC), add2(add2(mul_, mur), add2(muB, muD)));
            float2 div = v2(0);
            if constexpr (HYDRO) {
                float2 gu = gyA;
                if constexpr (!S) {
                    const float2 ng = sub2(v2(0), gyB);
                    gu = sel2(walls && fa + q4 == ny - 1, ng, walls && fb + q4 == ny - 1, ng, gu);
                }
                div = mul2(half, add2(sub2(gxr, gxl), sub2(gu, gyC)));
            }
            phn = fma2(v2(p.Gamma), lapmu, sub2(phi4, div));
        }

        spsi[qb] = psiA;
        smu[(m3 == 2 ? 0 : m3 + 1) * NT + t] = muA;
        if constexpr (HYDRO) {
            sPxx[qa] = pxx;
            sPxy[qa] = pxyA;
            sgx[qb] = gxv;
        }
        if (own) {
            // storage row offsets: lane .x at row bnd - 1 - q, lane .y at bnd + q
            auto ra = [&](int q) { return S ? (bnd - 1 - q) * pitch : off_a(fa + q); };
            auto rb = [&](int q) { return S ? (bnd + q) * pitch : off_b(fb + q); };
            if (S || (q1 >= 0 && q1 < ha)) { probe += Tn.x; io.T_out[ra(q1) + gx] = Tn.x; }
            if (S || (q1 >= 0 && q1 < hb)) { probe += Tn.y; io.T_out[rb(q1) + gx] = Tn.y; }
            if (S || (q4 >= 0 && q4 < ha)) { probe += phn.x; io.phi_out[ra(q4) + gx] = phn.x; }
            if (S || (q4 >= 0 && q4 < hb)) { probe += phn.y; io.phi_out[rb(q4) + gx] = phn.y; }
            if constexpr (HYDRO) {
                // frame population i of lane .x is storage population mirror_y(i);
                // bounce-back on the wall at the far end (frame row ny - 1),
                // periodic wrap in the frame otherwise
                const int cm = gxm - gx, cp = gxp - gx;
                auto push = [&](auto lane_tag, int q) {
                    constexpr int LN = decltype(lane_tag)::value;
                    auto P = [](int i) { return LN == 0 ? mirror_y(i) : i; };
                    auto pv = [&](int i) { return LN == 0 ? post[i].x : post[i].y; };
                    const int yf = (LN == 0 ? fa : fb) + q;
                    const int step = LN == 0 ? -pitch : pitch;
                    const int site = (LN == 0 ? ra(q) : rb(q)) + gx;
                    const int dn = site - step;
                    int up = site + step;
                    bool hi = false;
                    if constexpr (!S) {
                        hi = walls && yf == ny - 1;
                        if (yf + 1 == ny) up = (LN == 0 ? (ny - 1) * pitch : 0) + gx;
                    }
                    out[P(0) * plane + site] = pv(0);
                    out[P(1) * plane + site + cp] = pv(1);
                    out[P(3) * plane + site + cm] = pv(3);
                    out[P(4) * plane + dn] = pv(4);
                    out[P(7) * plane + dn + cm] = pv(7);
                    out[P(8) * plane + dn + cp] = pv(8);
                    if (hi) {
                        out[P(4) * plane + site] = pv(2);
                        out[P(7) * plane + site] = pv(5);
                        out[P(8) * plane + site] = pv(6);
                    } else {
                        out[P(2) * plane + up] = pv(2);
                        out[P(5) * plane + up + cp] = pv(5);
                        out[P(6) * plane + up + cm] = pv(6);
                    }
                };
                if (S || col_a) { probe += n.x; push(std::integral_constant<int, 0>{}, q3); }
                if (S || col_b) { probe += n.y; push(std::integral_constant<int, 1>{}, q3); }
            }
        }

        phi4 = phi3; phi3 = phi2; phi2 = phi1; phi1 = phi0;
        T2 = T1; T1 = T0;
        psiC = psiB; psiB = psiA;
        pxyC = pxyB; pxyB = pxyA; pyyC = pyyB; pyyB = pyyA;
        muD = muC; muC = muB; muB = muA;
        gyC = gyB; gyB = gyA;
        sk = (sk + 1 == M::SIN) ? 0 : sk + 1;
        m3 = (m3 == 2) ? 0 : m3 + 1;
    };

    for (int jj = 4 - D; jj < 4; ++jj) issue(jj);
    const int jend = hmax + 7;                      // last iteration: phi of row hmax - 1
    const int js0 = 9, js1 = hmin + 4;              // steady iterations
#pragma unroll 1
    for (j = 4; j <= jend; ++j) {
        if (HYDRO && j >= js0 && j <= js1) body(std::true_type{});
        else body(std::false_type{});
    }
    cp_wait<0>();
    if (__any_sync(0xffffffffu, !isfinite(probe)) && (t & 31) == 0) *reinterpret_cast<volatile int*>(io.flag) = 1;
}

}  // namespace march
}  // namespace lf
