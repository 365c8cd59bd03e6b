// lf_march2d.cuh -- the row-marching D2Q9 step of one (strip, segment) of
// a lattice, shared by the single-lattice kernel (lf_step2d.cu) and the
// ensemble kernel (lf_ens.cu), so both run exactly the same arithmetic.
#pragma once

#include "lf_internal.cuh"

namespace lf {
namespace march {

__device__ __forceinline__ int wrap_any(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Row index of an unwrapped y along an axis that is either periodic or
// bounded by two mirror planes (period 2n reflection).
__device__ __forceinline__ int map_axis(int v, int n, int walls)
{
    if (!walls) return wrap_any(v, n);
    int m = wrap_any(v, 2 * n);
    return m < n ? m : 2 * n - 1 - m;
}

// ===========================================================================
// Row-marching variant of the same step (the default for lf_step).
//
// A CTA of NT threads owns NT - 8 columns (one per thread) plus a 4-column
// halo on each side, and marches down a segment of H rows.  At iteration k
// the inputs of row k (phi, T) and the populations of row k - 3 arrive in a
// shared-memory ring through cp.async issued D iterations earlier; the
// stages then run one row apart:
//   row k-1: psi = nabla^2 phi, and T(t+1)
//   row k-2: lam = nabla^4 phi, P_ab, mu
//   row k-3: F = -d_a P_ab, n, u, g = phi u; collide and push (own rows)
//   row k-4: phi(t+1)
// Neighbours along y come from per-thread register windows; neighbours along
// x from small shared rings of rows that were written in earlier iterations,
// so one barrier per row orders everything.
// ===========================================================================
__device__ __forceinline__ unsigned smem_u32(const void* ptr)
{
    return (unsigned)__cvta_generic_to_shared(ptr);
}

template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src)
{
    if constexpr (B == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename R, int NT, int D>
struct March {
    static constexpr int U = NT - 8;          // columns written per CTA
    static constexpr int SIN = D + 3;         // phi / T rows in flight or in use
    static constexpr int SF = D + 1;          // population rows in flight or in use
    static constexpr int PHI = 0;
    static constexpr int TT = PHI + SIN * NT;
    static constexpr int F = TT + SIN * NT;
    static constexpr int PSI = F + SF * 9 * NT;
    static constexpr int PXX = PSI + 2 * NT;
    static constexpr int PXY = PXX + 2 * NT;
    static constexpr int MU = PXY + 2 * NT;
    static constexpr int GX = MU + 3 * NT;
    static constexpr int TOTAL = GX + 2 * NT;
    static constexpr size_t BYTES = sizeof(R) * TOTAL;
};

template <typename R>
__device__ __forceinline__ R recip(R x) { return R(1) / x; }
template <>
__device__ __forceinline__ float recip<float>(float x) { return __frcp_rn(x); }

// Storage row of an unwrapped row index: the direct cases without division,
// the general reflection / wrap only for lattices smaller than the halo.
__device__ __forceinline__ int map_row(int v, int n, int walls)
{
    if (v >= 0 && v < n) return v;
    const int m = walls ? (v < 0 ? -1 - v : 2 * n - 1 - v) : (v < 0 ? v + n : v - n);
    if (m >= 0 && m < n) return m;
    return map_axis(v, n, walls);
}

// Periodic index with the same shortcut: one add or subtract for v in
// [-n, 2n), the division only beyond.
__device__ __forceinline__ int wrap_near(int v, int n)
{
    if (v >= 0 && v < n) return v;
    const int m = v < 0 ? v + n : v - n;
    if (m >= 0 && m < n) return m;
    return wrap_any(v, n);
}

template <typename R, int NT, int D>
__device__ __forceinline__ void march2d_segment(const Geom& g, const Phys<R>& p, const StepIO<R>& io, int strip, int seg,
                                                int H, unsigned char* smem_raw)
{
    using L = D2Q9;
    using M = March<R, NT, D>;
    static_assert(M::SF == 4, "population ring indexed with & 3");
    R* sm = reinterpret_cast<R*>(smem_raw);
    R* sphi = sm + M::PHI;
    R* sT = sm + M::TT;
    R* sf = sm + M::F;
    R* spsi = sm + M::PSI;
    R* sPxx = sm + M::PXX;
    R* sPxy = sm + M::PXY;
    R* smu = sm + M::MU;
    R* sgx = sm + M::GX;

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
    const bool has_u = t >= 3 && t < NT - 3;        // columns whose velocity is needed
    const R half = R(0.5);
    const R omega = p.inv_tau, keep = R(1) - p.inv_tau;
    const int kbeg = y0 - 4, kend = y1 + 3;        // phi / T rows read by this segment

    // register windows along y (suffix = lag behind the newest row k)
    R phi0 = 0, phi1 = 0, phi2 = 0, phi3 = 0, phi4 = 0;
    R T1 = 0, T2 = 0;
    R psiB = 0, psiC = 0;
    R pxyB = 0, pxyC = 0, pyyB = 0, pyyC = 0;
    R muB = 0, muC = 0, muD = 0;
    R gyB = 0, gyC = 0;
    R probe = 0;              // sum of the outputs: NaN / Inf anywhere make it non-finite

    // ring positions: sk = (k - kbeg) mod SIN, m3 = (k - kbeg) mod 3
    int s_issue = 0;                                 // slot of the next phi / T row to fetch
    auto issue = [&](int j) {
        const int r = j + D;                         // phi / T row
        if (r <= kend) {
            const int off = map_row(r, ny, walls) * pitch + gx;
            cp_async<sizeof(R)>(&sphi[s_issue * NT + t], io.phi_in + off);
            cp_async<sizeof(R)>(&sT[s_issue * NT + t], io.T_in + off);
        }
        s_issue = (s_issue + 1 == M::SIN) ? 0 : s_issue + 1;
        const int rf = j + D - 3;                    // population row
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

    int sk = 0, m3 = 0;
#pragma unroll 2
    for (int k = kbeg; k <= kend; ++k) {
        cp_wait<D - 1>();
        __syncthreads();
        issue(k);
        const int s1 = sk == 0 ? M::SIN - 1 : sk - 1;
        const int s2 = s1 == 0 ? M::SIN - 1 : s1 - 1;
        const int par = (k - kbeg) & 1;              // parity ring position of row k
        phi0 = sphi[sk * NT + t];
        const R T0 = sT[sk * NT + t];

        // ---- row k-1: psi, and the temperature update ----------------------
        const int r1 = k - 1;
        R psiA = 0;
        if (r1 >= y0 - 3 && r1 <= y1 + 2 && t >= 1 && t < NT - 1) {
            psiA = sphi[s1 * NT + t - 1] + sphi[s1 * NT + t + 1] + phi2 + phi0 - R(4) * phi1;
            spsi[(par ^ 1) * NT + t] = psiA;
        }
        if (own && r1 >= y0 && r1 < y1) {
            R Tn = T1;
            if (p.t_update) {
                if (walls && g.t_mode == LF_TWALL_LAYERS && (r1 == 0 || r1 == ny - 1)) {
                    Tn = p.T_w;
                } else {
                    R tu = T0, td = T2;
                    if (walls && g.t_mode == LF_TWALL_HALFWAY) {
                        if (r1 == 0) td = R(2) * p.T_w - T1;
                        if (r1 == ny - 1) tu = R(2) * p.T_w - T1;
                    }
                    Tn = T1 + p.dxi * (sT[s1 * NT + t - 1] + sT[s1 * NT + t + 1] + tu + td - R(4) * T1);
                }
            }
            probe += Tn;
            io.T_out[r1 * pitch + gx] = Tn;
        }

        // ---- row k-2: lam, P, mu --------------------------------------------
        const int r2 = k - 2;
        const int mu_slot2 = m3 == 2 ? 0 : m3 + 1;   // (k - 2 - kbeg) mod 3
        R muA = 0, pxyA = 0, pyyA = 0;
        if (r2 >= y0 - 2 && r2 <= y1 + 1 && t >= 2 && t < NT - 2) {
            const int q = par * NT + t;              // row k-2 has the parity of row k
            const R ps = psiB;
            const R lam = spsi[q - 1] + spsi[q + 1] + psiA + psiC - R(4) * ps;
            const R ph = phi2;
            const R av = (T2 - p.Tc) * p.inv_Tc;
            muA = av * ph + p.b * ph * ph * ph - p.kappa * ps + p.c * lam;
            smu[mu_slot2 * NT + t] = muA;
            if (p.hydro) {
                const R dpx = half * (sphi[s2 * NT + t + 1] - sphi[s2 * NT + t - 1]);
                const R dpy = half * (phi1 - phi3);
                const R dsx = half * (spsi[q + 1] - spsi[q - 1]);
                const R dsy = half * (psiA - psiC);
                const R ph2 = ph * ph;
                const R iso = av * ph2 * half + R(0.75) * p.b * ph2 * ph2
                            - p.kappa * (ph * ps + half * (dpx * dpx + dpy * dpy))
                            + p.c * (ph * lam + half * ps * ps + dpx * dsx + dpy * dsy);
                sPxx[q] = iso + p.kappa * dpx * dpx - R(2) * p.c * dpx * dsx;
                pyyA = iso + p.kappa * dpy * dpy - R(2) * p.c * dpy * dsy;
                pxyA = p.kappa * dpx * dpy - p.c * (dpx * dsy + dpy * dsx);
                sPxy[q] = pxyA;
            }
        }

        // ---- row k-3: F, u, g; collide and push -----------------------------
        const int r3 = k - 3;
        R gyA = 0;
        if (p.hydro && r3 >= y0 - 1 && r3 <= y1 && has_u) {
            const bool ghost = walls && (r3 < 0 || r3 >= ny);
            R gxv = 0;
            if (!ghost) {
                const int qp = (par ^ 1) * NT + t;   // row k-3
                const R Fx = -(half * (sPxx[qp + 1] - sPxx[qp - 1]) + half * (pxyA - pxyC));
                const R Fy = -(half * (sPxy[qp + 1] - sPxy[qp - 1]) + half * (pyyA - pyyC));
                const R* fr = sf + ((r3 - kbeg) & 3) * L::Q * NT + t;
                R df[L::Q];
#pragma unroll
                for (int i = 0; i < L::Q; ++i) df[i] = fr[i * NT];
                const R dn = ((df[0] + df[1]) + (df[2] + df[3])) + ((df[4] + df[5]) + (df[6] + df[7])) + df[8];
                const R jx = (df[1] - df[3]) + (df[5] - df[6]) + (df[8] - df[7]);
                const R jy = (df[2] - df[4]) + (df[5] - df[8]) + (df[6] - df[7]);
                const R n = p.n0 + dn;
                const R inv_n = recip(n);
                const R vx = (jx + half * Fx) * inv_n, vy = (jy + half * Fy) * inv_n;
                gxv = phi3 * vx;
                gyA = phi3 * vy;
                if (own && r3 >= y0 && r3 < y1) {
                    probe += n;
                    // Eq. evoleqn with the Qian equilibrium and Guo's term, written
                    // per opposite pair (i, i'): f*_i = (1 - w) df_i + w_i (sym +- anti)
                    const R on = omega * n;
                    const R C0 = omega * dn - R(1.5) * on * (vx * vx + vy * vy) - R(3) * p.guo * (vx * Fx + vy * Fy);
                    const R a3 = R(3) * on, a45 = R(4.5) * on, g3 = R(3) * p.guo, g9 = R(9) * p.guo;
                    const int site = r3 * pitch + gx;
                    const int up = ((r3 + 1 == ny) ? 0 : r3 + 1) * pitch;
                    const int dn_ = ((r3 == 0) ? ny - 1 : r3 - 1) * pitch;
                    const int mid = r3 * pitch;
                    const bool wall_lo = walls && r3 == 0, wall_hi = walls && r3 == ny - 1;
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
            sgx[(par ^ 1) * NT + t] = gxv;
        }

        // ---- row k-4: phi(t+1) ------------------------------------------------
        const int r4 = k - 4;
        if (own && r4 >= y0 && r4 < y1) {
            const int qm = (m3 == 0 ? 2 : m3 - 1) * NT + t;     // (k - 4 - kbeg) mod 3
            const R lapmu = smu[qm - 1] + smu[qm + 1] + muB + muD - R(4) * muC;
            R div = 0;
            if (p.hydro) {
                const int qg = par * NT + t;                    // row k-4 has the parity of row k
                R gu = gyA, gd = gyC;
                if (walls) {
                    if (r4 == 0) gd = -gyB;
                    if (r4 == ny - 1) gu = -gyB;
                }
                div = half * (sgx[qg + 1] - sgx[qg - 1]) + half * (gu - gd);
            }
            const R phn = phi4 - div + p.Gamma * lapmu;
            probe += phn;
            io.phi_out[r4 * pitch + gx] = phn;
        }

        // ---- shift the windows -----------------------------------------------
        phi4 = phi3; phi3 = phi2; phi2 = phi1; phi1 = phi0;
        T2 = T1; T1 = T0;
        psiC = psiB; psiB = psiA;
        pxyC = pxyB; pxyB = pxyA; pyyC = pyyB; pyyB = pyyA;
        muD = muC; muC = muB; muB = muA;
        gyC = gyB; gyB = gyA;
        sk = (sk + 1 == M::SIN) ? 0 : sk + 1;
        m3 = (m3 == 2) ? 0 : m3 + 1;
    }
    cp_wait<0>();
    if (__any_sync(0xffffffffu, !isfinite(probe)) && (t & 31) == 0) *reinterpret_cast<volatile int*>(io.flag) = 1;
}


// One explicit temperature sub-step at site (x, y): T += dxi nabla^2 T with
// the wall rule of the context (layers held at T_w, or a halfway ghost).
template <typename R>
__device__ __forceinline__ void tsub2d_site(const Geom& g, const Phys<R>& p, const R* __restrict__ Tin,
                                            R* __restrict__ Tout, int x, int y)
{
    const int nx = g.nx, ny = g.ny, pitch = g.pitch;
    const int site = y * pitch + x;
    const R t0 = Tin[site];
    if (g.walls && g.t_mode == LF_TWALL_LAYERS && (y == 0 || y == ny - 1)) {
        Tout[site] = p.T_w;
        return;
    }
    const int xl = x == 0 ? nx - 1 : x - 1, xr = x == nx - 1 ? 0 : x + 1;
    R td, tu;
    if (g.walls) {
        td = y == 0 ? R(2) * p.T_w - t0 : Tin[site - pitch];
        tu = y == ny - 1 ? R(2) * p.T_w - t0 : Tin[site + pitch];
    } else {
        td = Tin[(y == 0 ? ny - 1 : y - 1) * pitch + x];
        tu = Tin[(y == ny - 1 ? 0 : y + 1) * pitch + x];
    }
    Tout[site] = t0 + p.dxi * (Tin[y * pitch + xl] + Tin[y * pitch + xr] + tu + td - R(4) * t0);
}

// Segment height for a lattice: about four CTAs of four warps per SM
// (param > 0 overrides).
inline int march_rows_for(int nx, int ny, int U, int param)
{
    if (param > 0) return param < ny ? param : ny;
    const int strips = (nx + U - 1) / U;
    const int target = 152 * 4;
    int h = (int)(((int64_t)ny * strips + target - 1) / target);
    if (h < 12) h = 12;
    if (h > ny) h = ny;
    return h;
}

// Rows per lane for the two-segment kernel.  Co-resident CTAs share an SM's
// issue rate, so the step takes about (CTAs per SM, rounded up) x (rows per
// lane + 4 pipeline iterations); the smallest such cost wins among heights
// that still give every SM about two CTAs (8 warps) when the lattice allows.
inline int march2_rows_for(int nx, int ny, int U, int param, int sms)
{
    if (param > 0) return param < ny ? param : ny;
    const int strips = (nx + U - 1) / U;
    int best = 1;
    int64_t best_cost = -1;
    // from one row per lane: on small lattices the step is a chain of H + 4
    // dependent row iterations, so short lanes cut its latency
    for (int h = 1; h <= ny && h <= 512; ++h) {
        int pairs = (ny + 2 * h - 1) / (2 * h);
        if (pairs > ny / 2) pairs = ny / 2;
        if (pairs < 1) break;
        const int64_t ctas = (int64_t)strips * pairs;
        if (10 * ctas < 18 * (int64_t)sms && h > 8) break;     // fewer than ~2 CTAs per SM
        const int lane = (ny + 2 * pairs - 1) / (2 * pairs);
        const int64_t cost = ((ctas + sms - 1) / sms) * (lane + 4);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = h; }
    }
    return best;
}

}  // namespace march
}  // namespace lf
