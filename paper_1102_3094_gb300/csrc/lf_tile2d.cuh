// lf_tile2d.cuh -- the tile form of the D2Q9 step (one TX x TY tile, every
// stage of the step in shared memory; the compact or the isotropic 9-point
// stencils) and the isotropic temperature sub-step, shared by the tile
// kernel (lf_step2d.cu) and the ensemble's persistent kernel (lf_ens.cu), so
// a run gives the same bits in both.
#pragma once

#include "lf_internal.cuh"
#include "lf_march2d.cuh"

namespace lf {
namespace tile {

using march::wrap_near;
using march::map_row;

// Stencils on a row-major shared-memory region of row length W, centre c.
template <typename R, int W, bool ISO>
__device__ __forceinline__ R lap_s(const R* a, int c)
{
    if constexpr (ISO)
        return (R(4) * (a[c - 1] + a[c + 1] + a[c - W] + a[c + W])
                + (a[c - W - 1] + a[c - W + 1] + a[c + W - 1] + a[c + W + 1]) - R(20) * a[c]) * R(1.0 / 6.0);
    else
        return a[c - 1] + a[c + 1] + a[c - W] + a[c + W] - R(4) * a[c];
}

template <typename R, int W, bool ISO>
__device__ __forceinline__ R dx_s(const R* a, int c)
{
    if constexpr (ISO)
        return (R(4) * (a[c + 1] - a[c - 1]) + (a[c + W + 1] - a[c + W - 1]) + (a[c - W + 1] - a[c - W - 1]))
               * R(1.0 / 12.0);
    else
        return R(0.5) * (a[c + 1] - a[c - 1]);
}

template <typename R, int W, bool ISO>
__device__ __forceinline__ R dy_s(const R* a, int c)
{
    if constexpr (ISO)
        return (R(4) * (a[c + W] - a[c - W]) + (a[c + W + 1] - a[c - W + 1]) + (a[c + W - 1] - a[c - W - 1]))
               * R(1.0 / 12.0);
    else
        return R(0.5) * (a[c + W] - a[c - W]);
}

template <typename R, int TX, int TY>
struct Tile {
    static constexpr int W4 = TX + 8, H4 = TY + 8;
    static constexpr int W3 = TX + 6, H3 = TY + 6;
    static constexpr int W2 = TX + 4, H2 = TY + 4;
    static constexpr int W1 = TX + 2, H1 = TY + 2;
    static constexpr int PHI = 0;
    static constexpr int T = PHI + W4 * H4;
    static constexpr int PSI = T + W2 * H2;
    static constexpr int LAM = PSI + W3 * H3;
    static constexpr int P = LAM + W2 * H2;       // Pxx, Pyy, Pxy
    static constexpr int F = P + 3 * W2 * H2;     // Fx, Fy
    static constexpr int MU = F + 2 * W1 * H1;
    static constexpr int G = P;                   // gx, gy reuse the P area
    static constexpr int TOTAL = MU + W1 * H1;
    static constexpr size_t BYTES = sizeof(R) * TOTAL;
    static_assert(2 * W1 * H1 <= 3 * W2 * H2, "g must fit in the P area");
};

// One TX x TY tile (bx, by) of the step, run by NT threads; smem_raw holds
// Tile<R, TX, TY>::BYTES.  Called once per CTA by the tile kernel and once per
// work item by the ensemble's persistent kernel, so both do the same arithmetic.
template <typename R, int TX, int TY, int NT, bool AUX, bool ISO>
__device__ __forceinline__ void step2d_tile(const Geom& g, const Phys<R>& p, const StepIO<R>& io, int bx, int by,
                                            unsigned char* smem_raw)
{
    using L = D2Q9;
    using TL = Tile<R, TX, TY>;
    constexpr int W4 = TL::W4, H4 = TL::H4, W3 = TL::W3, H3 = TL::H3;
    constexpr int W2 = TL::W2, H2 = TL::H2, W1 = TL::W1, H1 = TL::H1;

    R* sm = reinterpret_cast<R*>(smem_raw);
    R* sphi = sm + TL::PHI;
    R* sT = sm + TL::T;
    R* spsi = sm + TL::PSI;
    R* slam = sm + TL::LAM;
    R* sPxx = sm + TL::P;
    R* sPyy = sPxx + W2 * H2;
    R* sPxy = sPyy + W2 * H2;
    R* sFx = sm + TL::F;
    R* sFy = sFx + W1 * H1;
    R* smu = sm + TL::MU;
    R* sgx = sm + TL::G;
    R* sgy = sgx + W1 * H1;

    const int nx = g.nx, ny = g.ny, pitch = g.pitch, walls = g.walls;
    const int plane = (int)g.plane;        // 32-bit offsets: Q * padded sites < 2^31 (checked at creation)
    const int x0 = bx * TX, y0 = by * TY;
    const R half = R(0.5);
    bool bad = false;

    // ---- stage 1: phi (r = 4) and T (r = 2) -----------------------------
    for (int k = threadIdx.x; k < W4 * H4; k += NT) {
        const int ly = k / W4, lx = k - ly * W4;
        const int gx = wrap_near(x0 - 4 + lx, nx), gy = map_row(y0 - 4 + ly, ny, walls);
        sphi[k] = io.phi_in[gy * pitch + gx];
    }
    for (int k = threadIdx.x; k < W2 * H2; k += NT) {
        const int ly = k / W2, lx = k - ly * W2;
        const int gx = wrap_near(x0 - 2 + lx, nx), gy = map_row(y0 - 2 + ly, ny, walls);
        sT[k] = io.T_in[gy * pitch + gx];
    }
    __syncthreads();

    // ---- stage 2: psi = nabla^2 phi (r = 3) ------------------------------
    for (int k = threadIdx.x; k < W3 * H3; k += NT) {
        const int ly = k / W3, lx = k - ly * W3;
        const int c = (ly + 1) * W4 + lx + 1;
        spsi[k] = lap_s<R, W4, ISO>(sphi, c);
    }
    __syncthreads();

    // ---- stage 3: lam = nabla^4 phi and P_ab (r = 2) ---------------------
    for (int k = threadIdx.x; k < W2 * H2; k += NT) {
        const int ly = k / W2, lx = k - ly * W2;
        const int cp = (ly + 2) * W4 + lx + 2;
        const int cs = (ly + 1) * W3 + lx + 1;
        const R ph = sphi[cp], psi = spsi[cs];
        const R lam = lap_s<R, W3, ISO>(spsi, cs);
        slam[k] = lam;
        if (AUX || p.hydro) {
            const R av = (sT[k] - p.Tc) / p.Tc;
            const R dpx = dx_s<R, W4, ISO>(sphi, cp);
            const R dpy = dy_s<R, W4, ISO>(sphi, cp);
            const R dsx = dx_s<R, W3, ISO>(spsi, cs);
            const R dsy = dy_s<R, W3, ISO>(spsi, cs);
            const R ph2 = ph * ph;
            const R iso = av * ph2 * half + R(0.75) * p.b * ph2 * ph2
                        - p.kappa * (ph * psi + half * (dpx * dpx + dpy * dpy))
                        + p.c * (ph * lam + half * psi * psi + dpx * dsx + dpy * dsy);
            sPxx[k] = iso + p.kappa * dpx * dpx - R(2) * p.c * dpx * dsx;
            sPyy[k] = iso + p.kappa * dpy * dpy - R(2) * p.c * dpy * dsy;
            sPxy[k] = p.kappa * dpx * dpy - p.c * (dpx * dsy + dpy * dsx);
        }
    }
    __syncthreads();

    // ---- stage 4: mu and F (r = 1) --------------------------------------
    for (int k = threadIdx.x; k < W1 * H1; k += NT) {
        const int ly = k / W1, lx = k - ly * W1;
        const int c2 = (ly + 1) * W2 + lx + 1;
        const int cs = (ly + 2) * W3 + lx + 2;
        const int cp = (ly + 3) * W4 + lx + 3;
        const R ph = sphi[cp];
        const R av = (sT[c2] - p.Tc) / p.Tc;
        smu[k] = av * ph + p.b * ph * ph * ph - p.kappa * spsi[cs] + p.c * slam[c2];
        if (AUX || p.hydro) {
            sFx[k] = -(dx_s<R, W2, ISO>(sPxx, c2) + dy_s<R, W2, ISO>(sPxy, c2));
            sFy[k] = -(dx_s<R, W2, ISO>(sPxy, c2) + dy_s<R, W2, ISO>(sPyy, c2));
        } else {
            sFx[k] = R(0);
            sFy[k] = R(0);
        }
    }
    __syncthreads();

    // ---- stage 5: moments, flux g = phi u (r = 1, corners only for the
    //      isotropic divergence); interior sites collide and push -------------
    for (int k = threadIdx.x; k < W1 * H1; k += NT) {
        const int ly = k / W1, lx = k - ly * W1;
        const bool edge_x = (lx == 0 || lx == W1 - 1), edge_y = (ly == 0 || ly == H1 - 1);
        if (!ISO && edge_x && edge_y) continue;
        const int ux = x0 - 1 + lx, uy = y0 - 1 + ly;        // unwrapped position
        if (walls && (uy < 0 || uy >= ny)) continue;         // ghost row: see stage 6
        const bool inner = !edge_x && !edge_y;
        const bool real = inner && ux < nx && uy < ny;
        if (!p.hydro && !(AUX && real)) {
            sgx[k] = R(0);
            sgy[k] = R(0);
            continue;
        }
        const int gx = wrap_near(ux, nx), gy = walls ? uy : wrap_near(uy, ny);
        const int site = gy * pitch + gx;
        R df[L::Q];
        R dn = R(0), jx = R(0), jy = R(0);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            df[i] = io.f_in[i * plane + site];
            dn += df[i];
            jx += R(L::ex(i)) * df[i];
            jy += R(L::ey(i)) * df[i];
        }
        const R n = p.n0 + dn;
        const R Fx = sFx[k], Fy = sFy[k];
        const R inv_n = R(1) / n;
        const R vx = p.hydro ? (jx + half * Fx) * inv_n : R(0);
        const R vy = p.hydro ? (jy + half * Fy) * inv_n : R(0);
        const R ph = sphi[(ly + 3) * W4 + lx + 3];
        sgx[k] = ph * vx;
        sgy[k] = ph * vy;
        if (!real) continue;
        bad |= !isfinite(n);
        if (AUX) {
            io.rho[site] = n;
            io.u[0][site] = vx;
            io.u[1][site] = vy;
            continue;
        }
        if (!p.hydro) continue;
        // Eq. evoleqn with the Qian equilibrium and Guo's term, in deviation
        // form: df* = df - (df - dfeq)/tau + F_i,  dfeq = feq - w n0.
        const R uu = vx * vx + vy * vy;
        const R uF = vx * Fx + vy * Fy;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const R wi = R(L::w(i));
            const R eu = R(L::ex(i)) * vx + R(L::ey(i)) * vy;
            const R eF = R(L::ex(i)) * Fx + R(L::ey(i)) * Fy;
            const R dfeq = wi * (dn + n * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * uu));
            const R Fi = p.guo * wi * (R(3) * (eF - uF) + R(9) * eu * eF);
            const R post = df[i] - (df[i] - dfeq) * p.inv_tau + Fi;
            int tx = ux + L::ex(i);
            int ty = uy + L::ey(i);
            if (walls && (ty < 0 || ty >= ny)) {
                io.f_out[L::opp(i) * plane + site] = post;       // halfway bounce-back
            } else {
                tx = tx < 0 ? tx + nx : (tx >= nx ? tx - nx : tx);
                ty = ty < 0 ? ty + ny : (ty >= ny ? ty - ny : ty);
                io.f_out[i * plane + ty * pitch + tx] = post;
            }
        }
    }
    __syncthreads();

    // ---- stage 6: phi and T updates (r = 0) ------------------------------
    for (int k = threadIdx.x; k < TX * TY; k += NT) {
        const int ly = k / TX, lx = k - ly * TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        const int site = gy * pitch + gx;
        const int c1 = (ly + 1) * W1 + lx + 1;
        if (AUX) {
            io.mu[site] = smu[c1];
            io.F[0][site] = sFx[c1];
            io.F[1][site] = sFy[c1];
            continue;
        }
        const int cp = (ly + 4) * W4 + lx + 4;
        const int c2 = (ly + 2) * W2 + lx + 2;
        const R lapmu = lap_s<R, W1, ISO>(smu, c1);
        R div = R(0);
        if (p.hydro) {
            if constexpr (ISO) {
                // rows below / at / above: a row beyond a wall is the image of
                // the site's own row (g_x even, g_y odd: no flux through it)
                const bool lo = walls && gy == 0, hi = walls && gy == ny - 1;
                const int rd = lo ? c1 : c1 - W1, ru = hi ? c1 : c1 + W1;
                const R sd = lo ? R(-1) : R(1), su = hi ? R(-1) : R(1);
                const R dgx = R(4) * (sgx[c1 + 1] - sgx[c1 - 1]) + (sgx[ru + 1] - sgx[ru - 1])
                            + (sgx[rd + 1] - sgx[rd - 1]);
                const R dgy = R(4) * (su * sgy[ru] - sd * sgy[rd]) + (su * sgy[ru + 1] - sd * sgy[rd + 1])
                            + (su * sgy[ru - 1] - sd * sgy[rd - 1]);
                div = (dgx + dgy) * R(1.0 / 12.0);
            } else {
                R gyu = sgy[c1 + W1], gyd = sgy[c1 - W1];
                if (walls) {                                 // no flux through the walls
                    if (gy == 0) gyd = -sgy[c1];
                    if (gy == ny - 1) gyu = -sgy[c1];
                }
                div = half * (sgx[c1 + 1] - sgx[c1 - 1]) + half * (gyu - gyd);
            }
        }
        const R phn = sphi[cp] - div + p.Gamma * lapmu;
        const R Tc0 = sT[c2];
        R Tn = Tc0;
        if (p.t_update) {
            if (walls && g.t_mode == LF_TWALL_LAYERS && (gy == 0 || gy == ny - 1)) {
                Tn = p.T_w;
            } else if constexpr (ISO) {
                // halfway ghosts: 2 T_w minus the mirror image the halo row holds
                const bool lo = walls && g.t_mode == LF_TWALL_HALFWAY && gy == 0;
                const bool hi = walls && g.t_mode == LF_TWALL_HALFWAY && gy == ny - 1;
                const R* rd = sT + c2 - W2;
                const R* ru = sT + c2 + W2;
                const R d0 = lo ? R(2) * p.T_w - rd[0] : rd[0], dl = lo ? R(2) * p.T_w - rd[-1] : rd[-1];
                const R dr = lo ? R(2) * p.T_w - rd[1] : rd[1];
                const R u0 = hi ? R(2) * p.T_w - ru[0] : ru[0], ul = hi ? R(2) * p.T_w - ru[-1] : ru[-1];
                const R ur = hi ? R(2) * p.T_w - ru[1] : ru[1];
                const R lap = (R(4) * (sT[c2 - 1] + sT[c2 + 1] + u0 + d0) + (ul + ur + dl + dr) - R(20) * Tc0)
                              * R(1.0 / 6.0);
                Tn = Tc0 + p.dxi * lap;
            } else {
                R tu = sT[c2 + W2], td = sT[c2 - W2];
                if (walls && g.t_mode == LF_TWALL_HALFWAY) {
                    if (gy == 0) td = R(2) * p.T_w - Tc0;
                    if (gy == ny - 1) tu = R(2) * p.T_w - Tc0;
                }
                Tn = Tc0 + p.dxi * (sT[c2 - 1] + sT[c2 + 1] + tu + td - R(4) * Tc0);
            }
        }
        bad |= !isfinite(phn) || !isfinite(Tn);
        io.phi_out[site] = phn;
        io.T_out[site] = Tn;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
        *reinterpret_cast<volatile int*>(io.flag) = 1;
}

// The same sub-step with the isotropic 9-point Laplacian.  A row beyond a wall
// holds 2 T_w - T of the site's own row (halfway ghost); with held wall
// layers the interior never reaches past them.
template <typename R>
__device__ __forceinline__ void tsub2d_site_iso(const Geom& g, const Phys<R>& p, const R* __restrict__ Tin,
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
    const bool lo = g.walls && y == 0, hi = g.walls && y == ny - 1;
    const int yd = lo ? 0 : (y == 0 ? ny - 1 : y - 1);
    const int yu = hi ? y : (y == ny - 1 ? 0 : y + 1);
    const R* rd = Tin + yd * pitch;
    const R* r0 = Tin + y * pitch;
    const R* ru = Tin + yu * pitch;
    const R two_w = R(2) * p.T_w;
    const R d0 = lo ? two_w - rd[x] : rd[x], dl = lo ? two_w - rd[xl] : rd[xl], dr = lo ? two_w - rd[xr] : rd[xr];
    const R u0 = hi ? two_w - ru[x] : ru[x], ul = hi ? two_w - ru[xl] : ru[xl], ur = hi ? two_w - ru[xr] : ru[xr];
    const R lap = (R(4) * (r0[xl] + r0[xr] + u0 + d0) + (ul + ur + dl + dr) - R(20) * t0) * R(1.0 / 6.0);
    Tout[site] = t0 + p.dxi * lap;
}

}  // namespace tile
}  // namespace lf
