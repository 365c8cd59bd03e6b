// lf_step3d.cu -- one fused pass per time step of the hybrid LB/FD method of
// arXiv:1102.3094, Sec. 2, on the D3Q19 lattice (three dimensions, walls
// normal to z, x and y periodic).
//
// A CTA owns a TX x TY tile of the (x, y) plane and marches along z over a
// segment of planes.  At iteration k the next phi / T plane (k + 1, with a
// 4-site halo in x and y) is prefetched by cp.async while the stages run on
// shrinking in-plane regions, one plane apart:
//   plane k-1: psi = nabla^2 phi (r = 3);  T(t+1) (r = 0)
//   plane k-2: lam = nabla^4 phi, P_ab (6 components), mu (r = 2)
//   plane k-3: F = -d_a P_ab, n, u = (sum f e + F/2)/n, g = phi u (r = 1);
//              interior sites collide (BGK + Guo) and push their populations
//   plane k-4: phi(t+1) = phi - div(g) + Gamma nabla^2 mu (r = 0)
// Neighbours along z come from rings of planes in shared memory.  The wall
// rule is the one of the 2D kernel: halo planes beyond z = 0 and nz - 1 are
// read through the mirror map (even reflection of phi and T, hence of every
// derived scalar; tensors and the force follow), and the wall-normal flux
// g_z is odd, so plane 0 (nz - 1) uses -g_z(own) for its missing neighbour.
// Populations are stored as deviations f_i - w_i n0 and pushed with halfway
// bounce-back at the walls.
//
// With ISO set, every derivative takes the isotropic 19-point form (D3Q19
// weights: d_a = 3 sum w_i e_ia A(r + e_i), lap = 6 sum w_i [A(r + e_i) - A(r)]).
// Those reach the in-plane neighbours of the planes above and below, so the
// in-plane tensor components and the flux g keep three planes instead of two,
// the flux is computed on the corners of the r = 1 region too, and a plane
// beyond a wall is replaced by the image of the wall plane itself (g_z odd,
// the halfway temperature ghost 2 T_w - T).
#include "lf_internal.cuh"
#include "lf_iso3.cuh"

namespace lf {

namespace {

__device__ __forceinline__ int wrap_any3(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

template <typename R>
__device__ __forceinline__ R recip3(R x) { return R(1) / x; }
template <>
__device__ __forceinline__ float recip3<float>(float x) { return __frcp_rn(x); }

// Storage plane of an unwrapped z (periodic, or mirrored about the half-way
// walls with period 2n); the division only for v outside [-n, 2n).
__device__ __forceinline__ int map_axis3(int v, int n, int walls)
{
    if (v >= 0 && v < n) return v;
    const int d = walls ? (v < 0 ? -1 - v : 2 * n - 1 - v) : (v < 0 ? v + n : v - n);
    if (d >= 0 && d < n) return d;
    if (!walls) return wrap_any3(v, n);
    const int m = wrap_any3(v, 2 * n);
    return m < n ? m : 2 * n - 1 - m;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

template <int B>
__device__ __forceinline__ void cp_async3(void* dst, const void* src)
{
    if constexpr (B == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

template <typename R, int TX, int TY, bool ISO = false>
struct Plane3 {
    static constexpr int W4 = TX + 8, H4 = TY + 8, A4 = W4 * H4;   // phi region (r = 4)
    static constexpr int W3 = TX + 6, H3 = TY + 6, A3 = W3 * H3;   // psi
    static constexpr int W2 = TX + 4, H2 = TY + 4, A2 = W2 * H2;   // T, lam, P, mu
    static constexpr int W1 = TX + 2, H1 = TY + 2, A1 = W1 * H1;   // F, u, g, mu(use)
    static constexpr int NPHI = 6;     // planes k-4 .. k+1
    static constexpr int NT_ = 4;      // T planes k-2 .. k+1
    static constexpr int NPIN = ISO ? 3 : 2;          // planes of Pxx, Pxy, Pyy and of gx, gy
    static constexpr int PHI = 0;
    static constexpr int T = PHI + NPHI * A4;
    static constexpr int PSI = T + NT_ * A2;          // 3 planes
    static constexpr int PIN = PSI + 3 * A3;          // Pxx, Pxy, Pyy: NPIN planes each
    static constexpr int PZ = PIN + 3 * NPIN * A2;    // Pxz, Pyz, Pzz: 3 planes each
    static constexpr int MU = PZ + 9 * A2;            // 4 planes of the r = 1 region
    static constexpr int GXY = MU + 4 * A1;           // gx, gy: NPIN planes each
    static constexpr int GZ = GXY + 2 * NPIN * A1;    // gz: 3 planes
    static constexpr int TOTAL = GZ + 3 * A1;
    // wrapped storage column / row of every position of the r = 4 region
    static constexpr size_t MAPS = sizeof(R) * TOTAL;
    static constexpr size_t BYTES = MAPS + sizeof(int) * (W4 + H4);
};

template <typename R, int TX, int TY, int NT, bool AUX, bool ISO>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? (ISO ? 2 : 3) : 1)
    k_march3d(Geom g, Phys<R> p, StepIO<R> io, int Hz)
{
    using L = D3Q19;
    using P3 = Plane3<R, TX, TY, ISO>;
    constexpr int NPIN = P3::NPIN;
    constexpr int W4 = P3::W4, W3 = P3::W3, W2 = P3::W2, W1 = P3::W1;
    constexpr int A4 = P3::A4, A3 = P3::A3, A2 = P3::A2, A1 = P3::A1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    R* sphi = sm + P3::PHI;
    R* sT = sm + P3::T;
    R* spsi = sm + P3::PSI;
    R* sPin = sm + P3::PIN;   // [comp 0..2][plane mod NPIN][A2]: xx, xy, yy
    R* sPz = sm + P3::PZ;     // [comp 0..2][plane mod 3][A2]: xz, yz, zz
    R* smu = sm + P3::MU;     // [plane mod 4][A1]
    R* sgxy = sm + P3::GXY;   // [comp 0..1][plane mod NPIN][A1]
    R* sgz = sm + P3::GZ;     // [plane mod 3][A1]
    int* colmap = reinterpret_cast<int*>(smem_raw + P3::MAPS);   // x0 - 4 + lx -> storage column
    int* rowmap = colmap + W4;                                   // y0 - 4 + ly -> storage row

    const int nx = g.nx, ny = g.ny, nz = g.nz, pitch = g.pitch, walls = g.walls;
    const int plane = (int)g.plane;                  // one population field (Q * padded sites < 2^31)
    const int zs = ny * pitch;                      // one z plane
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * Hz, z1 = min(z0 + Hz, nz);
    const int kbeg = z0 - 4, kend = z1 + 3;
    const R half = R(0.5);
    bool bad = false;

    for (int q = threadIdx.x; q < W4 + P3::H4; q += NT) {
        if (q < W4) colmap[q] = wrap_any3(x0 - 4 + q, nx);
        else rowmap[q - W4] = wrap_any3(y0 - 4 + (q - W4), ny);
    }
    __syncthreads();

    // plane ring slots are counted from kbeg
    auto ring = [&](int z, int n) { return (z - kbeg) % n; };

    auto fetch = [&](int z) {             // phi (r = 4) and T (r = 2) of plane z
        if (z <= kend) {
            const int gz = map_axis3(z, nz, walls);
            R* dphi = sphi + ring(z, P3::NPHI) * A4;
            R* dT = sT + ring(z, P3::NT_) * A2;
            for (int q = threadIdx.x; q < A4; q += NT) {
                const int ly = q / W4, lx = q - ly * W4;
                const int off = gz * zs + rowmap[ly] * pitch + colmap[lx];
                cp_async3<sizeof(R)>(&dphi[q], io.phi_in + off);
                if (lx >= 2 && lx < W4 - 2 && ly >= 2 && ly < P3::H4 - 2)
                    cp_async3<sizeof(R)>(&dT[(ly - 2) * W2 + lx - 2], io.T_in + off);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    fetch(kbeg);
    for (int k = kbeg; k <= kend; ++k) {
        // plane k has landed (own copies), and after the barrier every thread's
        // copies are visible and every read of the previous iteration is done,
        // so the prefetch of plane k + 1 may overwrite the oldest slot.
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        fetch(k + 1);
        const R* phk = sphi + ring(k, P3::NPHI) * A4;
        const R* phm1 = sphi + ring(k + P3::NPHI - 1, P3::NPHI) * A4;   // plane k-1
        const R* phm2 = sphi + ring(k + P3::NPHI - 2, P3::NPHI) * A4;
        const R* phm3 = sphi + ring(k + P3::NPHI - 3, P3::NPHI) * A4;
        const R* phm4 = sphi + ring(k + P3::NPHI - 4, P3::NPHI) * A4;

        // ---- plane k-1: psi (r = 3), T(t+1) (r = 0) -------------------------
        const int z1p = k - 1;
        if (z1p >= z0 - 3 && z1p <= z1 + 2) {
            R* dst = spsi + ring(z1p, 3) * A3;
            for (int q = threadIdx.x; q < A3; q += NT) {
                const int ly = q / W3, lx = q - ly * W3;
                const int c = (ly + 1) * W4 + lx + 1;
                if constexpr (ISO)
                    dst[q] = lap19<R, W4>(phm2, phm1, phk, c);
                else
                    dst[q] = phm1[c - 1] + phm1[c + 1] + phm1[c - W4] + phm1[c + W4] + phm2[c] + phk[c]
                           - R(6) * phm1[c];
            }
        }
        if (!AUX && z1p >= z0 && z1p < z1) {
            const R* t0 = sT + ring(z1p, P3::NT_) * A2;
            const R* tu = sT + ring(k, P3::NT_) * A2;
            const R* td = sT + ring(z1p + P3::NT_ - 1, P3::NT_) * A2;
            for (int q = threadIdx.x; q < TX * TY; q += NT) {
                const int ly = q / TX, lx = q - ly * TX;
                const int gx = x0 + lx, gy = y0 + ly;
                if (gx >= nx || gy >= ny) continue;
                const int c = (ly + 2) * W2 + lx + 2;
                const R Tc0 = t0[c];
                R Tn = Tc0;
                if (p.t_update) {
                    if (walls && g.t_mode == LF_TWALL_LAYERS && (z1p == 0 || z1p == nz - 1)) {
                        Tn = p.T_w;
                    } else if constexpr (ISO) {
                        // halfway ghosts: 2 T_w minus the mirror image the halo plane holds
                        const bool lo = walls && g.t_mode == LF_TWALL_HALFWAY && z1p == 0;
                        const bool hi = walls && g.t_mode == LF_TWALL_HALFWAY && z1p == nz - 1;
                        const R tw2 = R(2) * p.T_w;
                        auto vd = [&](int o) { return lo ? tw2 - td[c + o] : td[c + o]; };
                        auto vu = [&](int o) { return hi ? tw2 - tu[c + o] : tu[c + o]; };
                        const R nn = t0[c - 1] + t0[c + 1] + t0[c - W2] + t0[c + W2] + vd(0) + vu(0);
                        const R ed = (t0[c - W2 - 1] + t0[c - W2 + 1] + t0[c + W2 - 1] + t0[c + W2 + 1])
                                   + (vd(-1) + vd(1) + vd(-W2) + vd(W2)) + (vu(-1) + vu(1) + vu(-W2) + vu(W2));
                        Tn = Tc0 + p.dxi * ((R(2) * nn + ed - R(24) * Tc0) * R(1.0 / 6.0));
                    } else {
                        R up = tu[c], dn = td[c];
                        if (walls && g.t_mode == LF_TWALL_HALFWAY) {
                            if (z1p == 0) dn = R(2) * p.T_w - Tc0;
                            if (z1p == nz - 1) up = R(2) * p.T_w - Tc0;
                        }
                        Tn = Tc0 + p.dxi * (t0[c - 1] + t0[c + 1] + t0[c - W2] + t0[c + W2] + up + dn - R(6) * Tc0);
                    }
                }
                bad |= !isfinite(Tn);
                io.T_out[z1p * zs + gy * pitch + gx] = Tn;
            }
        }
        __syncthreads();

        // ---- plane k-2: lam, P, mu (r = 2) ------------------------------------
        const int z2 = k - 2;
        if (z2 >= z0 - 2 && z2 <= z1 + 1) {
            const R* ps0 = spsi + ring(z2, 3) * A3;
            const R* psu = spsi + ring(z2 + 1, 3) * A3;
            const R* psd = spsi + ring(z2 + 2, 3) * A3;      // plane z2 - 1 (mod 3)
            const R* tz = sT + ring(z2, P3::NT_) * A2;
            const int pin = ring(z2, NPIN), pz = ring(z2, 3);
            R* mu_dst = smu + ring(z2, 4) * A1;
            for (int q = threadIdx.x; q < A2; q += NT) {
                const int ly = q / W2, lx = q - ly * W2;
                const int cp = (ly + 2) * W4 + lx + 2;
                const int cs = (ly + 1) * W3 + lx + 1;
                const R ph = phm2[cp], psi = ps0[cs];
                R lam;
                if constexpr (ISO)
                    lam = lap19<R, W3>(psd, ps0, psu, cs);
                else
                    lam = ps0[cs - 1] + ps0[cs + 1] + ps0[cs - W3] + ps0[cs + W3] + psu[cs] + psd[cs] - R(6) * psi;
                const R av = (tz[q] - p.Tc) * p.inv_Tc;
                const R mu = av * ph + p.b * ph * ph * ph - p.kappa * psi + p.c * lam;
                if (lx >= 1 && lx < W2 - 1 && ly >= 1 && ly < P3::H2 - 1) mu_dst[(ly - 1) * W1 + lx - 1] = mu;
                if (AUX || p.hydro) {
                    R d0, d1, d2, s0, s1, s2;
                    if constexpr (ISO) {
                        d0 = grad19<R, W4>(phm3, phm2, phm1, cp, 0);
                        d1 = grad19<R, W4>(phm3, phm2, phm1, cp, 1);
                        d2 = grad19<R, W4>(phm3, phm2, phm1, cp, 2);
                        s0 = grad19<R, W3>(psd, ps0, psu, cs, 0);
                        s1 = grad19<R, W3>(psd, ps0, psu, cs, 1);
                        s2 = grad19<R, W3>(psd, ps0, psu, cs, 2);
                    } else {
                        d0 = half * (phm2[cp + 1] - phm2[cp - 1]);
                        d1 = half * (phm2[cp + W4] - phm2[cp - W4]);
                        d2 = half * (phm1[cp] - phm3[cp]);
                        s0 = half * (ps0[cs + 1] - ps0[cs - 1]);
                        s1 = half * (ps0[cs + W3] - ps0[cs - W3]);
                        s2 = half * (psu[cs] - psd[cs]);
                    }
                    const R ph2 = ph * ph;
                    const R iso = av * ph2 * half + R(0.75) * p.b * ph2 * ph2
                                - p.kappa * (ph * psi + half * (d0 * d0 + d1 * d1 + d2 * d2))
                                + p.c * (ph * lam + half * psi * psi + d0 * s0 + d1 * s1 + d2 * s2);
                    sPin[(0 * NPIN + pin) * A2 + q] = iso + p.kappa * d0 * d0 - R(2) * p.c * d0 * s0;
                    sPin[(1 * NPIN + pin) * A2 + q] = p.kappa * d0 * d1 - p.c * (d0 * s1 + d1 * s0);
                    sPin[(2 * NPIN + pin) * A2 + q] = iso + p.kappa * d1 * d1 - R(2) * p.c * d1 * s1;
                    sPz[(0 * 3 + pz) * A2 + q] = p.kappa * d0 * d2 - p.c * (d0 * s2 + d2 * s0);
                    sPz[(1 * 3 + pz) * A2 + q] = p.kappa * d1 * d2 - p.c * (d1 * s2 + d2 * s1);
                    sPz[(2 * 3 + pz) * A2 + q] = iso + p.kappa * d2 * d2 - R(2) * p.c * d2 * s2;
                }
            }
        }
        __syncthreads();

        // ---- plane k-3: F, u, g (r = 1); collide and push (r = 0) -------------
        const int z3 = k - 3;
        if ((AUX || p.hydro) && z3 >= z0 - 1 && z3 <= z1) {
            const bool ghost = walls && (z3 < 0 || z3 >= nz);
            const int pin = ring(z3, NPIN);
            const int pz0 = ring(z3, 3), pzu = ring(z3 + 1, 3), pzd = ring(z3 + 2, 3);
            R* gx_dst = sgxy + (0 * NPIN + ring(z3, NPIN)) * A1;
            R* gy_dst = sgxy + (1 * NPIN + ring(z3, NPIN)) * A1;
            R* gz_dst = sgz + ring(z3, 3) * A1;
            const int gzp = ghost ? 0 : (walls ? z3 : map_axis3(z3, nz, 0));
            for (int q = threadIdx.x; q < A1; q += NT) {
                const int ly = q / W1, lx = q - ly * W1;
                const bool ex_ = (lx == 0 || lx == W1 - 1), ey_ = (ly == 0 || ly == P3::H1 - 1);
                if (!ISO && ex_ && ey_) continue;            // corners: only the isotropic divergence reads them
                R gxv = 0, gyv = 0, gzv = 0;
                if (!ghost) {
                    const int c2 = (ly + 1) * W2 + lx + 1;
                    const R* Pxx = sPin + (0 * NPIN + pin) * A2;
                    const R* Pxy = sPin + (1 * NPIN + pin) * A2;
                    const R* Pyy = sPin + (2 * NPIN + pin) * A2;
                    R Fx, Fy, Fz;
                    if constexpr (ISO) {
                        // F_b = -d_a P_ab on the planes z3 - 1, z3, z3 + 1 of every component
                        const int pu = ring(z3 + 1, NPIN), pd = ring(z3 + 2, NPIN);
                        auto Pin3 = [&](int comp, int slot) { return sPin + (comp * NPIN + slot) * A2; };
                        auto Pz3 = [&](int comp, int slot) { return sPz + (comp * 3 + slot) * A2; };
                        Fx = -(grad19<R, W2>(Pin3(0, pd), Pxx, Pin3(0, pu), c2, 0)
                               + grad19<R, W2>(Pin3(1, pd), Pxy, Pin3(1, pu), c2, 1)
                               + grad19<R, W2>(Pz3(0, pzd), Pz3(0, pz0), Pz3(0, pzu), c2, 2));
                        Fy = -(grad19<R, W2>(Pin3(1, pd), Pxy, Pin3(1, pu), c2, 0)
                               + grad19<R, W2>(Pin3(2, pd), Pyy, Pin3(2, pu), c2, 1)
                               + grad19<R, W2>(Pz3(1, pzd), Pz3(1, pz0), Pz3(1, pzu), c2, 2));
                        Fz = -(grad19<R, W2>(Pz3(0, pzd), Pz3(0, pz0), Pz3(0, pzu), c2, 0)
                               + grad19<R, W2>(Pz3(1, pzd), Pz3(1, pz0), Pz3(1, pzu), c2, 1)
                               + grad19<R, W2>(Pz3(2, pzd), Pz3(2, pz0), Pz3(2, pzu), c2, 2));
                    } else {
                        Fx = -(half * (Pxx[c2 + 1] - Pxx[c2 - 1]) + half * (Pxy[c2 + W2] - Pxy[c2 - W2])
                               + half * (sPz[(0 * 3 + pzu) * A2 + c2] - sPz[(0 * 3 + pzd) * A2 + c2]));
                        Fy = -(half * (Pxy[c2 + 1] - Pxy[c2 - 1]) + half * (Pyy[c2 + W2] - Pyy[c2 - W2])
                               + half * (sPz[(1 * 3 + pzu) * A2 + c2] - sPz[(1 * 3 + pzd) * A2 + c2]));
                        Fz = -(half * (sPz[(0 * 3 + pz0) * A2 + c2 + 1] - sPz[(0 * 3 + pz0) * A2 + c2 - 1])
                               + half * (sPz[(1 * 3 + pz0) * A2 + c2 + W2] - sPz[(1 * 3 + pz0) * A2 + c2 - W2])
                               + half * (sPz[(2 * 3 + pzu) * A2 + c2] - sPz[(2 * 3 + pzd) * A2 + c2]));
                    }
                    const int ux = x0 - 1 + lx, uy = y0 - 1 + ly;
                    const int gx = colmap[lx + 3], gy = rowmap[ly + 3];
                    const int site = gzp * zs + gy * pitch + gx;
                    R df[L::Q];
                    R dn = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
                    for (int i = 0; i < L::Q; ++i) {
                        df[i] = io.f_in[i * plane + site];
                        dn += df[i];
                        jx += R(L::ex(i)) * df[i];
                        jy += R(L::ey(i)) * df[i];
                        jz += R(L::ez(i)) * df[i];
                    }
                    const R n = p.n0 + dn;
                    const R inv_n = recip3(n);
                    const bool hyd = p.hydro != 0;
                    const R vx = hyd ? (jx + half * Fx) * inv_n : R(0);
                    const R vy = hyd ? (jy + half * Fy) * inv_n : R(0);
                    const R vz = hyd ? (jz + half * Fz) * inv_n : R(0);
                    const R ph = phm3[(ly + 3) * W4 + lx + 3];
                    gxv = ph * vx;
                    gyv = ph * vy;
                    gzv = ph * vz;
                    const bool inner = !ex_ && !ey_ && ux < nx && uy < ny && z3 >= z0 && z3 < z1;
                    if (inner) {
                        bad |= !isfinite(n);
                        if (AUX) {
                            io.rho[site] = n;
                            io.u[0][site] = vx; io.u[1][site] = vy; io.u[2][site] = vz;
                            io.F[0][site] = Fx; io.F[1][site] = Fy; io.F[2][site] = Fz;
                        } else if (hyd) {
                            // Eq. evoleqn with the Qian equilibrium and Guo's term, written per
                            // opposite pair (i, i'): f*_i = (1 - w) df_i + w_i (sym +- anti)
                            const R omega = p.inv_tau, keep = R(1) - p.inv_tau;
                            const R on = omega * n;
                            const R C0 = omega * dn - R(1.5) * on * (vx * vx + vy * vy + vz * vz)
                                       - R(3) * p.guo * (vx * Fx + vy * Fy + vz * Fz);
                            const R a3 = R(3) * on, a45 = R(4.5) * on, g3 = R(3) * p.guo, g9 = R(9) * p.guo;
                            const int gxp = colmap[lx + 4], gxm = colmap[lx + 2];
                            const int gyp = rowmap[ly + 4], gym = rowmap[ly + 2];
                            const int gzu = gzp + 1 == nz ? 0 : gzp + 1, gzd = gzp == 0 ? nz - 1 : gzp - 1;
                            const bool wall_lo = walls && gzp == 0, wall_hi = walls && gzp == nz - 1;
                            R* out = io.f_out;
                            out[site] = keep * df[0] + R(L::w(0)) * C0;
                            auto dest = [&](int ex, int ey, int ez) -> int {
                                const int tx = ex > 0 ? gxp : (ex < 0 ? gxm : gx);
                                const int ty = ey > 0 ? gyp : (ey < 0 ? gym : gy);
                                const int tz = ez > 0 ? gzu : (ez < 0 ? gzd : gzp);
                                return tz * zs + ty * pitch + tx;
                            };
#pragma unroll
                            for (int i = 1; i < L::Q; i += 2) {           // (i, i + 1) are opposite
                                const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
                                const R sv = R(ex) * vx + R(ey) * vy + R(ez) * vz;
                                const R ev = R(ex) * Fx + R(ey) * Fy + R(ez) * Fz;
                                const R sym = C0 + sv * (a45 * sv + g9 * ev);
                                const R anti = a3 * sv + g3 * ev;
                                const R wi = R(L::w(i));
                                const R pi = keep * df[i] + wi * (sym + anti);
                                const R pj = keep * df[i + 1] + wi * (sym - anti);
                                const bool bb_i = (ez > 0 && wall_hi) || (ez < 0 && wall_lo);
                                const bool bb_j = (ez < 0 && wall_hi) || (ez > 0 && wall_lo);
                                if (bb_i) out[(i + 1) * plane + site] = pi;   // halfway bounce-back
                                else out[i * plane + dest(ex, ey, ez)] = pi;
                                if (bb_j) out[i * plane + site] = pj;
                                else out[(i + 1) * plane + dest(-ex, -ey, -ez)] = pj;
                            }
                        }
                    }
                }
                gx_dst[q] = gxv;
                gy_dst[q] = gyv;
                gz_dst[q] = gzv;
            }
        }
        __syncthreads();

        // ---- plane k-4: phi(t+1) (r = 0) ---------------------------------------
        const int z4 = k - 4;
        if (z4 >= z0 && z4 < z1) {
            const R* mu0 = smu + ring(z4, 4) * A1;
            const R* muu = smu + ring(z4 + 1, 4) * A1;
            const R* mud = smu + ring(z4 + 3, 4) * A1;        // plane z4 - 1 (mod 4)
            const R* gx0 = sgxy + (0 * NPIN + ring(z4, NPIN)) * A1;
            const R* gy0 = sgxy + (1 * NPIN + ring(z4, NPIN)) * A1;
            const R* gz0 = sgz + ring(z4, 3) * A1;
            const R* gzu = sgz + ring(z4 + 1, 3) * A1;
            const R* gzd = sgz + ring(z4 + 2, 3) * A1;        // plane z4 - 1 (mod 3)
            for (int q = threadIdx.x; q < TX * TY; q += NT) {
                const int ly = q / TX, lx = q - ly * TX;
                const int gx = x0 + lx, gy = y0 + ly;
                if (gx >= nx || gy >= ny) continue;
                const int c1 = (ly + 1) * W1 + lx + 1;
                const int site = z4 * zs + gy * pitch + gx;
                if (AUX) {
                    io.mu[site] = mu0[c1];
                    continue;
                }
                if constexpr (ISO) {
                    const R lapmu = lap19<R, W1>(mud, mu0, muu, c1);
                    R div = 0;
                    if (p.hydro) {
                        // planes beyond a wall: the image of the wall plane (g_x, g_y even, g_z odd)
                        const bool lo = walls && z4 == 0, hi = walls && z4 == nz - 1;
                        const int su = ring(z4 + 1, NPIN), sd = ring(z4 + NPIN - 1, NPIN);
                        const R* gxd = lo ? gx0 : sgxy + (0 * NPIN + sd) * A1;
                        const R* gxu = hi ? gx0 : sgxy + (0 * NPIN + su) * A1;
                        const R* gyd = lo ? gy0 : sgxy + (1 * NPIN + sd) * A1;
                        const R* gyu = hi ? gy0 : sgxy + (1 * NPIN + su) * A1;
                        const R* gzd_ = lo ? gz0 : gzd;
                        const R* gzu_ = hi ? gz0 : gzu;
                        const R sgd = lo ? R(-1) : R(1), sgu = hi ? R(-1) : R(1);
                        auto zd = [&](int o) { return sgd * gzd_[c1 + o]; };
                        auto zu = [&](int o) { return sgu * gzu_[c1 + o]; };
                        const R dz = (R(2) * (zu(0) - zd(0)) + (zu(1) - zd(1)) + (zu(-1) - zd(-1))
                                      + (zu(W1) - zd(W1)) + (zu(-W1) - zd(-W1))) * R(1.0 / 12.0);
                        div = grad19<R, W1>(gxd, gx0, gxu, c1, 0) + grad19<R, W1>(gyd, gy0, gyu, c1, 1) + dz;
                    }
                    const R phn = phm4[(ly + 4) * W4 + lx + 4] - div + p.Gamma * lapmu;
                    bad |= !isfinite(phn);
                    io.phi_out[site] = phn;
                    continue;
                }
                const R lapmu = mu0[c1 - 1] + mu0[c1 + 1] + mu0[c1 - W1] + mu0[c1 + W1] + muu[c1] + mud[c1]
                              - R(6) * mu0[c1];
                R div = 0;
                if (p.hydro) {
                    R up = gzu[c1], dn = gzd[c1];
                    if (walls) {                                  // no flux through the walls
                        if (z4 == 0) dn = -gz0[c1];
                        if (z4 == nz - 1) up = -gz0[c1];
                    }
                    div = half * (gx0[c1 + 1] - gx0[c1 - 1]) + half * (gy0[c1 + W1] - gy0[c1 - W1])
                        + half * (up - dn);
                }
                const R phn = phm4[(ly + 4) * W4 + lx + 4] - div + p.Gamma * lapmu;
                bad |= !isfinite(phn);
                io.phi_out[site] = phn;
            }
        }
        // the barrier at the top of the next iteration orders the rings
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *reinterpret_cast<volatile int*>(io.flag) = 1;
}

template <typename R, int TX, int TY, int NT, bool AUX, bool ISO>
cudaError_t launch_cfg3(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s)
{
    using P3 = Plane3<R, TX, TY, ISO>;
    auto kern = k_march3d<R, TX, TY, NT, AUX, ISO>;
    static unsigned long long attr_done = 0;      // per instantiation and device
    const cudaError_t e = raise_smem_limit(kern, (int)P3::BYTES, &attr_done);
    if (e != cudaSuccess) return e;
    const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    int Hz = g.tune > 0 ? g.tune : g.nz;
    if (g.tune <= 0) {   // about eight waves of three CTAs per SM, segments of at least 16 planes
        const int want = (8 * 3 * 152 + tiles - 1) / tiles;
        Hz = (g.nz + want - 1) / want;
        if (Hz < 16) Hz = 16;
    }
    if (Hz > g.nz) Hz = g.nz;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + Hz - 1) / Hz);
    kern<<<grid, NT, P3::BYTES, s>>>(g, p, io, Hz);
    return cudaGetLastError();
}

template <typename R>
__global__ void k_tsub3d(Geom g, Phys<R> p, const R* __restrict__ Tin, R* __restrict__ Tout)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int nx = g.nx, ny = g.ny, nz = g.nz, pitch = g.pitch;
    const int zs = ny * pitch;                   // 32-bit offsets: Q * padded sites < 2^31 (checked at creation)
    const int site = z * zs + y * pitch + x;
    const R t0 = Tin[site];
    if (g.walls && g.t_mode == LF_TWALL_LAYERS && (z == 0 || z == nz - 1)) {
        Tout[site] = p.T_w;
        return;
    }
    const int xl = x == 0 ? nx - 1 : x - 1, xr = x == nx - 1 ? 0 : x + 1;
    const int yl = y == 0 ? ny - 1 : y - 1, yr = y == ny - 1 ? 0 : y + 1;
    R td, tu;
    if (g.walls) {
        td = z == 0 ? R(2) * p.T_w - t0 : Tin[site - zs];
        tu = z == nz - 1 ? R(2) * p.T_w - t0 : Tin[site + zs];
    } else {
        td = Tin[(z == 0 ? nz - 1 : z - 1) * zs + y * pitch + x];
        tu = Tin[(z == nz - 1 ? 0 : z + 1) * zs + y * pitch + x];
    }
    const int row = z * zs;
    Tout[site] = t0 + p.dxi * (Tin[row + y * pitch + xl] + Tin[row + y * pitch + xr] +
                               Tin[row + yl * pitch + x] + Tin[row + yr * pitch + x] + tu + td -
                               R(6) * t0);
}

// The same sub-step with the isotropic 19-point Laplacian; a plane beyond a
// wall holds 2 T_w - T of the wall plane (halfway ghost).
template <typename R>
__global__ void k_tsub3d_iso(Geom g, Phys<R> p, const R* __restrict__ Tin, R* __restrict__ Tout)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int nx = g.nx, ny = g.ny, nz = g.nz, pitch = g.pitch;
    const int zs = ny * pitch;                   // 32-bit offsets: Q * padded sites < 2^31 (checked at creation)
    const int site = z * zs + y * pitch + x;
    const R t0 = Tin[site];
    if (g.walls && g.t_mode == LF_TWALL_LAYERS && (z == 0 || z == nz - 1)) {
        Tout[site] = p.T_w;
        return;
    }
    const int xl = x == 0 ? nx - 1 : x - 1, xr = x == nx - 1 ? 0 : x + 1;
    const int yl = y == 0 ? ny - 1 : y - 1, yr = y == ny - 1 ? 0 : y + 1;
    const bool lo = g.walls && z == 0, hi = g.walls && z == nz - 1;
    const int zd = lo ? 0 : (z == 0 ? nz - 1 : z - 1);
    const int zu = hi ? z : (z == nz - 1 ? 0 : z + 1);
    const R tw2 = R(2) * p.T_w;
    auto at = [&](int zz, int yy, int xx) { return Tin[zz * zs + yy * pitch + xx]; };
    auto dn = [&](int yy, int xx) { return lo ? tw2 - at(zd, yy, xx) : at(zd, yy, xx); };
    auto up = [&](int yy, int xx) { return hi ? tw2 - at(zu, yy, xx) : at(zu, yy, xx); };
    const R nn = at(z, y, xl) + at(z, y, xr) + at(z, yl, x) + at(z, yr, x) + dn(y, x) + up(y, x);
    const R ed = (at(z, yl, xl) + at(z, yl, xr) + at(z, yr, xl) + at(z, yr, xr))
               + (dn(y, xl) + dn(y, xr) + dn(yl, x) + dn(yr, x)) + (up(y, xl) + up(y, xr) + up(yl, x) + up(yr, x));
    Tout[site] = t0 + p.dxi * ((R(2) * nn + ed - R(24) * t0) * R(1.0 / 6.0));
}

}  // namespace

template <typename R>
cudaError_t launch_step3d(const Geom& g, const Phys<R>& p, const StepIO<R>& io, bool aux, cudaStream_t s)
{
    if (!aux && g.variant == LF_VARIANT_SPLIT3) return launch_split3d<R>(g, p, io, s);
    if (g.stencil == LF_STENCIL_ISOTROPIC) {
        if constexpr (sizeof(R) == 4)
            return aux ? launch_cfg3<R, 32, 8, 256, true, true>(g, p, io, s)
                       : launch_cfg3<R, 32, 8, 256, false, true>(g, p, io, s);
        else
            return aux ? launch_cfg3<R, 16, 16, 256, true, true>(g, p, io, s)
                       : launch_cfg3<R, 16, 16, 256, false, true>(g, p, io, s);
    }
    if constexpr (sizeof(R) == 4) {
        return aux ? launch_cfg3<R, 32, 8, 256, true, false>(g, p, io, s)
                   : launch_cfg3<R, 32, 8, 256, false, false>(g, p, io, s);
    } else {
        return aux ? launch_cfg3<R, 16, 16, 256, true, false>(g, p, io, s)
                   : launch_cfg3<R, 16, 16, 256, false, false>(g, p, io, s);
    }
}

template <typename R>
cudaError_t launch_tsub3d(const Geom& g, const Phys<R>& p, const R* Tin, R* Tout, cudaStream_t s)
{
    dim3 blk(32, 8), grd((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    if (g.stencil == LF_STENCIL_ISOTROPIC)
        k_tsub3d_iso<R><<<grd, blk, 0, s>>>(g, p, Tin, Tout);
    else
        k_tsub3d<R><<<grd, blk, 0, s>>>(g, p, Tin, Tout);
    return cudaGetLastError();
}

template cudaError_t launch_step3d<float>(const Geom&, const Phys<float>&, const StepIO<float>&, bool, cudaStream_t);
template cudaError_t launch_step3d<double>(const Geom&, const Phys<double>&, const StepIO<double>&, bool, cudaStream_t);
template cudaError_t launch_tsub3d<float>(const Geom&, const Phys<float>&, const float*, float*, cudaStream_t);
template cudaError_t launch_tsub3d<double>(const Geom&, const Phys<double>&, const double*, double*, cudaStream_t);

}  // namespace lf
