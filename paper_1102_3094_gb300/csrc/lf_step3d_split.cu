// lf_step3d_split.cu -- the D3Q19 time step of arXiv:1102.3094, Sec. 2, as
// three passes (LF_VARIANT_SPLIT3):
//   A  k_force3d: mu and F = -d_a P_ab from phi(t), T(t) (Eqs. chem, ff);
//      a plane march along z over an (x, y) tile, the stencil chain
//      psi (r = 2) -> lam, P (r = 1) -> F, mu (r = 0) in shared memory;
//   B  k_lb3d: n, u = (sum f e + F/2)/n, BGK + Guo collision and push
//      streaming with halfway bounce-back (Eqs. moment, evoleqn,
//      latticeforceterm), one thread per site; writes u(t);
//   C  k_phi3d: phi(t+1) = phi - div(phi u) + Gamma lap(mu) (Eq. massdiff)
//      and the first temperature sub-step, one thread per site.
// mu, F and u pass through the context's aux planes.  The arithmetic per site
// is that of the fused plane march (lf_step3d.cu), with the same wall rules:
// even reflection of phi, T and every derived scalar about the half-way
// planes (so mu(-1) = mu(0)), odd reflection of the wall-normal flux, halfway
// bounce-back of the populations.  Every stage covers only the region its
// consumer needs: psi on the tile + 2, P on the tile + 1, F and mu on the
// tile, against + 3 / + 2 / + 1 in the fused kernel, and no population is
// read outside its own site.
#include "lf_internal.cuh"

namespace lf {

namespace {

__device__ __forceinline__ int wrap_s(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

__device__ __forceinline__ int map_z(int v, int n, int walls)
{
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

template <typename R, int TX, int TY>
struct Force3 {
    static constexpr int W3 = TX + 6, H3 = TY + 6, A3 = W3 * H3;   // phi (r = 3)
    static constexpr int W2 = TX + 4, H2 = TY + 4, A2 = W2 * H2;   // psi (r = 2)
    static constexpr int W1 = TX + 2, H1 = TY + 2, A1 = W1 * H1;   // T, lam, P (r = 1)
    static constexpr int NPHI = 5;                                  // planes k-3 .. k+1
    static constexpr int NT = 4;                                    // T planes k-2 .. k+1
    static constexpr int PHI = 0;
    static constexpr int TT = PHI + NPHI * A3;
    static constexpr int PSI = TT + NT * A1;                        // 3 planes
    static constexpr int PIN = PSI + 3 * A2;                        // xx, xy, yy: 2 planes each
    static constexpr int PZ = PIN + 6 * A1;                         // xz, yz, zz: 3 planes each
    static constexpr int TOTAL = PZ + 9 * A1;
    static constexpr size_t MAPS = sizeof(R) * TOTAL;
    static constexpr size_t BYTES = MAPS + sizeof(int) * (W3 + H3);
};

// Pass A.  A CTA owns a TX x TY tile and marches along z over [z0, z1):
// iteration k prefetches phi / T of plane k + 1 and runs psi on plane k - 1,
// lam / P / mu on plane k - 2 and F on plane k - 3.
template <typename R, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) k_force3d(Geom g, Phys<R> p, StepIO<R> io, int Hz)
{
    using P3 = Force3<R, TX, TY>;
    constexpr int W3 = P3::W3, W2 = P3::W2, W1 = P3::W1;
    constexpr int A3 = P3::A3, A2 = P3::A2, A1 = P3::A1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    R* sphi = sm + P3::PHI;
    R* sT = sm + P3::TT;
    R* spsi = sm + P3::PSI;
    R* sPin = sm + P3::PIN;   // [comp 0..2][plane parity][A1]: xx, xy, yy
    R* sPz = sm + P3::PZ;     // [comp 0..2][plane mod 3][A1]: xz, yz, zz
    int* colmap = reinterpret_cast<int*>(smem_raw + P3::MAPS);   // x0 - 3 + lx -> storage column
    int* rowmap = colmap + W3;                                   // y0 - 3 + ly -> storage row

    const int nx = g.nx, ny = g.ny, nz = g.nz, pitch = g.pitch, walls = g.walls;
    const int64_t zs = (int64_t)ny * pitch;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * Hz, z1 = min(z0 + Hz, nz);
    const int kbeg = z0 - 3, kend = z1 + 2;
    const R half = R(0.5);
    bool bad = false;

    for (int q = threadIdx.x; q < W3 + P3::H3; q += NT) {
        if (q < W3) colmap[q] = wrap_s(x0 - 3 + q, nx);
        else rowmap[q - W3] = wrap_s(y0 - 3 + (q - W3), ny);
    }
    __syncthreads();

    auto ring = [&](int z, int n) { return (z - kbeg + 3 * n) % n; };
    auto fetch = [&](int z) {             // phi (r = 3) and T (r = 1) of plane z
        if (z <= kend) {
            const int gz = map_z(z, nz, walls);
            R* dphi = sphi + ring(z, P3::NPHI) * A3;
            R* dT = sT + ring(z, P3::NT) * A1;
            for (int q = threadIdx.x; q < A3; q += NT) {
                const int ly = q / W3, lx = q - ly * W3;
                const int64_t off = gz * zs + (int64_t)rowmap[ly] * pitch + colmap[lx];
                cp_async_s<sizeof(R)>(&dphi[q], io.phi_in + off);
                if (lx >= 2 && lx < W3 - 2 && ly >= 2 && ly < P3::H3 - 2)
                    cp_async_s<sizeof(R)>(&dT[(ly - 2) * W1 + lx - 2], io.T_in + off);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    fetch(kbeg);
    for (int k = kbeg; k <= kend; ++k) {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        fetch(k + 1);
        const R* phk = sphi + ring(k, P3::NPHI) * A3;
        const R* phm1 = sphi + ring(k - 1, P3::NPHI) * A3;
        const R* phm2 = sphi + ring(k - 2, P3::NPHI) * A3;
        const R* phm3 = sphi + ring(k - 3, P3::NPHI) * A3;

        // ---- plane k-1: psi (r = 2) ------------------------------------------
        const int z1p = k - 1;
        if (z1p >= z0 - 2 && z1p <= z1 + 1) {
            R* dst = spsi + ring(z1p, 3) * A2;
            for (int q = threadIdx.x; q < A2; q += NT) {
                const int ly = q / W2, lx = q - ly * W2;
                const int c = (ly + 1) * W3 + lx + 1;
                dst[q] = phm1[c - 1] + phm1[c + 1] + phm1[c - W3] + phm1[c + W3] + phm2[c] + phk[c]
                       - R(6) * phm1[c];
            }
        }
        __syncthreads();

        // ---- plane k-2: lam, P (r = 1), mu (r = 0) ------------------------------
        const int z2 = k - 2;
        if (z2 >= z0 - 1 && z2 <= z1) {
            const R* ps0 = spsi + ring(z2, 3) * A2;
            const R* psu = spsi + ring(z2 + 1, 3) * A2;
            const R* psd = spsi + ring(z2 - 1, 3) * A2;
            const R* tz = sT + ring(z2, P3::NT) * A1;
            const int pin = ring(z2, 2), pz = ring(z2, 3);
            const bool mu_plane = z2 >= z0 && z2 < z1;
            for (int q = threadIdx.x; q < A1; q += NT) {
                const int ly = q / W1, lx = q - ly * W1;
                const int cp = (ly + 2) * W3 + lx + 2;
                const int cs = (ly + 1) * W2 + lx + 1;
                const R ph = phm2[cp], psi = ps0[cs];
                const R lam = ps0[cs - 1] + ps0[cs + 1] + ps0[cs - W2] + ps0[cs + W2] + psu[cs] + psd[cs] - R(6) * psi;
                const R av = (tz[q] - p.Tc) * p.inv_Tc;
                if (mu_plane && lx >= 1 && lx < W1 - 1 && ly >= 1 && ly < P3::H1 - 1) {
                    const int gx = x0 + lx - 1, gy = y0 + ly - 1;
                    if (gx < nx && gy < ny) {
                        const R mu = av * ph + p.b * ph * ph * ph - p.kappa * psi + p.c * lam;
                        bad |= !isfinite(mu);
                        io.mu[z2 * zs + (int64_t)gy * pitch + gx] = mu;
                    }
                }
                if (p.hydro) {
                    const R d0 = half * (phm2[cp + 1] - phm2[cp - 1]);
                    const R d1 = half * (phm2[cp + W3] - phm2[cp - W3]);
                    const R d2 = half * (phm1[cp] - phm3[cp]);
                    const R s0 = half * (ps0[cs + 1] - ps0[cs - 1]);
                    const R s1 = half * (ps0[cs + W2] - ps0[cs - W2]);
                    const R s2 = half * (psu[cs] - psd[cs]);
                    const R ph2 = ph * ph;
                    const R iso = av * ph2 * half + R(0.75) * p.b * ph2 * ph2
                                - p.kappa * (ph * psi + half * (d0 * d0 + d1 * d1 + d2 * d2))
                                + p.c * (ph * lam + half * psi * psi + d0 * s0 + d1 * s1 + d2 * s2);
                    sPin[(0 * 2 + pin) * A1 + q] = iso + p.kappa * d0 * d0 - R(2) * p.c * d0 * s0;
                    sPin[(1 * 2 + pin) * A1 + q] = p.kappa * d0 * d1 - p.c * (d0 * s1 + d1 * s0);
                    sPin[(2 * 2 + pin) * A1 + q] = iso + p.kappa * d1 * d1 - R(2) * p.c * d1 * s1;
                    sPz[(0 * 3 + pz) * A1 + q] = p.kappa * d0 * d2 - p.c * (d0 * s2 + d2 * s0);
                    sPz[(1 * 3 + pz) * A1 + q] = p.kappa * d1 * d2 - p.c * (d1 * s2 + d2 * s1);
                    sPz[(2 * 3 + pz) * A1 + q] = iso + p.kappa * d2 * d2 - R(2) * p.c * d2 * s2;
                }
            }
        }
        __syncthreads();

        // ---- plane k-3: F (r = 0) -----------------------------------------------
        const int z3 = k - 3;
        if (p.hydro && z3 >= z0 && z3 < z1) {
            const int pin = ring(z3, 2);
            const int pz0 = ring(z3, 3), pzu = ring(z3 + 1, 3), pzd = ring(z3 - 1, 3);
            const R* Pxx = sPin + (0 * 2 + pin) * A1;
            const R* Pxy = sPin + (1 * 2 + pin) * A1;
            const R* Pyy = sPin + (2 * 2 + pin) * A1;
            for (int q = threadIdx.x; q < TX * TY; q += NT) {
                const int ly = q / TX, lx = q - ly * TX;
                const int gx = x0 + lx, gy = y0 + ly;
                if (gx >= nx || gy >= ny) continue;
                const int c = (ly + 1) * W1 + lx + 1;
                const R Fx = -(half * (Pxx[c + 1] - Pxx[c - 1]) + half * (Pxy[c + W1] - Pxy[c - W1])
                               + half * (sPz[(0 * 3 + pzu) * A1 + c] - sPz[(0 * 3 + pzd) * A1 + c]));
                const R Fy = -(half * (Pxy[c + 1] - Pxy[c - 1]) + half * (Pyy[c + W1] - Pyy[c - W1])
                               + half * (sPz[(1 * 3 + pzu) * A1 + c] - sPz[(1 * 3 + pzd) * A1 + c]));
                const R Fz = -(half * (sPz[(0 * 3 + pz0) * A1 + c + 1] - sPz[(0 * 3 + pz0) * A1 + c - 1])
                               + half * (sPz[(1 * 3 + pz0) * A1 + c + W1] - sPz[(1 * 3 + pz0) * A1 + c - W1])
                               + half * (sPz[(2 * 3 + pzu) * A1 + c] - sPz[(2 * 3 + pzd) * A1 + c]));
                const int64_t site = z3 * zs + (int64_t)gy * pitch + gx;
                io.F[0][site] = Fx;
                io.F[1][site] = Fy;
                io.F[2][site] = Fz;
            }
        }
        // the barrier at the top of the next iteration orders the rings
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *reinterpret_cast<volatile int*>(io.flag) = 1;
}

// Pass B: one thread per site.  Moments of f(t) with the half-force shift,
// collision per opposite pair, push to the neighbours (halfway bounce-back on
// the walls at z = 0 and nz - 1); u(t) to the aux planes.
template <typename R>
__global__ void __launch_bounds__(128) k_lb3d(Geom g, Phys<R> p, StepIO<R> io)
{
    using L = D3Q19;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int nx = g.nx, ny = g.ny, nz = g.nz, pitch = g.pitch, walls = g.walls;
    const int64_t plane = g.plane, zs = (int64_t)ny * pitch;
    const int64_t site = z * zs + (int64_t)y * pitch + x;
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
    const R half = R(0.5);
    const R Fx = io.F[0][site], Fy = io.F[1][site], Fz = io.F[2][site];
    const R n = p.n0 + dn;
    const R inv_n = rcp_s(n);
    const R vx = (jx + half * Fx) * inv_n, vy = (jy + half * Fy) * inv_n, vz = (jz + half * Fz) * inv_n;
    io.u[0][site] = vx;
    io.u[1][site] = vy;
    io.u[2][site] = vz;
    const R omega = p.inv_tau, keep = R(1) - p.inv_tau;
    const R on = omega * n;
    const R C0 = omega * dn - R(1.5) * on * (vx * vx + vy * vy + vz * vz) - R(3) * p.guo * (vx * Fx + vy * Fy + vz * Fz);
    const R a3 = R(3) * on, a45 = R(4.5) * on, g3 = R(3) * p.guo, g9 = R(9) * p.guo;
    const int gxp = x + 1 == nx ? 0 : x + 1, gxm = x == 0 ? nx - 1 : x - 1;
    const int gyp = y + 1 == ny ? 0 : y + 1, gym = y == 0 ? ny - 1 : y - 1;
    const int gzu = z + 1 == nz ? 0 : z + 1, gzd = z == 0 ? nz - 1 : z - 1;
    const bool wall_lo = walls && z == 0, wall_hi = walls && z == nz - 1;
    R* out = io.f_out;
    out[site] = keep * df[0] + R(L::w(0)) * C0;
    auto dest = [&](int ex, int ey, int ez) -> int64_t {
        const int tx = ex > 0 ? gxp : (ex < 0 ? gxm : x);
        const int ty = ey > 0 ? gyp : (ey < 0 ? gym : y);
        const int tz = ez > 0 ? gzu : (ez < 0 ? gzd : z);
        return tz * zs + (int64_t)ty * pitch + tx;
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
    if (!isfinite(n)) *reinterpret_cast<volatile int*>(io.flag) = 1;
}

// Pass C.  A 32 x 8 block marches a column segment of ZC planes: each thread
// keeps the planes z - 1, z, z + 1 of mu, T and the wall-normal flux
// g_z = phi u_z in registers, so along z only the plane z + 1 is loaded;
// the in-plane neighbours come through L1.  phi(t+1) from the fluxes
// g = phi u of the neighbours and lap(mu) (mu even, g_z odd across the
// walls); the first temperature sub-step with the wall rule of the context.
constexpr int kZC = 16;

template <typename R>
__global__ void __launch_bounds__(256) k_phi3d(Geom g, Phys<R> p, StepIO<R> io)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int za = blockIdx.z * kZC, zb = min(za + kZC, g.nz);
    if (x >= g.nx || y >= g.ny) return;
    const int nx = g.nx, ny = g.ny, nz = g.nz, pitch = g.pitch, walls = g.walls;
    const int64_t zs = (int64_t)ny * pitch;
    const int64_t row = (int64_t)y * pitch;
    const int xl = x == 0 ? nx - 1 : x - 1, xr = x + 1 == nx ? 0 : x + 1;
    const int64_t ryl = (int64_t)(y == 0 ? ny - 1 : y - 1) * pitch, ryr = (int64_t)(y + 1 == ny ? 0 : y + 1) * pitch;
    const R half = R(0.5);
    const R* mu = io.mu;
    const R* ph = io.phi_in;
    const R* T = io.T_in;
    const R* uz = io.u[2];
    // plane index of the neighbour below / above: wrap (periodic) or the plane itself (walls)
    auto below = [&](int z) { return z == 0 ? (walls ? 0 : nz - 1) : z - 1; };
    auto above = [&](int z) { return z + 1 == nz ? (walls ? z : 0) : z + 1; };
    const bool hyd = p.hydro != 0;
    int64_t o = below(za) * zs + row + x;
    R mu_d = mu[o], T_d = T[o], gz_d = hyd ? ph[o] * uz[o] : R(0);
    o = (int64_t)za * zs + row + x;
    R mu_c = mu[o], T_c = T[o], gz_c = hyd ? ph[o] * uz[o] : R(0);
    bool bad = false;
    for (int z = za; z < zb; ++z) {
        const int64_t pz = (int64_t)z * zs;
        const int64_t site = pz + row + x;
        const int64_t ou = above(z) * zs + row + x;
        const R mu_u = mu[ou], T_u = T[ou], gz_u = hyd ? ph[ou] * uz[ou] : R(0);
        const R lapmu = mu[pz + row + xl] + mu[pz + row + xr] + mu[pz + ryl + x] + mu[pz + ryr + x] + mu_u + mu_d
                      - R(6) * mu_c;
        R div = 0;
        if (hyd) {
            const R gxl = ph[pz + row + xl] * io.u[0][pz + row + xl];
            const R gxr = ph[pz + row + xr] * io.u[0][pz + row + xr];
            const R gyl = ph[pz + ryl + x] * io.u[1][pz + ryl + x];
            const R gyr = ph[pz + ryr + x] * io.u[1][pz + ryr + x];
            R up = gz_u, dn = gz_d;
            if (walls) {                                   // no flux through the walls
                if (z == 0) dn = -gz_c;
                if (z == nz - 1) up = -gz_c;
            }
            div = half * (gxr - gxl) + half * (gyr - gyl) + half * (up - dn);
        }
        const R phn = ph[site] - div + p.Gamma * lapmu;
        io.phi_out[site] = phn;
        R Tn = T_c;
        if (p.t_update) {
            if (walls && g.t_mode == LF_TWALL_LAYERS && (z == 0 || z == nz - 1)) {
                Tn = p.T_w;
            } else {
                R tu = T_u, td = T_d;
                if (walls && g.t_mode == LF_TWALL_HALFWAY) {
                    if (z == 0) td = R(2) * p.T_w - T_c;
                    if (z == nz - 1) tu = R(2) * p.T_w - T_c;
                }
                Tn = T_c + p.dxi * (T[pz + row + xl] + T[pz + row + xr] + T[pz + ryl + x] + T[pz + ryr + x] + tu + td -
                                    R(6) * T_c);
            }
        }
        io.T_out[site] = Tn;
        bad |= !isfinite(phn) || !isfinite(Tn);
        mu_d = mu_c; mu_c = mu_u;
        T_d = T_c; T_c = T_u;
        gz_d = gz_c; gz_c = gz_u;
    }
    if (bad) *reinterpret_cast<volatile int*>(io.flag) = 1;
}

template <typename R, int TX, int TY, int NT>
cudaError_t launch_force(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s)
{
    using P3 = Force3<R, TX, TY>;
    auto kern = k_force3d<R, TX, TY, NT>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P3::BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    int Hz = (g.tune & 0xFFFF) > 0 ? (g.tune & 0xFFFF) : 0;
    if (Hz <= 0) {   // about eight waves of four CTAs per SM, segments of at least 16 planes
        const int want = (8 * 4 * 152 + tiles - 1) / tiles;
        Hz = (g.nz + want - 1) / want;
        if (Hz < 16) Hz = 16;
    }
    if (Hz > g.nz) Hz = g.nz;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + Hz - 1) / Hz);
    kern<<<grid, NT, P3::BYTES, s>>>(g, p, io, Hz);
    return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_split3d(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s)
{
    cudaError_t e;
    if constexpr (sizeof(R) == 4)
        e = (g.tune >> 16) == 1 ? launch_force<R, 32, 16, 512>(g, p, io, s) : launch_force<R, 32, 8, 256>(g, p, io, s);
    else
        e = launch_force<R, 16, 8, 128>(g, p, io, s);
    if (e != cudaSuccess) return e;
    if (p.hydro) {
        dim3 grid((g.nx + 127) / 128, g.ny, g.nz);
        k_lb3d<R><<<grid, 128, 0, s>>>(g, p, io);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    dim3 gc((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + kZC - 1) / kZC);
    k_phi3d<R><<<gc, 256, 0, s>>>(g, p, io);
    return cudaGetLastError();
}

template cudaError_t launch_split3d<float>(const Geom&, const Phys<float>&, const StepIO<float>&, cudaStream_t);
template cudaError_t launch_split3d<double>(const Geom&, const Phys<double>&, const StepIO<double>&, cudaStream_t);

}  // namespace lf
