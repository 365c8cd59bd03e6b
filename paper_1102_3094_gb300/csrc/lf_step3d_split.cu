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
//
// lf_step3d_passes.cu launches the three passes in order; with the isotropic
// stencils passes A and C are those of lf_step3d_iso.cu.
#include "lf_step3d_common.cuh"
#include "lf_march2d_x2.cuh"      // packed FP32x2 helpers

#include <type_traits>

namespace lf {

namespace {

// Pass A layout.  A CTA owns a TX x TY tile and one thread per column of the
// tile grown by 2 on every side ((TX + 4) x (TY + 4) threads), marching
// along z.  Shared memory holds in-plane neighbours only: a ring of phi planes
// (tile + 3), the psi plane and the five in-plane components of P (tile + 1),
// each of the last two double-buffered; values along z stay in registers.
template <typename R, int TX, int TY>
struct Force3 {
    static constexpr int CW = TX + 4, CH = TY + 4, NTH = CW * CH;   // threads = columns of the psi region
    static constexpr int W3 = TX + 6, H3 = TY + 6, A3 = W3 * H3;    // phi (r = 3)
    static constexpr int A2 = CW * CH;                              // psi (r = 2)
    static constexpr int NPHI = 4;                                  // phi planes k-2 .. k+1
    static constexpr int NPSI = 2;                                  // psi planes
    static constexpr int NPC = 5;                                   // stored components of P
    static constexpr int NPP = 2;                                   // planes of P
    static constexpr int PHI = 0;
    static constexpr int PSI = PHI + NPHI * A3;
    static constexpr int PP = PSI + NPSI * A2;                      // [plane][comp][A2], psi-region indexing
    static constexpr int TOTAL = PP + NPC * NPP * A2;
    static constexpr size_t MAPS = sizeof(R) * TOTAL;
    static constexpr size_t BYTES = MAPS + sizeof(int) * (W3 + H3);
};

// Pass A.  Iteration k: phi plane k + 1 is prefetched (cp.async) while
//   psi   = lap(phi)                    on plane k - 1 (every column, r = 2),
//   lam, P, mu                          on plane k - 2 (r = 1; mu stored on r = 0),
//   F = -d_a P_ab                       on plane k - 3 (r = 0, stored)
// run one plane apart; each stage reads only what earlier iterations wrote,
// so one barrier per plane orders everything.
template <typename R, int TX, int TY>
__global__ void __launch_bounds__(Force3<R, TX, TY>::NTH) k_force3d(Geom g, Phys<R> p, StepIO<R> io, int Hz)
{
    using P3 = Force3<R, TX, TY>;
    constexpr int W3 = P3::W3, CW = P3::CW, A3 = P3::A3, A2 = P3::A2, NTH = P3::NTH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    R* sphi = sm + P3::PHI;
    R* spsi = sm + P3::PSI;
    R* sP = sm + P3::PP;      // [plane slot][comp xx, xy, yy, xz, yz][A2]
    int* colmap = reinterpret_cast<int*>(smem_raw + P3::MAPS);   // x0 - 3 + i -> storage column
    int* rowmap = colmap + W3;                                   // y0 - 3 + j -> storage row

    const int t = threadIdx.x;
    const int cx = t % CW, cy = t / CW;                  // column of the psi region
    const int nx = g.nx, ny = g.ny, nz = g.nz, pitch = g.pitch, walls = g.walls;
    const int zs = ny * pitch;                   // 32-bit offsets: Q * padded sites < 2^31 (checked at creation)
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * Hz, z1 = min(z0 + Hz, nz);
    const int kbeg = z0 - 3, kend = z1 + 2;
    const R half = R(0.5);
    const bool in1 = cx >= 1 && cx < CW - 1 && cy >= 1 && cy < P3::CH - 1;   // r = 1 region
    const bool in0 = cx >= 2 && cx < CW - 2 && cy >= 2 && cy < P3::CH - 2;   // the tile
    const int gx = x0 - 2 + cx, gy = y0 - 2 + cy;
    const bool own = in0 && gx < nx && gy < ny;
    bool bad = false;

    for (int q = t; q < W3 + P3::H3; q += NTH) {
        if (q < W3) colmap[q] = wrap_s(x0 - 3 + q, nx);
        else rowmap[q - W3] = wrap_s(y0 - 3 + (q - W3), ny);
    }
    __syncthreads();
    // storage offset of this column inside a plane (wrapped)
    const int col_off = rowmap[cy + 1] * pitch + colmap[cx + 1];
    const int c3 = (cy + 1) * W3 + cx + 1;               // own position in a phi plane
    const int c2 = t;                                    // own position in a psi / P plane
    // the phi elements this thread copies into every plane of the ring:
    // q = t and q = t + NTH (when inside the r = 3 region), as in-plane offsets
    static_assert(A3 <= 2 * NTH, "at most two phi elements per thread");
    const int qe = t + NTH;
    const bool two = qe < A3;
    const int oe0 = rowmap[t / W3] * pitch + colmap[t % W3];
    const int oe1 = two ? rowmap[qe / W3] * pitch + colmap[qe % W3] : 0;

    auto slot = [&](int z) { return (z - kbeg + 4 * P3::NPHI) % P3::NPHI; };
    // pz: storage offset of plane z (z in [kbeg, kend])
    auto fetch = [&](int z, int pz) {
        if (z <= kend) {
            R* d = sphi + slot(z) * A3;
            cp_async_s<sizeof(R)>(&d[t], io.phi_in + (pz + oe0));
            if (two) cp_async_s<sizeof(R)>(&d[qe], io.phi_in + (pz + oe1));
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    auto Tload = [&](int z, int pz) -> R {               // T of this column (r = 1 columns only)
        if (!in1 || z > kend) return R(0);
        return io.T_in[pz + col_off];
    };

    // register windows along z (suffix = plane offset from k)
    R phm1 = 0, phm2 = 0, phm3 = 0;          // own-column phi(k-1), phi(k-2), phi(k-3)
    R psm1 = 0, psm2 = 0;                    // own-column psi(k-2), psi(k-3) (psi(k-1) is computed in iteration k)
    R xzA = 0, xzB = 0, xzC = 0, yzA = 0, yzB = 0, yzC = 0, zzA = 0, zzB = 0, zzC = 0;   // P_az at k-2 .. k-4
    const int pz0 = map_z(kbeg, nz, walls) * zs;
    R Tq0 = Tload(kbeg, pz0), Tq1 = 0, Tq2 = 0, Tq3 = 0;   // T(k) .. T(k-3)

    fetch(kbeg, pz0);
    for (int k = kbeg; k <= kend; ++k) {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        const int pzn = k + 1 <= kend ? map_z(k + 1, nz, walls) * zs : 0;
        fetch(k + 1, pzn);
        const R Tnext = Tload(k + 1, pzn);               // consumed three iterations later
        const R* pk = sphi + slot(k) * A3;
        const R* p1 = sphi + slot(k - 1) * A3;
        const R* p2 = sphi + slot(k - 2) * A3;
        const R phk = pk[c3];

        // ---- plane k-1: psi (r = 2) ---------------------------------------------
        const R psi_new = p1[c3 - 1] + p1[c3 + 1] + p1[c3 - W3] + p1[c3 + W3] + phm2 + phk - R(6) * phm1;
        spsi[((k - 1 - kbeg) & 1) * A2 + c2] = psi_new;

        // ---- plane k-2: lam, P, mu (r = 1) -----------------------------------------
        R xz = 0, yz = 0, zz = 0;
        const int z2 = k - 2;
        if (in1 && z2 >= z0 - 1 && z2 <= z1) {
            const R* ps = spsi + ((z2 - kbeg) & 1) * A2;   // psi(k-2), written one iteration ago
            const R ph = phm2, psi = psm1;                  // phi(k-2), psi(k-2)
            const R lam = ps[c2 - 1] + ps[c2 + 1] + ps[c2 - CW] + ps[c2 + CW] + psi_new + psm2 - R(6) * psi;
            const R av = (Tq2 - p.Tc) * p.inv_Tc;
            if (own && z2 >= z0 && z2 < z1) {
                const R mu = av * ph + p.b * ph * ph * ph - p.kappa * psi + p.c * lam;
                bad |= !isfinite(mu);
                io.mu[z2 * zs + gy * pitch + gx] = mu;
            }
            if (p.hydro) {
                const R d0 = half * (p2[c3 + 1] - p2[c3 - 1]);
                const R d1 = half * (p2[c3 + W3] - p2[c3 - W3]);
                const R d2 = half * (phm1 - phm3);
                const R s0 = half * (ps[c2 + 1] - ps[c2 - 1]);
                const R s1 = half * (ps[c2 + CW] - ps[c2 - CW]);
                const R s2 = half * (psi_new - psm2);
                const R ph2 = ph * ph;
                const R iso = av * ph2 * half + R(0.75) * p.b * ph2 * ph2
                            - p.kappa * (ph * psi + half * (d0 * d0 + d1 * d1 + d2 * d2))
                            + p.c * (ph * lam + half * psi * psi + d0 * s0 + d1 * s1 + d2 * s2);
                R* P = sP + ((z2 - kbeg) & 1) * 5 * A2;
                P[0 * A2 + c2] = iso + p.kappa * d0 * d0 - R(2) * p.c * d0 * s0;
                P[1 * A2 + c2] = p.kappa * d0 * d1 - p.c * (d0 * s1 + d1 * s0);
                P[2 * A2 + c2] = iso + p.kappa * d1 * d1 - R(2) * p.c * d1 * s1;
                xz = p.kappa * d0 * d2 - p.c * (d0 * s2 + d2 * s0);
                yz = p.kappa * d1 * d2 - p.c * (d1 * s2 + d2 * s1);
                zz = iso + p.kappa * d2 * d2 - R(2) * p.c * d2 * s2;
                P[3 * A2 + c2] = xz;
                P[4 * A2 + c2] = yz;
            }
        }

        // ---- plane k-3: F (r = 0) ---------------------------------------------------
        const int z3 = k - 3;
        if (p.hydro && own && z3 >= z0 && z3 < z1) {
            const R* P = sP + ((z3 - kbeg) & 1) * 5 * A2;  // P(k-3), written one iteration ago
            const R Fx = -(half * (P[0 * A2 + c2 + 1] - P[0 * A2 + c2 - 1]) + half * (P[1 * A2 + c2 + CW] - P[1 * A2 + c2 - CW])
                           + half * (xz - xzC));
            const R Fy = -(half * (P[1 * A2 + c2 + 1] - P[1 * A2 + c2 - 1]) + half * (P[2 * A2 + c2 + CW] - P[2 * A2 + c2 - CW])
                           + half * (yz - yzC));
            const R Fz = -(half * (P[3 * A2 + c2 + 1] - P[3 * A2 + c2 - 1]) + half * (P[4 * A2 + c2 + CW] - P[4 * A2 + c2 - CW])
                           + half * (zz - zzC));
            const int site = z3 * zs + gy * pitch + gx;
            io.F[0][site] = Fx;
            io.F[1][site] = Fy;
            io.F[2][site] = Fz;
        }

        // shift the windows
        phm3 = phm2; phm2 = phm1; phm1 = phk;
        psm2 = psm1; psm1 = psi_new;
        xzC = xzB; xzB = xz; yzC = yzB; yzB = yz; zzC = zzB; zzB = zz;
        Tq3 = Tq2; Tq2 = Tq1; Tq1 = Tq0; Tq0 = Tnext;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (__any_sync(0xffffffffu, bad) && (t & 31) == 0) *reinterpret_cast<volatile int*>(io.flag) = 1;
}

// Pass A on two z-segments at once (FP32): lane .x marches planes
// [z0, z0 + H), lane .y planes [z0 + H, z0 + 2H) (shorter or empty at the top
// of the lattice), both with the same lags, and all arithmetic runs on packed
// FP32x2 instructions.  Layout and stages as in k_force3d, with float2
// shared-memory planes.
template <int TX, int TY>
struct Force3x2 {
    static constexpr int CW = TX + 4, CH = TY + 4, NTH = CW * CH;
    static constexpr int W3 = TX + 6, H3 = TY + 6, A3 = W3 * H3;
    static constexpr int A2 = CW * CH;
    static constexpr int NPHI = 4;
    static constexpr int PHI = 0;
    static constexpr int PSI = PHI + NPHI * A3;
    static constexpr int PP = PSI + 2 * A2;
    static constexpr int TOTAL = PP + 10 * A2;                      // float2 elements
    static constexpr size_t MAPS = sizeof(float2) * TOTAL;
    static constexpr size_t BYTES = MAPS + sizeof(int) * (W3 + H3);
};

template <int TX, int TY>
__global__ void __launch_bounds__(Force3x2<TX, TY>::NTH, 2) k_force3d_x2(Geom g, Phys<float> p, StepIO<float> io, int H)
{
    using namespace march;
    using P3 = Force3x2<TX, TY>;
    constexpr int W3 = P3::W3, CW = P3::CW, A3 = P3::A3, A2 = P3::A2, NTH = P3::NTH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);
    float2* sphi = sm + P3::PHI;
    float2* spsi = sm + P3::PSI;
    float2* sP = sm + P3::PP;
    int* colmap = reinterpret_cast<int*>(smem_raw + P3::MAPS);
    int* rowmap = colmap + W3;

    const int t = threadIdx.x;
    const int cx = t % CW, cy = t / CW;
    const int nx = g.nx, ny = g.ny, nz = g.nz, pitch = g.pitch, walls = g.walls;
    const int zs = ny * pitch;                   // 32-bit offsets: Q * padded sites < 2^31 (checked at creation)
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int za0 = blockIdx.z * 2 * H, zb0 = za0 + H;                    // first plane of each lane
    const int ha = min(H, nz - za0), hb = max(0, min(H, nz - zb0));     // planes per lane
    const int hmax = ha > hb ? ha : hb;
    const int nit = hmax + 6;                                            // relative iterations 0 .. nit-1
    const float2 half = v2(0.5f), six = v2(6.f);
    const bool in1 = cx >= 1 && cx < CW - 1 && cy >= 1 && cy < P3::CH - 1;
    const bool in0 = cx >= 2 && cx < CW - 2 && cy >= 2 && cy < P3::CH - 2;
    const int gx = x0 - 2 + cx, gy = y0 - 2 + cy;
    const bool own = in0 && gx < nx && gy < ny;
    bool bad = false;

    for (int q = t; q < W3 + P3::H3; q += NTH) {
        if (q < W3) colmap[q] = wrap_s(x0 - 3 + q, nx);
        else rowmap[q - W3] = wrap_s(y0 - 3 + (q - W3), ny);
    }
    __syncthreads();
    const int col_off = rowmap[cy + 1] * pitch + colmap[cx + 1];
    const int c3 = (cy + 1) * W3 + cx + 1;
    const int c2 = t;
    const int own_off = gy * pitch + gx;
    // the phi elements this thread copies into every plane of the ring:
    // q = t and q = t + NTH (when inside the r = 3 region), as in-plane offsets
    static_assert(A3 <= 2 * NTH, "at most two phi elements per thread");
    const int qe = t + NTH;
    const bool two = qe < A3;
    const int oe0 = rowmap[t / W3] * pitch + colmap[t % W3];
    const int oe1 = two ? rowmap[qe / W3] * pitch + colmap[qe % W3] : 0;

    // relative plane j (iteration k = j + 3 loads relative plane k + 1 - 3 ... ): plane of lane L = z0_L + j
    auto slot = [&](int j) { return (j + 4 * P3::NPHI) % P3::NPHI; };
    // storage offsets pa, pb of relative plane j in the two lanes, j = -3 .. hmax + 2
    auto fetch_s = [&](int sl, int j, int pa, int pb) {      // into ring slot sl
        if (j <= hmax + 2) {
            float* d = reinterpret_cast<float*>(sphi + sl * A3);
            cp_async_s<4>(d + 2 * t, io.phi_in + (pa + oe0));
            cp_async_s<4>(d + 2 * t + 1, io.phi_in + (pb + oe0));
            if (two) {
                cp_async_s<4>(d + 2 * qe, io.phi_in + (pa + oe1));
                cp_async_s<4>(d + 2 * qe + 1, io.phi_in + (pb + oe1));
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    auto Tload = [&](int j, int pa, int pb) -> float2 {
        if (!in1 || j > hmax + 2) return v2(0.f);
        return make_float2(io.T_in[pa + col_off], io.T_in[pb + col_off]);
    };

    float2 phm1 = v2(0), phm2 = v2(0), phm3 = v2(0);
    float2 psm1 = v2(0), psm2 = v2(0);
    float2 xzB = v2(0), xzC = v2(0), yzB = v2(0), yzC = v2(0), zzB = v2(0), zzC = v2(0);
    const int pa0 = map_z(za0 - 3, nz, walls) * zs, pb0 = map_z(zb0 - 3, nz, walls) * zs;
    float2 Tq0 = Tload(-3, pa0, pb0), Tq1 = v2(0), Tq2 = v2(0);

    fetch_s(slot(-3), -3, pa0, pb0);
    // iteration j handles relative plane j as "k": fetch j + 1, psi on j - 1, P on j - 2, F on j - 3.
    // Four iterations per trip with j = U - 3 (mod 4) in sub-iteration U, so
    // ring slots and buffer parities are constants and the register windows
    // of depth two need no copies; iterations past the last plane (up to three
    // in the last trip) do only guarded-off work.
    auto iter = [&](const int j, auto utag) {
        constexpr int U = decltype(utag)::value;
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        int pan = 0, pbn = 0;
        if (j + 1 <= hmax + 2) {
            pan = map_z(za0 + j + 1, nz, walls) * zs;
            pbn = map_z(zb0 + j + 1, nz, walls) * zs;
        }
        fetch_s((2 + U) & 3, j + 1, pan, pbn);
        const float2 Tnext = Tload(j + 1, pan, pbn);
        const float2* pk = sphi + ((1 + U) & 3) * A3;
        const float2* p1 = sphi + (U & 3) * A3;
        const float2* p2 = sphi + ((U + 3) & 3) * A3;
        const float2 phk = pk[c3];

        // psi of plane j - 1
        const float2 psi_new = fma2(six, sub2(v2(0), phm1),
                                    add2(add2(add2(p1[c3 - 1], p1[c3 + 1]), add2(p1[c3 - W3], p1[c3 + W3])), add2(phm2, phk)));
        spsi[(U & 1) * A2 + c2] = psi_new;

        // lam, P, mu of plane j - 2
        float2 xz = v2(0), yz = v2(0), zz = v2(0);
        const int r2 = j - 2;                              // relative plane
        if (in1 && r2 >= -1 && r2 <= hmax) {
            const float2* ps = spsi + ((U + 1) & 1) * A2;
            const float2 ph = phm2, psi = psm1;
            const float2 lam = fma2(six, sub2(v2(0), psi),
                                    add2(add2(add2(ps[c2 - 1], ps[c2 + 1]), add2(ps[c2 - CW], ps[c2 + CW])), add2(psi_new, psm2)));
            const float2 av = mul2(sub2(Tq2, v2(p.Tc)), v2(p.inv_Tc));
            const float2 ph2 = mul2(ph, ph);
            if (own && r2 >= 0) {
                // mu = a phi + b phi^3 - kappa psi + c lam
                const float2 mu = fma2(v2(p.c), lam, fma2(v2(-p.kappa), psi, mul2(ph, fma2(v2(p.b), ph2, av))));
                if (r2 < ha) { bad |= !isfinite(mu.x); io.mu[(za0 + r2) * zs + own_off] = mu.x; }
                if (r2 < hb) { bad |= !isfinite(mu.y); io.mu[(zb0 + r2) * zs + own_off] = mu.y; }
            }
            if (p.hydro) {
                const float2 d0 = mul2(half, sub2(p2[c3 + 1], p2[c3 - 1]));
                const float2 d1 = mul2(half, sub2(p2[c3 + W3], p2[c3 - W3]));
                const float2 d2 = mul2(half, sub2(phm1, phm3));
                const float2 s0 = mul2(half, sub2(ps[c2 + 1], ps[c2 - 1]));
                const float2 s1 = mul2(half, sub2(ps[c2 + CW], ps[c2 - CW]));
                const float2 s2 = mul2(half, sub2(psi_new, psm2));
                const float2 gp2 = fma2(d0, d0, fma2(d1, d1, mul2(d2, d2)));
                const float2 gpgs = fma2(d0, s0, fma2(d1, s1, mul2(d2, s2)));
                // iso = a phi^2/2 + 3b phi^4/4 - kappa (phi psi + gp2/2) + c (phi lam + psi^2/2 + gpgs)
                float2 iso = mul2(ph2, fma2(v2(0.75f * p.b), ph2, mul2(half, av)));
                iso = fma2(v2(-p.kappa), fma2(half, gp2, mul2(ph, psi)), iso);
                iso = fma2(v2(p.c), add2(fma2(ph, lam, mul2(half, mul2(psi, psi))), gpgs), iso);
                const float2 k_ = v2(p.kappa), mc = v2(-p.c), m2c = v2(-2.f * p.c);
                float2* P = sP + ((U + 1) & 1) * 5 * A2;
                P[0 * A2 + c2] = fma2(k_, mul2(d0, d0), fma2(m2c, mul2(d0, s0), iso));
                P[1 * A2 + c2] = fma2(k_, mul2(d0, d1), mul2(mc, fma2(d0, s1, mul2(d1, s0))));
                P[2 * A2 + c2] = fma2(k_, mul2(d1, d1), fma2(m2c, mul2(d1, s1), iso));
                xz = fma2(k_, mul2(d0, d2), mul2(mc, fma2(d0, s2, mul2(d2, s0))));
                yz = fma2(k_, mul2(d1, d2), mul2(mc, fma2(d1, s2, mul2(d2, s1))));
                zz = fma2(k_, mul2(d2, d2), fma2(m2c, mul2(d2, s2), iso));
                P[3 * A2 + c2] = xz;
                P[4 * A2 + c2] = yz;
            }
        }

        // F of plane j - 3
        const int r3 = j - 3;
        if (p.hydro && own && r3 >= 0 && r3 < hmax) {
            const float2* P = sP + (U & 1) * 5 * A2;
            const float2 Fx = sub2(v2(0), mul2(half, add2(add2(sub2(P[0 * A2 + c2 + 1], P[0 * A2 + c2 - 1]),
                                                               sub2(P[1 * A2 + c2 + CW], P[1 * A2 + c2 - CW])), sub2(xz, xzC))));
            const float2 Fy = sub2(v2(0), mul2(half, add2(add2(sub2(P[1 * A2 + c2 + 1], P[1 * A2 + c2 - 1]),
                                                               sub2(P[2 * A2 + c2 + CW], P[2 * A2 + c2 - CW])), sub2(yz, yzC))));
            const float2 Fz = sub2(v2(0), mul2(half, add2(add2(sub2(P[3 * A2 + c2 + 1], P[3 * A2 + c2 - 1]),
                                                               sub2(P[4 * A2 + c2 + CW], P[4 * A2 + c2 - CW])), sub2(zz, zzC))));
            if (r3 < ha) {
                const int site = (za0 + r3) * zs + own_off;
                io.F[0][site] = Fx.x; io.F[1][site] = Fy.x; io.F[2][site] = Fz.x;
            }
            if (r3 < hb) {
                const int site = (zb0 + r3) * zs + own_off;
                io.F[0][site] = Fx.y; io.F[1][site] = Fy.y; io.F[2][site] = Fz.y;
            }
        }

        phm3 = phm2; phm2 = phm1; phm1 = phk;
        psm2 = psm1; psm1 = psi_new;
        xzC = xzB; xzB = xz; yzC = yzB; yzB = yz; zzC = zzB; zzB = zz;
        Tq2 = Tq1; Tq1 = Tq0; Tq0 = Tnext;
    };
#pragma unroll 1
    for (int j = -3; j < nit - 3; j += 4) {
        iter(j, std::integral_constant<int, 0>{});
        iter(j + 1, std::integral_constant<int, 1>{});
        iter(j + 2, std::integral_constant<int, 2>{});
        iter(j + 3, std::integral_constant<int, 3>{});
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (__any_sync(0xffffffffu, bad) && (t & 31) == 0) *reinterpret_cast<volatile int*>(io.flag) = 1;
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
    const int plane = (int)g.plane, zs = ny * pitch;   // 32-bit offsets: Q * padded sites < 2^31 (checked at creation)
    const int site = z * zs + y * pitch + x;
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
    // neighbour offsets per axis, indexed by the velocity component + 1
    const int rx[3] = {gxm, x, gxp};
    const int ry[3] = {gym * pitch, y * pitch, gyp * pitch};
    const int rz[3] = {gzd * zs, z * zs, gzu * zs};
    auto dest = [&](int ex, int ey, int ez) -> int { return rz[ez + 1] + ry[ey + 1] + rx[ex + 1]; };
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

template <typename R>
__global__ void __launch_bounds__(256) k_phi3d(Geom g, Phys<R> p, StepIO<R> io, int zc)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int za = blockIdx.z * zc, zb = min(za + zc, g.nz);
    if (x >= g.nx || y >= g.ny) return;
    const int nx = g.nx, ny = g.ny, nz = g.nz, pitch = g.pitch, walls = g.walls;
    const int64_t zs = (int64_t)ny * pitch;
    const int64_t row = (int64_t)y * pitch;
    const int xl = x == 0 ? nx - 1 : x - 1, xr = x + 1 == nx ? 0 : x + 1;
    const int64_t ryl = (int64_t)(y == 0 ? ny - 1 : y - 1) * pitch, ryr = (int64_t)(y + 1 == ny ? 0 : y + 1) * pitch;
    const R half = R(0.5);
    const R* __restrict__ mu = io.mu;
    const R* __restrict__ ph = io.phi_in;
    const R* __restrict__ T = io.T_in;
    const R* __restrict__ ux = io.u[0];
    const R* __restrict__ uy = io.u[1];
    const R* __restrict__ uz = io.u[2];
    R* __restrict__ phi_out = io.phi_out;
    R* __restrict__ T_out = io.T_out;
    // plane index of the neighbour below / above: wrap (periodic) or the plane itself (walls)
    auto below = [&](int z) { return z == 0 ? (walls ? 0 : nz - 1) : z - 1; };
    auto above = [&](int z) { return z + 1 == nz ? (walls ? z : 0) : z + 1; };
    const bool hyd = p.hydro != 0;
    // in-plane neighbours of plane z, loaded one plane ahead of their use so
    // that two planes of loads are in flight per thread
    struct Nb {
        R mxl, mxr, myl, myr, txl, txr, tyl, tyr, gxl, gxr, gyl, gyr, pc;
    };
    auto load_nb = [&](int z) {
        Nb v;
        const int64_t pz = (int64_t)z * zs;
        v.mxl = mu[pz + row + xl]; v.mxr = mu[pz + row + xr];
        v.myl = mu[pz + ryl + x]; v.myr = mu[pz + ryr + x];
        v.txl = T[pz + row + xl]; v.txr = T[pz + row + xr];
        v.tyl = T[pz + ryl + x]; v.tyr = T[pz + ryr + x];
        v.pc = ph[pz + row + x];
        if (hyd) {
            v.gxl = ph[pz + row + xl] * ux[pz + row + xl];
            v.gxr = ph[pz + row + xr] * ux[pz + row + xr];
            v.gyl = ph[pz + ryl + x] * uy[pz + ryl + x];
            v.gyr = ph[pz + ryr + x] * uy[pz + ryr + x];
        } else {
            v.gxl = v.gxr = v.gyl = v.gyr = R(0);
        }
        return v;
    };
    int64_t o = below(za) * zs + row + x;
    R mu_d = mu[o], T_d = T[o], gz_d = hyd ? ph[o] * uz[o] : R(0);
    o = (int64_t)za * zs + row + x;
    R mu_c = mu[o], T_c = T[o], gz_c = hyd ? ph[o] * uz[o] : R(0);
    Nb nb = load_nb(za);
    bool bad = false;
    for (int z = za; z < zb; ++z) {
        const int64_t site = (int64_t)z * zs + row + x;
        const int64_t ou = above(z) * zs + row + x;
        const R mu_u = mu[ou], T_u = T[ou], gz_u = hyd ? ph[ou] * uz[ou] : R(0);
        const Nb nxt = load_nb(z + 1 < zb ? z + 1 : z);
        const R lapmu = nb.mxl + nb.mxr + nb.myl + nb.myr + mu_u + mu_d - R(6) * mu_c;
        R div = 0;
        if (hyd) {
            R up = gz_u, dn = gz_d;
            if (walls) {                                   // no flux through the walls
                if (z == 0) dn = -gz_c;
                if (z == nz - 1) up = -gz_c;
            }
            div = half * (nb.gxr - nb.gxl) + half * (nb.gyr - nb.gyl) + half * (up - dn);
        }
        const R phn = nb.pc - div + p.Gamma * lapmu;
        phi_out[site] = phn;
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
                Tn = T_c + p.dxi * (nb.txl + nb.txr + nb.tyl + nb.tyr + tu + td - R(6) * T_c);
            }
        }
        T_out[site] = Tn;
        bad |= !isfinite(phn) || !isfinite(Tn);
        mu_d = mu_c; mu_c = mu_u;
        T_d = T_c; T_c = T_u;
        gz_d = gz_c; gz_c = gz_u;
        nb = nxt;
    }
    if (bad) *reinterpret_cast<volatile int*>(io.flag) = 1;
}

template <typename R, int TX, int TY>
cudaError_t launch_force(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s)
{
    using P3 = Force3<R, TX, TY>;
    auto kern = k_force3d<R, TX, TY>;
    static unsigned long long attr_done = 0;      // per instantiation and device
    const cudaError_t e = raise_smem_limit(kern, (int)P3::BYTES, &attr_done);
    if (e != cudaSuccess) return e;
    const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    int Hz = (g.tune & 0xFFFF) > 0 ? (g.tune & 0xFFFF) : 0;
    if (Hz <= 0) {   // about eight waves of two CTAs per SM, segments of at least 16 planes
        const int want = (8 * 2 * 152 + tiles - 1) / tiles;
        Hz = (g.nz + want - 1) / want;
        if (Hz < 16) Hz = 16;
    }
    if (Hz > g.nz) Hz = g.nz;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + Hz - 1) / Hz);
    kern<<<grid, P3::NTH, P3::BYTES, s>>>(g, p, io, Hz);
    return cudaGetLastError();
}

template <int TX, int TY>
cudaError_t launch_force_x2(const Geom& g, const Phys<float>& p, const StepIO<float>& io, cudaStream_t s)
{
    using P3 = Force3x2<TX, TY>;
    auto kern = k_force3d_x2<TX, TY>;
    static unsigned long long attr_done = 0;      // per instantiation and device
    const cudaError_t e = raise_smem_limit(kern, (int)P3::BYTES, &attr_done);
    if (e != cudaSuccess) return e;
    const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    int H = (g.tune & 0xFFFF) > 0 ? (g.tune & 0xFFFF) : 0;     // planes per lane
    if (H <= 0) {   // about eight CTAs per SM (two resident), lanes of at least 16 planes
        const int want = (8 * 152 + tiles - 1) / tiles;
        H = (g.nz + 2 * want - 1) / (2 * want);
        if (H < 16) H = 16;
        H += (6 - H % 4) % 4;   // H + 6 iterations: whole trips of four
    }
    if (H > g.nz) H = g.nz;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + 2 * H - 1) / (2 * H));
    kern<<<grid, P3::NTH, P3::BYTES, s>>>(g, p, io, H);
    return cudaGetLastError();
}

}  // namespace

// The compact passes, one launcher each (the three-pass step, with the pass
// boundaries, is put together by lf_step3d_passes.cu).
template <typename R>
cudaError_t launch_force3d_compact(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s)
{
    if constexpr (sizeof(R) == 4) {
        // (param >> 16) & 15: 0 = two z-lanes in packed FP32x2, 1 / 2 = one lane on 60x4 / 28x12 tiles
        const int sel = (g.tune >> 16) & 15;
        return sel == 1 ? launch_force<R, 60, 4>(g, p, io, s)
             : sel == 2 ? launch_force<R, 28, 12>(g, p, io, s)
                        : launch_force_x2<28, 12>(g, p, io, s);
    } else {
        return launch_force<R, 28, 12>(g, p, io, s);
    }
}

template <typename R>
cudaError_t launch_lb3d(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s)
{
    dim3 grid((g.nx + 127) / 128, g.ny, g.nz);
    k_lb3d<R><<<grid, 128, 0, s>>>(g, p, io);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_phi3d_compact(const Geom& g, const Phys<R>& p, const StepIO<R>& io, int zc, cudaStream_t s)
{
    dim3 gc((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + zc - 1) / zc);
    k_phi3d<R><<<gc, 256, 0, s>>>(g, p, io, zc);
    return cudaGetLastError();
}

#define LF_INST(R)                                                                                              \
    template cudaError_t launch_force3d_compact<R>(const Geom&, const Phys<R>&, const StepIO<R>&, cudaStream_t); \
    template cudaError_t launch_lb3d<R>(const Geom&, const Phys<R>&, const StepIO<R>&, cudaStream_t);           \
    template cudaError_t launch_phi3d_compact<R>(const Geom&, const Phys<R>&, const StepIO<R>&, int, cudaStream_t);
LF_INST(float)
LF_INST(double)
#undef LF_INST

}  // namespace lf
