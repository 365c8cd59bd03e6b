// lf_step3d_iso.cu -- passes A and C of the three-pass D3Q19 step
// (lf_step3d_split.cu, LF_VARIANT_SPLIT3) with the isotropic 19-point
// stencils (LF_STENCIL_ISOTROPIC), as column marches along z whose 19-point
// operators are split by plane into sliding sums (Plane19 / Slide19 in
// lf_iso3.cuh):
//   A  mu and F = -d_a P_ab (Eqs. chem, ff): k_force3d_iso (one lane, FP32
//      and FP64) or k_force3d_iso_x2 (two z-lanes in packed FP32x2);
//   C  phi(t+1) = phi - div(phi u) + Gamma lap(mu) (Eq. massdiff) and the
//      first temperature sub-step: k_phi3d_isoz (fields staged through
//      registers) or k_phi3d_isoa (raw fields staged by cp.async).
// Pass B (collision and streaming) is the same for both stencils.  The wall
// rules are those of the compact passes: phi, T and every derived scalar
// even about the half-way planes, the wall-normal flux odd, T with its
// ghost or held layers.
#include "lf_step3d_common.cuh"
#include "lf_march2d_x2.cuh"      // packed FP32x2 helpers
#include "lf_iso3.cuh"

#include <type_traits>

namespace lf {

namespace {

// Pass A with the isotropic stencils as a column march with sliding sums.
// Every 19-point operator is split by plane (Plane19 in lf_iso3.cuh): each
// thread loads the in-plane neighbours of one new plane of phi, psi and P per
// iteration and keeps the partial sums of the centres still open in
// registers, so shared memory holds one plane of each field (two with the
// plane in flight) and each neighbour is loaded once per column rather than
// once per operator and centre.  Iteration k, after one barrier:
//   phi plane k (prefetched in iteration k - 1)   -> psi, grad phi at k - 1   (every column, r = 2)
//   psi plane k - 2 (stored in iteration k - 1)   -> lam, grad psi at k - 3, then mu and P at k - 3 (r = 1)
//   P plane k - 4 (stored in iteration k - 1)     -> F at k - 5 (the tile)
// Each stage reads only planes written before the barrier and writes the slot
// its readers left in the previous iteration, so one barrier per plane
// orders everything; the march runs z1 - z0 + 8 iterations.
template <typename R, int TX, int TY>
struct Force3Iso {
    static constexpr int CW = TX + 4, CH = TY + 4, NTH = CW * CH;   // threads = columns of the psi region
    static constexpr int W3 = TX + 6, H3 = TY + 6, A3 = W3 * H3;    // phi (r = 3)
    static constexpr int A2 = CW * CH;                              // psi, P (r = 2 / r = 1, psi-region indexing)
    static constexpr int PHI = 0;                                   // [2][A3]
    static constexpr int PSI = PHI + 2 * A3;                        // [2][A2]
    static constexpr int PP = PSI + 2 * A2;                         // [2][xx, xy, yy, xz, yz, zz][A2]
    static constexpr int TOTAL = PP + 12 * A2;
    static constexpr size_t MAPS = sizeof(R) * TOTAL;
    static constexpr size_t BYTES = MAPS + sizeof(int) * (W3 + H3);
};

template <typename R, int TX, int TY, int MINB>
__global__ void __launch_bounds__(Force3Iso<R, TX, TY>::NTH, MINB) k_force3d_iso(Geom g, Phys<R> p, StepIO<R> io, int Hz)
{
    using P3 = Force3Iso<R, TX, TY>;
    constexpr int W3 = P3::W3, CW = P3::CW, A3 = P3::A3, A2 = P3::A2, NTH = P3::NTH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    R* sphi = sm + P3::PHI;
    R* spsi = sm + P3::PSI;
    R* sP = sm + P3::PP;
    int* colmap = reinterpret_cast<int*>(smem_raw + P3::MAPS);   // x0 - 3 + i -> storage column
    int* rowmap = colmap + W3;                                   // y0 - 3 + j -> storage row

    const int t = threadIdx.x;
    const int cx = t % CW, cy = t / CW;
    const int nx = g.nx, ny = g.ny, nz = g.nz, pitch = g.pitch, walls = g.walls;
    const int zs = ny * pitch;                   // 32-bit offsets: Q * padded sites < 2^31 (checked at creation)
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * Hz, z1 = min(z0 + Hz, nz);
    const int kbeg = z0 - 3, kphi = z1 + 2, kend = z1 + 4;   // phi planes kbeg .. kphi
    const R half = R(0.5);
    const bool in0 = cx >= 2 && cx < CW - 2 && cy >= 2 && cy < P3::CH - 2;
    const bool row1 = cy >= 1 && cy < P3::CH - 1, row0 = cy >= 2 && cy < P3::CH - 2;
    const int gx = x0 - 2 + cx, gy = y0 - 2 + cy;
    const bool own = in0 && gx < nx && gy < ny;
    const bool hyd = p.hydro != 0;
    bool bad = false;

    for (int q = t; q < W3 + P3::H3; q += NTH) {
        if (q < W3) colmap[q] = wrap_s(x0 - 3 + q, nx);
        else rowmap[q - W3] = wrap_s(y0 - 3 + (q - W3), ny);
    }
    __syncthreads();
    const int col_off = rowmap[cy + 1] * pitch + colmap[cx + 1];
    const int c3 = (cy + 1) * W3 + cx + 1;
    const int c2 = t;
    static_assert(A3 <= 2 * NTH, "at most two phi elements per thread");
    const int qe = t + NTH;
    const bool two = qe < A3;
    const int oe0 = rowmap[t / W3] * pitch + colmap[t % W3];
    const int oe1 = two ? rowmap[qe / W3] * pitch + colmap[qe % W3] : 0;

    auto fetch = [&](int z, int slot) {
        if (z <= kphi) {
            const int pz = map_z(z, nz, walls) * zs;
            R* d = sphi + slot * A3;
            cp_async_s<sizeof(R)>(&d[t], io.phi_in + (pz + oe0));
            if (two) cp_async_s<sizeof(R)>(&d[qe], io.phi_in + (pz + oe1));
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    Slide19<R> sphi19, spsi19;
    R ph1 = 0, ph2 = 0, ph3 = 0;                     // own phi(k-1), phi(k-2), phi(k-3)
    R ps1 = 0, ps2 = 0;                              // own psi(k-2), psi(k-3)
    R dx1 = 0, dy1 = 0, dz1 = 0, dx2 = 0, dy2 = 0, dz2 = 0;   // grad phi(k-2), grad phi(k-3)
    R oxz = 0, oyz = 0, ozz = 0;                     // own P_xz, P_yz, P_zz of plane k-4
    R aFx = 0, aFy = 0, aFz = 0, bFx = 0, bFy = 0, bFz = 0;   // -12 F: open sums of centre k-5, parts of plane k-5 for k-4

    // iteration k; PAR = (k - kbeg) & 1 selects the ring slots.  The stage
    // predicates depend on the row of the column only (a warp is one row of
    // the psi region): the halo lanes of a row run the stage too, on
    // neighbours that stay inside the shared allocation, and neither their
    // mu nor their F is stored (their P lands in columns nobody reads).
    auto iter = [&](int k, auto par_c) {
        constexpr int PAR = decltype(par_c)::value;
        const int z2 = k - 3;                            // mu / P plane of this iteration
        const bool st2 = row1 && k >= z0 && k <= z1 + 3;
        R Tc = R(0);
        if (st2 && z2 >= z0 - 1) Tc = io.T_in[map_z(z2, nz, walls) * zs + col_off];
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        fetch(k + 1, PAR ^ 1);

        // ---- phi plane k: psi and grad phi at k - 1 (every column) ------------------
        R phk = R(0), psk = R(0), dxk = R(0), dyk = R(0), dzk = R(0);
        if (k <= kphi) {
            const R* a = sphi + PAR * A3;
            phk = a[c3];
            sphi19.push(plane19<R, W3>(a, c3, phk), psk, dxk, dyk, dzk);
            spsi[(PAR ^ 1) * A2 + c2] = psk;             // slot of psi(k - 1)
        }

        // ---- psi plane k - 2: lam, grad psi, mu, P at k - 3 (r = 1) --------------------
        R nxz = R(0), nyz = R(0), nzz = R(0);
        if (st2) {
            const R* b = spsi + PAR * A2;                // psi(k - 2)
            R lam, s0, s1, s2;
            spsi19.push(plane19<R, CW>(b, c2, ps1), lam, s0, s1, s2);
            if (z2 >= z0 - 1) {
                const R ph = ph3, psi = ps2;
                const R av = (Tc - p.Tc) * p.inv_Tc;
                if (own && z2 >= z0 && z2 < z1) {
                    const R mu = av * ph + p.b * ph * ph * ph - p.kappa * psi + p.c * lam;
                    bad |= !isfinite(mu);
                    io.mu[z2 * zs + gy * pitch + gx] = mu;
                }
                if (hyd) {
                    const R d0 = dx2, d1 = dy2, d2 = dz2;
                    const R ph2_ = ph * ph;
                    const R iso = av * ph2_ * half + R(0.75) * p.b * ph2_ * ph2_
                                - p.kappa * (ph * psi + half * (d0 * d0 + d1 * d1 + d2 * d2))
                                + p.c * (ph * lam + half * psi * psi + d0 * s0 + d1 * s1 + d2 * s2);
                    R* P = sP + (PAR ^ 1) * 6 * A2;          // slot of P(k - 3)
                    nxz = p.kappa * d0 * d2 - p.c * (d0 * s2 + d2 * s0);
                    nyz = p.kappa * d1 * d2 - p.c * (d1 * s2 + d2 * s1);
                    nzz = iso + p.kappa * d2 * d2 - R(2) * p.c * d2 * s2;
                    P[0 * A2 + c2] = iso + p.kappa * d0 * d0 - R(2) * p.c * d0 * s0;
                    P[1 * A2 + c2] = p.kappa * d0 * d1 - p.c * (d0 * s1 + d1 * s0);
                    P[2 * A2 + c2] = iso + p.kappa * d1 * d1 - R(2) * p.c * d1 * s1;
                    P[3 * A2 + c2] = nxz;
                    P[4 * A2 + c2] = nyz;
                    P[5 * A2 + c2] = nzz;
                }
            }
        }

        // ---- P plane k - 4: F at k - 5 (the tile) --------------------------------------
        if (hyd && row0 && k >= z0 + 3 && k <= kend) {
            const R* P = sP + PAR * 6 * A2;              // P(k - 4)
            const Plane19<R> xx = plane19<R, CW>(P + 0 * A2, c2, R(0));
            const Plane19<R> xy = plane19<R, CW>(P + 1 * A2, c2, R(0));
            const Plane19<R> yy = plane19<R, CW>(P + 2 * A2, c2, R(0));
            const Plane19<R> xz = plane19<R, CW>(P + 3 * A2, c2, oxz);
            const Plane19<R> yz = plane19<R, CW>(P + 4 * A2, c2, oyz);
            const R zc = (P[5 * A2 + c2 + 1] + P[5 * A2 + c2 - 1]) + (P[5 * A2 + c2 + CW] + P[5 * A2 + c2 - CW]);
            const R szz = R(2) * ozz + zc;
            // -12 F(m) = O(m) + [A(m - 1) - s(m - 1)] + [A(m + 1) + s(m + 1)], per component
            const R Ox = xx.gx + xy.gy, Ax = xx.ax + xy.ay;
            const R Oy = xy.gx + yy.gy, Ay = xy.ax + yy.ay;
            const R Oz = xz.gx + yz.gy, Az = xz.ax + yz.ay;
            if (own && k >= z0 + 5) {
                const int site = (k - 5) * zs + gy * pitch + gx;
                io.F[0][site] = -(aFx + (Ax + xz.s)) * R(1.0 / 12.0);
                io.F[1][site] = -(aFy + (Ay + yz.s)) * R(1.0 / 12.0);
                io.F[2][site] = -(aFz + (Az + szz)) * R(1.0 / 12.0);
            }
            aFx = Ox + bFx; aFy = Oy + bFy; aFz = Oz + bFz;
            bFx = Ax - xz.s; bFy = Ay - yz.s; bFz = Az - szz;
        }

        // shift the windows
        ph3 = ph2; ph2 = ph1; ph1 = phk;
        ps2 = ps1; ps1 = psk;
        dx2 = dx1; dy2 = dy1; dz2 = dz1; dx1 = dxk; dy1 = dyk; dz1 = dzk;
        oxz = nxz; oyz = nyz; ozz = nzz;
    };

    fetch(kbeg, 0);
    // two iterations per trip, so that slots and window shifts are fixed in
    // each copy; an odd count ends with one more iteration whose stages are all
    // out of range (only its barrier runs)
    for (int k = kbeg; k <= kend; k += 2) {
        iter(k, std::integral_constant<int, 0>{});
        iter(k + 1, std::integral_constant<int, 1>{});
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (__any_sync(0xffffffffu, bad) && (t & 31) == 0) *reinterpret_cast<volatile int*>(io.flag) = 1;
}

// The sliding-sum isotropic pass A on two z-segments at once (FP32): lane .x
// marches planes [z0, z0 + H), lane .y planes [z0 + H, z0 + 2H) (shorter or
// empty at the top of the lattice), with the stages and lags of
// k_force3d_iso, float2 shared planes (one 64-bit load brings a neighbour of
// both lanes) and packed FP32x2 arithmetic throughout.
template <int TX, int TY>
struct Force3IsoX2 {
    static constexpr int CW = TX + 4, CH = TY + 4, NTH = CW * CH;
    static constexpr int W3 = TX + 6, H3 = TY + 6, A3 = W3 * H3;
    static constexpr int A2 = CW * CH;
    static constexpr int PHI = 0;                                   // [2][A3] float2
    static constexpr int PSI = PHI + 2 * A3;                        // [2][A2]
    static constexpr int PP = PSI + 2 * A2;                         // [2][6][A2]
    static constexpr int TOTAL = PP + 12 * A2;
    static constexpr size_t MAPS = sizeof(float2) * TOTAL;
    static constexpr size_t BYTES = MAPS + sizeof(int) * (W3 + H3);
};

namespace iso2 {
using namespace march;
struct Plane {
    float2 s, l, gx, gy, ax, ay;
};
template <int W>
__device__ __forceinline__ Plane plane(const float2* a, int c, float2 ac)
{
    const float2 e = a[c + 1], w = a[c - 1], n = a[c + W], so = a[c - W];
    const float2 ne = a[c + W + 1], nw = a[c + W - 1], se = a[c - W + 1], sw = a[c - W - 1];
    const float2 cross = add2(add2(e, w), add2(n, so));
    Plane r;
    r.s = fma2(v2(2.f), ac, cross);
    r.l = fma2(v2(-24.f), ac, fma2(v2(2.f), cross, add2(add2(ne, nw), add2(se, sw))));
    r.ax = sub2(e, w);
    r.ay = sub2(n, so);
    r.gx = fma2(v2(2.f), r.ax, add2(sub2(ne, nw), sub2(se, sw)));
    r.gy = fma2(v2(2.f), r.ay, add2(sub2(ne, se), sub2(nw, sw)));
    return r;
}
struct Slide {
    float2 l = v2(0.f), gx = v2(0.f), gy = v2(0.f), s_prev = v2(0.f), s = v2(0.f), ax = v2(0.f), ay = v2(0.f);
    __device__ __forceinline__ void push(const Plane& q, float2& lap, float2& dx, float2& dy, float2& dz)
    {
        lap = mul2(add2(l, q.s), v2(1.f / 6.f));
        dx = mul2(add2(gx, q.ax), v2(1.f / 12.f));
        dy = mul2(add2(gy, q.ay), v2(1.f / 12.f));
        dz = mul2(sub2(q.s, s_prev), v2(1.f / 12.f));
        l = add2(q.l, s);
        gx = add2(q.gx, ax);
        gy = add2(q.gy, ay);
        s_prev = s;
        s = q.s;
        ax = q.ax;
        ay = q.ay;
    }
};
}  // namespace iso2

template <int TX, int TY>
__global__ void __launch_bounds__(Force3IsoX2<TX, TY>::NTH, 1) k_force3d_iso_x2(Geom g, Phys<float> p, StepIO<float> io, int H)
{
    using namespace march;
    using P3 = Force3IsoX2<TX, TY>;
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
    // relative plane j of lane L is plane z0_L + j; phi planes j = -3 .. hmax + 2,
    // iterations j = -3 .. hmax + 4
    const int jphi = hmax + 2, jend = hmax + 4;
    const bool in0 = cx >= 2 && cx < CW - 2 && cy >= 2 && cy < P3::CH - 2;
    const bool row1 = cy >= 1 && cy < P3::CH - 1, row0 = cy >= 2 && cy < P3::CH - 2;
    const int gx = x0 - 2 + cx, gy = y0 - 2 + cy;
    const bool own = in0 && gx < nx && gy < ny;
    const int own_off = gy * pitch + gx;
    const bool hyd = p.hydro != 0;
    bool bad = false;

    for (int q = t; q < W3 + P3::H3; q += NTH) {
        if (q < W3) colmap[q] = wrap_s(x0 - 3 + q, nx);
        else rowmap[q - W3] = wrap_s(y0 - 3 + (q - W3), ny);
    }
    __syncthreads();
    const int col_off = rowmap[cy + 1] * pitch + colmap[cx + 1];
    const int c3 = (cy + 1) * W3 + cx + 1;
    const int c2 = t;
    static_assert(A3 <= 2 * NTH, "at most two phi elements per thread");
    const int qe = t + NTH;
    const bool two = qe < A3;
    const int oe0 = rowmap[t / W3] * pitch + colmap[t % W3];
    const int oe1 = two ? rowmap[qe / W3] * pitch + colmap[qe % W3] : 0;

    // storage offsets pa, pb of the planes to fetch into ring slot `slot`
    auto fetch_at = [&](int pa, int pb, int slot) {
        float* d = reinterpret_cast<float*>(sphi + slot * A3);
        cp_async_s<4>(d + 2 * t, io.phi_in + (pa + oe0));
        cp_async_s<4>(d + 2 * t + 1, io.phi_in + (pb + oe0));
        if (two) {
            cp_async_s<4>(d + 2 * qe, io.phi_in + (pa + oe1));
            cp_async_s<4>(d + 2 * qe + 1, io.phi_in + (pb + oe1));
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    auto fetch = [&](int j, int slot) {
        if (j <= jphi) {
            fetch_at(map_z(za0 + j, nz, walls) * zs, map_z(zb0 + j, nz, walls) * zs, slot);
            return;
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    const int zs3 = 3 * zs, zs5 = 5 * zs;

    iso2::Slide sphi19, spsi19;
    float2 ph1 = v2(0.f), ph2 = v2(0.f), ph3 = v2(0.f);        // own phi(j-1), phi(j-2), phi(j-3)
    float2 ps1 = v2(0.f), ps2 = v2(0.f);                       // own psi(j-2), psi(j-3)
    float2 dx1 = v2(0.f), dy1 = v2(0.f), dz1 = v2(0.f), dx2 = v2(0.f), dy2 = v2(0.f), dz2 = v2(0.f);
    float2 oxz = v2(0.f), oyz = v2(0.f), ozz = v2(0.f);        // own P_xz, P_yz, P_zz of plane j-4
    float2 aFx = v2(0.f), aFy = v2(0.f), aFz = v2(0.f), bFx = v2(0.f), bFy = v2(0.f), bFz = v2(0.f);
    const float2 half = v2(0.5f), k_ = v2(p.kappa), mc = v2(-p.c), m2c = v2(-2.f * p.c);

    // iteration j; PAR = (j + 3) & 1 selects the ring slots.  FULL: an
    // iteration of the steady state (j in [5, hmin - 2]), in which every stage
    // runs, every plane it touches lies inside both lanes' ranges and inside
    // the lattice, and all its outputs are stored: no range checks, no plane
    // mapping.
    const int hmin = ha < hb ? ha : hb;
    auto iter = [&](int j, auto par_c, auto full_c) {
        constexpr int PAR = decltype(par_c)::value;
        constexpr bool FULL = decltype(full_c)::value;
        const int r2 = j - 3;                               // mu / P plane of this iteration
        const int ba = (za0 + j) * zs, bb = (zb0 + j) * zs; // plane j of each lane (FULL only)
        const bool st2 = FULL ? row1 : row1 && j >= 0 && j <= hmax + 3;
        float2 Tc = v2(0.f);
        if constexpr (FULL) {
            if (row1) Tc = make_float2(io.T_in[ba - zs3 + col_off], io.T_in[bb - zs3 + col_off]);
        } else if (st2 && r2 >= -1) {
            Tc = make_float2(io.T_in[map_z(za0 + r2, nz, walls) * zs + col_off],
                             io.T_in[map_z(zb0 + r2, nz, walls) * zs + col_off]);
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        if constexpr (FULL) fetch_at(ba + zs, bb + zs, PAR ^ 1);
        else fetch(j + 1, PAR ^ 1);

        // phi plane j: psi and grad phi at j - 1 (every column)
        float2 phk, psk, dxk, dyk, dzk;
        if (FULL || j <= jphi) {
            const float2* a = sphi + PAR * A3;
            phk = a[c3];
            sphi19.push(iso2::plane<W3>(a, c3, phk), psk, dxk, dyk, dzk);
            spsi[(PAR ^ 1) * A2 + c2] = psk;
        } else {
            phk = psk = dxk = dyk = dzk = v2(0.f);
        }

        // psi plane j - 2: lam, grad psi, mu, P at j - 3 (rows of the r = 1 region)
        float2 nxz = v2(0.f), nyz = v2(0.f), nzz = v2(0.f);
        if (st2) {
            float2 lam, s0, s1, s2;
            spsi19.push(iso2::plane<CW>(spsi + PAR * A2, c2, ps1), lam, s0, s1, s2);
            if (FULL || r2 >= -1) {
                const float2 ph = ph3, psi = ps2;
                const float2 av = mul2(sub2(Tc, v2(p.Tc)), v2(p.inv_Tc));
                const float2 phsq = mul2(ph, ph);
                if (own && (FULL || r2 >= 0)) {
                    const float2 mu = fma2(v2(p.c), lam, fma2(v2(-p.kappa), psi, mul2(ph, fma2(v2(p.b), phsq, av))));
                    if constexpr (FULL) {
                        bad |= !isfinite(mu.x) || !isfinite(mu.y);
                        io.mu[ba - zs3 + own_off] = mu.x;
                        io.mu[bb - zs3 + own_off] = mu.y;
                    } else {
                        if (r2 < ha) { bad |= !isfinite(mu.x); io.mu[(za0 + r2) * zs + own_off] = mu.x; }
                        if (r2 < hb) { bad |= !isfinite(mu.y); io.mu[(zb0 + r2) * zs + own_off] = mu.y; }
                    }
                }
                if (hyd) {
                    const float2 d0 = dx2, d1 = dy2, d2 = dz2;
                    const float2 gp2 = fma2(d0, d0, fma2(d1, d1, mul2(d2, d2)));
                    const float2 gpgs = fma2(d0, s0, fma2(d1, s1, mul2(d2, s2)));
                    float2 iso = mul2(phsq, fma2(v2(0.75f * p.b), phsq, mul2(half, av)));
                    iso = fma2(v2(-p.kappa), fma2(half, gp2, mul2(ph, psi)), iso);
                    iso = fma2(v2(p.c), add2(fma2(ph, lam, mul2(half, mul2(psi, psi))), gpgs), iso);
                    float2* P = sP + (PAR ^ 1) * 6 * A2;
                    nxz = fma2(k_, mul2(d0, d2), mul2(mc, fma2(d0, s2, mul2(d2, s0))));
                    nyz = fma2(k_, mul2(d1, d2), mul2(mc, fma2(d1, s2, mul2(d2, s1))));
                    nzz = fma2(k_, mul2(d2, d2), fma2(m2c, mul2(d2, s2), iso));
                    P[0 * A2 + c2] = fma2(k_, mul2(d0, d0), fma2(m2c, mul2(d0, s0), iso));
                    P[1 * A2 + c2] = fma2(k_, mul2(d0, d1), mul2(mc, fma2(d0, s1, mul2(d1, s0))));
                    P[2 * A2 + c2] = fma2(k_, mul2(d1, d1), fma2(m2c, mul2(d1, s1), iso));
                    P[3 * A2 + c2] = nxz;
                    P[4 * A2 + c2] = nyz;
                    P[5 * A2 + c2] = nzz;
                }
            }
        }

        // P plane j - 4: F at j - 5 (rows of the tile)
        if (hyd && row0 && (FULL || (j >= 3 && j <= jend))) {
            const float2* P = sP + PAR * 6 * A2;
            const iso2::Plane xx = iso2::plane<CW>(P + 0 * A2, c2, v2(0.f));
            const iso2::Plane xy = iso2::plane<CW>(P + 1 * A2, c2, v2(0.f));
            const iso2::Plane yy = iso2::plane<CW>(P + 2 * A2, c2, v2(0.f));
            const iso2::Plane xz = iso2::plane<CW>(P + 3 * A2, c2, oxz);
            const iso2::Plane yz = iso2::plane<CW>(P + 4 * A2, c2, oyz);
            const float2* pz = P + 5 * A2;
            const float2 szz = fma2(v2(2.f), ozz, add2(add2(pz[c2 + 1], pz[c2 - 1]), add2(pz[c2 + CW], pz[c2 - CW])));
            const float2 Ox = add2(xx.gx, xy.gy), Ax = add2(xx.ax, xy.ay);
            const float2 Oy = add2(xy.gx, yy.gy), Ay = add2(xy.ax, yy.ay);
            const float2 Oz = add2(xz.gx, yz.gy), Az = add2(xz.ax, yz.ay);
            const int r5 = j - 5;
            if (own && (FULL || r5 >= 0)) {
                const float2 m12 = v2(-1.f / 12.f);
                const float2 Fx = mul2(add2(aFx, add2(Ax, xz.s)), m12);
                const float2 Fy = mul2(add2(aFy, add2(Ay, yz.s)), m12);
                const float2 Fz = mul2(add2(aFz, add2(Az, szz)), m12);
                if (FULL || r5 < ha) {
                    const int site = (FULL ? ba - zs5 : (za0 + r5) * zs) + own_off;
                    io.F[0][site] = Fx.x; io.F[1][site] = Fy.x; io.F[2][site] = Fz.x;
                }
                if (FULL || r5 < hb) {
                    const int site = (FULL ? bb - zs5 : (zb0 + r5) * zs) + own_off;
                    io.F[0][site] = Fx.y; io.F[1][site] = Fy.y; io.F[2][site] = Fz.y;
                }
            }
            aFx = add2(Ox, bFx); aFy = add2(Oy, bFy); aFz = add2(Oz, bFz);
            bFx = sub2(Ax, xz.s); bFy = sub2(Ay, yz.s); bFz = sub2(Az, szz);
        }

        ph3 = ph2; ph2 = ph1; ph1 = phk;
        ps2 = ps1; ps1 = psk;
        dx2 = dx1; dy2 = dy1; dz2 = dz1; dx1 = dxk; dy1 = dyk; dz1 = dzk;
        oxz = nxz; oyz = nyz; ozz = nzz;
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using GEN = std::false_type;
    using STEADY = std::true_type;

    fetch(-3, 0);
    int j = -3;
    // warm-up iterations -3 .. 4, the steady state in pairs, then the rest
    // (an odd count ends with one iteration whose stages are all out of range)
#pragma unroll 1
    for (; j < 5; j += 2) {
        iter(j, I0{}, GEN{});
        iter(j + 1, I1{}, GEN{});
    }
#pragma unroll 1
    for (; j + 1 <= hmin - 2; j += 2) {
        iter(j, I0{}, STEADY{});
        iter(j + 1, I1{}, STEADY{});
    }
#pragma unroll 1
    for (; j <= jend; j += 2) {
        iter(j, I0{}, GEN{});
        iter(j + 1, I1{}, GEN{});
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (__any_sync(0xffffffffu, bad) && (t & 31) == 0) *reinterpret_cast<volatile int*>(io.flag) = 1;
}

constexpr int kIsoTW = 34, kIsoTA = kIsoTW * 10, kIsoNF = 5;   // tile + 1 (32 x 8 + halo); mu, T, g_x, g_y, g_z

// Pass C with the isotropic stencils as a column march with sliding sums
// (Plane19 in lf_iso3.cuh).  A 32 x 8 block stages one plane of mu, T and the
// fluxes g = phi u on the tile grown by one site in a two-slot shared ring;
// each thread loads the in-plane neighbours of the new plane k once, keeps the
// open sums of its column in registers and completes phi(t+1) and the first
// temperature sub-step at k - 1.  Plane k + 1 is loaded into registers before
// the arithmetic of plane k and stored into the slot of plane k - 1 after it,
// so one barrier per plane orders the ring.  A plane beyond a wall holds the
// wall plane, and its parts enter the sums transformed: mu, g_x and g_y even
// (unchanged), g_z odd (s negated), T the halfway ghost 2 T_w - T (s -> 12 T_w - s).
template <typename R>
__global__ void __launch_bounds__(256) k_phi3d_isoz(Geom g, Phys<R> p, StepIO<R> io, int zc)
{
    constexpr int TW = kIsoTW, TA = kIsoTA, NF = kIsoNF;
    extern __shared__ __align__(16) unsigned char smem_iso[];
    R (*sm)[NF][TA] = reinterpret_cast<R (*)[NF][TA]>(smem_iso);     // [2 slots][NF][TA]
    const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8;
    const int za = blockIdx.z * zc, zb = min(za + zc, g.nz);
    const int nx = g.nx, ny = g.ny, nz = g.nz, pitch = g.pitch, walls = g.walls;
    const int64_t zs = (int64_t)ny * pitch;
    const bool hyd = p.hydro != 0;
    const bool halfway = walls && g.t_mode == LF_TWALL_HALFWAY;
    const R* __restrict__ mu = io.mu;
    const R* __restrict__ ph = io.phi_in;
    const R* __restrict__ T = io.T_in;
    const R* __restrict__ ux = io.u[0];
    const R* __restrict__ uy = io.u[1];
    const R* __restrict__ uz = io.u[2];
    auto zmap = [&](int zl) -> int64_t {
        int z = zl;
        if (walls) z = z < 0 ? 0 : (z >= nz ? nz - 1 : z);
        else z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
        return (int64_t)z * zs;
    };
    int64_t off[2];
    bool has[2];
    for (int i = 0; i < 2; ++i) {
        const int q = t + 256 * i;
        has[i] = q < TA;
        const int ly = has[i] ? q / TW : 0, lx = has[i] ? q - ly * TW : 0;
        int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
        gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
        off[i] = (int64_t)gy * pitch + gx;
    }
    R v[2][NF];
    auto fetch = [&](int zl) {
        const int64_t pz = zmap(zl);
        for (int i = 0; i < 2; ++i) {
            if (!has[i]) continue;
            const int64_t o = pz + off[i];
            v[i][0] = mu[o];
            v[i][1] = T[o];
            const R f = ph[o];
            v[i][2] = hyd ? f * ux[o] : R(0);
            v[i][3] = hyd ? f * uy[o] : R(0);
            v[i][4] = hyd ? f * uz[o] : R(0);
        }
    };
    auto put = [&](int zl) {
        const int sl = (zl - za + 1) & 1;
        for (int i = 0; i < 2; ++i)
            if (has[i])
                for (int f = 0; f < NF; ++f) sm[sl][f][t + 256 * i] = v[i][f];
    };
    const int x = x0 + tx, y = y0 + ty;
    const bool act = x < nx && y < ny;
    const int c = (ty + 1) * TW + tx + 1;
    const int64_t col = (int64_t)y * pitch + x;
    Slide19<R> smu, sT, sgx, sgy, sgz;
    R Tc1 = R(0);                                           // own T of plane k - 1
    bool bad = false;
    fetch(za - 1);
    put(za - 1);
    for (int k = za - 1; k <= zb; ++k) {
        __syncthreads();                                    // plane k is in its slot
        if (k < zb) fetch(k + 1);                           // in flight during the arithmetic below
        const int s0 = (k - za + 1) & 1;
        const bool ghost = walls && (k < 0 || k >= nz);
        const R Tck = sm[s0][1][c];
        Plane19<R> qm = plane19<R, TW>(sm[s0][0], c, sm[s0][0][c]);
        Plane19<R> qT = plane19<R, TW>(sm[s0][1], c, Tck);
        Plane19<R> qx = plane19<R, TW>(sm[s0][2], c, R(0));
        Plane19<R> qy = plane19<R, TW>(sm[s0][3], c, R(0));
        Plane19<R> qz = plane19<R, TW>(sm[s0][4], c, sm[s0][4][c]);
        if (ghost) {
            qz.s = -qz.s;
            if (halfway) qT.s = R(12) * p.T_w - qT.s;
        }
        R lapmu, lapT, dgx, dgy, dgz, u0, u1, u2;
        smu.push(qm, lapmu, u0, u1, u2);
        sT.push(qT, lapT, u0, u1, u2);
        sgx.push(qx, u0, dgx, u1, u2);
        sgy.push(qy, u0, u1, dgy, u2);
        sgz.push(qz, u0, u1, u2, dgz);
        const int m = k - 1;                                // the plane completed by plane k
        if (act && k > za) {
            const int64_t site = (int64_t)m * zs + col;
            const R div = hyd ? (dgx + dgy) + dgz : R(0);
            const R phn = ph[site] - div + p.Gamma * lapmu;
            io.phi_out[site] = phn;
            R Tn = Tc1;
            if (p.t_update) {
                if (walls && g.t_mode == LF_TWALL_LAYERS && (m == 0 || m == nz - 1)) Tn = p.T_w;
                else Tn = Tc1 + p.dxi * lapT;
            }
            io.T_out[site] = Tn;
            bad |= !isfinite(phn) || !isfinite(Tn);
        }
        Tc1 = Tck;
        if (k < zb) put(k + 1);                             // slot of plane k - 1, read by nobody now
    }
    if (__any_sync(0xffffffffu, bad) && (t & 31) == 0) *reinterpret_cast<volatile int*>(io.flag) = 1;
}

// Pass C with the raw fields staged by cp.async: mu, T, phi, u_x, u_y, u_z of
// the tile grown by one site go straight from global to a three-slot shared
// ring, two planes ahead of their use, and the fluxes g = phi u are formed
// where they are read.  The sums and wall rules are those of k_phi3d_isoz.
constexpr int kIsoNR = 6;   // mu, T, phi, u_x, u_y, u_z

template <typename R>
__global__ void __launch_bounds__(256) k_phi3d_isoa(Geom g, Phys<R> p, StepIO<R> io, int zc)
{
    constexpr int TW = kIsoTW, TA = kIsoTA, NF = kIsoNR;
    extern __shared__ __align__(16) unsigned char smem_iso[];
    R (*sm)[NF][TA] = reinterpret_cast<R (*)[NF][TA]>(smem_iso);     // [3 slots][NF][TA]
    const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8;
    const int za = blockIdx.z * zc, zb = min(za + zc, g.nz);
    const int nx = g.nx, ny = g.ny, nz = g.nz, pitch = g.pitch, walls = g.walls;
    const int64_t zs = (int64_t)ny * pitch;
    const bool hyd = p.hydro != 0;
    const bool halfway = walls && g.t_mode == LF_TWALL_HALFWAY;
    auto zmap = [&](int zl) -> int64_t {
        int z = zl;
        if (walls) z = z < 0 ? 0 : (z >= nz ? nz - 1 : z);
        else z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
        return (int64_t)z * zs;
    };
    int64_t off[2];
    bool has[2];
    for (int i = 0; i < 2; ++i) {
        const int q = t + 256 * i;
        has[i] = q < TA;
        const int ly = has[i] ? q / TW : 0, lx = has[i] ? q - ly * TW : 0;
        int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
        gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
        off[i] = (int64_t)gy * pitch + gx;
    }
    const R* src[NF] = {io.mu, io.T_in, io.phi_in, io.u[0], io.u[1], io.u[2]};
    const int nf = hyd ? NF : 2;
    // plane zl (za - 1 .. zb) into slot (zl - za + 1) mod 3; one commit group per call
    auto fetch = [&](int zl) {
        if (zl <= zb) {
            const int sl = (zl - za + 1) % 3;
            const int64_t pz = zmap(zl);
            for (int i = 0; i < 2; ++i)
                if (has[i])
                    for (int f = 0; f < nf; ++f) cp_async_s<sizeof(R)>(&sm[sl][f][t + 256 * i], src[f] + (pz + off[i]));
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    const int x = x0 + tx, y = y0 + ty;
    const bool act = x < nx && y < ny;
    const int c = (ty + 1) * TW + tx + 1;
    const int64_t col = (int64_t)y * pitch + x;
    Slide19<R> smu, sT, sgx, sgy, sgz;
    R Tc1 = R(0);
    bool bad = false;
    fetch(za - 1);
    fetch(za);
    for (int k = za - 1; k <= zb; ++k) {
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // plane k has landed (k + 1 may be in flight)
        __syncthreads();
        fetch(k + 2);                                       // into the slot of plane k - 1
        const int s0 = (k - za + 1) % 3;
        const bool ghost = walls && (k < 0 || k >= nz);
        const R* M = sm[s0][0];
        const R* TT = sm[s0][1];
        const R Tck = TT[c];
        Plane19<R> qm = plane19<R, TW>(M, c, M[c]);
        Plane19<R> qT = plane19<R, TW>(TT, c, Tck);
        Plane19<R> qx{}, qy{}, qz{};
        if (hyd) {
            const R* F = sm[s0][2];
            const R* UX = sm[s0][3];
            const R* UY = sm[s0][4];
            const R* UZ = sm[s0][5];
            auto gxa = [&](int o) { return F[c + o] * UX[c + o]; };
            auto gya = [&](int o) { return F[c + o] * UY[c + o]; };
            auto gza = [&](int o) { return F[c + o] * UZ[c + o]; };
            const R xe = gxa(1), xw = gxa(-1), xne = gxa(TW + 1), xnw = gxa(TW - 1), xse = gxa(-TW + 1),
                    xsw = gxa(-TW - 1);
            qx.ax = xe - xw;
            qx.gx = R(2) * qx.ax + (xne - xnw) + (xse - xsw);
            const R yn = gya(TW), ys = gya(-TW), yne = gya(TW + 1), ynw = gya(TW - 1), yse = gya(-TW + 1),
                    ysw = gya(-TW - 1);
            qy.ay = yn - ys;
            qy.gy = R(2) * qy.ay + (yne - yse) + (ynw - ysw);
            qz.s = R(2) * gza(0) + ((gza(1) + gza(-1)) + (gza(TW) + gza(-TW)));
        }
        if (ghost) {
            qz.s = -qz.s;
            if (halfway) qT.s = R(12) * p.T_w - qT.s;
        }
        R lapmu, lapT, dgx, dgy, dgz, u0, u1, u2;
        smu.push(qm, lapmu, u0, u1, u2);
        sT.push(qT, lapT, u0, u1, u2);
        sgx.push(qx, u0, dgx, u1, u2);
        sgy.push(qy, u0, u1, dgy, u2);
        sgz.push(qz, u0, u1, u2, dgz);
        const int m = k - 1;
        if (act && k > za) {
            const int64_t site = (int64_t)m * zs + col;
            const R div = hyd ? (dgx + dgy) + dgz : R(0);
            const R phn = io.phi_in[site] - div + p.Gamma * lapmu;
            io.phi_out[site] = phn;
            R Tn = Tc1;
            if (p.t_update) {
                if (walls && g.t_mode == LF_TWALL_LAYERS && (m == 0 || m == nz - 1)) Tn = p.T_w;
                else Tn = Tc1 + p.dxi * lapT;
            }
            io.T_out[site] = Tn;
            bad |= !isfinite(phn) || !isfinite(Tn);
        }
        Tc1 = Tck;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (__any_sync(0xffffffffu, bad) && (t & 31) == 0) *reinterpret_cast<volatile int*>(io.flag) = 1;
}

template <typename R, int TX, int TY, int MINB>
cudaError_t launch_force_iso(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s)
{
    using P3 = Force3Iso<R, TX, TY>;
    auto kern = k_force3d_iso<R, TX, TY, MINB>;
    static unsigned long long attr_done = 0;      // per instantiation and device
    const cudaError_t e = raise_smem_limit(kern, (int)P3::BYTES, &attr_done);
    if (e != cudaSuccess) return e;
    const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    int Hz = (g.tune & 0xFFFF) > 0 ? (g.tune & 0xFFFF) : 0;
    if (Hz <= 0) {   // about eight waves of the resident CTAs, segments of at least 16 planes
        const int want = (8 * MINB * 152 + tiles - 1) / tiles;
        Hz = (g.nz + want - 1) / want;
        if (Hz < 16) Hz = 16;
    }
    if (Hz > g.nz) Hz = g.nz;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + Hz - 1) / Hz);
    kern<<<grid, P3::NTH, P3::BYTES, s>>>(g, p, io, Hz);
    return cudaGetLastError();
}

template <int TX, int TY>
cudaError_t launch_force_iso_x2(const Geom& g, const Phys<float>& p, const StepIO<float>& io, cudaStream_t s)
{
    using P3 = Force3IsoX2<TX, TY>;
    auto kern = k_force3d_iso_x2<TX, TY>;
    static unsigned long long attr_done = 0;      // per instantiation and device
    const cudaError_t e = raise_smem_limit(kern, (int)P3::BYTES, &attr_done);
    if (e != cudaSuccess) return e;
    const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    int H = (g.tune & 0xFFFF) > 0 ? (g.tune & 0xFFFF) : 0;     // planes per lane
    if (H <= 0) {   // about eight waves of one CTA per SM, lanes of at least 16 planes
        const int want = (8 * 152 + tiles - 1) / tiles;
        H = (g.nz + 2 * want - 1) / (2 * want);
        if (H < 16) H = 16;
    }
    if (H > g.nz) H = g.nz;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + 2 * H - 1) / (2 * H));
    kern<<<grid, P3::NTH, P3::BYTES, s>>>(g, p, io, H);
    return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_force3d_iso(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s)
{
    // (param >> 16) & 15: 0 = one lane on 28x12 tiles (FP32: two CTAs per SM),
    // 1 = one lane on 28x28 tiles, 3 = one lane on 28x12 tiles at one CTA per
    // SM, 4 = two z-lanes in packed FP32x2 on 28x12 tiles (1, 3, 4: FP32 only)
    const int sel = (g.tune >> 16) & 15;
    if constexpr (sizeof(R) == 4) {
        return sel == 1 ? launch_force_iso<R, 28, 28, 1>(g, p, io, s)
             : sel == 3 ? launch_force_iso<R, 28, 12, 1>(g, p, io, s)
             : sel == 4 ? launch_force_iso_x2<28, 12>(g, p, io, s)
                        : launch_force_iso<R, 28, 12, 2>(g, p, io, s);
    } else {
        return launch_force_iso<R, 28, 12, 1>(g, p, io, s);
    }
}

template <typename R>
cudaError_t launch_phi3d_iso(const Geom& g, const Phys<R>& p, const StepIO<R>& io, int zc, cudaStream_t s)
{
    dim3 gc((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + zc - 1) / zc);
    if ((g.tune >> 28) & 1) {                           // param bit 28: the raw fields staged by cp.async
        constexpr size_t bytes = sizeof(R) * 3 * kIsoNR * kIsoTA;
        static unsigned long long attr_done = 0;
        const cudaError_t e = raise_smem_limit(k_phi3d_isoa<R>, (int)bytes, &attr_done);
        if (e != cudaSuccess) return e;
        k_phi3d_isoa<R><<<gc, 256, bytes, s>>>(g, p, io, zc);
        return cudaGetLastError();
    }
    constexpr size_t bytes = sizeof(R) * 2 * kIsoNF * kIsoTA;
    static unsigned long long attr_done = 0;
    const cudaError_t e = raise_smem_limit(k_phi3d_isoz<R>, (int)bytes, &attr_done);
    if (e != cudaSuccess) return e;
    k_phi3d_isoz<R><<<gc, 256, bytes, s>>>(g, p, io, zc);
    return cudaGetLastError();
}

template cudaError_t launch_force3d_iso<float>(const Geom&, const Phys<float>&, const StepIO<float>&, cudaStream_t);
template cudaError_t launch_force3d_iso<double>(const Geom&, const Phys<double>&, const StepIO<double>&, cudaStream_t);
template cudaError_t launch_phi3d_iso<float>(const Geom&, const Phys<float>&, const StepIO<float>&, int, cudaStream_t);
template cudaError_t launch_phi3d_iso<double>(const Geom&, const Phys<double>&, const StepIO<double>&, int, cudaStream_t);

}  // namespace lf
