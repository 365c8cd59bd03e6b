// lf_timplicit.cu -- implicit temperature step (lf_set_t_solver).
//
// The temperature obeys d_t T = xi lap T (arXiv:1102.3094, Sec. 2, after Eq.
// massdiff).  The explicit update needs xi / n_sub <= 1/(2d) per sub-step,
// i.e. hundreds of sub-steps per time step at the paper's largest xi.  The
// implicit option takes one backward-Euler step per time step,
//   (I - xi L) T(t+1) = T(t),
// with the same Laplacian L (compact 5-/7-point or isotropic 9-/19-point) and
// wall rules as the explicit update.  L is diagonal in a lattice Fourier basis
// along the periodic axes and couples only neighbouring layers along the wall
// normal, so the solve is: FP64 DFT along x (2D) or x and y (3D); for every
// Fourier mode a tridiagonal system along the wall normal (Thomas algorithm,
// one thread per mode) -- or a plain division when every axis is periodic;
// the inverse DFT as conj(DFT(conj(.))) / n; back to the state's precision.
//
// For a mode with in-plane wavenumbers (kx[, ky]) L acts on the layer
// amplitudes as alpha (A_{j+1} + A_{j-1}) + beta A_j:
//   compact:        alpha = 1,                 beta = -2 - sum 2 (1 - cos k)
//   isotropic, 2D:  alpha = (4 + 2 cx) / 6,     beta = (8 cx - 20) / 6
//   isotropic, 3D:  alpha = (2 + 2 cx + 2 cy)/6, beta = (4 cx + 4 cy + 4 cx cy - 24) / 6
// (c = cos k).  Every offset that crosses a wall has the wall-normal step of
// the axis neighbour, so the ghost rules enter with the same alpha.
#include <cmath>

#include "lf_ctx.cuh"
#include "lf_diag.cuh"

namespace lf {

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

template <typename R>
__global__ void k_t_load(Geom g, const R* __restrict__ T, double2* __restrict__ buf)
{
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = k / g.nx;
        const int x = (int)(k - row * g.nx);
        buf[k] = make_double2((double)T[row * g.pitch + x], 0.0);
    }
}

template <typename R>
__global__ void k_t_store(Geom g, const double2* __restrict__ buf, double scale, R* __restrict__ T,
                          int* __restrict__ flag)
{
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    bool bad = false;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = k / g.nx;
        const int x = (int)(k - row * g.nx);
        const double v = buf[k].x * scale;
        bad |= !isfinite(v);
        T[row * g.pitch + x] = (R)v;
    }
    if (bad) *reinterpret_cast<volatile int*>(flag) = 1;
}

// Cosines of the wavenumbers of the mode with packed index m over the
// periodic axes (x fastest); 1 for the others.
__device__ __forceinline__ void mode_cos(const Geom& g, int64_t m, int nper_axes, double c[3])
{
    c[0] = cos(kTwoPi * (int)(m % g.nx) / g.nx);
    c[1] = nper_axes >= 2 ? cos(kTwoPi * (int)((m / g.nx) % g.ny) / g.ny) : 1.0;
    c[2] = nper_axes >= 3 ? cos(kTwoPi * (int)(m / ((int64_t)g.nx * g.ny)) / g.nz) : 1.0;
}

// Every axis periodic: eigenvalue of -L for mode m.
__device__ __forceinline__ double lam_periodic(const Geom& g, int64_t m)
{
    double c[3];
    mode_cos(g, m, g.d, c);
    if (g.stencil == LF_STENCIL_ISOTROPIC) {
        if (g.d == 2) return -(8.0 * (c[0] + c[1]) + 4.0 * c[0] * c[1] - 20.0) / 6.0;
        return -(4.0 * (c[0] + c[1] + c[2]) + 4.0 * (c[0] * c[1] + c[0] * c[2] + c[1] * c[2]) - 24.0) / 6.0;
    }
    double lam = 0.0;
    for (int a = 0; a < g.d; ++a) lam += 2.0 * (1.0 - c[a]);
    return lam;
}

// Walls: L on the layer amplitudes of in-plane mode m is alpha (A_{j+1} +
// A_{j-1}) + beta A_j.
__device__ __forceinline__ void layer_coeffs(const Geom& g, int64_t m, double* alpha, double* beta)
{
    double c[3];
    mode_cos(g, m, g.d - 1, c);
    if (g.stencil == LF_STENCIL_ISOTROPIC) {
        if (g.d == 2) {
            *alpha = (4.0 + 2.0 * c[0]) / 6.0;
            *beta = (8.0 * c[0] - 20.0) / 6.0;
        } else {
            *alpha = (2.0 + 2.0 * c[0] + 2.0 * c[1]) / 6.0;
            *beta = (4.0 * c[0] + 4.0 * c[1] + 4.0 * c[0] * c[1] - 24.0) / 6.0;
        }
        return;
    }
    double lam = 2.0 * (1.0 - c[0]);
    if (g.d == 3) lam += 2.0 * (1.0 - c[1]);
    *alpha = 1.0;
    *beta = -2.0 - lam;
}

// The tridiagonal system of Fourier mode m along the wall normal: constant
// off-diagonal a, diagonal b (b0 / b1 on the first / last unknown layer with
// the halfway ghost), unknown layers j0 .. j1.
struct TriSys {
    double a, b, b0, b1;
    int j0, j1;
};

__device__ __forceinline__ TriSys tri_sys(const Geom& g, int64_t m, double xi, int t_mode, int L)
{
    double alpha, beta;
    layer_coeffs(g, m, &alpha, &beta);
    TriSys t;
    t.b = 1.0 - xi * beta;
    t.a = -xi * alpha;                       // sub- and super-diagonal
    t.b0 = t.b;
    t.b1 = t.b;
    t.j0 = 0;
    t.j1 = L - 1;
    if (t_mode == LF_TWALL_LAYERS) {         // held layers 0 and L-1 enter the right-hand side
        t.j0 = 1;
        t.j1 = L - 2;
    } else {                                 // ghost 2 T_w - T: +xi alpha on the diagonal
        t.b0 -= t.a;
        t.b1 -= t.a;
    }
    return t;
}

// Diagonal of unknown layer j.
__device__ __forceinline__ double tri_diag(const TriSys& t, int j, int t_mode)
{
    double bj = t.b;
    if (j == t.j0) bj = t_mode == LF_TWALL_LAYERS ? t.b : t.b0;
    if (j == t.j1 && t_mode != LF_TWALL_LAYERS) bj = (t.j0 == t.j1) ? t.b0 + (t.b1 - t.b) : t.b1;
    return bj;
}

// The part of the Thomas algorithm that does not depend on the right-hand
// side: c'_j = a / (b_j - a c'_{j-1}) and the reciprocal pivot
// 1 / (b_j - a c'_{j-1}) of every unknown layer of every mode, stored at
// j * M + m (c') and N + j * M + m (pivot).  The coefficients do not change
// from step to step, so the divisions leave the per-step recurrence.
__global__ void k_t_coef(Geom g, double* __restrict__ coef, double xi, int t_mode)
{
    const int d = g.d;
    const int64_t M = d == 2 ? (int64_t)g.nx : (int64_t)g.nx * g.ny;
    const int L = d == 2 ? g.ny : g.nz;
    const int64_t N = M * L;
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= M) return;
    const TriSys t = tri_sys(g, m, xi, t_mode, L);
    double cprev = 0.0;
    for (int j = t.j0; j <= t.j1; ++j) {
        const double inv = 1.0 / (tri_diag(t, j, t_mode) - t.a * cprev);
        const double cj = t.a * inv;
        coef[(int64_t)j * M + m] = cj;
        coef[N + (int64_t)j * M + m] = inv;
        cprev = cj;
    }
}

// Walls along the last axis: one thread per Fourier mode m of the periodic
// axes (M modes), the Thomas sweeps along the L layers of the wall normal
// with c' and the pivots from k_t_coef; element (j, m) at j * M + m.  The
// serial chain holds only multiply-adds: dp_j = (d_j - a dp_{j-1}) pivot_j,
// x_j = dp_j - c'_j x_{j+1}.  Writes the conjugate of the solution.
__global__ void k_t_thomas(Geom g, double2* __restrict__ buf, const double* __restrict__ coef, double xi,
                           double Tw_hat0, int t_mode)
{
    const int d = g.d;
    const int64_t M = d == 2 ? (int64_t)g.nx : (int64_t)g.nx * g.ny;
    const int L = d == 2 ? g.ny : g.nz;
    const int64_t N = M * L;
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= M) return;
    const TriSys t = tri_sys(g, m, xi, t_mode, L);
    const double a = t.a;
    const int j0 = t.j0, j1 = t.j1;
    auto at = [&](int j) -> double2& { return buf[(int64_t)j * M + m]; };
    double2 lo_add, hi_add;
    if (t_mode == LF_TWALL_LAYERS) {
        lo_add = make_double2(-a * at(0).x, -a * at(0).y);
        hi_add = make_double2(-a * at(L - 1).x, -a * at(L - 1).y);
    } else {                                 // 2 xi alpha T_w in the right-hand side of mode 0
        const double w = m == 0 ? -2.0 * a * Tw_hat0 : 0.0;
        lo_add = make_double2(w, 0.0);
        hi_add = make_double2(w, 0.0);
    }
    if (j1 < j0) {                           // no unknown layer
        for (int j = 0; j < L; ++j) at(j) = make_double2(at(j).x, -at(j).y);
        return;
    }
    // Forward sweep in blocks of kB layers: the right-hand sides and pivots of
    // block b + 1 are loaded while the recurrence runs over block b, so only
    // the multiply-adds sit in the serial chain.
    constexpr int kB = 8;
    double2 dv[kB], dn[kB];
    double pv[kB], pn[kB];
    auto load_fw = [&](int jb, double2* dd, double* pp) {
#pragma unroll
        for (int u = 0; u < kB; ++u)
            if (jb + u <= j1) {
                dd[u] = at(jb + u);
                pp[u] = coef[N + (int64_t)(jb + u) * M + m];
            }
    };
    load_fw(j0, dv, pv);
    double2 dprev = make_double2(0.0, 0.0);
    for (int jb = j0; jb <= j1; jb += kB) {
        if (jb + kB <= j1) load_fw(jb + kB, dn, pn);
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int j = jb + u;
            if (j > j1) break;
            double2 dj = dv[u];
            if (j == j0) { dj.x += lo_add.x; dj.y += lo_add.y; }
            if (j == j1) { dj.x += hi_add.x; dj.y += hi_add.y; }
            const double2 dp = make_double2((dj.x - a * dprev.x) * pv[u], (dj.y - a * dprev.y) * pv[u]);
            at(j) = dp;
            dprev = dp;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) { dv[u] = dn[u]; pv[u] = pn[u]; }
    }
    // back substitution x_j = dp_j - c'_j x_{j+1}, storing conj(x), in blocks
    // of kB layers downwards with the next block's loads in flight
    double2 xnext = at(j1);
    at(j1) = make_double2(xnext.x, -xnext.y);
    auto load_bw = [&](int jb, double* cc, double2* dd) {
#pragma unroll
        for (int u = 0; u < kB; ++u)
            if (jb - u >= j0) { cc[u] = coef[(int64_t)(jb - u) * M + m]; dd[u] = at(jb - u); }
    };
    if (j1 - 1 >= j0) load_bw(j1 - 1, pv, dv);
    for (int jb = j1 - 1; jb >= j0; jb -= kB) {
        if (jb - kB >= j0) load_bw(jb - kB, pn, dn);
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int j = jb - u;
            if (j < j0) break;
            const double2 x = make_double2(dv[u].x - pv[u] * xnext.x, dv[u].y - pv[u] * xnext.y);
            at(j) = make_double2(x.x, -x.y);
            xnext = x;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) { dv[u] = dn[u]; pv[u] = pn[u]; }
    }
    for (int j = 0; j < j0; ++j) at(j) = make_double2(at(j).x, -at(j).y);          // held layers
    for (int j = j1 + 1; j < L; ++j) at(j) = make_double2(at(j).x, -at(j).y);
}

// Every axis periodic: the mode is divided by 1 + xi lam; writes the conjugate.
__global__ void k_t_divide(Geom g, double2* __restrict__ buf, double xi)
{
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const double s = 1.0 / (1.0 + xi * lam_periodic(g, k));
        buf[k] = make_double2(buf[k].x * s, -buf[k].y * s);
    }
}

unsigned grid_t(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

bool t_implicit_supported(const Geom& g)
{
    if (!fft_supported(g.nx)) return false;
    if ((g.d == 3 || !g.walls) && !fft_supported(g.ny)) return false;
    if (g.d == 3 && !g.walls && !fft_supported(g.nz)) return false;
    return true;
}

template <typename R>
int t_implicit_step(lf_ctx* c, double xi, double T_w)
{
    const Geom& g = c->g;
    const cudaStream_t s = c->stream;
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    double2* buf = fft_buffer(g, c->scratch);
    R* T = (R*)c->T[c->tcur];
    const int nper_axes = g.walls ? g.d - 1 : g.d;
    int64_t nper = g.nx;
    if (nper_axes >= 2) nper *= g.ny;
    if (nper_axes >= 3) nper *= g.nz;
    k_t_load<R><<<grid_t(N), 256, 0, s>>>(g, T, buf);
    for (int a = 0; a < nper_axes; ++a)
        if (fft_forward_axis(g, buf, a, s) != cudaSuccess) return LF_ECUDA;
    if (g.walls) {
        const int64_t M = N / (g.d == 2 ? g.ny : g.nz);
        if (!c->tcoef) return LF_EINVAL;     // lf_set_t_solver allocates the tables
        if (!c->tcoef_valid || c->tcoef_xi != xi || c->tcoef_mode != g.t_mode || c->tcoef_stencil != g.stencil) {
            k_t_coef<<<(unsigned)((M + 31) / 32), 32, 0, s>>>(g, c->tcoef, xi, g.t_mode);
            c->tcoef_valid = true;
            c->tcoef_xi = xi;
            c->tcoef_mode = g.t_mode;
            c->tcoef_stencil = g.stencil;
        }
        k_t_thomas<<<(unsigned)((M + 31) / 32), 32, 0, s>>>(g, buf, c->tcoef, xi, T_w * (double)nper, g.t_mode);
    } else {
        k_t_divide<<<grid_t(N), 256, 0, s>>>(g, buf, xi);
    }
    for (int a = 0; a < nper_axes; ++a)
        if (fft_forward_axis(g, buf, a, s) != cudaSuccess) return LF_ECUDA;
    k_t_store<R><<<grid_t(N), 256, 0, s>>>(g, buf, 1.0 / (double)nper, T, c->flag_dev);
    return cudaGetLastError() == cudaSuccess ? LF_OK : LF_ECUDA;
}

template int t_implicit_step<float>(lf_ctx*, double, double);
template int t_implicit_step<double>(lf_ctx*, double, double);

}  // namespace lf
