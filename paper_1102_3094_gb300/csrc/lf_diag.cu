// lf_diag.cu -- diagnostics kernels.
//
// Sums are FP64 whatever the state precision: every site's contribution is
// converted to double, reduced within a CTA by warp shuffles, written as one
// partial per CTA, and the partials are reduced in a fixed order by a single
// CTA, so the result does not depend on scheduling.
//
// S(k) = |sum_r (phi - mean) e^{-i k.r}|^2 / N: the FFT runs in FP64 on the
// GPU, line by line along each axis, each line transformed in shared memory
// by a mixed-radix Cooley-Tukey (decimation in time, digit-reversed load).
// The k = 0 coefficient, the only one the mean affects, is left out of the
// shells.  Shells have width dk = 2 pi / L_min; bin b = floor(|k|/dk + 1/2),
// b = 1 .. L_min/2.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "lf_diag.cuh"

namespace lf {

namespace {

constexpr int kBlocks = 152 * 8;   // partial sums: a few waves on 152 SMs
constexpr int kThreads = 256;
constexpr int kMaxRadix = 32;
constexpr int kMaxStages = 40;
constexpr int kShellSmemBins = 4096;   // shell histogram kept in shared memory up to this many bins

struct Scratch {
    double* part;    // kBlocks * DQ_N
    double* res;     // DQ_N
    double* layers;  // L * 2
    double* bins;    // (B + 1) * 2: sum, count
    double2* fft;    // N
};

size_t a256(size_t v) { return (v + 255) / 256 * 256; }

Scratch carve(const Geom& g, void* base)
{
    Scratch s;
    unsigned char* p = (unsigned char*)base;
    const int64_t L = g.d == 2 ? g.ny : g.nz;
    int64_t lmin = g.nx < g.ny ? g.nx : g.ny;
    if (g.d == 3 && g.nz < lmin) lmin = g.nz;
    const int64_t B = lmin / 2;
    s.part = (double*)p; p += a256(sizeof(double) * kBlocks * DQ_N);
    s.res = (double*)p; p += a256(sizeof(double) * DQ_N);
    s.layers = (double*)p; p += a256(sizeof(double) * 2 * L);
    s.bins = (double*)p; p += a256(sizeof(double) * 2 * (B + 1));
    s.fft = (double2*)p;
    return s;
}

__device__ __forceinline__ int nb_index(int v, int step, int n, int mirror)
{
    int t = v + step;
    if (t < 0) return mirror ? 0 : n - 1;
    if (t >= n) return mirror ? n - 1 : 0;
    return t;
}

template <typename R>
__device__ __forceinline__ double at(const R* f, const Geom& g, int x, int y, int z)
{
    return (double)f[((int64_t)z * g.ny + y) * g.pitch + x];
}

// Central differences and the Laplacian of phi at (x, y, z); along the wall
// axis the neighbour beyond the last layer is the layer itself (even mirror).
// With `links` given, also the sum over the site's forward links of
// (phi(r + e) - phi(r))^2: the mirror neighbour makes the link out of the
// last layer vanish, so every nearest-neighbour link inside the lattice is
// counted once.
template <typename R>
__device__ void phi_derivs(const R* phi, const Geom& g, int x, int y, int z, double* grad, double* lap,
                           double* links = nullptr)
{
    const int wy = g.walls && g.d == 2, wz = g.walls && g.d == 3;
    const double c = at(phi, g, x, y, z);
    const double xp = at(phi, g, nb_index(x, 1, g.nx, 0), y, z), xm = at(phi, g, nb_index(x, -1, g.nx, 0), y, z);
    const double yp = at(phi, g, x, nb_index(y, 1, g.ny, wy), z), ym = at(phi, g, x, nb_index(y, -1, g.ny, wy), z);
    grad[0] = 0.5 * (xp - xm);
    grad[1] = 0.5 * (yp - ym);
    double l = xp + xm - 2.0 * c + yp + ym - 2.0 * c;
    double k2 = (xp - c) * (xp - c) + (yp - c) * (yp - c);
    grad[2] = 0.0;
    if (g.d == 3) {
        const double zp = at(phi, g, x, y, nb_index(z, 1, g.nz, wz)), zm = at(phi, g, x, y, nb_index(z, -1, g.nz, wz));
        grad[2] = 0.5 * (zp - zm);
        l += zp + zm - 2.0 * c;
        k2 += (zp - c) * (zp - c);
    }
    *lap = l;
    if (links) *links = k2;
}

template <int NQ>
__device__ void block_reduce_store(double (&v)[NQ], double* out, int max_slot)
{
    __shared__ double red[kThreads / 32][NQ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_down_sync(0xffffffffu, x, o);
            x = (q == max_slot) ? fmax(x, y) : x + y;
        }
        if (lane == 0) red[warp][q] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double x = lane < kThreads / 32 ? red[lane][q] : (q == max_slot ? 0.0 : 0.0);
            for (int o = 16; o > 0; o >>= 1) {
                const double y = __shfl_down_sync(0xffffffffu, x, o);
                x = (q == max_slot) ? fmax(x, y) : x + y;
            }
            if (lane == 0) out[q] = x;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_diag_partial(Geom g, const R* __restrict__ phi, const R* __restrict__ T,
                                                           const R* __restrict__ aux, double b, double kappa, double c,
                                                           double Tc, double* part)
{
    double v[DQ_N];
#pragma unroll
    for (int q = 0; q < DQ_N; ++q) v[q] = 0.0;
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    const int64_t P = g.plane;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % g.nx);
        const int64_t row = k / g.nx;
        const int y = (int)(row % g.ny), z = (int)(row / g.ny);
        const int64_t site = row * g.pitch + x;
        const double ph = (double)phi[site];
        double gr[3], lap, links;
        phi_derivs(phi, g, x, y, z, gr, &lap, &links);
        const double n = (double)aux[4 * P + site];
        const double ux = (double)aux[5 * P + site], uy = (double)aux[6 * P + site], uz = (double)aux[7 * P + site];
        const double a = ((double)T[site] - Tc) / Tc;
        v[DQ_MASS] += n;
        v[DQ_PHI] += ph;
        v[DQ_MX] += n * ux;
        v[DQ_MY] += n * uy;
        v[DQ_MZ] += n * uz;
        v[DQ_GX] += gr[0] * gr[0];
        v[DQ_GY] += gr[1] * gr[1];
        v[DQ_GZ] += gr[2] * gr[2];
        v[DQ_FE] += a * ph * ph / 2 + b * ph * ph * ph * ph / 4 + kappa * links / 2 + c * lap * lap / 2;
        v[DQ_U2MAX] = fmax(v[DQ_U2MAX], ux * ux + uy * uy + uz * uz);
    }
    block_reduce_store<DQ_N>(v, part + (int64_t)blockIdx.x * DQ_N, DQ_U2MAX);
}

__global__ void __launch_bounds__(kThreads) k_diag_final(const double* __restrict__ part, int nblk, double* res)
{
    double v[DQ_N];
#pragma unroll
    for (int q = 0; q < DQ_N; ++q) v[q] = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x)
#pragma unroll
        for (int q = 0; q < DQ_N; ++q)
            v[q] = (q == DQ_U2MAX) ? fmax(v[q], part[(int64_t)i * DQ_N + q]) : v[q] + part[(int64_t)i * DQ_N + q];
    block_reduce_store<DQ_N>(v, res, DQ_U2MAX);
}

// One CTA per layer along the wall normal: sum (d_perp phi)^2, |grad phi|^2.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_layers(Geom g, const R* __restrict__ phi, double* out)
{
    const int h = blockIdx.x;
    const int64_t per = g.d == 2 ? g.nx : (int64_t)g.nx * g.ny;
    double v[2] = {0.0, 0.0};
    for (int64_t k = threadIdx.x; k < per; k += blockDim.x) {
        int x, y, z;
        if (g.d == 2) { x = (int)k; y = h; z = 0; }
        else { x = (int)(k % g.nx); y = (int)(k / g.nx); z = h; }
        double gr[3], lap;
        phi_derivs(phi, g, x, y, z, gr, &lap);
        const double gp = g.d == 2 ? gr[1] : gr[2];
        v[0] += gp * gp;
        v[1] += gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
    }
    block_reduce_store<2>(v, out + 2 * h, -1);
}

// ---- FFT ------------------------------------------------------------------
struct FftPlan {
    int n;
    int nst;
    int radix[kMaxStages];
};

bool make_plan(int n, FftPlan* p)
{
    p->n = n;
    p->nst = 0;
    int m = n;
    while (m % 4 == 0) { p->radix[p->nst++] = 4; m /= 4; }
    for (int r = 2; r <= kMaxRadix && m > 1; ++r)
        while (m % r == 0) {
            if (p->nst >= kMaxStages) return false;
            p->radix[p->nst++] = r;
            m /= r;
        }
    return m == 1;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// multiply by -i
__device__ __forceinline__ double2 cmul_mi(double2 a) { return make_double2(a.y, -a.x); }

// C lines of length n per CTA; line l starts at (l / inner) * outer_stride +
// (l % inner) * inner_stride and has element stride `es`.  Shared memory:
// the twiddle table tw[j] = e^{-2 pi i j / n}, j < n, then the C lines.
__global__ void k_fft_lines(double2* data, FftPlan plan, int64_t es, int64_t nlines, int64_t inner,
                            int64_t inner_stride, int64_t outer_stride, int C)
{
    extern __shared__ double2 smem_fft[];
    const int n = plan.n;
    double2* tw = smem_fft;
    double2* buf = smem_fft + n;
    const int64_t l0 = (int64_t)blockIdx.x * C;
    const int nl = (int)((nlines - l0) < C ? (nlines - l0) : C);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)j / (double)n, &sn, &cs);
        tw[j] = make_double2(cs, sn);
    }
    // digit-reversed load
    for (int t = threadIdx.x; t < nl * n; t += blockDim.x) {
        int c, j;
        if (es == 1) { c = t / n; j = t - c * n; }
        else { j = t / nl; c = t - j * nl; }
        const int64_t l = l0 + c;
        const int64_t base = (l / inner) * outer_stride + (l % inner) * inner_stride;
        int pos = 0, rem = j, size = n;
        for (int st = plan.nst - 1; st >= 0; --st) {
            const int r = plan.radix[st];
            size /= r;
            pos += (rem % r) * size;
            rem /= r;
        }
        buf[c * n + pos] = data[base + (int64_t)j * es];
    }
    __syncthreads();
    int m = 1;
    for (int st = 0; st < plan.nst; ++st) {
        const int r = plan.radix[st];
        const int nb = n / r;
        const int stride = n / (m * r);          // tw index step of W_{m r}
        for (int t = threadIdx.x; t < nl * nb; t += blockDim.x) {
            const int c = t / nb, bi = t - c * nb;
            const int grp = bi / m, k = bi - grp * m;
            double2* b = buf + c * n + grp * m * r + k;
            if (r == 2) {
                const double2 y0 = b[0], y1 = cmul(b[m], tw[k * stride]);
                b[0] = cadd(y0, y1);
                b[m] = csub(y0, y1);
            } else if (r == 4) {
                const double2 y0 = b[0];
                const double2 y1 = cmul(b[m], tw[k * stride]);
                const double2 y2 = cmul(b[2 * m], tw[2 * k * stride]);
                const double2 y3 = cmul(b[3 * m], tw[3 * k * stride]);
                const double2 a0 = cadd(y0, y2), a1 = csub(y0, y2);
                const double2 b0 = cadd(y1, y3), b1 = cmul_mi(csub(y1, y3));
                b[0] = cadd(a0, b0);
                b[m] = cadd(a1, b1);
                b[2 * m] = csub(a0, b0);
                b[3 * m] = csub(a1, b1);
            } else {
                double2 y[kMaxRadix];
                y[0] = b[0];
                for (int s2 = 1; s2 < r; ++s2) y[s2] = cmul(b[s2 * m], tw[k * s2 * stride]);
                const int wr = n / r;            // tw index step of W_r
                for (int q = 0; q < r; ++q) {
                    double2 acc = y[0];
                    for (int s2 = 1; s2 < r; ++s2) acc = cadd(acc, cmul(y[s2], tw[((q * s2) % r) * wr]));
                    b[q * m] = acc;
                }
            }
        }
        __syncthreads();
        m *= r;
    }
    for (int t = threadIdx.x; t < nl * n; t += blockDim.x) {
        int c, j;
        if (es == 1) { c = t / n; j = t - c * n; }
        else { j = t / nl; c = t - j * nl; }
        const int64_t l = l0 + c;
        const int64_t base = (l / inner) * outer_stride + (l % inner) * inner_stride;
        data[base + (int64_t)j * es] = buf[c * n + j];
    }
}

template <typename R>
__global__ void k_fft_fill(Geom g, const R* __restrict__ phi, double2* out)
{
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = k / g.nx;
        const int x = (int)(k - row * g.nx);
        out[k] = make_double2((double)phi[row * g.pitch + x], 0.0);
    }
}

__device__ __forceinline__ double kfreq2(int64_t i, int64_t n, int64_t lmin)
{
    const int64_t f = (2 * i <= n) ? i : i - n;
    const double r = (double)f * (double)lmin / (double)n;   // |k| / dk along this axis
    return r * r;
}

__global__ void k_shells(Geom g, const double2* __restrict__ X, int64_t lmin, int64_t B, double* bins)
{
    extern __shared__ double hist[];            // 2 (B + 1) doubles when B <= kShellSmemBins
    const bool local = B <= kShellSmemBins;
    if (local) {
        for (int i = threadIdx.x; i < 2 * (B + 1); i += blockDim.x) hist[i] = 0.0;
        __syncthreads();
    }
    double* h = local ? hist : bins;
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        if (k == 0) continue;
        const int64_t ix = k % g.nx, row = k / g.nx;
        const int64_t iy = row % g.ny, iz = row / g.ny;
        double r2 = kfreq2(ix, g.nx, lmin) + kfreq2(iy, g.ny, lmin);
        if (g.d == 3) r2 += kfreq2(iz, g.nz, lmin);
        const int64_t b = (int64_t)floor(sqrt(r2) + 0.5);
        if (b < 1 || b > B) continue;
        const double2 v = X[k];
        atomicAdd(&h[2 * b], (v.x * v.x + v.y * v.y) / (double)N);
        atomicAdd(&h[2 * b + 1], 1.0);
    }
    if (local) {
        __syncthreads();
        for (int i = threadIdx.x; i < 2 * (B + 1); i += blockDim.x)
            if (hist[i] != 0.0) atomicAdd(&bins[i], hist[i]);
    }
}

unsigned grid_n(int64_t N)
{
    int64_t b = (N + kThreads - 1) / kThreads;
    if (b > kBlocks) b = kBlocks;
    return (unsigned)(b < 1 ? 1 : b);
}

int64_t lmin_of(const Geom& g)
{
    int64_t l = g.nx < g.ny ? g.nx : g.ny;
    if (g.d == 3 && g.nz < l) l = g.nz;
    return l;
}

// Forward DFT (kernel e^{-2 pi i j k / n}) of every line along axis a of a
// packed [nz][ny][nx] complex FP64 array, in place.
cudaError_t fft_lines_axis(const Geom& g, double2* data, int a, const FftPlan& plan, cudaStream_t s)
{
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    const int n = plan.n;
    int C = 4096 / n;
    if (C < 1) C = 1;
    if (C > 16) C = 16;
    int64_t nlines, inner, inner_stride, outer_stride, es;
    if (a == 0) { nlines = N / n; inner = 1; inner_stride = 0; outer_stride = n; es = 1; }
    else if (a == 1) { nlines = N / n; inner = g.nx; inner_stride = 1; outer_stride = (int64_t)g.nx * g.ny; es = g.nx; }
    else { nlines = N / n; inner = (int64_t)g.nx * g.ny; inner_stride = 1; outer_stride = 0; es = (int64_t)g.nx * g.ny; }
    const size_t smem = sizeof(double2) * (size_t)(C + 1) * n;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_fft_lines, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const unsigned blocks = (unsigned)((nlines + C - 1) / C);
    k_fft_lines<<<blocks, kThreads, smem, s>>>(data, plan, es, nlines, inner, inner_stride, outer_stride, C);
    return cudaGetLastError();
}

// FFT of phi into sc.fft and the shell sums into sc.bins (device).  Returns
// false when a lattice size has a prime factor above kMaxRadix or a line does
// not fit in shared memory.
bool enqueue_sk(const DiagInput& in, const Scratch& sc, cudaStream_t s, cudaError_t* err)
{
    const Geom& g = in.g;
    const int64_t lmin = lmin_of(g), B = lmin / 2;
    const int sizes[3] = {g.nx, g.ny, g.nz};
    FftPlan plans[3];
    for (int a = 0; a < g.d; ++a) {
        if (!make_plan(sizes[a], &plans[a]) || sizes[a] > 4096) return false;   // line + twiddles fit in smem
    }
    *err = cudaSuccess;
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    if (in.prec == LF_FP64) k_fft_fill<double><<<grid_n(N), kThreads, 0, s>>>(g, (const double*)in.phi, sc.fft);
    else k_fft_fill<float><<<grid_n(N), kThreads, 0, s>>>(g, (const float*)in.phi, sc.fft);
    for (int a = 0; a < g.d; ++a) {
        const cudaError_t e = fft_lines_axis(g, sc.fft, a, plans[a], s);
        if (e != cudaSuccess) { *err = e; return true; }
    }
    cudaMemsetAsync(sc.bins, 0, sizeof(double) * 2 * (B + 1), s);
    const size_t hs = B <= kShellSmemBins ? sizeof(double) * 2 * (B + 1) : 0;
    if (hs > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_shells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs);
        if (e != cudaSuccess) { *err = e; return true; }
    }
    k_shells<<<grid_n(N), kThreads, hs, s>>>(g, sc.fft, lmin, B, sc.bins);
    *err = cudaGetLastError();
    return true;
}

void peak_from_bins(const std::vector<double>& bins, int64_t B, int64_t lmin, double* k_peak, double* s_peak)
{
    const double dk = 2.0 * M_PI / (double)lmin;
    std::vector<double> S(B + 1, 0.0);
    double smax = 0.0;
    for (int64_t b = 1; b <= B; ++b) {
        S[b] = bins[2 * b + 1] > 0 ? bins[2 * b] / bins[2 * b + 1] : 0.0;
        if (S[b] > smax) smax = S[b];
    }
    double num = 0.0, den = 0.0;
    for (int64_t b = 1; b <= B; ++b)
        if (S[b] > 0.5 * smax) { num += b * dk * S[b]; den += S[b]; }
    *s_peak = smax;
    *k_peak = den > 0 ? num / den : 0.0;
}

}  // namespace

size_t diag_scratch_bytes(int d, int64_t nx, int64_t ny, int64_t nz)
{
    const int64_t L = d == 2 ? ny : nz;
    int64_t lmin = nx < ny ? nx : ny;
    if (d == 3 && nz < lmin) lmin = nz;
    const int64_t B = lmin / 2;
    return a256(sizeof(double) * kBlocks * DQ_N) + a256(sizeof(double) * DQ_N) + a256(sizeof(double) * 2 * L) +
           a256(sizeof(double) * 2 * (B + 1)) + a256(sizeof(double2) * (size_t)(nx * ny * nz));
}

double2* fft_buffer(const Geom& g, void* scratch) { return carve(g, scratch).fft; }

bool fft_supported(int n) { FftPlan p; return n <= 4096 && make_plan(n, &p); }

cudaError_t fft_forward_axis(const Geom& g, double2* data, int axis, cudaStream_t s)
{
    const int sizes[3] = {g.nx, g.ny, g.nz};
    FftPlan plan;
    if (!make_plan(sizes[axis], &plan) || sizes[axis] > 4096) return cudaErrorInvalidValue;
    return fft_lines_axis(g, data, axis, plan, s);
}

int run_diag(const DiagInput& in, DiagResult* r, cudaStream_t s)
{
    const Geom& g = in.g;
    const Scratch sc = carve(g, in.scratch);
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    const unsigned nblk = grid_n(N);
    if (in.prec == LF_FP64)
        k_diag_partial<double><<<nblk, kThreads, 0, s>>>(g, (const double*)in.phi, (const double*)in.T,
                                                         (const double*)in.aux, in.b, in.kappa, in.c, in.Tc, sc.part);
    else
        k_diag_partial<float><<<nblk, kThreads, 0, s>>>(g, (const float*)in.phi, (const float*)in.T,
                                                        (const float*)in.aux, in.b, in.kappa, in.c, in.Tc, sc.part);
    k_diag_final<<<1, kThreads, 0, s>>>(sc.part, (int)nblk, sc.res);
    if (cudaGetLastError() != cudaSuccess) return LF_ECUDA;
    cudaError_t e = cudaSuccess;
    const bool have_sk = enqueue_sk(in, sc, s, &e);
    if (e != cudaSuccess) return LF_ECUDA;
    const int64_t lmin = lmin_of(g), B = lmin / 2;
    std::vector<double> host(DQ_N + 2 * (B + 1));
    if (cudaMemcpyAsync(host.data(), sc.res, sizeof(double) * DQ_N, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return LF_ECUDA;
    if (have_sk && cudaMemcpyAsync(host.data() + DQ_N, sc.bins, sizeof(double) * 2 * (B + 1), cudaMemcpyDeviceToHost,
                                   s) != cudaSuccess)
        return LF_ECUDA;
    int rc = wait_stream(s);
    if (rc != LF_OK) return rc;
    std::memcpy(r->sums, host.data(), sizeof(double) * DQ_N);
    if (have_sk) {
        std::vector<double> bins(host.begin() + DQ_N, host.end());
        peak_from_bins(bins, B, lmin, &r->k_peak, &r->s_peak);
    } else {
        r->k_peak = r->s_peak = NAN;
    }
    return LF_OK;
}

int run_layers(const DiagInput& in, double* out_host, cudaStream_t s)
{
    const Geom& g = in.g;
    const Scratch sc = carve(g, in.scratch);
    const int L = g.d == 2 ? g.ny : g.nz;
    if (in.prec == LF_FP64) k_layers<double><<<L, kThreads, 0, s>>>(g, (const double*)in.phi, sc.layers);
    else k_layers<float><<<L, kThreads, 0, s>>>(g, (const float*)in.phi, sc.layers);
    if (cudaGetLastError() != cudaSuccess) return LF_ECUDA;
    std::vector<double> h(2 * (size_t)L);
    if (cudaMemcpyAsync(h.data(), sc.layers, sizeof(double) * 2 * L, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return LF_ECUDA;
    int rc = wait_stream(s);
    if (rc != LF_OK) return rc;
    const int d = g.d;
    for (int i = 0; i < L; ++i)
        out_host[i] = h[2 * i + 1] > 0 ? (d * h[2 * i] / h[2 * i + 1] - 1.0) / (d - 1) : 0.0;
    return LF_OK;
}

int run_sk_shells(const DiagInput& in, double* out_host, int64_t nb, cudaStream_t s)
{
    const Geom& g = in.g;
    const int64_t lmin = lmin_of(g), B = lmin / 2;
    if (nb != B + 1) return LF_EINVAL;
    const Scratch sc = carve(g, in.scratch);
    cudaError_t e = cudaSuccess;
    if (!enqueue_sk(in, sc, s, &e)) return LF_EINVAL;
    if (e != cudaSuccess) return LF_ECUDA;
    std::vector<double> bins(2 * (B + 1));
    if (cudaMemcpyAsync(bins.data(), sc.bins, sizeof(double) * 2 * (B + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return LF_ECUDA;
    int rc = wait_stream(s);
    if (rc != LF_OK) return rc;
    out_host[0] = 0.0;
    for (int64_t b = 1; b <= B; ++b) out_host[b] = bins[2 * b + 1] > 0 ? bins[2 * b] / bins[2 * b + 1] : 0.0;
    return LF_OK;
}

}  // namespace lf

// ===========================================================================
// Diagnostics without allocation (lf_diag_sums_noalloc in include/lf.h).
//
// For callers that cannot allocate device memory on the way: a reduction
// started while a CUDA graph is being captured, a real-time loop that must
// not stall on cudaMalloc's implicit synchronisation, or a host framework
// that owns every byte of device memory.  Same kernels as lf_diag's sums and
// layer sums; their scratch (per-CTA partial sums and per-layer sums) lives in
// the file-scope array below instead of a context's workspace.  Every GPU that
// loads this library holds the array (kNoAllocScratchBytes) until exit.
// ===========================================================================
namespace lf {
namespace {

constexpr int kNoAllocMaxLayers = 4096;
constexpr size_t kNoAllocPartDoubles = (size_t)kBlocks * DQ_N;
constexpr size_t kNoAllocScratchDoubles = kNoAllocPartDoubles + 2 * (size_t)kNoAllocMaxLayers;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// s(h) = (d sum(d_perp phi)^2 / sum |grad phi|^2 - 1) / (d - 1), per layer.
__global__ void k_layers_to_s(const double* __restrict__ sums, int L, int d, double* __restrict__ s)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= L) return;
    const double a = sums[2 * h], b = sums[2 * h + 1];
    s[h] = b > 0 ? (d * a / b - 1.0) / (d - 1) : 0.0;
}

// Device address of the scratch array on the current device, resolved once
// per device (the first call on a device does it; see the header).  The
// cached address belongs to the device's primary context: after that context
// is reset (cudaDeviceReset) the address is stale, so the entry point is not
// for use across a reset.
int noalloc_scratch(double** out)
{
    static std::mutex mu;
    static double* addr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LF_ECUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return LF_ECUDA;
        }
        addr[dev] = (double*)p;
    }
    *out = addr[dev];
    return LF_OK;
}

}  // namespace
}  // namespace lf

extern "C" int lf_diag_sums_noalloc(int d, int64_t nx, int64_t ny, int64_t nz, int walls, int precision,
                                    const void* phi, const void* T, const void* moments, double b, double kappa,
                                    double c, double Tc, double* out, void* stream)
{
    using namespace lf;
    if (d != 2 && d != 3) return LF_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || (d == 2 && nz != 1)) return LF_EINVAL;
    // bound each extent before forming the product, which could otherwise wrap
    if (nx > (1 << 24) || ny > (1 << 24) || nz > (1 << 24)) return LF_EINVAL;
    if (precision != LF_FP64 && precision != LF_FP32) return LF_EINVAL;
    if (!phi || !T || !moments || !out) return LF_EINVAL;
    if (!(Tc > 0)) return LF_EINVAL;
    const int64_t L = d == 2 ? ny : nz;
    if (L > kNoAllocMaxLayers) return LF_EINVAL;              // the layer sums would not fit
    if (nx * ny * nz >= ((int64_t)1 << 31)) return LF_EINVAL;
    double* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != LF_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    Geom g{};
    g.d = d;
    g.nx = (int)nx; g.ny = (int)ny; g.nz = (int)nz;
    g.pitch = (int)nx;                                     // caller fields are unpadded
    g.plane = nx * ny * nz;
    g.walls = walls ? 1 : 0;
    // The sums kernel reads n, ux, uy, uz as planes 4..7 of a context's aux
    // block; the caller's moments block holds exactly those four planes, so
    // it is addressed through a base four planes before it (only planes 4..7
    // are ever read).
    const size_t es = precision == LF_FP64 ? 8 : 4;
    const uintptr_t aux_addr = (uintptr_t)moments - 4 * (uintptr_t)g.plane * es;
    const void* aux = (const void*)aux_addr;
    const int64_t N = nx * ny * nz;
    const unsigned nblk = grid_n(N);
    double* part = scratch;
    double* lay = scratch + kNoAllocPartDoubles;
    if (precision == LF_FP64)
        k_diag_partial<double><<<nblk, kThreads, 0, s>>>(g, (const double*)phi, (const double*)T,
                                                         (const double*)aux, b, kappa, c, Tc, part);
    else
        k_diag_partial<float><<<nblk, kThreads, 0, s>>>(g, (const float*)phi, (const float*)T,
                                                        (const float*)aux, b, kappa, c, Tc, part);
    k_diag_final<<<1, kThreads, 0, s>>>(part, (int)nblk, out);
    if (precision == LF_FP64) k_layers<double><<<(unsigned)L, kThreads, 0, s>>>(g, (const double*)phi, lay);
    else k_layers<float><<<(unsigned)L, kThreads, 0, s>>>(g, (const float*)phi, lay);
    k_layers_to_s<<<(unsigned)((L + 127) / 128), 128, 0, s>>>(lay, (int)L, d, out + DQ_N);
    return cudaGetLastError() == cudaSuccess ? LF_OK : LF_ECUDA;
}
