// lf_api.cu -- host side of the C ABI declared in include/lf.h.
//
// The context holds two copies (ping-pong) of the state in one device block:
// populations f (Q planes, deviations f_i - w_i n0), phi and T, plus the aux
// fields (mu, F, n, u) that lf_fields / lf_diag derive from the current state,
// a staging area for host transfers and the reduction scratch of the
// diagnostics.  lf_step only enqueues kernels; every other call waits for the
// stream with a deadline.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "lf_ctx.cuh"
#include "lf_diag.cuh"
#include "lf_internal.cuh"

using namespace lf;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int check(cudaError_t e) { return e == cudaSuccess ? LF_OK : LF_ECUDA; }

int wall_len(const lf_grid* g) { return g->d == 2 ? (int)g->ny : (int)g->nz; }

int validate(const lf_grid* grid, const lf_walls* walls, const lf_params* p)
{
    if (!grid || !walls || !p) return LF_EINVAL;
    if (grid->d != 2 && grid->d != 3) return LF_EINVAL;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return LF_EINVAL;
    if (grid->d == 2 && grid->nz != 1) return LF_EINVAL;
    if (grid->nx > (1 << 24) || grid->ny > (1 << 24) || grid->nz > (1 << 24)) return LF_EINVAL;
    if (walls->walls != 0 && walls->walls != 1) return LF_EINVAL;
    if (walls->t_wall_mode != LF_TWALL_LAYERS && walls->t_wall_mode != LF_TWALL_HALFWAY) return LF_EINVAL;
    if (walls->walls && wall_len(grid) < 2) return LF_EINVAL;
    {   // kernels index populations with 32-bit offsets: Q * padded sites < 2^31
        const int64_t pitch = (grid->nx + 31) / 32 * 32;
        const int64_t Q = grid->d == 2 ? 9 : 19;
        if (Q * pitch * grid->ny * grid->nz >= ((int64_t)1 << 31)) return LF_EINVAL;
    }
    if (p->precision != LF_FP64 && p->precision != LF_FP32) return LF_EINVAL;
    if (p->hydro != 0 && p->hydro != 1) return LF_EINVAL;
    if (p->ideal_mode != 0) return LF_EINVAL;
    if (p->stencil != LF_STENCIL_COMPACT && p->stencil != LF_STENCIL_ISOTROPIC) return LF_EINVAL;
    const double vals[] = {p->b, p->kappa, p->c, p->Gamma, p->Tc, p->T0, p->tau, p->n0,
                           p->phi_amp, walls->T_w};
    for (double v : vals)
        if (!std::isfinite(v)) return LF_EINVAL;
    if (p->b < 0 || p->c < 0 || p->Gamma < 0 || p->Tc <= 0 || p->n0 <= 0 || p->phi_amp < 0) return LF_EINVAL;
    if (std::isnan(p->xi) || p->xi < 0) return LF_EINVAL;
    if (p->hydro && !(p->tau > 0.5)) return LF_EUNSTABLE;
    // Linear stability of the explicit phi update: a lattice eigenmode with
    // Laplacian eigenvalue lam in [0, lmax] is multiplied per step by
    // 1 - Gamma lam (a + kappa lam + c lam^2); require that factor > -1 at the
    // largest a the run can see.  lmax = 4d for the compact stencils and 16/3
    // for the isotropic ones (2D: at q = (pi, pi); 3D: at q = (pi, pi, 0)).
    const double amax = (std::fmax(p->T0, walls->T_w) - p->Tc) / p->Tc;
    const double lmax = p->stencil == LF_STENCIL_ISOTROPIC ? 16.0 / 3.0 : 4.0 * grid->d;
    for (int k = 0; k <= 4000; ++k) {
        const double lam = lmax * k / 4000.0;
        if (p->Gamma * lam * (amax + p->kappa * lam + p->c * lam * lam) >= 2.0) return LF_EUNSTABLE;
    }
    return LF_OK;
}

struct Layout {
    size_t f, phi, T, aux, stage, scratch, guard, total;
};

// Checked mode: LF_CHECKED=1 in the environment when the workspace is sized and
// the context created.
constexpr size_t kGuard = 64 * 1024;        // bytes per guard band
constexpr unsigned char kGuardByte = 0xA5;

bool checked_mode()
{
    const char* v = std::getenv("LF_CHECKED");
    return v && v[0] == '1';
}

// Every byte of the ten guard bands still holds kGuardByte; clears *bad otherwise.
struct GuardOffsets {
    unsigned long long off[10];
};

__global__ void k_guard_check(const unsigned char* __restrict__ base, GuardOffsets g, int* __restrict__ bad)
{
    constexpr int W = (int)(kGuard / 16);
    const uint4 want = make_uint4(0xA5A5A5A5u, 0xA5A5A5A5u, 0xA5A5A5A5u, 0xA5A5A5A5u);
    bool ok = true;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 10 * W; i += gridDim.x * blockDim.x) {
        const uint4 v = reinterpret_cast<const uint4*>(base + g.off[i / W])[i % W];
        ok &= v.x == want.x && v.y == want.y && v.z == want.z && v.w == want.w;
    }
    if (!ok) *reinterpret_cast<volatile int*>(bad) = 1;
}

// Checked mode: enqueue the verification of every guard band.
int check_guards(lf_ctx* c)
{
    if (!c->checked) return LF_OK;
    GuardOffsets g;
    for (int i = 0; i < 10; ++i) g.off[i] = c->guard_off[i];
    k_guard_check<<<152, 256, 0, c->stream>>>(c->base, g, c->guard_dev);
    return check(cudaGetLastError());
}

Layout layout_for(const lf_grid* grid, const lf_params* p, int64_t* plane_out, int* pitch_out)
{
    const int Q = grid->d == 2 ? 9 : 19;
    const size_t esz = p->precision == LF_FP64 ? 8 : 4;
    const int pitch = (int)align_up((size_t)grid->nx, 32);
    const int64_t plane = (int64_t)pitch * grid->ny * grid->nz;
    const int64_t N = grid->nx * grid->ny * grid->nz;
    Layout L;
    L.f = align_up((size_t)Q * plane * esz, kAlign);
    L.phi = align_up((size_t)plane * esz, kAlign);
    L.T = L.phi;
    L.aux = align_up((size_t)8 * plane * esz, kAlign);
    L.stage = align_up((size_t)N * 8, kAlign);
    L.scratch = align_up(diag_scratch_bytes(grid->d, grid->nx, grid->ny, grid->nz), kAlign);
    L.guard = checked_mode() ? kGuard : 0;
    L.total = 2 * L.f + 2 * L.phi + 2 * L.T + L.aux + L.stage + L.scratch + 10 * L.guard;
    if (plane_out) *plane_out = plane;
    if (pitch_out) *pitch_out = pitch;
    return L;
}

template <typename R>
Phys<R> phys_of(const lf_ctx* c)
{
    const lf_params& p = c->params;
    Phys<R> ph;
    ph.b = (R)p.b; ph.kappa = (R)p.kappa; ph.c = (R)p.c; ph.Gamma = (R)p.Gamma; ph.Tc = (R)p.Tc;
    ph.T_w = (R)c->walls.T_w;
    ph.inv_Tc = (R)(1.0 / p.Tc);
    ph.t_update = !(std::isinf(p.xi) || p.xi == 0.0);
    // the implicit solver takes the whole diffusion after the step kernel, which then keeps T
    ph.dxi = (ph.t_update && c->t_solver != LF_TSOLVER_IMPLICIT) ? (R)(p.xi / c->nsub) : R(0);
    ph.inv_tau = (R)(1.0 / p.tau);
    ph.guo = (R)(1.0 - 1.0 / (2.0 * p.tau));
    ph.n0 = (R)p.n0;
    ph.hydro = p.hydro;
    return ph;
}

template <typename R>
StepIO<R> io_of(lf_ctx* c, bool aux)
{
    StepIO<R> io{};
    io.f_in = (const R*)c->f[c->fcur];
    io.f_out = (R*)c->f[c->fcur ^ 1];
    io.phi_in = (const R*)c->phi[c->pcur];
    io.phi_out = (R*)c->phi[c->pcur ^ 1];
    io.T_in = (const R*)c->T[c->tcur];
    io.T_out = (R*)c->T[c->tcur ^ 1];
    io.flag = c->flag_dev;
    if (aux) {
        R* a = (R*)c->aux;
        const int64_t P = c->g.plane;
        io.mu = a;
        io.F[0] = a + P; io.F[1] = a + 2 * P; io.F[2] = a + 3 * P;
        io.rho = a + 4 * P;
        io.u[0] = a + 5 * P; io.u[1] = a + 6 * P; io.u[2] = a + 7 * P;
    }
    return io;
}

template <typename R>
cudaError_t launch_step_any(const Geom& g, const Phys<R>& p, const StepIO<R>& io, bool aux, cudaStream_t s,
                            cudaEvent_t* ev = nullptr)
{
    if (g.d == 2) return launch_step2d<R>(g, p, io, aux, s);
    if (!aux && g.variant == LF_VARIANT_SPLIT3) return launch_split3d<R>(g, p, io, s, ev);
    return launch_step3d<R>(g, p, io, aux, s);
}

template <typename R>
int do_steps(lf_ctx* c, int64_t n)
{
    const Phys<R> ph = phys_of<R>(c);
    for (int64_t k = 0; k < n; ++k) {
        StepIO<R> io = io_of<R>(c, true);      // the three-pass 3D step passes mu, F, u through aux
        const bool timed = c->pass_timing && c->g.d == 3 && c->g.variant == LF_VARIANT_SPLIT3;
        if (launch_step_any<R>(c->g, ph, io, false, c->stream, timed ? c->pass_ev : nullptr) != cudaSuccess)
            return LF_ECUDA;
        c->pass_recorded = timed;
        if (c->params.hydro) c->fcur ^= 1;
        c->pcur ^= 1;
        c->tcur ^= 1;
        if (ph.t_update && c->t_solver == LF_TSOLVER_IMPLICIT) {
            const int rc = t_implicit_step<R>(c, c->params.xi, c->walls.T_w);
            if (rc != LF_OK) return rc;
        } else if (ph.t_update) {
            for (int s = 1; s < c->nsub; ++s) {
                if (launch_tsub<R>(c->g, ph, (const R*)c->T[c->tcur], (R*)c->T[c->tcur ^ 1], c->stream) != cudaSuccess)
                    return LF_ECUDA;
                c->tcur ^= 1;
            }
        }
        c->step += 1;
    }
    c->aux_valid = false;
    return check_guards(c);
}

template <typename R>
int do_aux(lf_ctx* c)
{
    if (c->aux_valid) return LF_OK;
    StepIO<R> io = io_of<R>(c, true);
    if (launch_step_any<R>(c->g, phys_of<R>(c), io, true, c->stream) != cudaSuccess) return LF_ECUDA;
    c->aux_valid = true;
    return LF_OK;
}

int ensure_aux(lf_ctx* c) { return c->prec == LF_FP64 ? do_aux<double>(c) : do_aux<float>(c); }

// Device address of one plane of a field of the current state.
const void* field_plane(lf_ctx* c, int which, int q)
{
    const size_t P = (size_t)c->g.plane * c->esz;
    const unsigned char* a = (const unsigned char*)c->aux;
    switch (which) {
    case LF_FIELD_PHI: return c->phi[c->pcur];
    case LF_FIELD_T: return c->T[c->tcur];
    case LF_FIELD_POP: return (const unsigned char*)c->f[c->fcur] + (size_t)q * P;
    case LF_FIELD_MU: return a;
    case LF_FIELD_FX: return a + P;
    case LF_FIELD_FY: return a + 2 * P;
    case LF_FIELD_FZ: return a + 3 * P;
    case LF_FIELD_RHO: return a + 4 * P;
    case LF_FIELD_UX: return a + 5 * P;
    case LF_FIELD_UY: return a + 6 * P;
    case LF_FIELD_UZ: return a + 7 * P;
    default: return nullptr;
    }
}

double pop_weight(const lf_ctx* c, int q)
{
    return (c->g.d == 2 ? D2Q9::w(q) : D3Q19::w(q)) * c->params.n0;
}

// Address under which kernels of this device reach a host buffer: pinned or
// registered host memory is mapped into the device's address space, so the
// conversion kernels read or write it directly (no staging copy); null for
// pageable memory.
const void* mapped_host(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Planes [0, nplanes) of a field out (pack) or in (unpack).  Device buffers
// and host buffers mapped into the device's address space take one kernel
// for all planes; pageable host memory goes plane by plane through the stage
// with stream-ordered copies.  The caller waits once at the end.
template <typename R, typename D>
int pack_planes(lf_ctx* c, const void* src, void* dst, int nplanes, const PlaneAdd& add, int dst_on_device)
{
    void* target = dst_on_device ? dst : const_cast<void*>(mapped_host(dst));
    if (target) return launch_pack<R, D>(c->g, (const R*)src, (D*)target, nplanes, add, c->stream) == cudaSuccess
                           ? LF_OK : LF_ECUDA;
    for (int q = 0; q < nplanes; ++q) {
        PlaneAdd one{};
        one.v[0] = add.v[q];
        const R* s = (const R*)src + (size_t)q * c->g.plane;
        if (launch_pack<R, D>(c->g, s, (D*)c->stage, 1, one, c->stream) != cudaSuccess) return LF_ECUDA;
        if (cudaMemcpyAsync((D*)dst + (size_t)q * c->N, c->stage, (size_t)c->N * sizeof(D), cudaMemcpyDeviceToHost,
                            c->stream) != cudaSuccess)
            return LF_ECUDA;
    }
    return LF_OK;
}

template <typename R, typename D>
int unpack_planes(lf_ctx* c, const void* src, void* dst, int nplanes, const PlaneAdd& sub, int src_on_device)
{
    const void* from = src_on_device ? src : mapped_host(src);
    if (from) return launch_unpack<R, D>(c->g, (const D*)from, (R*)dst, nplanes, sub, c->stream) == cudaSuccess
                         ? LF_OK : LF_ECUDA;
    for (int q = 0; q < nplanes; ++q) {
        PlaneAdd one{};
        one.v[0] = sub.v[q];
        if (cudaMemcpyAsync(c->stage, (const D*)src + (size_t)q * c->N, (size_t)c->N * sizeof(D),
                            cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            return LF_ECUDA;
        if (launch_unpack<R, D>(c->g, (const D*)c->stage, (R*)dst + (size_t)q * c->g.plane, 1, one, c->stream) !=
            cudaSuccess)
            return LF_ECUDA;
    }
    return LF_OK;
}

template <typename R>
int pack_dispatch(lf_ctx* c, const void* src, void* dst, int np, const PlaneAdd& add, int on_dev, bool dbl)
{
    return dbl ? pack_planes<R, double>(c, src, dst, np, add, on_dev) : pack_planes<R, float>(c, src, dst, np, add, on_dev);
}

template <typename R>
int unpack_dispatch(lf_ctx* c, const void* src, void* dst, int np, const PlaneAdd& sub, int on_dev, bool dbl)
{
    return dbl ? unpack_planes<R, double>(c, src, dst, np, sub, on_dev)
               : unpack_planes<R, float>(c, src, dst, np, sub, on_dev);
}

PlaneAdd plane_offsets(const lf_ctx* c, int which)
{
    PlaneAdd a{};
    if (which == LF_FIELD_POP)
        for (int q = 0; q < c->Q; ++q) a.v[q] = pop_weight(c, q);
    return a;
}

int elem_from_bytes(const lf_ctx* c, int which, size_t bytes, bool* dbl)
{
    const size_t count = (size_t)c->N * (which == LF_FIELD_POP ? c->Q : 1);
    if (bytes == count * 8) { *dbl = true; return LF_OK; }
    if (bytes == count * 4) { *dbl = false; return LF_OK; }
    return LF_EINVAL;
}

int pending_status(lf_ctx* c)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return LF_ECUDA;
    if (c->guard_host && *c->guard_host) return LF_ECORRUPT;
    if (c->flag_host && *c->flag_host) return LF_ENONFINITE;
    return LF_OK;
}


}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
namespace lf {
// lf_fields / lf_fields_set between a context and device memory, enqueued on
// the context's stream without waiting (for code inside the library that
// chains several copies before one wait).
int fields_get_async(lf_ctx* c, int which, void* dst, size_t bytes)
{
    if (!c || !dst || which < 0 || which > LF_FIELD_FZ) return LF_EINVAL;
    bool dbl;
    int rc = elem_from_bytes(c, which, bytes, &dbl);
    if (rc != LF_OK) return rc;
    if (which != LF_FIELD_PHI && which != LF_FIELD_T && which != LF_FIELD_POP && (rc = ensure_aux(c)) != LF_OK)
        return rc;
    const int nplanes = which == LF_FIELD_POP ? c->Q : 1;
    const PlaneAdd add = plane_offsets(c, which);
    const void* src = field_plane(c, which, 0);
    return c->prec == LF_FP64 ? pack_dispatch<double>(c, src, dst, nplanes, add, 1, dbl)
                              : pack_dispatch<float>(c, src, dst, nplanes, add, 1, dbl);
}

int fields_set_async(lf_ctx* c, int which, const void* src, size_t bytes)
{
    if (!c || !src) return LF_EINVAL;
    if (which != LF_FIELD_PHI && which != LF_FIELD_T && which != LF_FIELD_POP) return LF_EINVAL;
    bool dbl;
    int rc = elem_from_bytes(c, which, bytes, &dbl);
    if (rc != LF_OK) return rc;
    const int nplanes = which == LF_FIELD_POP ? c->Q : 1;
    const PlaneAdd sub = plane_offsets(c, which);
    void* dst = const_cast<void*>(field_plane(c, which, 0));
    c->aux_valid = false;
    return c->prec == LF_FP64 ? unpack_dispatch<double>(c, src, dst, nplanes, sub, 1, dbl)
                              : unpack_dispatch<float>(c, src, dst, nplanes, sub, 1, dbl);
}
}  // namespace lf

extern "C" {

int lf_lattice(int d, int* e, double* w)
{
    if (d != 2 && d != 3) return LF_EINVAL;
    const int Q = d == 2 ? 9 : 19;
    for (int i = 0; i < Q; ++i) {
        if (e) {
            e[3 * i] = d == 2 ? D2Q9::ex(i) : D3Q19::ex(i);
            e[3 * i + 1] = d == 2 ? D2Q9::ey(i) : D3Q19::ey(i);
            e[3 * i + 2] = d == 2 ? D2Q9::ez(i) : D3Q19::ez(i);
        }
        if (w) w[i] = d == 2 ? D2Q9::w(i) : D3Q19::w(i);
    }
    return Q;
}

int lf_nsub(double xi, int d)
{
    if (d != 2 && d != 3) return LF_EINVAL;
    if (std::isinf(xi) || !(xi > 0.0)) return 1;
    const double n = std::ceil(xi / (0.8 / (2.0 * d)) - 1e-12);
    return n < 1 ? 1 : (int)n;
}

int lf_workspace_bytes(const lf_grid* grid, const lf_walls* walls, const lf_params* params, size_t* bytes)
{
    if (!bytes) return LF_EINVAL;
    int rc = validate(grid, walls, params);
    if (rc != LF_OK) return rc;
    *bytes = layout_for(grid, params, nullptr, nullptr).total;
    return LF_OK;
}

int lf_create(const lf_grid* grid, const lf_walls* walls, const lf_params* params, lf_ctx** out)
{
    if (!out) return LF_EINVAL;
    *out = nullptr;
    int rc = validate(grid, walls, params);
    if (rc != LF_OK) return rc;

    lf_ctx* c = new (std::nothrow) lf_ctx();
    if (!c) return LF_ENOMEM;
    c->grid = *grid;
    c->walls = *walls;
    c->params = *params;
    c->prec = params->precision;
    c->esz = c->prec == LF_FP64 ? 8 : 4;
    c->Q = grid->d == 2 ? 9 : 19;
    c->nsub = lf_nsub(params->xi, grid->d);
    c->N = grid->nx * grid->ny * grid->nz;
    c->stream = (cudaStream_t)params->stream;

    int64_t plane;
    int pitch;
    Layout L = layout_for(grid, params, &plane, &pitch);
    c->g.d = grid->d;
    c->g.nx = (int)grid->nx; c->g.ny = (int)grid->ny; c->g.nz = (int)grid->nz;
    c->g.pitch = pitch;
    c->g.plane = plane;
    c->g.walls = walls->walls;
    c->g.t_mode = walls->t_wall_mode;
    c->g.variant = grid->d == 3 ? LF_VARIANT_SPLIT3
                 : (params->precision == LF_FP32 ? LF_VARIANT_MARCH2 : LF_VARIANT_MARCH);
    c->g.tune = 0;
    c->g.stencil = params->stencil;
    c->t_solver = LF_TSOLVER_EXPLICIT;

    if (params->workspace) {
        if (params->workspace_bytes < L.total || ((uintptr_t)params->workspace % kAlign) != 0) {
            delete c;
            return LF_ENOMEM;
        }
        c->base = (unsigned char*)params->workspace;
        c->own = false;
    } else {
        if (cudaMalloc((void**)&c->base, L.total) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return LF_ENOMEM;
        }
        c->own = true;
    }
    c->bytes = L.total;
    c->checked = L.guard > 0;
    unsigned char* p = c->base;
    int ng = 0;
    auto guard = [&]() {                     // a guard band (checked mode only)
        if (!c->checked) return;
        c->guard_off[ng++] = (size_t)(p - c->base);
        p += L.guard;
    };
    guard();
    c->f[0] = p; p += L.f; guard();
    c->f[1] = p; p += L.f; guard();
    c->phi[0] = p; p += L.phi; guard();
    c->phi[1] = p; p += L.phi; guard();
    c->T[0] = p; p += L.T; guard();
    c->T[1] = p; p += L.T; guard();
    c->aux = p; p += L.aux; guard();
    c->stage = p; p += L.stage; guard();
    c->scratch = p; p += L.scratch; guard();
    c->scratch_bytes = L.scratch;

    int* fh = nullptr;
    if (cudaHostAlloc((void**)&fh, 2 * sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&c->flag_dev, fh, 0) != cudaSuccess) {
        cudaGetLastError();
        if (fh) cudaFreeHost(fh);
        if (c->own) cudaFree(c->base);
        delete c;
        return LF_ECUDA;
    }
    fh[0] = fh[1] = 0;
    c->flag_host = fh;
    c->guard_host = fh + 1;
    c->guard_dev = c->flag_dev + 1;

    rc = LF_OK;
    for (int i = 0; i < (c->checked ? 10 : 0) && rc == LF_OK; ++i)
        rc = check(cudaMemsetAsync(c->base + c->guard_off[i], kGuardByte, L.guard, c->stream));
    for (void* b : {c->f[0], c->f[1], c->phi[0], c->phi[1], c->T[0], c->T[1]})
        if (rc == LF_OK) rc = check(cudaMemsetAsync(b, 0, b == c->f[0] || b == c->f[1] ? L.f : L.phi, c->stream));
    if (rc == LF_OK) rc = check(cudaMemsetAsync(c->aux, 0, L.aux, c->stream));
    const int quench = std::isinf(params->xi) ? 1 : 0;
    if (rc == LF_OK) {
        if (c->prec == LF_FP64)
            rc = check(launch_init<double>(c->g, params->seed, params->phi_amp, params->T0, walls->T_w, quench,
                                           (double*)c->phi[0], (double*)c->T[0], c->stream));
        else
            rc = check(launch_init<float>(c->g, params->seed, params->phi_amp, params->T0, walls->T_w, quench,
                                          (float*)c->phi[0], (float*)c->T[0], c->stream));
    }
    if (rc == LF_OK) rc = wait_stream(c->stream);
    if (rc != LF_OK) {
        lf_destroy(c);
        return rc;
    }
    *out = c;
    return LF_OK;
}

int lf_step(lf_ctx* c, int64_t nsteps)
{
    lf::NvtxRange nvtx_range("lf_step");
    if (!c || nsteps < 0 || c->ens_member) return LF_EINVAL;
    int rc = pending_status(c);
    if (rc != LF_OK) return rc;
    return c->prec == LF_FP64 ? do_steps<double>(c, nsteps) : do_steps<float>(c, nsteps);
}


int lf_fields(lf_ctx* c, int which, void* dst, size_t bytes, int dst_on_device)
{
    lf::NvtxRange nvtx_range("lf_fields");
    if (!c || !dst || which < 0 || which > LF_FIELD_FZ) return LF_EINVAL;
    bool dbl;
    int rc = elem_from_bytes(c, which, bytes, &dbl);
    if (rc != LF_OK) return rc;
    if (which != LF_FIELD_PHI && which != LF_FIELD_T && which != LF_FIELD_POP) {
        rc = ensure_aux(c);
        if (rc != LF_OK) return rc;
    }
    const int nplanes = which == LF_FIELD_POP ? c->Q : 1;
    const PlaneAdd add = plane_offsets(c, which);
    const void* src = field_plane(c, which, 0);
    rc = c->prec == LF_FP64 ? pack_dispatch<double>(c, src, dst, nplanes, add, dst_on_device, dbl)
                            : pack_dispatch<float>(c, src, dst, nplanes, add, dst_on_device, dbl);
    if (rc == LF_OK) rc = wait_stream(c->stream);
    if (rc == LF_OK) rc = check(cudaGetLastError());
    return rc;
}

int lf_fields_set(lf_ctx* c, int which, const void* src, size_t bytes, int src_on_device)
{
    lf::NvtxRange nvtx_range("lf_fields_set");
    if (!c || !src) return LF_EINVAL;
    if (which != LF_FIELD_PHI && which != LF_FIELD_T && which != LF_FIELD_POP) return LF_EINVAL;
    bool dbl;
    int rc = elem_from_bytes(c, which, bytes, &dbl);
    if (rc != LF_OK) return rc;
    const int nplanes = which == LF_FIELD_POP ? c->Q : 1;
    const PlaneAdd sub = plane_offsets(c, which);
    void* dst = const_cast<void*>(field_plane(c, which, 0));
    rc = c->prec == LF_FP64 ? unpack_dispatch<double>(c, src, dst, nplanes, sub, src_on_device, dbl)
                            : unpack_dispatch<float>(c, src, dst, nplanes, sub, src_on_device, dbl);
    c->aux_valid = false;
    if (rc == LF_OK) rc = wait_stream(c->stream);
    if (rc == LF_OK) rc = check(cudaGetLastError());
    return rc;
}

int lf_diag(lf_ctx* c, lf_diag_t* out)
{
    lf::NvtxRange nvtx_range("lf_diag");
    if (!c || !out) return LF_EINVAL;
    std::memset(out, 0, sizeof(*out));
    int rc = ensure_aux(c);
    if (rc != LF_OK) return rc;
    DiagInput in;
    in.g = c->g;
    in.prec = c->prec;
    in.phi = c->phi[c->pcur];
    in.T = c->T[c->tcur];
    in.aux = c->aux;
    in.b = c->params.b; in.kappa = c->params.kappa; in.c = c->params.c; in.Tc = c->params.Tc;
    in.scratch = c->scratch;
    in.scratch_bytes = c->scratch_bytes;
    in.stage = c->stage;
    DiagResult r;
    rc = run_diag(in, &r, c->stream);
    if (rc != LF_OK) return rc;
    out->step = c->step;
    out->mass = r.sums[DQ_MASS];
    out->phi_sum = r.sums[DQ_PHI];
    out->mom[0] = r.sums[DQ_MX]; out->mom[1] = r.sums[DQ_MY]; out->mom[2] = r.sums[DQ_MZ];
    out->umax = std::sqrt(r.sums[DQ_U2MAX]);
    out->mach = out->umax * std::sqrt(3.0);
    out->free_energy = r.sums[DQ_FE];
    out->grad2[0] = r.sums[DQ_GX]; out->grad2[1] = r.sums[DQ_GY]; out->grad2[2] = r.sums[DQ_GZ];
    const int d = c->g.d;
    const double gall = r.sums[DQ_GX] + r.sums[DQ_GY] + r.sums[DQ_GZ];
    const double gperp = d == 2 ? r.sums[DQ_GY] : r.sums[DQ_GZ];
    out->orient_s = gall > 0 ? (d * gperp / gall - 1.0) / (d - 1) : 0.0;
    out->k_peak = r.k_peak;
    out->s_peak = r.s_peak;
    out->nonfinite = (c->flag_host && *c->flag_host) ? 1 : 0;
    bool finite = std::isfinite(out->mass) && std::isfinite(out->phi_sum) && std::isfinite(out->umax);
    if (!finite) {
        out->nonfinite = 1;
        *const_cast<int*>(c->flag_host) = 1;
    }
    return out->nonfinite ? LF_ENONFINITE : LF_OK;
}

int lf_diag_layers(lf_ctx* c, double* out, int64_t L)
{
    if (!c || !out || L != (c->g.d == 2 ? c->g.ny : c->g.nz)) return LF_EINVAL;
    DiagInput in;
    in.g = c->g;
    in.prec = c->prec;
    in.phi = c->phi[c->pcur];
    in.scratch = c->scratch;
    in.scratch_bytes = c->scratch_bytes;
    in.stage = c->stage;
    return run_layers(in, out, c->stream);
}

int lf_structure_factor(lf_ctx* c, double* out, int64_t nb)
{
    if (!c || !out) return LF_EINVAL;
    DiagInput in;
    in.g = c->g;
    in.prec = c->prec;
    in.phi = c->phi[c->pcur];
    in.scratch = c->scratch;
    in.scratch_bytes = c->scratch_bytes;
    in.stage = c->stage;
    return run_sk_shells(in, out, nb, c->stream);
}

int64_t lf_step_count(const lf_ctx* c) { return c ? c->step : -1; }

int lf_set_pass_timing(lf_ctx* c, int enable)
{
    if (!c || c->ens_member) return LF_EINVAL;
    if (enable && !c->pass_ev[0]) {
        for (int i = 0; i < 4; ++i)
            if (cudaEventCreate(&c->pass_ev[i]) != cudaSuccess) {
                for (int j = 0; j < i; ++j) {
                    cudaEventDestroy(c->pass_ev[j]);
                    c->pass_ev[j] = nullptr;
                }
                cudaGetLastError();
                return LF_ECUDA;
            }
    }
    c->pass_timing = enable != 0;
    c->pass_recorded = false;
    return LF_OK;
}

int lf_pass_times(lf_ctx* c, float* ms, int n, int* npasses)
{
    if (!c || n < 0 || (n > 0 && !ms)) return LF_EINVAL;
    int np = 0;
    if (c->pass_recorded) {
        const int rc = wait_stream(c->stream);
        if (rc != LF_OK) return rc;
        np = 3;
        for (int i = 0; i < np && i < n; ++i)
            if (cudaEventElapsedTime(&ms[i], c->pass_ev[i], c->pass_ev[i + 1]) != cudaSuccess) return LF_ECUDA;
    }
    if (npasses) *npasses = np;
    return LF_OK;
}

int lf_set_t_solver(lf_ctx* c, int solver)
{
    if (!c || (solver != LF_TSOLVER_EXPLICIT && solver != LF_TSOLVER_IMPLICIT) || c->ens_member) return LF_EINVAL;
    if (solver == LF_TSOLVER_IMPLICIT && !t_implicit_supported(c->g)) return LF_EINVAL;
    if (solver == LF_TSOLVER_IMPLICIT && c->g.walls && !c->tcoef) {
        void* t = nullptr;
        if (cudaMalloc(&t, sizeof(double) * 2 * (size_t)c->N) != cudaSuccess) {
            cudaGetLastError();
            return LF_ENOMEM;
        }
        c->tcoef = (double*)t;
        c->tcoef_valid = false;
    }
    c->t_solver = solver;
    return LF_OK;
}

int lf_set_stencil(lf_ctx* c, int stencil)
{
    if (!c || (stencil != LF_STENCIL_COMPACT && stencil != LF_STENCIL_ISOTROPIC) || c->ens_member) return LF_EINVAL;
    lf_params p = c->params;
    p.stencil = stencil;
    const int rc = validate(&c->grid, &c->walls, &p);
    if (rc != LF_OK) return rc;
    if (stencil != c->g.stencil) c->aux_valid = false;
    c->params.stencil = stencil;
    c->g.stencil = stencil;
    return LF_OK;
}

int lf_set_kernel_variant(lf_ctx* c, int variant, int param)
{
    if (!c || (variant != LF_VARIANT_MARCH && variant != LF_VARIANT_TILE && variant != LF_VARIANT_MARCH2 &&
               variant != LF_VARIANT_SPLIT3) ||
        param < 0)
        return LF_EINVAL;
    c->g.variant = variant;
    c->g.tune = param;
    return LF_OK;
}

// ---- checkpoints ----------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];
    int32_t version, d, precision, walls, t_mode, Q;
    int64_t nx, ny, nz, step;
    lf_params params;
    double T_w;
    int32_t stencil, t_solver;   // the scheme the state was advanced with
    int32_t pad_[2];
};
constexpr char kCkptMagic[8] = "LFCKPT2";
}  // namespace

// The file holds the state exactly as the context stores it: the population
// deviations f_i - w_i n0, phi and T, each unpadded, in the context precision,
// so that save + load + n steps is bit-identical to n steps.
namespace {
int raw_copy(lf_ctx* c, const void* plane_dev, void* host, bool to_host)
{
    int rc;
    const PlaneAdd zero{};
    if (to_host) {
        rc = c->prec == LF_FP64 ? pack_planes<double, double>(c, plane_dev, host, 1, zero, 0)
                                : pack_planes<float, float>(c, plane_dev, host, 1, zero, 0);
    } else {
        rc = c->prec == LF_FP64 ? unpack_planes<double, double>(c, host, const_cast<void*>(plane_dev), 1, zero, 0)
                                : unpack_planes<float, float>(c, host, const_cast<void*>(plane_dev), 1, zero, 0);
    }
    return rc;
}
}  // namespace

int lf_save(lf_ctx* c, const char* path)
{
    lf::NvtxRange nvtx_range("lf_save");
    if (!c || !path) return LF_EINVAL;
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 2; h.d = c->g.d; h.precision = c->prec; h.walls = c->g.walls; h.t_mode = c->g.t_mode;
    h.Q = c->Q; h.nx = c->g.nx; h.ny = c->g.ny; h.nz = c->g.nz; h.step = c->step;
    h.params = c->params;
    h.params.stream = nullptr; h.params.workspace = nullptr; h.params.workspace_bytes = 0;
    h.T_w = c->walls.T_w;
    h.stencil = c->g.stencil;
    h.t_solver = c->t_solver;
    const size_t nf = (size_t)c->N * c->esz;
    unsigned char* buf = (unsigned char*)std::malloc(nf * (c->Q + 2));
    if (!buf) return LF_ENOMEM;
    int rc = LF_OK;
    for (int q = 0; q < c->Q && rc == LF_OK; ++q) rc = raw_copy(c, field_plane(c, LF_FIELD_POP, q), buf + nf * q, true);
    if (rc == LF_OK) rc = raw_copy(c, field_plane(c, LF_FIELD_PHI, 0), buf + nf * c->Q, true);
    if (rc == LF_OK) rc = raw_copy(c, field_plane(c, LF_FIELD_T, 0), buf + nf * (c->Q + 1), true);
    if (rc == LF_OK) rc = wait_stream(c->stream);
    if (rc == LF_OK) {
        FILE* fp = std::fopen(path, "wb");
        if (!fp) rc = LF_EIO;
        else {
            if (std::fwrite(&h, sizeof(h), 1, fp) != 1 || std::fwrite(buf, nf, c->Q + 2, fp) != (size_t)(c->Q + 2))
                rc = LF_EIO;
            if (std::fclose(fp) != 0) rc = LF_EIO;
        }
    }
    std::free(buf);
    return rc;
}

int lf_load(lf_ctx* c, const char* path)
{
    lf::NvtxRange nvtx_range("lf_load");
    if (!c || !path) return LF_EINVAL;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return LF_EIO;
    CkptHeader h;
    int rc = LF_OK;
    // A checkpoint resumes only on the lattice and with the scheme it was
    // written with: a different stencil or temperature solver would silently
    // continue the run with another method, so it is refused.
    if (std::fread(&h, sizeof(h), 1, fp) != 1 || std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.d != c->g.d ||
        h.precision != c->prec || h.walls != c->g.walls || h.nx != c->g.nx || h.ny != c->g.ny || h.nz != c->g.nz ||
        h.Q != c->Q || h.stencil != c->g.stencil || h.t_solver != c->t_solver)
        rc = LF_EIO;
    const size_t nf = (size_t)c->N * c->esz;
    unsigned char* buf = nullptr;
    if (rc == LF_OK) {
        buf = (unsigned char*)std::malloc(nf * (c->Q + 2));
        if (!buf) rc = LF_ENOMEM;
        else if (std::fread(buf, nf, c->Q + 2, fp) != (size_t)(c->Q + 2)) rc = LF_EIO;
    }
    std::fclose(fp);
    for (int q = 0; q < c->Q && rc == LF_OK; ++q) rc = raw_copy(c, field_plane(c, LF_FIELD_POP, q), buf + nf * q, false);
    if (rc == LF_OK) rc = raw_copy(c, field_plane(c, LF_FIELD_PHI, 0), buf + nf * c->Q, false);
    if (rc == LF_OK) rc = raw_copy(c, field_plane(c, LF_FIELD_T, 0), buf + nf * (c->Q + 1), false);
    if (rc == LF_OK) rc = wait_stream(c->stream);
    if (rc == LF_OK) {
        c->step = h.step;
        c->aux_valid = false;
    }
    std::free(buf);
    return rc;
}

void lf_destroy(lf_ctx* c)
{
    if (!c) return;
    wait_stream(c->stream);
    if (c->own && c->base) cudaFree(c->base);
    if (c->tcoef) cudaFree(c->tcoef);
    for (cudaEvent_t ev : c->pass_ev)
        if (ev) cudaEventDestroy(ev);
    if (c->flag_host) cudaFreeHost(const_cast<int*>(c->flag_host));
    cudaGetLastError();
    delete c;
}

const char* lf_strerror(int code)
{
    switch (code) {
    case LF_OK: return "ok";
    case LF_EINVAL: return "invalid argument";
    case LF_EUNSTABLE: return "parameters outside the stability limits of the explicit schemes";
    case LF_ENOMEM: return "out of memory (or workspace too small / misaligned)";
    case LF_ECUDA: return "CUDA error";
    case LF_ENONFINITE: return "non-finite value (NaN/Inf) in the state";
    case LF_ETIMEOUT: return "timed out waiting for the GPU";
    case LF_EIO: return "checkpoint I/O error or mismatch";
    case LF_ECORRUPT: return "a guard band around a device buffer was overwritten (checked mode)";
    default: return "unknown error";
    }
}

}  // extern "C"
