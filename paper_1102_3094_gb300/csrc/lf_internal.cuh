// lf_internal.cuh -- state layout and kernel entry points shared by the CUDA
// translation units of the library.  Not part of the public C ABI (lf.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <cstdlib>
#include <thread>

#include "lf.h"

#include <nvtx3/nvToolsExt.h>

namespace lf {

// A named NVTX range for the duration of a scope (one per public call, so that
// profilers can filter and attribute the kernels a call launches).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// Velocity sets (Sec. 2: moduli 0, c, sqrt(2) c; weights 4/9, 1/9, 1/36).
// D2Q9 order: rest, +x, +y, -x, -y, (+x+y), (-x+y), (-x-y), (+x-y).
// D3Q19 order: rest, +-x, +-y, +-z, then the 12 edge diagonals.
// ---------------------------------------------------------------------------
// Tables are constexpr functions so that, inside fully unrolled loops, every
// entry folds to an immediate in device code.
struct D2Q9 {
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int ex(int i)
    { constexpr int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}; return t[i]; }
    __host__ __device__ static constexpr int ey(int i)
    { constexpr int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1}; return t[i]; }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i)
    { constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6}; return t[i]; }
    __host__ __device__ static constexpr double w(int i)
    { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
};

struct D3Q19 {
    static constexpr int Q = 19;
    __host__ __device__ static constexpr int ex(int i)
    { constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0}; return t[i]; }
    __host__ __device__ static constexpr int ey(int i)
    { constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1}; return t[i]; }
    __host__ __device__ static constexpr int ez(int i)
    { constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1}; return t[i]; }
    __host__ __device__ static constexpr int opp(int i)
    { constexpr int t[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17}; return t[i]; }
    __host__ __device__ static constexpr double w(int i)
    { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
};

// ---------------------------------------------------------------------------
// Geometry of one lattice in device memory.
//   Scalar field: [nz][ny][pitch] with pitch = nx rounded up to 32 elements,
//   so every row starts on a 128-byte (FP32) / 256-byte (FP64) boundary.
//   Populations: Q such planes back to back (structure of arrays).
//   The wall axis is the slowest one of the lattice (y in 2D, z in 3D).
// ---------------------------------------------------------------------------
struct Geom {
    int d;
    int nx, ny, nz;
    int pitch;
    int64_t plane;   // pitch * ny * nz elements
    int walls;
    int t_mode;
    int variant;     // LF_VARIANT_MARCH or LF_VARIANT_TILE
    int tune;        // march: rows per segment (0 = automatic)
    int stencil;     // LF_STENCIL_COMPACT or LF_STENCIL_ISOTROPIC
};

// Physical parameters in the precision of the arithmetic.
template <typename R>
struct Phys {
    R b, kappa, c, Gamma, Tc, T_w;
    R inv_Tc;     // 1 / Tc
    R dxi;        // xi / nsub: explicit Euler step of the temperature
    R inv_tau;    // 1 / tau
    R guo;        // 1 - 1/(2 tau)
    R n0;
    int hydro;
    int t_update; // 0 when xi = 0 or +inf
};

// Pointers of one step.
template <typename R>
struct StepIO {
    const R* f_in;   R* f_out;
    const R* phi_in; R* phi_out;
    const R* T_in;   R* T_out;
    // Derived fields at time t (aux mode only): mu, F[3], n, u[3].
    R* mu; R* F[3]; R* rho; R* u[3];
    int* flag;       // set to 1 when a NaN/Inf is produced (host-mapped)
};

// ---------------------------------------------------------------------------
// Launchers (all enqueue on `s` and return the launch status).
// ---------------------------------------------------------------------------
template <typename R>
cudaError_t launch_step2d(const Geom& g, const Phys<R>& p, const StepIO<R>& io, bool aux,
                          cudaStream_t s);
template <typename R>
cudaError_t launch_step3d(const Geom& g, const Phys<R>& p, const StepIO<R>& io, bool aux,
                          cudaStream_t s);
// the three-pass 3D step (lf_step3d_passes.cu); ev: nullptr, or four events
// recorded before pass A and after passes A, B and C
template <typename R>
cudaError_t launch_split3d(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s,
                           cudaEvent_t* ev = nullptr);
// its passes with the compact stencils (lf_step3d_split.cu)
template <typename R>
cudaError_t launch_force3d_compact(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s);
template <typename R>
cudaError_t launch_lb3d(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s);
template <typename R>
cudaError_t launch_phi3d_compact(const Geom& g, const Phys<R>& p, const StepIO<R>& io, int zc, cudaStream_t s);
// passes A and C of the three-pass step with the isotropic stencils (lf_step3d_iso.cu)
template <typename R>
cudaError_t launch_force3d_iso(const Geom& g, const Phys<R>& p, const StepIO<R>& io, cudaStream_t s);
template <typename R>
cudaError_t launch_phi3d_iso(const Geom& g, const Phys<R>& p, const StepIO<R>& io, int zc, cudaStream_t s);
template <typename R>
cudaError_t launch_tsub3d(const Geom& g, const Phys<R>& p, const R* Tin, R* Tout, cudaStream_t s);
template <typename R>
cudaError_t launch_tsub(const Geom& g, const Phys<R>& p, const R* Tin, R* Tout, cudaStream_t s);
template <typename R>
cudaError_t launch_init(const Geom& g, uint64_t seed, double amp, double T0, double T_w,
                        int quench, R* phi, R* T, cudaStream_t s);
// Per-plane offsets of a layout conversion (population weights w_q n0).
struct PlaneAdd {
    double v[19];
};
// Planes q < nplanes: dst[q N + k] = (D)(src[q plane + site k] + add[q]), k
// over the unpadded lattice (x fastest), N = nx ny nz.
template <typename R, typename D>
cudaError_t launch_pack(const Geom& g, const R* src, D* dst, int nplanes, const PlaneAdd& add, cudaStream_t s);
// dst[q plane + site k] = (R)(src[q N + k] - sub[q]).
template <typename R, typename D>
cudaError_t launch_unpack(const Geom& g, const D* src, R* dst, int nplanes, const PlaneAdd& sub, cudaStream_t s);

// ---------------------------------------------------------------------------
// Bounded wait: polls an event recorded on `s` so that a GPU that stops
// answering turns into LF_ETIMEOUT instead of a hang.  The limit is 120 s, or
// LF_WAIT_TIMEOUT_S seconds when that environment variable is set.
// ---------------------------------------------------------------------------
inline int wait_stream(cudaStream_t s)
{
    const char* env = std::getenv("LF_WAIT_TIMEOUT_S");
    double lim = env ? std::atof(env) : 120.0;
    if (!(lim > 0)) lim = 120.0;
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return LF_ECUDA;
    if (cudaEventRecord(ev, s) != cudaSuccess) { cudaEventDestroy(ev); return LF_ECUDA; }
    const auto t0 = std::chrono::steady_clock::now();
    int rc = LF_OK;
    for (;;) {
        const cudaError_t q = cudaEventQuery(ev);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) { rc = LF_ECUDA; break; }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > lim) { rc = LF_ETIMEOUT; break; }
        // poll without sleeping for the first 2 ms (a sleep of a few us
        // overshoots by tens of us, which dominates short waits), then back off
        if (el < 0.002) continue;
        std::this_thread::sleep_for(std::chrono::microseconds(el < 0.05 ? 20 : 200));
    }
    cudaEventDestroy(ev);
    return rc;
}

// A kernel's dynamic shared-memory limit and the SM count belong to the
// current device, and one process may drive several devices: both are kept
// per device ordinal (0 .. 63; beyond that the attribute is set on every call).
constexpr int kMaxDevices = 64;

template <typename K>
cudaError_t raise_smem_limit(K kern, int bytes, unsigned long long* done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < kMaxDevices ? 1ull << dev : 0ull;
    if (bit && (__atomic_load_n(done, __ATOMIC_ACQUIRE) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) __atomic_fetch_or(done, bit, __ATOMIC_RELEASE);
    return e;
}

inline cudaError_t device_sms(int* sms)
{
    static int cache[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < kMaxDevices) {
        const int c = __atomic_load_n(&cache[dev], __ATOMIC_ACQUIRE);
        if (c > 0) { *sms = c; return cudaSuccess; }
    }
    int n = 0;
    if ((e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    n = n > 0 ? n : 1;
    if (dev < kMaxDevices) __atomic_store_n(&cache[dev], n, __ATOMIC_RELEASE);
    *sms = n;
    return cudaSuccess;
}

}  // namespace lf
