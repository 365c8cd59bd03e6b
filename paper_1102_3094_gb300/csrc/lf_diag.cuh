// lf_diag.cuh -- diagnostics of the current state: FP64 conservation sums,
// |u|_max (Mach check of arXiv:1102.3094 Sec. 2), gradient sums for the
// orientation order parameter, the phi part of the free energy (Eq. fren) and
// the shell-averaged structure factor S(k).
#pragma once

#include "lf_internal.cuh"

namespace lf {

enum {
    DQ_MASS = 0,   // sum n
    DQ_PHI,        // sum phi
    DQ_MX, DQ_MY, DQ_MZ,   // sum n u
    DQ_GX, DQ_GY, DQ_GZ,   // sum (d_a phi)^2, central differences
    DQ_FE,         // sum a phi^2/2 + b phi^4/4 + c (nabla^2 phi)^2/2, plus kappa/2 sum_links (dphi)^2
    DQ_U2MAX,      // max |u|^2
    DQ_N
};

struct DiagInput {
    Geom g;
    int prec;
    const void* phi;
    const void* T;
    const void* aux;          // mu, F[3], n, u[3] planes (see lf_api.cu)
    double b, kappa, c, Tc;
    void* scratch;            // diag_scratch_bytes() of device memory
    size_t scratch_bytes;
    void* stage;              // unused by the diagnostics; kept for symmetry
};

struct DiagResult {
    double sums[DQ_N];
    double k_peak, s_peak;    // NaN when the FFT cannot handle the lattice sizes
};

size_t diag_scratch_bytes(int d, int64_t nx, int64_t ny, int64_t nz);

// The N complex doubles of FFT scratch inside a context's diagnostics area.
double2* fft_buffer(const Geom& g, void* scratch);
// Whether a line of length n is within the FFT's reach (prime factors up to 31, n <= 4096).
bool fft_supported(int n);
// Forward DFT along one axis of a packed [nz][ny][nx] complex FP64 array, in place.
cudaError_t fft_forward_axis(const Geom& g, double2* data, int axis, cudaStream_t s);

// Blocking (bounded wait) runs; results land in host memory.
int run_diag(const DiagInput& in, DiagResult* r, cudaStream_t s);
int run_layers(const DiagInput& in, double* out_host, cudaStream_t s);
int run_sk_shells(const DiagInput& in, double* out_host, int64_t nb, cudaStream_t s);

}  // namespace lf
