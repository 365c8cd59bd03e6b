// lf_ctx.cuh -- the context behind the opaque lf_ctx handle of lf.h, shared
// by the single-lattice API (lf_api.cu) and the ensemble (lf_ens.cu).
#pragma once

#include "lf_internal.cuh"

struct lf_ctx {
    lf_grid grid;
    lf_walls walls;
    lf_params params;
    lf::Geom g;
    int Q, nsub, prec;
    size_t esz;
    int64_t N;            // sites
    cudaStream_t stream;
    unsigned char* base;  // device block
    size_t bytes;
    bool own;
    void* f[2];
    void* phi[2];
    void* T[2];
    int fcur, pcur, tcur;
    void* aux;            // 8 planes: mu, Fx, Fy, Fz, rho, ux, uy, uz
    void* stage;          // N doubles
    void* scratch;        // diagnostics reduction scratch
    size_t scratch_bytes;
    int* flag_dev;
    volatile int* flag_host;
    // checked mode (LF_CHECKED=1 at creation): guard bands around every buffer
    bool checked;
    int* guard_dev;                 // set to 1 by the guard check when a band changed
    volatile int* guard_host;
    size_t guard_off[10];           // offsets of the guard bands from base
    int64_t step;
    bool aux_valid;
    bool ens_member;      // stepped by an ensemble; lf_step on it is refused
    int t_solver;         // LF_TSOLVER_EXPLICIT (n_sub sub-steps) or LF_TSOLVER_IMPLICIT
    // implicit solver with walls: c'_j and the reciprocal pivots of the
    // tridiagonal solve, per Fourier mode and layer (2 N doubles, allocated by
    // lf_set_t_solver), valid for the xi, wall rule and stencil recorded here
    double* tcoef;
    bool tcoef_valid;
    double tcoef_xi;
    int tcoef_mode, tcoef_stencil;
    // pass timing (lf_set_pass_timing): events before and after the passes of
    // the last three-pass step, and whether that step recorded them
    cudaEvent_t pass_ev[4];
    bool pass_timing;
    bool pass_recorded;
};

namespace lf {
// lf_fields / lf_fields_set with device memory on the other side, enqueued
// on the context's stream without waiting (library-internal).
int fields_get_async(lf_ctx* c, int which, void* dst, size_t bytes);
int fields_set_async(lf_ctx* c, int which, const void* src, size_t bytes);
}  // namespace lf

namespace lf {
// Implicit (backward-Euler) temperature step of the current T, in place
// (lf_timplicit.cu); requires t_implicit_supported(g).
bool t_implicit_supported(const Geom& g);
template <typename R>
int t_implicit_step(lf_ctx* c, double xi, double T_w);
}  // namespace lf
