/*
 * lf.h -- C ABI of the GB300 library for the hybrid lattice-Boltzmann /
 * finite-difference time step of Gonnella, Lamura & Tiribocchi, "Thermal and
 * hydrodynamic effects in the ordering of lamellar fluids" (arXiv:1102.3094).
 *
 * One call of lf_step advances, per lattice site and per step (Sec. 2):
 *   a    = (T - Tc)/Tc                                       (Eq. aterm)
 *   mu   = a phi + b phi^3 - kappa nabla^2 phi + c nabla^4 phi (Eq. chem)
 *   P_ab = phi-dependent pressure tensor of the free energy    (Eq. fren, P_ab)
 *   F_b  = -d_a P_ab                                           (Eq. ff)
 *   n, n u = sum f_i, sum f_i e_i + F/2                        (Eq. moment)
 *   f_i(r + e_i, t+1) = f_i - (f_i - f_i^eq)/tau + F_i         (Eqs. evoleqn,
 *                                                               latticeforceterm)
 *   phi(t+1) = phi - d_a(phi u_a) + Gamma nabla^2 mu           (Eq. massdiff)
 *   T(t+1)   = T + xi nabla^2 T                                (Sec. 2, after
 *                                                               Eq. massdiff)
 * on a D2Q9 (d = 2) or D3Q19 (d = 3) lattice with dx = dt = c = 1, c_s^2 = 1/3.
 * Walls (Sec. 2, boundary paragraph) sit half a spacing outside the first and
 * last layer along the last axis (y in 2D, z in 3D); the other axes are
 * periodic.  At the walls: halfway bounce-back for the populations; even
 * reflection of phi, nabla^2 phi, nabla^4 phi, mu and a (neutral wetting and
 * exact conservation of phi); no flux of phi through the wall; T held at T_w.
 *
 * Conventions for every entry point:
 *   - Return 0 (LF_OK) or a negative LF_E* code; nothing exits, aborts or
 *     throws across this boundary.  lf_strerror maps a code to a message.
 *   - "Device" pointers are CUDA device (or managed) addresses of the current
 *     device, e.g. a torch tensor's data_ptr(); "host" pointers are ordinary
 *     (pageable or pinned) CPU memory.
 *   - Field layout is row-major [nz][ny][nx] (x fastest), nz = 1 in 2D;
 *     populations are [Q][nz][ny][nx] in the order lf_lattice reports.
 *   - The context owns its device state; no pointer into it escapes.  Caller
 *     buffers are only read or written during the call that receives them.
 *   - Work is enqueued on params.stream (a cudaStream_t; 0 = legacy default
 *     stream).  lf_step returns without waiting; lf_fields, lf_fields_set,
 *     lf_diag, lf_save and lf_load wait for the stream, with a time limit
 *     (LF_ETIMEOUT: 120 s, or LF_WAIT_TIMEOUT_S seconds from the
 *     environment).  After LF_ETIMEOUT the context stays usable, but a copy
 *     to or from a device or pinned caller buffer may still be in flight on
 *     the stream: synchronize the stream before reusing that buffer.
 *   - Checked mode: with LF_CHECKED=1 in the environment when
 *     lf_workspace_bytes and lf_create run, every device buffer of the
 *     context is followed by a 64 KiB guard band (one more before the first)
 *     filled with the byte 0xA5, and every lf_step call ends with a kernel
 *     that verifies all of them; the next call that reports pending errors
 *     (lf_step) returns LF_ECORRUPT if any guard byte changed.  The workspace
 *     grows by 640 KiB; the state, its layout and the results are unchanged.
 */
#ifndef LF_H
#define LF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define LF_OK          0
#define LF_EINVAL     -1  /* bad argument (sizes, pointers, enum values)           */
#define LF_EUNSTABLE  -2  /* parameters outside the explicit schemes' stability    */
#define LF_ENOMEM     -3  /* device or host allocation failed / workspace too small */
#define LF_ECUDA      -4  /* a CUDA runtime call or kernel launch failed            */
#define LF_ENONFINITE -5  /* a NaN or Inf appeared in phi, T or the density         */
#define LF_ETIMEOUT   -6  /* a bounded wait for the GPU ran out                     */
#define LF_EIO        -7  /* checkpoint file could not be written / read / matched  */
#define LF_ECORRUPT   -8  /* checked mode: a guard band of a buffer was overwritten */

/* ---- enumerations ------------------------------------------------------ */
#define LF_FP64 0         /* all state and arithmetic in double                     */
#define LF_FP32 1         /* state and arithmetic in float; populations stored as
                             deviations f_i - w_i n0; diagnostics sums in double   */

#define LF_TWALL_LAYERS  0 /* T = T_w held on the first and last layer (default)    */
#define LF_TWALL_HALFWAY 1 /* every layer evolves; ghost T = 2 T_w - T at the wall  */

#define LF_FIELD_PHI 0    /* order parameter phi                       [N]          */
#define LF_FIELD_T   1    /* temperature T                             [N]          */
#define LF_FIELD_RHO 2    /* density n = sum f_i                       [N]          */
#define LF_FIELD_UX  3    /* velocity u (Eq. moment, with F/2)         [N]          */
#define LF_FIELD_UY  4
#define LF_FIELD_UZ  5
#define LF_FIELD_POP 6    /* populations f_i (full, not deviations)    [Q][N]       */
#define LF_FIELD_MU  7    /* chemical potential mu (Eq. chem)          [N]          */
#define LF_FIELD_FX  8    /* force density F (Eq. ff)                  [N]          */
#define LF_FIELD_FY  9
#define LF_FIELD_FZ  10

/* ---- configuration ----------------------------------------------------- */
typedef struct {
    int     d;            /* 2 or 3                                               */
    int     pad_;
    int64_t nx, ny, nz;   /* lattice sizes; nz must be 1 when d = 2               */
} lf_grid;

typedef struct {
    int    walls;         /* 1: walls normal to the last axis; 0: fully periodic  */
    int    t_wall_mode;   /* LF_TWALL_LAYERS or LF_TWALL_HALFWAY                  */
    double T_w;           /* wall temperature                                     */
} lf_walls;

typedef struct {
    double   b, kappa, c; /* free-energy coefficients, Eq. fren (b, c > 0)        */
    double   Gamma;       /* mobility, Eq. massdiff                               */
    double   Tc;          /* critical temperature, Eq. aterm (> 0)                */
    double   T0;          /* initial temperature away from the walls              */
    double   xi;          /* thermal conductivity; +INFINITY = instant quench     */
    double   tau;         /* BGK relaxation time (> 1/2)                          */
    double   n0;          /* initial (reference) density                          */
    double   phi_amp;     /* initial phi i.i.d. uniform in [-phi_amp, phi_amp)    */
    uint64_t seed;        /* SplitMix64 seed of the initial phi                   */
    int      precision;   /* LF_FP64 or LF_FP32                                   */
    int      hydro;       /* 1: LB coupled; 0: Eq. massdiff without convection    */
    int      ideal_mode;  /* must be 0: ideal pressure n c_s^2 kept by the LB     */
    int      stencil;     /* LF_STENCIL_COMPACT (0) or LF_STENCIL_ISOTROPIC (1)  */
    void*    stream;      /* cudaStream_t to enqueue on (borrowed, not owned)     */
    void*    workspace;   /* optional caller device buffer for all state          */
    size_t   workspace_bytes; /* its size; see lf_workspace_bytes                 */
} lf_params;

typedef struct {
    int64_t step;         /* steps taken since lf_create / the loaded checkpoint  */
    double  mass;         /* sum n                        (FP64 reduction)        */
    double  phi_sum;      /* sum phi                                              */
    double  mom[3];       /* sum n u                                              */
    double  umax;         /* max |u|                                              */
    double  mach;         /* umax / c_s (Sec. 2: must stay < 0.1)                 */
    double  free_energy;  /* phi part of Eq. fren on the lattice: sum a phi^2/2 +
                             b phi^4/4 + c (lap phi)^2/2 (5-/7-point lap) plus
                             kappa/2 sum over nearest-neighbour links inside the
                             lattice of (dphi)^2; its phi-derivative is mu of
                             Eq. chem with the compact stencils                */
    double  grad2[3];     /* sum (d_x phi)^2, (d_y phi)^2, (d_z phi)^2 (central)  */
    double  orient_s;     /* (d <(d_perp phi)^2>/<|grad phi|^2> - 1)/(d - 1)      */
    double  k_peak;       /* first moment of S(k) over shells above S_peak / 2    */
    double  s_peak;       /* largest shell average of S(k)                        */
    int     nonfinite;    /* 1 if a NaN/Inf was seen since creation               */
    int     pad_;
} lf_diag_t;

typedef struct lf_ctx lf_ctx;

/* ---- lattice ----------------------------------------------------------- */
/* Velocity set of the library: fills e[Q*3] (integer components, z = 0 in 2D)
 * and w[Q] when non-NULL and returns Q (9 for d = 2, 19 for d = 3), or
 * LF_EINVAL.  Populations in LF_FIELD_POP follow this order.  Sec. 2, text
 * around Eqs. evoleqn and latticeforceterm (moduli 0, c, sqrt(2) c; weights
 * 4/9, 1/9, 1/36 in 2D; 1/3, 1/18, 1/36 for D3Q19). */
int lf_lattice(int d, int* e, double* w);

/* Number of explicit temperature sub-steps per step for this xi and d: the
 * smallest n with xi/n <= 0.8/(2d) (1 for xi = 0 or +INFINITY). */
int lf_nsub(double xi, int d);

/* Bytes of device memory one context needs for its state (both ping-pong
 * copies of f, phi, T, the aux fields and the reduction scratch). */
int lf_workspace_bytes(const lf_grid* grid, const lf_walls* walls,
                       const lf_params* params, size_t* bytes);

/* ---- life cycle -------------------------------------------------------- */
/* Validates the arguments (LF_EINVAL), the stability of the explicit schemes
 * (LF_EUNSTABLE: tau <= 1/2 with hydro, or Gamma lam (a + kappa lam + c lam^2)
 * >= 2 for some Laplacian eigenvalue lam of the chosen stencils at the
 * largest a in the run), places
 * the state in params->workspace (if given; LF_ENOMEM if too small) or in its
 * own device allocation, and enqueues the initial state: phi from SplitMix64,
 * T = T0 (T_w on the wall layers; T_w everywhere for xi = +INFINITY),
 * f_i = w_i n0 (u = 0).  *out receives the context (NULL on failure). */
int lf_create(const lf_grid* grid, const lf_walls* walls, const lf_params* params,
              lf_ctx** out);

/* Enqueues nsteps time steps on the context's stream and returns without
 * waiting.  Returns LF_ENONFINITE if an earlier, completed step saw a NaN/Inf,
 * LF_ECUDA if a launch failed (including errors of earlier async work). */
int lf_step(lf_ctx* ctx, int64_t nsteps);

/* Copies one field of the state at the current step into dst.  `bytes`
 * selects the element type: N*8 (or Q*N*8 for LF_FIELD_POP) gives double,
 * N*4 (Q*N*4) gives float; anything else is LF_EINVAL.  dst_on_device says
 * whether dst is a device or a host pointer.  Derived fields (RHO, U*, MU,
 * F*) are computed from the current state by the same device code the step
 * uses.  Waits for completion.  Copies whatever the state holds: a NaN/Inf
 * is reported by lf_step and lf_diag, not here. */
int lf_fields(lf_ctx* ctx, int which, void* dst, size_t bytes, int dst_on_device);

/* Overwrites PHI, T or POP (full f_i) of the current state from src, with the
 * same size/type rule as lf_fields.  Used for tests, restarts and fault
 * injection.  Waits for completion. */
int lf_fields_set(lf_ctx* ctx, int which, const void* src, size_t bytes, int src_on_device);

/* Diagnostics of the current state (FP64 reductions on the GPU, S(k) by an
 * FP64 FFT on the GPU).  Waits, bounded.  Returns LF_ENONFINITE (and fills
 * out) when a NaN/Inf is present. */
int lf_diag(lf_ctx* ctx, lf_diag_t* out);

/* Per-layer orientation s(h) along the wall normal, h = 0 .. L-1, into the
 * host array out[L] (L = ny in 2D, nz in 3D). */
int lf_diag_layers(lf_ctx* ctx, double* out, int64_t L);

/* Shell-averaged structure factor S_b, b = 0 .. nb-1, into host out[nb]
 * (nb = min lattice size / 2 + 1; S_0 = 0). */
int lf_structure_factor(lf_ctx* ctx, double* out, int64_t nb);

/* Diagnostics sums without any allocation.  The paper has no counterpart:
 * this serves callers that cannot allocate device memory at the point of the
 * call -- inside CUDA graph capture, in a loop that must not stall on
 * cudaMalloc's implicit device synchronisation, or in a host framework that
 * owns all device memory.  It computes what lf_diag and lf_diag_layers
 * report, from fields the caller holds on the device:
 *   phi, T:   [nz][ny][nx] (unpadded, nz = 1 in 2D) of double (LF_FP64) or
 *             float (LF_FP32);
 *   moments:  [4][nz][ny][nx] of the same type: n, ux, uy, uz (uz zero in 2D),
 *             e.g. from lf_fields(LF_FIELD_RHO / UX / UY / UZ);
 *   out:      device array of 10 + L doubles (L = ny in 2D, nz in 3D):
 *             out[0..9] = sum n, sum phi, sum n ux, sum n uy, sum n uz,
 *             sum (d_x phi)^2, sum (d_y phi)^2, sum (d_z phi)^2, free energy
 *             (phi part), max |u|^2; out[10 + h] = orientation s of layer h.
 * Work is enqueued on `stream` (cudaStream_t) and the call returns without
 * waiting; nothing is allocated and no CUDA allocation routine is called.
 * Scratch: a fixed device array of 162,816 bytes in this library (1216 x 10
 * partial sums and 2 x 4096 layer sums), present on every GPU that loads
 * the library until the process exits; an extent above 2^24, L above 4096,
 * or 2^31 or more sites is rejected with LF_EINVAL.  The first call on a
 * device resolves that array's device address (cudaGetSymbolAddress) and
 * keeps it for the life of the process; make it before any stream capture,
 * and do not use this call after the device's primary context has been
 * reset (cudaDeviceReset), which leaves the kept address stale.  Each device
 * has its own copy of the array, and all calls on one device share it: calls
 * on the same device whose work overlaps on the GPU (for instance on two
 * streams) race and corrupt each other's partial sums -- serialise them.
 * No state carries over between calls (every partial read is written by the
 * same call). */
int lf_diag_sums_noalloc(int d, int64_t nx, int64_t ny, int64_t nz, int walls, int precision,
                         const void* phi, const void* T, const void* moments, double b, double kappa,
                         double c, double Tc, double* out, void* stream);

/* Checkpoint: writes / reads grid, walls, params (except pointers), the
 * stencil and temperature solver in use, step and the full state in the
 * context's precision.  lf_load requires a context with the same grid, walls,
 * precision, stencil (lf_set_stencil) and temperature solver
 * (lf_set_t_solver), and returns LF_EIO otherwise, so that a resumed run
 * cannot continue with another scheme; set those before loading. */
int lf_save(lf_ctx* ctx, const char* path);
int lf_load(lf_ctx* ctx, const char* path);

/* Kernel variant of the step.  All compute the same step (parity-tested
 * against the oracle); they differ in how work is mapped to the GPU:
 *   LF_VARIANT_MARCH (default for 2D FP64): one thread per column, a CTA
 *     marches down a segment of (param & 0xFFFF) rows (0 = chosen from the
 *     lattice size), inputs prefetched with cp.async; (param >> 16) == 1
 *     selects CTAs of 64 threads (56 columns) instead of 128 (120 columns);
 *     with the isotropic stencils this one-lane march runs with sliding row
 *     sums;
 *   LF_VARIANT_TILE: one CTA per 2D tile, each stage of the step on the whole
 *     tile in shared memory (`param` ignored);
 *   LF_VARIANT_MARCH2 (default for 2D FP32; FP64 contexts run LF_VARIANT_MARCH
 *     instead): a CTA owns two vertically adjacent segments of a strip that
 *     march away from their common row, carried in the two lanes of packed
 *     FP32x2 arithmetic; (param & 0xFFFF) = rows per segment (0 = chosen from
 *     the lattice size and the SM count), (param >> 16) == 1 selects CTAs of
 *     64 threads (56 columns) instead of 128 (120 columns); with the
 *     isotropic stencils the two segments are the lower and upper halves of a
 *     pair, both marching upwards, with sliding row sums;
 *   LF_VARIANT_SPLIT3 (3D default): three passes per step -- mu and F by a
 *     plane march ((param & 0xFFFF) = planes per segment, 0 = automatic),
 *     then collision and streaming, then the phi and T updates by a column
 *     march over (param >> 20) & 255 planes per segment (0 = 16); mu, F and
 *     u pass through the context's derived-field planes.  (param >> 16) & 15
 *     selects the force pass's form: with the compact stencils, in FP32, 0 =
 *     two segments in the lanes of packed FP32x2 arithmetic, 1 / 2 = one lane
 *     on 60x4 / 28x12 tiles; with the isotropic stencils (both passes as
 *     column marches with sliding plane sums), 0 = one lane on 28x12 tiles
 *     (FP32: two CTAs per SM), 1 = on 28x28 tiles, 3 = on 28x12 tiles at one
 *     CTA per SM, 4 = two segments in packed FP32x2 lanes (1, 3 and 4 in FP32
 *     only; FP64 takes 0); with the isotropic stencils bit 28 selects the
 *     phi pass that stages its raw fields by cp.async.  For 3D contexts every
 *     other variant runs the fused plane march (param = planes per segment).
 * Returns LF_EINVAL for an unknown variant or a negative param. */
#define LF_VARIANT_MARCH  0
#define LF_VARIANT_TILE   1
#define LF_VARIANT_MARCH2 2
#define LF_VARIANT_SPLIT3 3
int lf_set_kernel_variant(lf_ctx* ctx, int variant, int param);

/* Autotuner of the step's mapping to the GPU.  Times every candidate kernel
 * variant and shape for this lattice -- 2D: CTA width (120 or 56 columns) and
 * rows per segment of the row marches, and the tile kernel; 3D: tile shape and
 * planes per segment of the three-pass step's force pass, and the fused plane
 * march -- `reps` timed steps each (CUDA events) on a scratch context of the
 * same lattice, stencil, precision, parameters and temperature solver, each
 * candidate from the same initial state, and sets the fastest on ctx as by
 * lf_set_kernel_variant.  ctx's state is not touched.  The choice is cached per
 * (device, lattice sizes, precision, stencil, walls, hydrodynamics) for the
 * life of the process, so later calls with the same key only set it.  The
 * scratch context allocates as much device memory as ctx, plus one copy of
 * its state, for the duration of the call; it waits for ctx's stream.  Any of
 * variant, param, ms_per_step may be NULL; on success they receive the choice
 * and its time per step in milliseconds.  For the isotropic 2D step the
 * candidates are the two-lane (FP32) and one-lane row marches and the tile
 * kernel.  Returns LF_EINVAL
 * for reps < 1 or an ensemble member. */
int lf_tune(lf_ctx* ctx, int reps, int* variant, int* param, double* ms_per_step);

/* Time discretisation of the temperature (d_t T = xi lap T, Sec. 2 after Eq.
 * massdiff):
 *   LF_TSOLVER_EXPLICIT (default): explicit Euler in n_sub = lf_nsub(xi, d)
 *     sub-steps of xi / n_sub, the first fused into the step kernel;
 *   LF_TSOLVER_IMPLICIT: one backward-Euler step (I - xi L) T(t+1) = T(t) per
 *     time step with the same Laplacian L and wall rules, solved by an FP64
 *     DFT along the periodic axes and a tridiagonal solve along the wall
 *     normal (a division when every axis is periodic).  Unconditionally
 *     stable: one solve per step at any xi.  Needs the periodic lattice sizes
 *     to be at most 4096 with prime factors up to 31.
 * The phi, f update always uses T(t).  With walls, switching to the implicit
 * solver allocates 16 bytes per site of device memory for the tridiagonal
 * coefficients (c' and the reciprocal pivots of every Fourier mode, rebuilt
 * when xi, the wall rule or the stencil change; freed by lf_destroy).
 * Returns LF_EINVAL for an unknown solver, an unsupported size, or an
 * ensemble member (ensembles always take explicit sub-steps), LF_ENOMEM if
 * the coefficient tables cannot be allocated.  Not stored in checkpoints. */
#define LF_TSOLVER_EXPLICIT 0
#define LF_TSOLVER_IMPLICIT 1
int lf_set_t_solver(lf_ctx* ctx, int solver);

/* Finite-difference stencils of every derivative of the step (Sec. 2 names a
 * "second-order finite-difference scheme" without fixing it); chosen at
 * lf_create by params->stencil, or changed later by lf_set_stencil:
 *   LF_STENCIL_COMPACT (default): 5-point (2D) / 7-point (3D) Laplacian and
 *     central first differences along the axes;
 *   LF_STENCIL_ISOTROPIC: the operators built from the lattice weights,
 *     d_a A = 3 sum_i w_i e_ia A(r + e_i) and lap A = 6 sum_i w_i [A(r + e_i) -
 *     A(r)] (D2Q9: the 9-point Laplacian [4 (nearest) + (diagonal) - 20 A]/6),
 *     second order with an isotropic leading error (Thampi et al., J. Comput.
 *     Phys. 234 (2013) 1).  Applies to psi, lam, grad phi, grad psi, F, the
 *     flux divergence, lap mu and lap T; the wall images are those of the
 *     compact stencils, applied to the diagonal neighbours too.  In 2D the
 *     march variants run a row march whose 9-point operators are split into
 *     sliding row sums, LF_VARIANT_TILE the tile kernel; in 3D the variant
 *     set (three passes by default, or the fused plane march).  Its
 *     largest Laplacian eigenvalue is 16/3 in 2D and 3D (8 and 12 for the
 *     compact stencils), which the stability check of lf_create uses.
 * Returns LF_EINVAL for an unknown stencil or an ensemble member (an
 * ensemble's runs take their stencil from params at lf_ens_create), and
 * LF_EUNSTABLE if the context's parameters are unstable with the new stencil
 * (the context keeps its stencil then).  lf_load refuses a checkpoint
 * written with another stencil. */
#define LF_STENCIL_COMPACT   0
#define LF_STENCIL_ISOTROPIC 1
int lf_set_stencil(lf_ctx* ctx, int stencil);

/* Current step counter. */
int64_t lf_step_count(const lf_ctx* ctx);

/* Timing of the passes of the three-pass 3D step (LF_VARIANT_SPLIT3, Sec. 2:
 * pass A mu and F, Eqs. chem and ff; pass B collision and streaming, Eqs.
 * moment, evoleqn, latticeforceterm; pass C phi(t+1), Eq. massdiff, and the
 * first temperature sub-step).  With enable != 0, every later lf_step of such
 * a context records CUDA events on its stream before pass A and after each
 * pass (it creates four events on the first call; lf_destroy releases them).
 * lf_pass_times waits for the context's stream and writes the durations in
 * milliseconds of the passes of the last step taken, in launch order, into
 * ms[0 .. min(n, 3) - 1], and their count into *npasses (may be NULL): 3, or
 * 0 when that step recorded none (timing off, 2D, another variant).  Further
 * temperature sub-steps are not part of the passes.  LF_EINVAL for a NULL
 * context, an ensemble member, n < 0 or ms NULL with n > 0; the bounded
 * stream wait's LF_ETIMEOUT / LF_ECUDA. */
int lf_set_pass_timing(lf_ctx* ctx, int enable);
int lf_pass_times(lf_ctx* ctx, float* ms, int n, int* npasses);

/* Frees the context's own allocations (not a caller workspace).  NULL is a no-op. */
void lf_destroy(lf_ctx* ctx);

const char* lf_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* LF_H */
