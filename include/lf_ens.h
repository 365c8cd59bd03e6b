/*
 * lf_ens.h -- batched ensembles of independent 2D runs of the hybrid
 * LB/FD step of arXiv:1102.3094 (Sec. 2) in one launch per time step.
 *
 * The paper itself runs one lattice at a time; an ensemble advances many
 * independent lattices of uneven sizes and parameters (xi, tau, seed, ...)
 * together.  Each run is an ordinary lf_ctx (so lf_fields, lf_fields_set,
 * lf_diag, lf_save and lf_load work on it) whose steps are taken by the
 * ensemble: one persistent kernel per time step walks a work list of
 * (run, strip, segment pair) items, and the steps are replayed from a CUDA
 * graph.  Results are bit-identical to stepping every run alone with lf_step
 * under LF_VARIANT_MARCH2 with param = lf_ens_param(e, r) (the per-site
 * arithmetic is the same code and the rows are split the same way).  Runs
 * created with params.stencil = LF_STENCIL_ISOTROPIC are (run, strip, segment
 * pair) items of a second persistent kernel, the two-lane isotropic march a
 * single isotropic FP32 run takes under LF_VARIANT_MARCH2, and are
 * bit-identical to that run stepped alone with the same param.
 *
 * Restrictions: every run is two-dimensional (d = 2), LF_FP32, ny >= 2.
 * Conventions (return codes, layouts, ownership) are those of lf.h.
 */
#ifndef LF_ENS_H
#define LF_ENS_H

#include "lf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lf_ens lf_ens;

/* Creates nruns contexts, run r from grids[r], walls[r], params[r] (the
 * stream, workspace and workspace_bytes fields of params are ignored), all in
 * one device arena, enqueued on `stream` (a cudaStream_t; 0 = a private
 * stream the ensemble creates).  LF_EINVAL if a run is not d = 2 / LF_FP32 /
 * ny >= 2 or fails lf_create's checks (then nothing is allocated).  Runs of
 * either stencil may be mixed. */
int lf_ens_create(int nruns, const lf_grid* grids, const lf_walls* walls, const lf_params* params,
                  void* stream, lf_ens** out);

/* Autotuner: for every distinct (lattice size, stencil) class of the runs in turn,
 * times the whole batch -- a scratch ensemble of the same runs, which holds
 * as much device memory as this one for the duration of the call -- with that
 * size's runs set to every CTA width (64 threads = 56-column strips, 128
 * threads = 120-column strips) and segment height (1 .. 128 rows, at most
 * ny / 2), reps timed steps each (CUDA events), and keeps the shape of the
 * fastest batch.  The objective is the ensemble's throughput, not one run's
 * latency.  The runs' states are not touched.  Rebuilds the work lists and
 * the graphs. */
int lf_ens_tune(lf_ens* e, int reps);

/* Rows per segment the work list uses for run r (after tuning, or the
 * default min(16, ny / 2)). */
int lf_ens_rows(const lf_ens* e, int run);

/* The LF_VARIANT_MARCH2 param of run r's shape: (1 << 16 for 64-thread CTAs,
 * 0 for 128) | rows per segment; lf_step of a single context with this param
 * reproduces the run bit for bit.  Default: 64-thread CTAs. */
int lf_ens_param(const lf_ens* e, int run);

/* Enqueues nsteps steps of every run on the ensemble's stream (graph
 * replays) and returns without waiting. */
int lf_ens_step(lf_ens* e, int64_t nsteps);

/* Retires every run whose state went non-finite (the flag lf_diag reports
 * as `nonfinite`; set by the step kernels): its work items leave the work
 * lists, so later steps cost nothing for it, and its state and step count
 * stay as they were when it was retired (a run may have taken a few steps
 * past its first NaN before the call).  Waits for the stream; rebuilds the
 * work lists and graphs when a run was retired.  nactive (may be NULL)
 * receives the number of runs still stepped. */
int lf_ens_prune(lf_ens* e, int* nactive);

/* 1 while run r is stepped, 0 after lf_ens_prune retired it. */
int lf_ens_active(const lf_ens* e, int run);

/* Borrowed context of run r (valid until lf_ens_destroy).  lf_step on it
 * returns LF_EINVAL: only the ensemble advances its runs. */
int lf_ens_run(lf_ens* e, int run, lf_ctx** ctx);

/* Waits (bounded) for the ensemble's stream. */
int lf_ens_sync(lf_ens* e);

void lf_ens_destroy(lf_ens* e);

#ifdef __cplusplus
}
#endif

#endif /* LF_ENS_H */
