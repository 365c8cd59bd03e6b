/*
 * lf_sur.h -- a learned surrogate for the hybrid LB/FD step of arXiv:1102.3094
 * (Sec. 2): a small residual convolutional network that advances the 2D state
 * (phi, T, ux, uy) by K time steps at once, trained on trajectories of the
 * plain method, run interleaved with plain steps, and checked against the
 * plain method (which takes over whenever the surrogate's error is too large).
 *
 * The paper has no surrogate; this is an addition on top of its method.
 *
 * Network (layers 1..6, 3x3 convolutions, BF16 weights and activations, FP32
 * accumulation on the tensor cores):
 *   x  = normalised state, 4 channels padded to 16 with zeros
 *   h1 = relu(conv(x) + b1)                       16 -> 64
 *   h_{l+1} = h_l + relu(conv(h_l) + b_l)         64 -> 64, l = 2..5
 *   y  = x[0..3] + (conv(h6) + b6)[0..3]          64 -> 16 (4 used)
 * Padding follows the lattice: periodic in x, zero beyond the walls in y.
 *
 * Activation layout ("padded NHWC"): BF16 [B][NY + 2][NX + 2][C] with a
 * one-pixel halo; halo columns 0 and NX + 1 hold copies of columns NX - 1 and
 * 0, halo rows 0 and NY + 1 are zero.  Weights: BF16 [9][COUT][CIN], tap
 * t = 3 (dy + 1) + (dx + 1) multiplies the input at (y + dy, x + dx).
 * Conventions (return codes, device pointers, streams) are those of lf.h.
 */
#ifndef LF_SUR_H
#define LF_SUR_H

#include "lf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lf_sur lf_sur;

/* Per-channel normalisation of (phi, T, ux, uy): network input and target are
 * (field - offset) / scale. */
typedef struct {
    double scale[4];
    double offset[4];
} lf_sur_norm;

typedef struct {
    int    windows_done;      /* windows completed (surrogate and plain)              */
    int    surrogate_windows; /* surrogate windows whose prediction was kept          */
    int    shadow_checks;     /* surrogate windows checked by a plain shadow window   */
    int    fallbacks;         /* checked windows replaced by the plain result         */
    double max_phi_l2_err;    /* largest ||phi_sur - phi_plain|| / ||phi_plain||     */
    double max_sk_err;        /* largest relative error of S(k) peak position/height  */
    double last_err;          /* error of the last checked window                     */
    double t_surrogate_s;     /* device time in surrogate predictions                 */
    double t_shadow_s;        /* device time in shadow windows and comparisons        */
    double t_plain_s;         /* device time in plain windows                         */
    int    rejected;          /* predictions not finite or with |u| > 0.2: plain window taken instead */
} lf_sur_report;

/* ---- network ------------------------------------------------------------- */

/* Creates the network for NY x NX lattices (NX a multiple of 128) and batches
 * of up to max_batch states, weights drawn (He-uniform, last layer x 0.1)
 * from SplitMix64(seed), Adam state zero.  Allocates its device memory once. */
int lf_sur_create(int NY, int NX, int max_batch, uint64_t seed, const lf_sur_norm* norm, void* stream,
                  lf_sur** out);

/* Number of FP32 parameters (per layer: weights [9][cout][cin], then bias [cout]). */
size_t lf_sur_param_count(void);

/* Master (FP32) parameters to / from host memory, layer by layer in the
 * order of lf_sur_param_count; set also refreshes the BF16 copies. */
int lf_sur_get_params(lf_sur* s, float* host);
int lf_sur_set_params(lf_sur* s, const float* host);

/* Loss of a batch: x, y raw states [B][4][NY][NX] FP32 on the device (y the
 * target K steps later); loss = mean over B NY NX 4 of (net(x) - y)^2 in
 * normalised units.  With grads_host non-NULL also the gradient of the loss
 * with respect to every parameter (same order as the parameters).  Waits. */
int lf_sur_grads(lf_sur* s, const float* x, const float* y, int B, double* loss, float* grads_host);

/* One training step: loss, gradients (tensor cores), Adam (lr, 0.9, 0.999)
 * on the gradients scaled by min(1, max_norm / ||g||) with ||g|| the global
 * norm over all parameters (lf_sur_set_clip; 1.0 after lf_sur_create). */
int lf_sur_train_step(lf_sur* s, const float* x, const float* y, int B, float lr, double* loss);

/* Global-norm gradient clipping threshold of lf_sur_train_step (0 = none). */
int lf_sur_set_clip(lf_sur* s, float max_norm);

/* y = net(x) in raw units, [B][4][NY][NX] FP32 device arrays; enqueued. */
int lf_sur_predict(lf_sur* s, const float* x, float* y, int B);

/* Runs nwindows windows of K steps on ctx (2D, LF_FP32, hydrodynamics on,
 * NY x NX): even windows by the surrogate, odd windows by lf_step.  Every
 * shadow_every-th surrogate window is also advanced by the plain method from
 * the same state; if max(phi relative L2 error, relative error of the S(k)
 * peak position or height) exceeds threshold, the plain result replaces the
 * prediction.  A prediction with a non-finite value or |u| > 0.2 is never
 * handed over: that window is advanced by lf_step instead (rep->rejected).
 * Kept predictions set phi and T and move the equilibrium part of the
 * populations from the current to the predicted velocity at the current
 * density (the non-equilibrium part is kept).  Waits; fills *rep. */
int lf_sur_run(lf_sur* s, lf_ctx* ctx, int K, int nwindows, int shadow_every, double threshold,
               lf_sur_report* rep);

void lf_sur_destroy(lf_sur* s);

/* ---- building blocks (used by the trainer; exposed for verification) ---- */

/* One 3x3 convolution on the tensor cores, (cin, cout) in {(16, 64), (64, 64),
 * (64, 16)}, NX a multiple of 128.  Per output pixel and channel:
 *   v = sum over taps and cin + bias;  zout = v;  v = relu(v) if relu;
 *   v += resid;  out = v;  out2 = v * (mask > 0);
 *   y4[0..3] = x4[0..3] + (sum + bias)[0..3]  (FP32, unpadded [B][NY][NX][4]).
 * Every non-null BF16 output is written in the padded layout, halo included.
 * The outputs must not overlap the inputs (other CTAs still read rows that a
 * CTA writes).  resid may be the input itself (resid == in, cin == cout):
 * it is then read from the input rows the kernel already holds in shared
 * memory.  The input rows and the weights are read by TMA (tensor maps
 * encoded per call through the driver's cuTensorMapEncodeTiled; LF_ECUDA if
 * the driver lacks it).  err (device int) is set to 1 if a bounded wait
 * inside the kernel gave up or the shared-memory window is not aligned for
 * the swizzled layouts.  Enqueued on stream; pointers 16-byte aligned. */
int lf_sur_conv3x3(int B, int NY, int NX, int cin, int cout, const void* in, const void* w,
                   const float* bias, int relu, const void* resid, const void* mask, void* out,
                   void* out2, void* zout, const float* x4, float* y4, int* err, void* stream);

/* Weight gradient of one such convolution: dW[t][o][i] = sum over pixels p of
 * h[p + off_t][i] g[p][o] (FP32 [9][cout][cin]), h in the padded NHWC layout
 * with cin channels, g with cout channels (halo of g unused).  `part` is FP32
 * device scratch of at least lf_sur_wgrad_scratch_floats(cin, cout) floats
 * for the per-CTA partial sums (tensor cores), reduced in a second kernel.
 * For (64, 64) the rows of h and g are read by TMA (as above). */
int lf_sur_conv3x3_wgrad(int B, int NY, int NX, int cin, int cout, const void* h, const void* g,
                         float* part, size_t part_floats, float* dW, int* err, void* stream);
size_t lf_sur_wgrad_scratch_floats(int cin, int cout);

#ifdef __cplusplus
}
#endif

#endif /* LF_SUR_H */
