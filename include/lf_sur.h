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

/* ---- building blocks (used by the trainer; exposed for verification) ---- */

/* One 3x3 convolution on the tensor cores, (cin, cout) in {(16, 64), (64, 64),
 * (64, 16)}, NX a multiple of 128.  Per output pixel and channel:
 *   v = sum over taps and cin + bias;  zout = v;  v = relu(v) if relu;
 *   v += resid;  out = v;  out2 = v * (mask > 0);
 *   y4[0..3] = x4[0..3] + (sum + bias)[0..3]  (FP32, unpadded [B][NY][NX][4]).
 * Every non-null BF16 output is written in the padded layout, halo included.
 * err (device int) is set to 1 if a bounded wait inside the kernel gave up.
 * Enqueued on stream; pointers 16-byte aligned. */
int lf_sur_conv3x3(int B, int NY, int NX, int cin, int cout, const void* in, const void* w,
                   const float* bias, int relu, const void* resid, const void* mask, void* out,
                   void* out2, void* zout, const float* x4, float* y4, int* err, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LF_SUR_H */
