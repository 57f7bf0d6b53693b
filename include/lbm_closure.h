/*
 * lbm_closure.h -- learned closure for the D3Q27 cumulant step of
 * liblbm.so: a per-cell MLP, fused into the stream + collide kernel, that
 * sets the free relaxation rates of the cumulants of orders 3, 4, 5 and 6
 * (the rates the paper's regularised methods fix at 1, Sec. 4.2), and the
 * trainer that fits it on the GPU.  This part is not in the paper.
 *
 * Inputs of the network, per cell, from the pre-collision populations:
 * with Pi = kappa_2 / rho - I/3 (normalised second-order central moments,
 * Sec. 2.3.2), S = -(3 omega_shear / 2) Pi (the non-equilibrium estimate of
 * the strain rate) and D = Pi - tr(Pi)/3 I,
 *   raw = {tr S, I2(S)/|S|, det S/|S|^2, I2(D)/|D|, det D/|D|^2, |Pi|, rho - 1},
 *   I2(A) = ((tr A)^2 - tr(A A)) / 2, |.| the Frobenius norm,
 * each quotient 0 where its norm is 0: the principal invariants, divided by
 * powers of the norm so that every input but the density is of degree 1 in
 * Pi (same scale for all, Lipschitz, no amplified rounding near zero);
 * normalised x_i = (raw_i - shift_i) * scale_i.  Network:
 *   h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), z = W3 h2 + b3,
 *   omega_{3..6} = clamp(2 sigmoid(z), 1e-3, 1.999);
 * with any normalised input non-finite or outside FP16's range
 * (|x_i| > 65504), or any non-finite output, all four rates fall back to 1
 * (the plain regularised cumulant method).  Weights are BF16 numbers; FP64
 * lattices apply them in FP64, FP32 lattices on the tensor cores as FP16
 * operands (exact for BF16 values of magnitude 2^-17 .. 65504) with the
 * activations split into two FP16 parts and FP32 accumulation.
 *
 * Parameter vector layout (LBM_CLOSURE_NPARAM values): W1[32][7], b1[32],
 * W2[32][32], b2[32], W3[4][32], b3[4], row-major.
 *
 * Training target: with snapshots f_c(s) of a coarse lattice (typically the
 * 4^3 block average of a fine run, one snapshot every 4 fine steps), the
 * loss of window s with unroll K is
 *   L = (1/K) sum_{k=1..K} mean over cells of |u(step_theta^k(f_c(s))) - u(f_c(s+k))|^2,
 * K coarse steps with the network's rates from snapshot s (K = 1: one-step
 * teacher forcing).  Its gradient is computed by hand-written kernels,
 * backwards through the K steps: the adjoint of streaming and of the
 * velocity, tangents of the post-collision populations with respect to the
 * four rates, the network's backward pass (weights and inputs), and the
 * transposed per-cell Jacobian of the collision (27 forward-mode dual-number
 * passes per cell) that carries dL/df to the step before; weight gradients
 * are reduced per block and folded in a fixed order.  Adam updates FP32
 * master weights; the forward uses their BF16 rounding.
 */
#ifndef LBM_CLOSURE_H
#define LBM_CLOSURE_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_CLOSURE_NIN 7
#define LBM_CLOSURE_NHIDDEN 32
#define LBM_CLOSURE_NOUT 4
#define LBM_CLOSURE_NPARAM 1444
#define LBM_CLOSURE_MAX_UNROLL 64

typedef struct {
  float shift[LBM_CLOSURE_NIN];
  float scale[LBM_CLOSURE_NIN];
  uint16_t w[LBM_CLOSURE_NPARAM]; /* BF16 bit patterns, layout above */
} lbm_closure_weights;

/* Enable (w != NULL) or disable (NULL) the learned rates on a context.
 * Served for D3Q27 cumulant contexts with pull streaming and FP32 or FP64
 * storage (others: LBM_ERR_UNSUPPORTED).  While enabled, lbm_step runs the
 * fused kernel; the context's rates for orders 3..6 are ignored.  The
 * weights are copied to the device.  Errors: INVALID (also a weight that is
 * not finite or of magnitude above 65504), UNSUPPORTED, OOM, CUDA. */
int lbm_set_closure(lbm_ctx* ctx, const lbm_closure_weights* w);

typedef struct lbm_trainer lbm_trainer;

/* Trainer for a coarse lattice of coarse_dims (each >= 1, product < 2^31)
 * with the given shear and bulk rates, holding at most max_snapshots
 * snapshots (27 * N FP32 values each; at least 2, a training pair).  Parameters start at zero (rates 1,
 * the plain method), shift 0, scale 1.  Errors: INVALID, OOM, CUDA. */
int lbm_trainer_create(lbm_trainer** out, const int64_t coarse_dims[3],
                       double omega_shear, double omega_bulk,
                       int max_snapshots, void* stream);

/* Append a snapshot: the 4^3 block average of the canonical populations of
 * a D3Q27 context whose dims are 4 x coarse_dims (any zero-centered
 * storage, pull or AA streaming; the esoteric patterns -> UNSUPPORTED). */
int lbm_trainer_add_restricted(lbm_trainer* t, lbm_ctx* fine);

/* Append a snapshot given as canonical FP64 populations df[27 * N]. */
int lbm_trainer_add_snapshot(lbm_trainer* t, const double* df, int on_device);

int lbm_trainer_snapshot_count(const lbm_trainer* t);
int lbm_trainer_get_snapshot(lbm_trainer* t, int s, double* df, int on_device);

/* Raw (unnormalised) network inputs of snapshot s, feat[7 * N] FP64. */
int lbm_trainer_features(lbm_trainer* t, int s, double* feat, int on_device);

/* Set the FP32 master parameters and the input normalisation; resets the
 * Adam moments and step counter. */
int lbm_trainer_set_params(lbm_trainer* t, const float* params,
                           const float shift[7], const float scale[7]);
int lbm_trainer_get_params(lbm_trainer* t, float* params);

/* Steps K of the rollout loss (1 <= K <= LBM_CLOSURE_MAX_UNROLL, K + 1 <=
 * max_snapshots; 1 at creation).  Allocates K post-collision fields and,
 * for K > 1, two adjoint fields (27 N FP32 each).  Errors: INVALID, OOM (the
 * previous K stays). */
int lbm_trainer_set_unroll(lbm_trainer* t, int K);

/* Loss of the window s .. s+K (snapshots s+1 .. s+K the targets; s + K <
 * count) and its gradient with respect to the parameters
 * (grad[LBM_CLOSURE_NPARAM] FP64 host, or NULL).  Synchronises. */
int lbm_trainer_loss_grad(lbm_trainer* t, int s, double* loss, double* grad);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on window s with
 * learning rate lr; returns the loss before the update.  Synchronises. */
int lbm_trainer_adam_step(lbm_trainer* t, int s, double lr, double* loss);

/* The current weights in inference form (BF16 bits + normalisation). */
int lbm_trainer_export(lbm_trainer* t, lbm_closure_weights* out);

void lbm_trainer_destroy(lbm_trainer* t);

#ifdef __cplusplus
}
#endif
#endif /* LBM_CLOSURE_H */
