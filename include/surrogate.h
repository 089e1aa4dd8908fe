/*
 * surrogate.h -- C ABI of the learned r-cell stress surrogate (GB300).
 *
 * The paper has no learned component: every quadrature point runs MD
 * (Sec. 2.1, Fig. 1).  This surrogate replaces the r-cell MD of a quadrature
 * point by a recurrent MLP that maps the strain-increment history to the stress,
 * with plain r-cell MD as the fallback whenever the ensemble disagrees.
 *
 * Architecture per time step (all members identical, weights differ):
 *   z_t = [u_t / u_scale (15), h_{t-1} (128), 0]                 (144)
 *   a_1 = gelu(z_t W1 + b1), a_2 = gelu(a_1 W2 + b2), a_3 = gelu(a_2 W3 + b3)   (256 each)
 *   o_t = a_3 W4 + b4 (144):  s_t = o_t[0:6] * s_scale,  h_t = tanh(o_t[6:134])
 * with u_t = (Delta F_t row-major (9), Green strain E_t = (F^T F - I)/2 in
 * Voigt order xx yy zz xy xz yz (6)), h_0 = 0, gelu(x) = x/2 (1 + erf(x/sqrt 2)).
 * Parameters: one flat FP32 vector per member, order W1 b1 W2 b2 W3 b3 W4 b4,
 * weights row-major K x N (SUR_N_PARAMS floats).
 * Precision: BF16 weights and activations on tensor cores with FP32
 * accumulation; FP32 master weights, biases, AdamW moments, losses.
 * Training loss: mean over (batch, time, 6) of (s_t / s_scale - y_t / s_scale)^2.
 *
 * Conventions as in rcell.h: rc_status return codes, device pointers unless
 * stated, work enqueued on the stream given at creation.
 */
#ifndef SURROGATE_H
#define SURROGATE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SUR_N_IN 15
#define SUR_N_H 128
#define SUR_N_OUT 6
#define SUR_WIDTH 256
#define SUR_N_PARAMS (144 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 144 + 144)

typedef struct sur_ctx sur_ctx;

/* Create n_members networks (seeded init: uniform +-1/sqrt(fan_in) weights,
 * zero biases, member m seeded with seed + m), with work buffers for up to
 * max_batch sequences of up to max_steps increments.  The BPTT buffers are
 * held once per member (about 5.2 KB per sequence-increment and member:
 * inputs, pre-activations, activations and their gradients in BF16), so that
 * the members train side by side.  u_scale = 1, s_scale = 1.  Synchronous.
 * Errors: RC_EINVAL, RC_ENOMEM, RC_ECUDA. */
int sur_create(int n_members, int max_batch, int max_steps, uint64_t seed, void *stream, sur_ctx **out);

/* Feature and stress scales (host, 15 and 6 floats, all > 0). */
int sur_set_scaling(sur_ctx *s, const float *u_scale, const float *s_scale);

/* Copy one member's parameters to / from host memory (SUR_N_PARAMS floats).
 * Setting parameters also resets that member's AdamW moments and step count.
 * Synchronous. */
int sur_get_params(sur_ctx *s, int member, float *theta);
int sur_set_params(sur_ctx *s, int member, const float *theta);

/* Loss and gradient of one member on a batch, no update.  U: B x T x 15,
 * Y: B x T x 6 (device, FP32, raw units).  loss (host, may be NULL) and grad
 * (host, SUR_N_PARAMS floats, may be NULL).  Synchronous. */
int sur_loss_grad(sur_ctx *s, int member, const float *U, const float *Y, int B, int T, double *loss, float *grad);

/* One AdamW step (beta1 0.9, beta2 0.999, eps 1e-8, decoupled weight decay wd)
 * of every member on the same batch (BPTT through all T increments).
 * loss: host, n_members doubles (loss before the update) or NULL (then no
 * synchronisation).  */
int sur_train_step(sur_ctx *s, const float *U, const float *Y, int B, int T, float lr, float wd, double *loss);

/* Predict whole sequences: S (device) n_members x B x T x 6, raw units. */
int sur_predict(sur_ctx *s, const float *U, int B, int T, float *S);

/* Time the phases of one training step of every member without applying it
 * (the parameters and optimiser state are unchanged; the gradient buffers are
 * overwritten): ms_out[0] the forward with the BPTT tape, ms_out[1] the data
 * gradients (the backward through time, with the loss), ms_out[2] the weight
 * and bias gradients, from CUDA events on the context's stream.  U, Y device
 * arrays as for sur_train_step.  Synchronises.  RC_EINVAL on a bad size. */
int sur_profile_step(sur_ctx *s, const float *U, const float *Y, int B, int T, double *ms_out);

/* One increment for n independent quadrature points and every member:
 *   u       device, n x 15 raw features of this increment
 *   h       device, n_members x n x 128 FP32 recurrent state (read, then
 *           overwritten with the new state; zero it to start a sequence)
 *   s_mean  device, n x 6: ensemble mean stress (raw units)
 *   spread  device, n: ||std over members|| / max(||mean||, s_floor)
 * Asynchronous. */
int sur_step(sur_ctx *s, const float *u, int n, float *h, float s_floor, float *s_mean, float *spread);

/* Surrogate input of one increment for n points: u = (F - F_prev row-major (9),
 * Green strain E = (F^T F - I)/2 in Voigt order xx yy zz xy xz yz (6)).
 * F_prev, F: device n x 9 doubles; u: device n x 15 floats.  Asynchronous on
 * `stream`. */
int sur_features(const double *F_prev, const double *F, int n, float *u, void *stream);

/* Tensor-core engine: 2 = the whole recurrent forward and the whole BPTT
 * data-gradient chain (all layers, all steps) each in one 5th-generation
 * tensor-core (tcgen05) kernel per 128-row tile, with the operands on chip,
 * and the members trained side by side (the default); 1 = one tcgen05 GEMM
 * per layer and step; 0 = warp-level BF16 instructions (mma.sync).  Weight
 * gradients use a tcgen05 kernel for engines 1 and 2, mma.sync for 0.  Same
 * results up to summation order and the rounding of the GELU' evaluation.
 * RC_EINVAL for another value. */
int sur_set_backend(sur_ctx *s, int backend);

/* Wait for the stream; return RC_ETIMEOUT if a bounded tensor-core wait gave up,
 * else RC_OK. */
int sur_sync(sur_ctx *s);

/* Number of members and the stream of a surrogate context (either may be NULL). */
int sur_info(const sur_ctx *s, int *n_members, void **stream);

void sur_destroy(sur_ctx *s);

#ifdef __cplusplus
}
#endif
#endif /* SURROGATE_H */
