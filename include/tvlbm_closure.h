/* Learned coarse-grid closure for D2Q16 TVLBM runs: a small network, trained and evaluated
 * by the library's own BF16 tensor-core (tcgen05) kernels, that corrects the collision of a
 * coarse run towards the block average of a 4x finer run.
 *
 * The paper has no learned part.  This extends its method (Sec. "The TVLBM model": BGK with a
 * Hermite equilibrium on a Gauss-Hermite velocity set); the correction is built so that the
 * conservation the paper insists on (Introduction, Conclusions) stays exact:
 *
 *   Delta f_l = w_l sum_{k<12} o_k psi_k(c_l),   psi_k = He_a(c_x) He_b(c_y) / sqrt(a! b!)
 *
 * over the 12 D2Q16 Hermite tensor vectors orthogonal (in sum_l w_l g_l h_l) to the collision
 * invariants 1, c_x, c_y, |c|^2, in this order:
 *   k = 0: (He_2(c_x) - He_2(c_y)) / 2,  then (a, b) = (1,1), (3,0), (2,1), (1,2), (0,3), (3,1),
 *   (2,2), (1,3), (3,2), (2,3), (3,3).
 * Such a correction adds no mass, momentum or energy.  The learned coarse step is the method's
 * pull-gather (Sec. "The TVLBM model") followed by a learned collision: every cell becomes
 * f_eq(rho, u, T) (the method's equilibrium at the cell's own moments) plus the correction,
 * whose coefficients the network predicts from the streamed (pre-collision) state.  The
 * conserved moments come from the streaming, the non-conserved ones from the network.
 *
 * Network: 54 inputs -> 128 GELU -> 128 GELU -> 12 outputs, GELU(z) = z Phi(z), Phi by the
 * erf approximation of Abramowitz & Stegun eq. 7.1.26 (|error| <= 1.5e-7; see
 * tvlbm_mlp_activation).
 * Inputs of cell (x, y): for (dy, dx) in {-1,0,1}^2 (row-major, dy outer) the 6 features
 * (rho, u_x, u_y, T, Pi^neq_xy, Pi^neq_xx - Pi^neq_yy) of cell (x+dx, y+dy) (periodic), each
 * normalised as (value - mu_q) * inv_sigma_q; Pi^neq = sum_l f_l c c - rho u u.
 * Outputs y_k; the correction uses o_k = out_scale_k y_k.
 * Parameters (TVLBM_MLP_PARAMS floats, this order, row-major [out][in]):
 *   W1[128][54], b1[128], W2[128][128], b2[128], W3[12][128], b3[12].
 * Arithmetic: BF16 weights, inputs and hidden activations, FP32 accumulation and outputs;
 * FP32 master parameters and Adam moments.
 *
 * Device buffers passed to these calls are the caller's (device pointers, 16-byte aligned).
 * Row counts must be multiples of 128 and at most the max_rows given at creation.  Errors:
 * TVLBM_EINVAL (arguments), TVLBM_ECUDA (a CUDA failure), TVLBM_ETIMEOUT (a bounded device
 * wait gave up).  tvlbm_mlp_last_error describes the last failure of a network call.
 */
#ifndef TVLBM_CLOSURE_H
#define TVLBM_CLOSURE_H

#include <stddef.h>

#include "tvlbm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define TVLBM_MLP_IN 54
#define TVLBM_MLP_IN_PAD 64 /* row length of the BF16 input matrix (entries 54..63 are zero) */
#define TVLBM_MLP_HIDDEN 128
#define TVLBM_MLP_OUT 12
#define TVLBM_MLP_OUT_PAD 16 /* row length of output / target matrices (entries 12..15 unused) */
#define TVLBM_MLP_PARAMS 25100

typedef struct tvlbm_mlp tvlbm_mlp;

/* Network with device storage for batches of up to max_rows rows (a multiple of 128) on the
 * current device; parameters start at zero.  Errors: EINVAL, ENOMEM, ECUDA. */
int tvlbm_mlp_create(int max_rows, tvlbm_mlp **out);
int tvlbm_mlp_destroy(tvlbm_mlp *m); /* synchronises its stream; NULL accepted */
/* Queue later work on `stream` (a cudaStream_t of the network's device; NULL = legacy default). */
int tvlbm_mlp_set_stream(tvlbm_mlp *m, void *stream);
/* Copy parameters from / to host memory (TVLBM_MLP_PARAMS floats).  Setting them also clears
 * the Adam moments and step count.  Both synchronise. */
int tvlbm_mlp_set_params(tvlbm_mlp *m, const float *params);
int tvlbm_mlp_get_params(tvlbm_mlp *m, float *params);

/* Inference: y[r][k] = network(x[r]) for r < rows.  x: device BF16 [rows][64]; y: device FP32
 * [rows][16] (entries 12..15 written as 0).  Asynchronous on the network's stream. */
int tvlbm_mlp_forward(tvlbm_mlp *m, const void *x, int rows, float *y);

/* Training pass: loss L = mean over rows r and k < 12 of (y[r][k] - ystar[r][k])^2 and its
 * gradient with respect to every parameter (kept on the device for tvlbm_mlp_adam).
 * x: device BF16 [rows][64]; ystar: device FP32 [rows][16].  loss (host, may be NULL) and grad
 * (host, TVLBM_MLP_PARAMS floats, may be NULL) make the call synchronous. */
int tvlbm_mlp_loss_grad(tvlbm_mlp *m, const void *x, const float *ystar, int rows, double *loss, float *grad);

/* One Adam step (bias-corrected moments) with the gradient of the last tvlbm_mlp_loss_grad:
 * theta -= lr mhat / (sqrt(vhat) + eps).  Refreshes the BF16 weight copies. */
int tvlbm_mlp_adam(tvlbm_mlp *m, float lr, float beta1, float beta2, float eps);

const char *tvlbm_mlp_last_error(const tvlbm_mlp *m);

/* The network's activation as its kernels evaluate it, on n device values: g[i] = GELU(z[i]) (as
 * the forward epilogues compute it, pairs of entries in packed FP32) and dg[i] = GELU'(z[i]) =
 * Phi(z) + z phi(z) (either output may be NULL).  z, g, dg: device FP32
 * arrays of n entries, caller-owned.  Asynchronous on `stream` (a cudaStream_t; NULL = legacy
 * default).  Errors: EINVAL (n < 0, z NULL), ECUDA. */
int tvlbm_mlp_activation(const float *z, float *g, float *dg, int n, void *stream);

/* ---- closure on a context (D2Q16, periodic, storage FP64 / FP32 / FP32_DEV, default
 * deviation reference); asynchronous on the context's stream unless stated ---------------- */

/* Raw per-cell features of the current state: m6[q][y][x] (device FP32 [6][ny][nx]) =
 * (rho, u_x, u_y, T, Pi^neq_xy, Pi^neq_xx - Pi^neq_yy), computed in FP64. */
int tvlbm_closure_moments(tvlbm_ctx *ctx, float *m6);

/* Network inputs of every cell of the current state: x (device BF16 [nx*ny][64], row
 * y*nx + x), normalised with host arrays mu[6], inv_sigma[6]; entries 54..63 set to 0. */
int tvlbm_closure_features(tvlbm_ctx *ctx, const float *mu, const float *inv_sigma, void *x);

/* Projection of the difference of two states on the basis: o[c][k] = inv_scale_k sum_l
 * (f_a - f_b)_l(c) psi_k(c_l) for k < 12 (device FP32 [nx*ny][16], entries 12..15 set to 0),
 * computed in FP64; inv_scale: host array of 12, or NULL for 1.  a and b: same grid, velocity
 * set and storage.  Unscaled, o is the least-squares correction coefficient vector that takes
 * b towards a. */
int tvlbm_closure_project(tvlbm_ctx *a, tvlbm_ctx *b, const float *inv_scale, float *o);

/* Non-equilibrium coefficients of the current state: o[c][k] = inv_scale_k sum_l (f - f_eq)_l(c)
 * psi_k(c_l) with f_eq at the cell's own (rho, u, T) (device FP32 [nx*ny][16], entries 12..15
 * set to 0; inv_scale host [12] or NULL), computed in FP64 (a diagnostic of a state's
 * non-equilibrium part in the basis). */
int tvlbm_closure_noneq(tvlbm_ctx *ctx, const float *inv_scale, float *o);

/* Coarse graining: the current state of `coarse` becomes the block average of the current
 * state of `fine` over m x m cells, m = fine nx / coarse nx = fine ny / coarse ny (>= 1).
 * Same velocity set; any two supported storages.  Conserves mass, momentum and energy. */
int tvlbm_downsample(tvlbm_ctx *fine, tvlbm_ctx *coarse);

/* Copy the current state of src into dst (same grid, velocity set and storage). */
int tvlbm_copy_state(tvlbm_ctx *src, tvlbm_ctx *dst);

/* n learned coarse steps: each streams, computes the network's coefficients o = out_scale * y
 * from the streamed state (features normalised with mu, inv_sigma; host arrays) and sets every
 * cell to f_eq(rho, u, T) + w sum_k o_k psi_k (the context's tau is not used).  The network's
 * stream is set to the context's.  Needs nx*ny to be a multiple of 128 and at most the
 * network's max_rows. */
int tvlbm_step_closure(tvlbm_ctx *ctx, tvlbm_mlp *m, const float *mu, const float *inv_sigma, const float *out_scale,
                       int n);

#ifdef __cplusplus
}
#endif

#endif /* TVLBM_CLOSURE_H */
