/*
 * libtled surrogate MLP -- a small fully connected network (GELU hidden
 * layers, linear output) trained with Adam on mean squared error, used to map
 * thermal-ablation scenario parameters to temperature and damage at probe
 * points, with the coupled solver (include/tled.h) as its data source and
 * fallback.  The paper mentions learned acceleration only as related work
 * (Section 7); this component is an extension of the method, not part of it.
 *
 * Numerics: BF16 weights and activations as tensor-core operands, FP32
 * accumulation (tcgen05 on sm_103a), FP32 master parameters, Adam moments,
 * biases, loss and gradients.
 *
 * Conventions as in tled.h: int status codes (TLED_OK / TLED_E_*), no
 * exceptions, no device allocation (caller workspace), all work on the
 * stream given at creation.  Device pointers are float32, row-major.
 * Parameters are one float32 vector: for each layer W [N][K] (row-major)
 * then b [N].
 */
#ifndef TLED_MLP_H
#define TLED_MLP_H
#include <stdint.h>

#include "tled.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tled_mlp tled_mlp;

/* dims[0] inputs, dims[1..n_layers-1] hidden widths, dims[n_layers] outputs;
 * hidden widths and outputs must be multiples of 128 (inputs are zero padded
 * to a multiple of 64).  max_batch: largest batch, a multiple of 128.
 * Errors: E_ARG. */
int tled_mlp_create(tled_mlp **out, int device, void *cuda_stream, int32_t n_layers, const int32_t *dims,
                    int32_t max_batch);
int tled_mlp_destroy(tled_mlp *m);
const char *tled_mlp_last_error(const tled_mlp *m);
/* total number of float32 parameters */
int tled_mlp_num_params(tled_mlp *m, int64_t *n);
/* bytes of device workspace (parameters, Adam moments, activations) */
int tled_mlp_workspace_size(tled_mlp *m, int64_t *bytes);
/* place the network in the workspace (256-byte aligned) and zero it */
int tled_mlp_init(tled_mlp *m, void *dev_workspace, int64_t bytes);
/* copy all parameters from / to host float32 memory; setting resets Adam */
int tled_mlp_set_params(tled_mlp *m, const float *params);
int tled_mlp_get_params(tled_mlp *m, float *params);
/* Affine map of the inputs, applied inside every forward pass before the
 * first layer: x' = (x - shift) * scale, shift and scale host float32 arrays
 * of dims[0] entries (copied; synchronises).  Both NULL: identity (the
 * default after tled_mlp_init).  Errors: E_ARG (only one given, non-finite). */
int tled_mlp_set_input_scaling(tled_mlp *m, const float *shift, const float *scale);
/* y [B][outputs] = network(x [B][inputs]); B a multiple of 128 <= max_batch */
int tled_mlp_forward(tled_mlp *m, const float *x, int32_t B, float *y);
/* gradient of the MSE loss mean((y - t)^2) over B x outputs into grad
 * [n_params] (device, may be NULL) and the loss into *loss (device float, may
 * be NULL); parameters unchanged */
int tled_mlp_gradients(tled_mlp *m, const float *x, const float *t, int32_t B, float *grad, float *loss);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr */
int tled_mlp_train_step(tled_mlp *m, const float *x, const float *t, int32_t B, float lr, float *loss);
/* the same on the batch of rows rows[0..B) (device int32) of a data set
 * x [n][inputs], t [n][outputs] resident on the device (an epoch's shuffled
 * mini-batches without copying them); rows must lie in [0, n) */
int tled_mlp_train_step_rows(tled_mlp *m, const float *x, const float *t, const int32_t *rows, int32_t B, float lr,
                             float *loss);
/* Ensemble statistics of n_members (1..16) network outputs y[k] [B][n_out]
 * (device float32, e.g. tled_mlp_forward of each member on the same inputs),
 * enqueued on `stream` of `device`; no context, nothing allocated.  Each
 * output is first mapped to z = (y * out_scale + out_shift) * r_b + out_offset
 * (out_scale, out_shift, out_offset: device [n_out], NULL = 1, 0, 0), where
 * the row factor r_b = row_src[b * row_stride] * row_mult applies to the
 * first n_row_scaled outputs only (row_src NULL: r_b = 1) -- e.g. a network
 * that learned temperature rise per unit source power, scaled back by each
 * scenario's power read from its raw input row -- then, over the members in
 * order:
 *   mean [B][n_out]  ensemble mean of z
 *   std  [B][n_out]  population standard deviation of z (two-pass)
 *   spread [B]       max of std over outputs [0, n_spread)
 *   fallback [B]     1 where spread > tol, else 0 (uint8; a negative tol flags every row)
 * Any of the four outputs may be NULL.  n_out must be a multiple of 4 and y,
 * mean and std 16-byte aligned (rows are read and written as float4).  Used to accept a surrogate answer or
 * send the scenario back to the solver.  Errors: E_ARG, E_CUDA. */
int tled_mlp_ensemble(int device, void *stream, int32_t n_members, const float *const *y, int32_t B, int32_t n_out,
                      const float *out_scale, const float *out_shift, const float *row_src, int32_t row_stride,
                      float row_mult, int32_t n_row_scaled, const float *out_offset, int32_t n_spread, float tol,
                      float *mean, float *std, float *spread, uint8_t *fallback);
/* wait for the stream; E_TIMEOUT if a bounded pipeline wait gave up */
int tled_mlp_sync(tled_mlp *m);
/* enqueue the network's later work on another stream of its device (e.g. to run the
 * members of an ensemble side by side); ordering against the previous stream is the
 * caller's.  Errors: E_ARG for a NULL network. */
int tled_mlp_set_stream(tled_mlp *m, void *cuda_stream);

/* ---- the surrogate: an ensemble of these networks with its data handling ----
 * (The paper has no learned component; this is the learned extension named in
 * the header comment above.)  tled_sur holds n_members networks [n_in, width x
 * (depth - 1), n_out] (tled_mlp_create's limits apply), each with its own CUDA
 * stream so that the members train and infer side by side; all results are
 * ordered on the stream given at creation.  Workspace as for the networks
 * (caller-provided, nothing allocated on the device by the library).
 * max_rows: largest training set; max_epochs: most epochs of one tled_sur_train. */
typedef struct tled_sur tled_sur;
/* Input features (computed by a library kernel before the first layer): every raw
 * input mapped to v in [-1, 1] (tled_sur_set_inputs), then for every input column j
 * whose bit is set in enc_cols and every octave f < n_freq the pair sin(pi 2^f v_j),
 * cos(pi 2^f v_j) -- e.g. the source position, on which the answer depends through a
 * peak that moves with it; n_freq = 0: the raw inputs only.  n_in <= 32, n_freq <= 12. */
int tled_sur_create(tled_sur **out, int device, void *cuda_stream, int32_t n_members, int32_t n_in, int32_t width,
                    int32_t depth, int32_t n_out, int32_t n_T, int32_t max_batch, int64_t max_rows,
                    int32_t max_epochs, int32_t n_freq, uint32_t enc_cols, int32_t max_sym);
/* Symmetries of the scenario family, used to augment the training data (e.g. the
 * reflections of a cube that leave the problem unchanged, with the probe lattice
 * reflected with them): n_sym <= max_sym maps g, each taking an input row x to x'
 * with x'_j = in_a[g][j] x[in_src[g][j]] + in_b[g][j] and an output row y to y' with
 * y'_o = y[out_perm[g][o]] (host arrays [n_sym][n_in] and [n_sym][n_out], copied; the
 * identity should be one of them).  tled_sur_train then trains on the n x n_sym rows
 * of the augmented set (row g n + i: map g applied to data row i); max_rows bounds
 * that count.  n_sym = 0: no augmentation.  Errors: E_ARG, E_STATE. */
int tled_sur_set_symmetries(tled_sur *s, int32_t n_sym, const int32_t *in_src, const float *in_a, const float *in_b,
                            const int32_t *out_perm);
int tled_sur_destroy(tled_sur *s);
const char *tled_sur_last_error(const tled_sur *s);
int tled_sur_workspace_size(tled_sur *s, int64_t *bytes);
/* place the networks and buffers in the workspace (256-byte aligned) */
int tled_sur_init(tled_sur *s, void *dev_workspace, int64_t bytes);
/* inputs mapped to [-1, 1] over [lo, hi] (host float32 [n_in] each; identity until set) */
int tled_sur_set_inputs(tled_sur *s, const float *lo, const float *hi);
/* Output transform.  power_col >= 0: the first n_T outputs are temperatures T (C) and
 * are learned as the rise per unit source power, (T - T_ref) / (x[power_col] /
 * power_ref) -- the bioheat problem is linear in the source power when c and k do
 * not depend on T -- and mapped back per row at inference.  Every output is then
 * standardised: norm 0, per output (mean and standard deviation of its column);
 * norm 1, mean per output but one scale per group of outputs (the temperatures
 * [0, n_T), the rest), so that the training loss weighs errors of the same
 * physical size alike.  Errors: E_ARG. */
int tled_sur_set_outputs(tled_sur *s, int32_t power_col, float power_ref, float T_ref, int32_t norm);
/* Train every member from a seeded He-normal initialisation with Adam (beta 0.9,
 * 0.999, eps 1e-8) on the mean squared error of the standardised targets: x
 * [n][n_in] raw inputs and y [n][n_out] outputs in physical units, both device
 * float32; `epochs` passes, each over a permutation of the rows (member k's from the
 * splitmix64 stream seeded by `seed`) in mini-batches of `batch` (a multiple of 128;
 * the last partial batch is dropped).  Learning rate: lr, decaying by a cosine to
 * lr_end over the whole run (lr_end = lr: constant).  bootstrap != 0: member k
 * trains on n rows drawn with replacement (once; every epoch permutes them), so the
 * members' spread also reflects the sampling of the data.  Each member replays a
 * CUDA graph of one epoch on its own stream.  loss_history: host float32
 * [n_members][epochs] of mean training losses, or NULL.  Synchronises.
 * Errors: E_ARG, E_STATE, E_CUDA. */
int tled_sur_train(tled_sur *s, const float *x, const float *y, int64_t n, int32_t epochs, int32_t batch, float lr,
                   float lr_end, int32_t bootstrap, uint64_t seed, float *loss_history);
/* Ensemble answer for B <= max_batch scenario rows x [B][n_in] (device float32),
 * enqueued: mean and std [B][n_out] in physical units (population std over the
 * members), spread [B] = max of std over outputs [0, n_spread), fallback_mask [B]
 * = 1 where spread > spread_tol_K (those scenarios go to the solver); any output
 * may be NULL.  Errors: E_ARG, E_STATE. */
int tled_sur_predict(tled_sur *s, const float *x, int32_t B, int32_t n_spread, float spread_tol_K, float *mean,
                     float *std, float *spread, uint8_t *fallback_mask);
/* Calibrate the spread threshold against solver answers y [n][n_out] (device) for
 * the scenarios x [n][n_in]: the largest threshold tau <= tol_K such that among the
 * scenarios with spread <= tau at least a `coverage` fraction have max over outputs
 * [0, n_spread) of |mean - y| <= tol_K; *tau = -1 if none qualifies; *accepted =
 * the fraction of the n scenarios with spread <= tau.  Synchronises. */
int tled_sur_calibrate(tled_sur *s, const float *x, const float *y, int64_t n, int32_t n_spread, float tol_K,
                       float coverage, float *tau, float *accepted);
/* The threshold rule of tled_sur_calibrate on host arrays spread [n] and err [n]
 * (no GPU needed): the longest prefix of the scenarios sorted by spread whose
 * fraction with err <= tol_K is at least `coverage`, capped at tol_K. */
int tled_sur_spread_threshold(int64_t n, const float *spread, const float *err, float tol_K, float coverage,
                              float *tau, float *accepted);
/* member k's network (parameters, gradients, single-member inference) */
int tled_sur_member(tled_sur *s, int32_t k, tled_mlp **member);
int tled_sur_sync(tled_sur *s);

#ifdef __cplusplus
}
#endif
#endif
