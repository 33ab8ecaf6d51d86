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
/* y [B][outputs] = network(x [B][inputs]); B a multiple of 128 <= max_batch */
int tled_mlp_forward(tled_mlp *m, const float *x, int32_t B, float *y);
/* gradient of the MSE loss mean((y - t)^2) over B x outputs into grad
 * [n_params] (device, may be NULL) and the loss into *loss (device float, may
 * be NULL); parameters unchanged */
int tled_mlp_gradients(tled_mlp *m, const float *x, const float *t, int32_t B, float *grad, float *loss);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr */
int tled_mlp_train_step(tled_mlp *m, const float *x, const float *t, int32_t B, float lr, float *loss);
/* wait for the stream; E_TIMEOUT if a bounded pipeline wait gave up */
int tled_mlp_sync(tled_mlp *m);

#ifdef __cplusplus
}
#endif
#endif
