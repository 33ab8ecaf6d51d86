// Internal declarations of the surrogate MLP kernels (not part of the C ABI).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace tmlp {

enum { kEpiBiasF32 = 0, kEpiGelu = 1, kEpiGeluGrad = 2, kEpiF32 = 3 };
constexpr int kLossBlocks = 296;

struct GemmArgs {
    int M, N, K;                 // D[M][N] = A[M][K] B[N][K]^T; M % 128 == 0, N % BN == 0, K % 64 == 0
    const float *bias;           // [N]
    float *out_f32;              // kEpiBiasF32 / kEpiF32
    int ld_f32;
    __nv_bfloat16 *out_bf;       // kEpiGelu / kEpiGeluGrad: [M][ld_bf]
    int ld_bf;
    __nv_bfloat16 *out_bfT;      // and its transpose [N][ld_bfT]
    int ld_bfT;
    float *z_out;                // kEpiGelu: pre-activation [M][ld_z]
    const float *z_in;           // kEpiGeluGrad: previous layer's pre-activation [M][ld_z]
    int ld_z;
    unsigned int *status;        // error word (bit 0: a bounded wait timed out)
};

constexpr int kMaxMembers = 16;
struct EnsembleArgs {
    const float *y[kMaxMembers];  // member outputs [B][n_out]
    int n_members, n_out, n_spread;
    const float *scale, *shift;   // [n_out] or NULL
    const float *row_src;         // per-row factor r_b = row_src[b * row_stride] * row_mult, or NULL (r_b = 1)
    int row_stride, n_row_scaled; // r_b multiplies outputs [0, n_row_scaled)
    float row_mult;
    const float *offset;          // [n_out] added after the row factor, or NULL
    float tol;
    float *mean, *std, *spread;   // [B][n_out], [B][n_out], [B]; each may be NULL
    uint8_t *fallback;            // [B] or NULL
};
cudaError_t launch_ensemble(const EnsembleArgs &e, int B, cudaStream_t s);

cudaError_t launch_gemm(const CUtensorMap &a, const CUtensorMap &b, const GemmArgs &g, int bn, int mode,
                        cudaStream_t s);
cudaError_t launch_input(const float *x, const int32_t *rows, int B, int n_in, int ld, const float *shift,
                         const float *scale, __nv_bfloat16 *xb, __nv_bfloat16 *xt, cudaStream_t s);
cudaError_t launch_loss(const float *y, const float *t, const int32_t *rows, int B, int N, __nv_bfloat16 *dy,
                        __nv_bfloat16 *dyt, double *partials, float *loss, cudaStream_t s);
cudaError_t launch_bias_grad(const __nv_bfloat16 *dzt, int B, int N, float *db, cudaStream_t s);
// bc: device (bc1, bc2) of a device step counter, overriding the scalars (NULL: use them)
cudaError_t launch_adam(float *w, float *m, float *v, const float *grad, int64_t n, float lr, float b1, float b2,
                        float eps, float bc1, float bc2, int N, int K, int ld, __nv_bfloat16 *wb, __nv_bfloat16 *wt,
                        cudaStream_t s, const float *bc = nullptr);
cudaError_t launch_adam_tick(int64_t *t, float *bc, float lr, float lr_end, int64_t n_decay, cudaStream_t s);
// surrogate data: temperature rise per unit source power, column statistics, standardisation,
// per-row maximum error, mean of per-step losses
cudaError_t launch_sur_encode(const float *x, int ld_x, int64_t n, int64_t n_rows, int n_in, const float *shift,
                              const float *scale, int n_freq, unsigned enc_cols, int n_feat, float *feat,
                              cudaStream_t s);
cudaError_t launch_sur_augment(const float *x, const float *y, int64_t n, int n_in, int n_out, int n_sym,
                               const int32_t *src, const float *a, const float *b, const int32_t *perm, float *xa,
                               float *ya, cudaStream_t s);
cudaError_t launch_sur_transform(const float *x, int ld_x, const float *y, int64_t n, int n_out, int n_T,
                                 int power_col, float T_ref, float inv_Pref, float *z, cudaStream_t s);
cudaError_t launch_column_stats(const float *z, int64_t n, int n_out, double *mean, double *m2, cudaStream_t s);
cudaError_t launch_standardize(float *z, int64_t n, int n_out, const float *shift, const float *scale,
                               cudaStream_t s);
cudaError_t launch_row_max_abs_diff(const float *a, const float *b, int64_t n, int n_out, int n_cmp, float *err,
                                    cudaStream_t s);
cudaError_t launch_mean_losses(const float *losses, int k, float *out, cudaStream_t s);
cudaError_t launch_gather_grad(const float *G, const float *db, int N, int K, int ld, float *grad, cudaStream_t s);

}  // namespace tmlp

// Internal entry of the MLP (mlp_capi.cpp) for the surrogate engine: one Adam step
// on rows of a device-resident data set, enqueued on `stream`, with Adam's step
// counter on the device (t_dev, bc_dev [3]: advanced by the step itself, the
// learning rate decaying from lr to lr_end over n_decay steps by a cosine, or
// constant for n_decay <= 0), so that a sequence of steps can be captured in a
// CUDA graph.
struct tled_mlp;
int tmlp_train_step_graphable(tled_mlp *m, cudaStream_t stream, const float *x, const float *t, const int32_t *rows,
                              int B, float lr, float lr_end, int64_t n_decay, float *loss, int64_t *t_dev,
                              float *bc_dev);
int tmlp_forward_on(tled_mlp *m, cudaStream_t stream, const float *x, int B, float *y);
