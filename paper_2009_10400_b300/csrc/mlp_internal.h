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
cudaError_t launch_adam(float *w, float *m, float *v, const float *grad, int64_t n, float lr, float b1, float b2,
                        float eps, float bc1, float bc2, int N, int K, int ld, __nv_bfloat16 *wb, __nv_bfloat16 *wt,
                        cudaStream_t s);
cudaError_t launch_gather_grad(const float *G, const float *db, int N, int K, int ld, float *grad, cudaStream_t s);

}  // namespace tmlp
