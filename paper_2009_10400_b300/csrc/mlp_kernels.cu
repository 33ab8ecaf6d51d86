// Surrogate MLP on the 5th-generation tensor cores (sm_103a): BF16 operands,
// FP32 accumulation in tensor memory, GELU activations, MSE loss, Adam.
//
// GEMM: D[M][N] = A[M][K] * B[N][K]^T with both operands K-major BF16 in
// global memory.  Persistent CTAs (two per SM) take 128 x BN tiles in turn: warp
// 0 streams 128 x 64 and BN x 64 operand boxes with TMA (128-byte swizzle)
// through a 2-stage mbarrier pipeline, one thread of warp 1 issues tcgen05.mma
// (K = 16 each) into one of two TMEM accumulators and commits stage releases,
// and warps 2-5 read the other accumulator with tcgen05.ld (one row per thread)
// and apply the epilogue:
//   kEpiBiasF32   Y = D + b                        (float output)
//   kEpiGelu      Z = D + b, A = GELU(Z)           (Z float; A bf16 and its transpose)
//   kEpiGeluGrad  dZ = D * GELU'(Zprev)            (bf16 and its transpose)
//   kEpiF32       G = D                            (float, weight gradients)
// Every mbarrier wait is bounded; a time-out sets an error word and the CTA
// drains its copies, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "mlp_internal.h"

namespace tmlp {

constexpr int kBM = 128;
constexpr int kEpiLd = 33;  // padded row of the per-warp epilogue transpose buffer (conflict-free)
constexpr int kBK = 64;  // 64 bf16 = 128 bytes = one swizzle row

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(su32(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// bounded wait: about 2^31 cycles (around a second) before giving up
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity) {
    const long long t0 = clock64();
    while (!bar_try(b, parity))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

// UMMA shared-memory descriptor, K-major operand in the canonical 128-byte
// swizzled layout: rows of 128 B, 8-row atoms 1024 B apart (SBO), version 1,
// layout type 2 (SWIZZLE_128B); the tile base is 1024-byte aligned.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused with 128-byte swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, M = 128, N = BN
template <int BN>
__device__ __forceinline__ constexpr uint32_t idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// shared memory of one CTA: the operand ring (1024-byte aligned) and four 32 x 33
// float transpose buffers of the epilogue warps
template <int BN, int STAGES>
constexpr int gemm_smem_bytes() {
    return STAGES * (kBM + BN) * kBK * 2 + 1024 + 4 * 32 * kEpiLd * 4;
}

// Epilogue of one 128 x BN tile for the calling warp (rows row0 .. row0 + 31 = TMEM lanes
// 32 lg .. + 31, one row per lane), from TMEM columns tcol .. tcol + BN - 1.  Row-major
// traffic goes through a per-warp 32 x 33 transpose buffer so that a warp's loads and
// stores cover 32 consecutive columns of one row.
template <int BN, int MODE>
__device__ __forceinline__ void epilogue_tile(const GemmArgs &g, uint32_t tmem, uint32_t tcol, int lg, int lane,
                                              float *buf, int m0, int n0) {
    const int row0 = m0 + lg * 32;
    const int row = row0 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(lg * 32) << 16) + tcol + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int col0 = n0 + c0;
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; j++) v[j] = __uint_as_float(r[j]);
        if constexpr (MODE == kEpiGeluGrad) {  // Z of the previous layer: coalesced rows in, transposed
#pragma unroll 4
            for (int rr = 0; rr < 32; rr++) buf[rr * kEpiLd + lane] = g.z_in[(int64_t)(row0 + rr) * g.ld_z + col0 + lane];
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 32; j++) v[j] *= gelu_grad(buf[lane * kEpiLd + j]);
            __syncwarp();
        } else if constexpr (MODE == kEpiBiasF32 || MODE == kEpiGelu) {
#pragma unroll
            for (int j = 0; j < 32; j++) v[j] += g.bias[col0 + j];
        }
        // row-major float output (Y, Z or G): stage and write rows
        float *out_rm = MODE == kEpiGelu ? g.z_out : g.out_f32;
        const int ld_rm = MODE == kEpiGelu ? g.ld_z : g.ld_f32;
        if constexpr (MODE != kEpiGeluGrad) {
#pragma unroll
            for (int j = 0; j < 32; j++) buf[lane * kEpiLd + j] = v[j];
            __syncwarp();
#pragma unroll 4
            for (int rr = 0; rr < 32; rr++) out_rm[(int64_t)(row0 + rr) * ld_rm + col0 + lane] = buf[rr * kEpiLd + lane];
            __syncwarp();
        }
        if constexpr (MODE == kEpiGelu || MODE == kEpiGeluGrad) {
            // bf16 activation (or gradient): transposed copy straight from registers
            // (consecutive lanes = consecutive rows), row-major copy through the buffer
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const __nv_bfloat16 h = __float2bfloat16_rn(MODE == kEpiGelu ? gelu(v[j]) : v[j]);
                g.out_bfT[(int64_t)(col0 + j) * g.ld_bfT + row] = h;
                buf[lane * kEpiLd + j] = __bfloat162float(h);
            }
            __syncwarp();
#pragma unroll 4
            for (int rr = 0; rr < 32; rr++)
                g.out_bf[(int64_t)(row0 + rr) * g.ld_bf + col0 + lane] = __float2bfloat16_rn(buf[rr * kEpiLd + lane]);
            __syncwarp();
        }
    }
}

// Persistent GEMM: CTA b takes the 128 x BN tiles b, b + gridDim.x, ... (M-major order, so
// that neighbouring CTAs share the weight tile).  The accumulator is double-buffered in
// TMEM (2 BN columns): the MMA warp fills one buffer while the epilogue warps drain the
// other; tfull[a] (MMA -> epilogue, a tcgen05 commit) and tempty[a] (epilogue -> MMA, one
// arrival per epilogue warp) hand the buffers over.
template <int BN, int MODE, int kStages>
__global__ void __launch_bounds__(192, 2)
    umma_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs g) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full[kStages], empty[kStages], tfull[2], tempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    uint8_t *smem = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int kABytes = kBM * kBK * 2, kBBytes = BN * kBK * 2;
    uint8_t *sA = smem, *sB = smem + kStages * kABytes;
    float *sEpi = reinterpret_cast<float *>(sB + kStages * kBBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_mt = g.M / kBM, n_tiles = n_mt * (g.N / BN);
    const int KB = g.K / kBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; a++) {
            bar_init(&tfull[a], 1);
            bar_init(&tempty[a], 4);  // one arrival per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"((uint32_t)(2 * BN)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    int issued = 0, consumed = 0;  // producer: k-blocks whose loads were issued / known to have landed

    if (warp == 0 && lane == 0) {
        // ---- TMA producer over all the CTA's tiles
        int it = 0;
        bool dead = false;
        for (int t = blockIdx.x; t < n_tiles && !dead; t += gridDim.x) {
            const int m0 = (t % n_mt) * kBM, n0 = (t / n_mt) * BN;
            for (int kb = 0; kb < KB; kb++, it++) {
                const int s = it % kStages;
                if (it >= kStages) {
                    if (!bar_wait(&empty[s], ((it / kStages) - 1) & 1)) {
                        s_fail = 1;
                        dead = true;
                        break;
                    }
                    consumed = it - kStages + 1;
                }
                bar_expect(&full[s], kABytes + kBBytes);
                tma_load_2d(sA + s * kABytes, &tmA, kb * kBK, m0, &full[s]);
                tma_load_2d(sB + s * kBBytes, &tmB, kb * kBK, n0, &full[s]);
                issued = it + 1;
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        constexpr uint32_t idesc = idesc_bf16<BN>();
        int it = 0, i = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, i++) {
            const int a = i & 1;
            if (i >= 2 && !bar_wait(&tempty[a], ((i >> 1) - 1) & 1)) {  // the epilogue drained buffer a
                s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc_t = tmem + (uint32_t)(a * BN);
            bool ok = true;
            for (int kb = 0; kb < KB; kb++, it++) {
                const int s = it % kStages;
                if (!bar_wait(&full[s], (it / kStages) & 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = su32(sA + s * kABytes), b0 = su32(sB + s * kBBytes);
#pragma unroll
                for (int kk = 0; kk < kBK / 16; kk++)  // advance 16 elements = 32 bytes along K inside the swizzle row
                    umma(acc_t, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc, (kb | kk) != 0);
                umma_commit(&empty[s]);  // stage reusable once these MMAs completed
            }
            if (!ok) {
                s_fail = 1;
                break;
            }
            umma_commit(&tfull[a]);  // buffer a complete once every MMA of the tile has
        }
    } else if (warp >= 2) {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31
        const int lg = warp & 3;
        float *buf = sEpi + (warp - 2) * 32 * kEpiLd;
        int i = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, i++) {
            const int a = i & 1;
            if (!bar_wait(&tfull[a], (i >> 1) & 1)) {
                s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            epilogue_tile<BN, MODE>(g, tmem, (uint32_t)(a * BN), lg, lane, buf, (t % n_mt) * kBM, (t / n_mt) * BN);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&tempty[a])) : "memory");
        }
    }
    __syncthreads();
    if (s_fail) {
        if (threadIdx.x == 0) {
            atomicOr(g.status, 1u);
            // let this CTA's issued copies land before its shared memory is released
            for (int it = consumed; it < issued; it++) bar_wait(&full[it % kStages], (it / kStages) & 1);
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN)));
}

// ---------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------
// batch row b = x[rows[b]] (rows NULL: x[b]) of x [*][n_in] float, mapped to
// (x - shift) * scale (NULL: identity), -> bf16 [B][ld] (zero padded) and its transpose [ld][B]
__global__ void input_kernel(const float *__restrict__ x, const int32_t *__restrict__ rows, int B, int n_in, int ld,
                             const float *__restrict__ shift, const float *__restrict__ scale, __nv_bfloat16 *xb,
                             __nv_bfloat16 *xt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * ld) return;
    const int b = (int)(i / ld), k = (int)(i % ld);
    float v = 0.f;
    if (k < n_in) {
        const int64_t r = rows ? (int64_t)rows[b] : (int64_t)b;
        v = x[r * n_in + k];
        if (shift) v = (v - shift[k]) * scale[k];
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    xb[i] = h;
    xt[(int64_t)k * B + b] = h;
}

// MSE loss 1/(B N) sum (y - t)^2 and dY = 2 (y - t) / (B N) in bf16 (+ transpose);
// per-block partial sums of the loss (fixed order, reduced by loss_final_kernel)
// (targets of batch row b: t[rows[b]], or t[b] when rows is NULL)
__global__ void loss_kernel(const float *__restrict__ y, const float *__restrict__ t, const int32_t *__restrict__ rows,
                            int B, int N, __nv_bfloat16 *dy, __nv_bfloat16 *dyt, double *partials) {
    __shared__ double sh[256];
    const double scale = 1.0 / ((double)B * N);
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)B * N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / N), n = (int)(i % N);
        const int64_t r = rows ? (int64_t)rows[b] : (int64_t)b;
        const float d = y[i] - t[r * N + n];
        acc += (double)d * d;
        const __nv_bfloat16 g = __float2bfloat16_rn((float)(2.0 * scale) * d);
        dy[i] = g;
        dyt[(int64_t)n * B + b] = g;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0] * scale;
}
__global__ void loss_final_kernel(const double *partials, int n, float *loss) {
    if (threadIdx.x) return;
    double s = 0;
    for (int i = 0; i < n; i++) s += partials[i];
    *loss = (float)s;
}

// bias gradient: db[n] = sum_b dZ[b][n], read from the transposed copy dZt [N][B]
__global__ void bias_grad_kernel(const __nv_bfloat16 *__restrict__ dzt, int B, int N, float *db) {
    const int n = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (n >= N) return;
    float s = 0.f;
    for (int b = lane; b < B; b += 32) s += __bfloat162float(dzt[(int64_t)n * B + b]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) db[n] = s;
}

// Adam on FP32 master parameters; refresh the bf16 weights W [N][ld] and W^T [ld][N]
__global__ void adam_kernel(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ grad, int64_t n, float lr, float b1, float b2, float eps,
                            float bc1, float bc2, const float *__restrict__ bc, int N, int K, int ld,
                            __nv_bfloat16 *wb, __nv_bfloat16 *wt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (bc) {  // the device step counter's bias corrections and learning rate (graph-captured training)
        bc1 = bc[0];
        bc2 = bc[1];
        lr = bc[2];
    }
    const float gr = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gr;
    const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    w[i] = wi;
    if (wb && i < (int64_t)N * K) {  // weight matrix part (the bias follows it)
        const int r = (int)(i / K), c = (int)(i % K);
        const __nv_bfloat16 h = __float2bfloat16_rn(wi);
        wb[(int64_t)r * ld + c] = h;
        wt[(int64_t)c * N + r] = h;
    }
}

// gradient of a layer's weights from the padded FP32 GEMM output G [N][ld]
__global__ void gather_grad_kernel(const float *__restrict__ G, const float *__restrict__ db, int N, int K, int ld,
                                   float *grad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)N * K + N) return;
    if (i < (int64_t)N * K) {
        const int r = (int)(i / K), c = (int)(i % K);
        grad[i] = G[(int64_t)r * ld + c];
    } else {
        grad[i] = db[i - (int64_t)N * K];
    }
}

// Ensemble statistics, one block per batch row b: z_k = (y_k * scale + shift)
// * r_b + offset for the members k (r_b only on the first n_row_scaled outputs;
// summed in member order), mean and population standard deviation (two
// passes), spread = max of std over the first n_spread outputs, fallback =
// spread > tol.
__global__ void __launch_bounds__(256) ensemble_kernel(const EnsembleArgs E) {
    const int b = blockIdx.x;
    const float rb = E.row_src ? E.row_src[(int64_t)b * E.row_stride] * E.row_mult : 1.f;
    float smax = 0.f;
    // four consecutive outputs per thread and iteration (n_out is a multiple of 128)
    for (int n = 4 * threadIdx.x; n < E.n_out; n += 4 * blockDim.x) {
        const int64_t i = (int64_t)b * E.n_out + n;
        float4 z[kMaxMembers];
#pragma unroll
        for (int k = 0; k < kMaxMembers; k++)
            if (k < E.n_members) z[k] = *reinterpret_cast<const float4 *>(E.y[k] + i);
        float mean[4], sd[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int nc = n + c;
            const float sc = E.scale ? E.scale[nc] : 1.f, sh = E.shift ? E.shift[nc] : 0.f;
            const float r = nc < E.n_row_scaled ? rb : 1.f, off = E.offset ? E.offset[nc] : 0.f;
            float zc[kMaxMembers];
            float sum = 0.f;
#pragma unroll
            for (int k = 0; k < kMaxMembers; k++) {
                if (k < E.n_members) {
                    const float y = c == 0 ? z[k].x : c == 1 ? z[k].y : c == 2 ? z[k].z : z[k].w;
                    zc[k] = fmaf(fmaf(y, sc, sh), r, off);
                    sum += zc[k];
                }
            }
            mean[c] = sum / (float)E.n_members;
            float var = 0.f;
#pragma unroll
            for (int k = 0; k < kMaxMembers; k++) {
                if (k < E.n_members) {
                    const float d = zc[k] - mean[c];
                    var = fmaf(d, d, var);
                }
            }
            sd[c] = sqrtf(var / (float)E.n_members);
            if (nc < E.n_spread) smax = fmaxf(smax, sd[c]);
        }
        if (E.mean) *reinterpret_cast<float4 *>(E.mean + i) = make_float4(mean[0], mean[1], mean[2], mean[3]);
        if (E.std) *reinterpret_cast<float4 *>(E.std + i) = make_float4(sd[0], sd[1], sd[2], sd[3]);
    }
    for (int o = 16; o > 0; o >>= 1) smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = smax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = fmaxf(m, red[w]);
        if (E.spread) E.spread[b] = m;
        if (E.fallback) E.fallback[b] = m > E.tol ? 1 : 0;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
constexpr int kGemmStages = 2;  // two persistent CTAs per SM, each overlapping its epilogue with its next MMAs
template <int BN, int MODE>
static cudaError_t launch_one(const CUtensorMap &a, const CUtensorMap &b, const GemmArgs &g, cudaStream_t s) {
    const int smem = gemm_smem_bytes<BN, kGemmStages>();
    auto kern = umma_gemm_kernel<BN, MODE, kGemmStages>;
    static int set_device = -1, n_sm = 0;  // the attribute is per device: set it on first use there
    int dev = 0;
    cudaGetDevice(&dev);
    if (set_device != dev) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        set_device = dev;
    }
    const int n_tiles = (g.M / kBM) * (g.N / BN);
    kern<<<std::min(n_tiles, 2 * n_sm), 192, smem, s>>>(a, b, g);
    return cudaGetLastError();
}

cudaError_t launch_gemm(const CUtensorMap &a, const CUtensorMap &b, const GemmArgs &g, int bn, int mode,
                        cudaStream_t s) {
    if (bn == 64) {
        switch (mode) {
            case kEpiBiasF32: return launch_one<64, kEpiBiasF32>(a, b, g, s);
            case kEpiGelu: return launch_one<64, kEpiGelu>(a, b, g, s);
            case kEpiGeluGrad: return launch_one<64, kEpiGeluGrad>(a, b, g, s);
            default: return launch_one<64, kEpiF32>(a, b, g, s);
        }
    }
    switch (mode) {
        case kEpiBiasF32: return launch_one<128, kEpiBiasF32>(a, b, g, s);
        case kEpiGelu: return launch_one<128, kEpiGelu>(a, b, g, s);
        case kEpiGeluGrad: return launch_one<128, kEpiGeluGrad>(a, b, g, s);
        default: return launch_one<128, kEpiF32>(a, b, g, s);
    }
}

cudaError_t launch_input(const float *x, const int32_t *rows, int B, int n_in, int ld, const float *shift,
                         const float *scale, __nv_bfloat16 *xb, __nv_bfloat16 *xt, cudaStream_t s) {
    const int64_t n = (int64_t)B * ld;
    input_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(x, rows, B, n_in, ld, shift, scale, xb, xt);
    return cudaGetLastError();
}

cudaError_t launch_loss(const float *y, const float *t, const int32_t *rows, int B, int N, __nv_bfloat16 *dy,
                        __nv_bfloat16 *dyt, double *partials, float *loss, cudaStream_t s) {
    loss_kernel<<<kLossBlocks, 256, 0, s>>>(y, t, rows, B, N, dy, dyt, partials);
    loss_final_kernel<<<1, 32, 0, s>>>(partials, kLossBlocks, loss);
    return cudaGetLastError();
}

cudaError_t launch_bias_grad(const __nv_bfloat16 *dzt, int B, int N, float *db, cudaStream_t s) {
    bias_grad_kernel<<<(N + 7) / 8, 256, 0, s>>>(dzt, B, N, db);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *w, float *m, float *v, const float *grad, int64_t n, float lr, float b1, float b2,
                        float eps, float bc1, float bc2, int N, int K, int ld, __nv_bfloat16 *wb, __nv_bfloat16 *wt,
                        cudaStream_t s, const float *bc) {
    adam_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(w, m, v, grad, n, lr, b1, b2, eps, bc1, bc2, bc, N, K, ld, wb,
                                                       wt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// device step counter of Adam, and the surrogate's data kernels
// ---------------------------------------------------------------------------
// t += 1; bc = (1 - 0.9^t, 1 - 0.999^t, lr_t) in FP64 like the host path, with the learning
// rate lr_t = lr_end + (lr - lr_end) (1 + cos(pi min(t - 1, n_decay) / n_decay)) / 2 over
// n_decay steps (cosine decay; n_decay <= 0: constant lr)
__global__ void adam_tick_kernel(int64_t *t, float *bc, float lr, float lr_end, int64_t n_decay) {
    const int64_t n = ++*t;
    bc[0] = (float)(1.0 - pow(0.9, (double)n));
    bc[1] = (float)(1.0 - pow(0.999, (double)n));
    if (n_decay > 0) {
        const double x = (double)min(n - 1, n_decay) / (double)n_decay;
        bc[2] = (float)(lr_end + (lr - lr_end) * 0.5 * (1.0 + cospi(x)));
    } else {
        bc[2] = lr;
    }
}
cudaError_t launch_adam_tick(int64_t *t, float *bc, float lr, float lr_end, int64_t n_decay, cudaStream_t s) {
    adam_tick_kernel<<<1, 1, 0, s>>>(t, bc, lr, lr_end, n_decay);
    return cudaGetLastError();
}

// z[i][j] = (y[i][j] - T_ref) / (x[i][power_col] inv_Pref) for j < n_T, else y[i][j]
__global__ void sur_transform_kernel(const float *__restrict__ x, int ld_x, const float *__restrict__ y, int64_t n,
                                     int n_out, int n_T, int power_col, float T_ref, float inv_Pref, float *z) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * n_out;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / n_out;
        const int j = (int)(i % n_out);
        const float v = y[i];
        z[i] = (j < n_T && power_col >= 0) ? (v - T_ref) / (x[r * ld_x + power_col] * inv_Pref) : v;
    }
}
// column means and centred sums of squares over n rows (FP64, rows in order), one thread per column
__global__ void column_stats_kernel(const float *__restrict__ z, int64_t n, int n_out, double *mean, double *m2) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_out) return;
    double s = 0.0;
    for (int64_t r = 0; r < n; r++) s += (double)z[r * n_out + j];
    const double mu = s / (double)n;
    double q = 0.0;
    for (int64_t r = 0; r < n; r++) {
        const double d = (double)z[r * n_out + j] - mu;
        q += d * d;
    }
    mean[j] = mu;
    m2[j] = q;
}
__global__ void standardize_kernel(float *z, int64_t n, int n_out, const float *__restrict__ shift,
                                   const float *__restrict__ scale) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * n_out;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % n_out);
        z[i] = (z[i] - shift[j]) / scale[j];
    }
}
// err[r] = max over j < n_cmp of |a[r][j] - b[r][j]|; one block per row
__global__ void row_max_abs_diff_kernel(const float *__restrict__ a, const float *__restrict__ b, int n_out, int n_cmp,
                                        float *err) {
    const int64_t r = blockIdx.x;
    float m = 0.f;
    for (int j = threadIdx.x; j < n_cmp; j += blockDim.x) m = fmaxf(m, fabsf(a[r * n_out + j] - b[r * n_out + j]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float q = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) q = fmaxf(q, red[w]);
        err[r] = q;
    }
}
// out = mean of losses[0..k) (FP64 sum in order)
__global__ void mean_losses_kernel(const float *losses, int k, float *out) {
    double s = 0.0;
    for (int i = 0; i < k; i++) s += losses[i];
    *out = (float)(s / k);
}

// Input features of the surrogate: v = (x - shift) * scale for every raw column, then
// for every column j in enc_cols and octave f < n_freq the pair sin(pi 2^f v_j),
// cos(pi 2^f v_j); rows [n, n_rows) (padding) are zero.  feat [n_rows][n_feat].
__global__ void sur_encode_kernel(const float *__restrict__ x, int ld_x, int64_t n, int64_t n_rows, int n_in,
                                  const float *__restrict__ shift, const float *__restrict__ scale, int n_freq,
                                  unsigned enc_cols, int n_feat, float *feat) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rows * n_feat;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / n_feat;
        const int c = (int)(i % n_feat);
        float out = 0.f;
        if (r < n) {
            if (c < n_in) {
                out = (x[r * ld_x + c] - shift[c]) * scale[c];
            } else {
                int k = (c - n_in) >> 1;  // which (column, octave) pair
                const bool cosine = ((c - n_in) & 1) != 0;
                int j = 0;
                for (; j < n_in; j++)
                    if (enc_cols & (1u << j)) {
                        if (k < n_freq) break;
                        k -= n_freq;
                    }
                const float v = (x[r * ld_x + j] - shift[j]) * scale[j];
                float sv, cv;
                sincospif(ldexpf(v, k), &sv, &cv);
                out = cosine ? cv : sv;
            }
        }
        feat[i] = out;
    }
}
cudaError_t launch_sur_encode(const float *x, int ld_x, int64_t n, int64_t n_rows, int n_in, const float *shift,
                              const float *scale, int n_freq, unsigned enc_cols, int n_feat, float *feat,
                              cudaStream_t s) {
    sur_encode_kernel<<<592, 256, 0, s>>>(x, ld_x, n, n_rows, n_in, shift, scale, n_freq, enc_cols, n_feat, feat);
    return cudaGetLastError();
}

// Augmented rows under n_sym symmetries: row g n + i of the augmented set is symmetry g
// applied to data row i: x'[j] = a[g][j] x[i][src[g][j]] + b[g][j], y'[o] = y[i][perm[g][o]].
__global__ void sur_augment_x_kernel(const float *__restrict__ x, int64_t n, int n_in, int n_sym,
                                     const int32_t *__restrict__ src, const float *__restrict__ a,
                                     const float *__restrict__ b, float *xa) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)n_sym * n * n_in;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(q % n_in);
        const int64_t r = q / n_in;
        const int g = (int)(r / n);
        const int64_t i = r % n;
        const int k = g * n_in + j;
        xa[q] = a[k] * x[i * n_in + src[k]] + b[k];
    }
}
__global__ void sur_augment_y_kernel(const float *__restrict__ y, int64_t n, int n_out, int n_sym,
                                     const int32_t *__restrict__ perm, float *ya) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)n_sym * n * n_out;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(q % n_out);
        const int64_t r = q / n_out;
        const int g = (int)(r / n);
        const int64_t i = r % n;
        ya[q] = y[i * n_out + perm[(int64_t)g * n_out + o]];
    }
}
cudaError_t launch_sur_augment(const float *x, const float *y, int64_t n, int n_in, int n_out, int n_sym,
                               const int32_t *src, const float *a, const float *b, const int32_t *perm, float *xa,
                               float *ya, cudaStream_t s) {
    sur_augment_x_kernel<<<592, 256, 0, s>>>(x, n, n_in, n_sym, src, a, b, xa);
    sur_augment_y_kernel<<<2368, 256, 0, s>>>(y, n, n_out, n_sym, perm, ya);
    return cudaGetLastError();
}

cudaError_t launch_sur_transform(const float *x, int ld_x, const float *y, int64_t n, int n_out, int n_T,
                                 int power_col, float T_ref, float inv_Pref, float *z, cudaStream_t s) {
    sur_transform_kernel<<<1184, 256, 0, s>>>(x, ld_x, y, n, n_out, n_T, power_col, T_ref, inv_Pref, z);
    return cudaGetLastError();
}
cudaError_t launch_column_stats(const float *z, int64_t n, int n_out, double *mean, double *m2, cudaStream_t s) {
    column_stats_kernel<<<(n_out + 127) / 128, 128, 0, s>>>(z, n, n_out, mean, m2);
    return cudaGetLastError();
}
cudaError_t launch_standardize(float *z, int64_t n, int n_out, const float *shift, const float *scale,
                               cudaStream_t s) {
    standardize_kernel<<<1184, 256, 0, s>>>(z, n, n_out, shift, scale);
    return cudaGetLastError();
}
cudaError_t launch_row_max_abs_diff(const float *a, const float *b, int64_t n, int n_out, int n_cmp, float *err,
                                    cudaStream_t s) {
    if (n > 0) row_max_abs_diff_kernel<<<(unsigned)n, 256, 0, s>>>(a, b, n_out, n_cmp, err);
    return cudaGetLastError();
}
cudaError_t launch_mean_losses(const float *losses, int k, float *out, cudaStream_t s) {
    mean_losses_kernel<<<1, 1, 0, s>>>(losses, k, out);
    return cudaGetLastError();
}

cudaError_t launch_ensemble(const EnsembleArgs &e, int B, cudaStream_t s) {
    if (B > 0) ensemble_kernel<<<B, 256, 0, s>>>(e);
    return cudaGetLastError();
}

cudaError_t launch_gather_grad(const float *G, const float *db, int N, int K, int ld, float *grad, cudaStream_t s) {
    const int64_t n = (int64_t)N * K + N;
    gather_grad_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(G, db, N, K, ld, grad);
    return cudaGetLastError();
}

}  // namespace tmlp
