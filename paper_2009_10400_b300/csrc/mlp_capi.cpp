// C ABI of the surrogate MLP (include/tled_mlp.h): parameters, workspace
// layout, tensor maps, and the forward / backward / Adam sequences built from
// the tcgen05 GEMM and the elementwise kernels of mlp_kernels.cu.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/tled_mlp.h"
#include "mlp_internal.h"

using namespace tmlp;

namespace {

struct Layer {
    int K = 0, Kp = 0, N = 0;  // inputs (padded to 64), outputs
    int64_t poff = 0;          // offset of W [N][K] then b [N] in the parameter vector
    size_t wb = 0, wt = 0, G = 0, db = 0, z = 0, a = 0, at = 0, dz = 0, dzt = 0;  // workspace offsets
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

}  // namespace

struct tled_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int L = 0, Bmax = 0;
    int n_sm = 148;  // multiprocessors of the device (tile-width choice)
    std::vector<Layer> layer;
    int64_t n_params = 0;
    size_t p_w = 0, p_m = 0, p_v = 0, p_g = 0, x_b = 0, x_t = 0, y = 0, loss_part = 0, loss = 0, status = 0, total = 0;
    size_t in_shift = 0, in_scale = 0;  // input affine map (x - shift) * scale, [n_in] each
    bool has_scaling = false;
    char *ws = nullptr;
    bool inited = false;
    int64_t adam_t = 0;
    // tensor maps of the workspace operands, keyed by (address, rows, cols, box rows): every
    // GEMM operand lives at a fixed workspace offset, so each map is encoded once
    std::map<std::tuple<uintptr_t, int, int, int>, CUtensorMap> maps;
};

namespace {

int fail(tled_mlp *m, int code, const std::string &s) {
    if (m) m->err = s;
    return code;
}
#define MCUDA(m, expr)                                                                             \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e != cudaSuccess) return fail(m, TLED_E_CUDA, std::string(#expr ": ") + cudaGetErrorString(_e)); \
    } while (0)

template <class T>
T *P(tled_mlp *m, size_t off) {
    return reinterpret_cast<T *>(m->ws + off);
}

int get_encoder(tled_mlp *m) {
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode ? TLED_OK : fail(m, TLED_E_CUDA, "cuTensorMapEncodeTiled unavailable");
}

// tensor map of a row-major bf16 matrix [rows][cols], boxes of box_rows x 64 (128-byte swizzle)
int make_map(tled_mlp *m, CUtensorMap *map, const void *base, int rows, int cols, int box_rows) {
    const auto key = std::make_tuple((uintptr_t)base, rows, cols, box_rows);
    auto it = m->maps.find(key);
    if (it != m->maps.end()) {
        *map = it->second;
        return TLED_OK;
    }
    if (int rc = get_encoder(m)) return rc;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(m, TLED_E_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    m->maps[key] = *map;
    return TLED_OK;
}

// D[M][N] = A[M][K] B[N][K]^T with the given epilogue
int gemm(tled_mlp *m, const void *A, const void *B, int M, int N, int K, GemmArgs g, int mode) {
    // 128-wide N tiles, or 64-wide when the 128-wide grid would leave SMs without two CTAs
    const int bn = (N % 128 == 0 && (int64_t)(M / 128) * (N / 128) >= 2 * m->n_sm) ? 128 : 64;
    CUtensorMap ta, tb;
    if (int rc = make_map(m, &ta, A, M, K, 128)) return rc;
    if (int rc = make_map(m, &tb, B, N, K, bn)) return rc;
    g.M = M;
    g.N = N;
    g.K = K;
    g.status = P<unsigned>(m, m->status);
    MCUDA(m, launch_gemm(ta, tb, g, bn, mode, m->stream));
    return TLED_OK;
}

int check_batch(tled_mlp *m, int B) {
    if (B <= 0 || B > m->Bmax || B % 128) return fail(m, TLED_E_ARG, "batch must be a positive multiple of 128 up to max_batch");
    return TLED_OK;
}

int forward(tled_mlp *m, const float *x, const int32_t *rows, int B, float *y) {
    const Layer &l0 = m->layer[0];
    const float *sh = m->has_scaling ? P<float>(m, m->in_shift) : nullptr;
    const float *sc = m->has_scaling ? P<float>(m, m->in_scale) : nullptr;
    MCUDA(m, launch_input(x, rows, B, l0.K, l0.Kp, sh, sc, P<__nv_bfloat16>(m, m->x_b), P<__nv_bfloat16>(m, m->x_t),
                          m->stream));
    for (int l = 0; l < m->L; l++) {
        const Layer &ly = m->layer[l];
        const void *Ain = l == 0 ? (const void *)P<char>(m, m->x_b) : (const void *)P<char>(m, m->layer[l - 1].a);
        GemmArgs g{};
        g.bias = P<float>(m, m->p_w) + ly.poff + (int64_t)ly.N * ly.K;
        if (l < m->L - 1) {
            g.z_out = P<float>(m, ly.z);
            g.ld_z = ly.N;
            g.out_bf = P<__nv_bfloat16>(m, ly.a);
            g.ld_bf = ly.N;
            g.out_bfT = P<__nv_bfloat16>(m, ly.at);
            g.ld_bfT = B;
            if (int rc = gemm(m, Ain, P<char>(m, ly.wb), B, ly.N, ly.Kp, g, kEpiGelu)) return rc;
        } else {
            g.out_f32 = y;
            g.ld_f32 = ly.N;
            if (int rc = gemm(m, Ain, P<char>(m, ly.wb), B, ly.N, ly.Kp, g, kEpiBiasF32)) return rc;
        }
    }
    return TLED_OK;
}

// gradients of the mean squared error into p_g (and the loss into `loss`)
int backward(tled_mlp *m, const float *t, const int32_t *rows, int B, float *loss) {
    const Layer &last = m->layer[m->L - 1];
    MCUDA(m, launch_loss(P<float>(m, m->y), t, rows, B, last.N, P<__nv_bfloat16>(m, last.dz), P<__nv_bfloat16>(m, last.dzt),
                         P<double>(m, m->loss_part), loss ? loss : P<float>(m, m->loss), m->stream));
    for (int l = m->L - 1; l >= 0; l--) {
        const Layer &ly = m->layer[l];
        const void *At = l == 0 ? (const void *)P<char>(m, m->x_t) : (const void *)P<char>(m, m->layer[l - 1].at);
        GemmArgs g{};
        g.out_f32 = P<float>(m, ly.G);
        g.ld_f32 = ly.Kp;
        // dW[N][Kp] = dZ^T[N][B] * (A_prev^T[Kp][B])^T
        if (int rc = gemm(m, P<char>(m, ly.dzt), At, ly.N, ly.Kp, B, g, kEpiF32)) return rc;
        MCUDA(m, launch_bias_grad(P<__nv_bfloat16>(m, ly.dzt), B, ly.N, P<float>(m, ly.db), m->stream));
        MCUDA(m, launch_gather_grad(P<float>(m, ly.G), P<float>(m, ly.db), ly.N, ly.K, ly.Kp,
                                    P<float>(m, m->p_g) + ly.poff, m->stream));
        if (l > 0) {
            const Layer &pv = m->layer[l - 1];
            GemmArgs h{};
            h.z_in = P<float>(m, pv.z);
            h.ld_z = pv.N;
            h.out_bf = P<__nv_bfloat16>(m, pv.dz);
            h.ld_bf = pv.N;
            h.out_bfT = P<__nv_bfloat16>(m, pv.dzt);
            h.ld_bfT = B;
            // dA_prev[B][Kp] = dZ[B][N] * (W^T[Kp][N])^T, times GELU'(Z_prev)
            if (int rc = gemm(m, P<char>(m, ly.dz), P<char>(m, ly.wt), B, ly.Kp, ly.N, h, kEpiGeluGrad)) return rc;
        }
    }
    return TLED_OK;
}

// refresh the bf16 weights and their transposes from the FP32 master copy
int refresh_bf16(tled_mlp *m) {
    // an Adam step with zero learning rate and zero moments only rewrites the bf16 copies
    for (int l = 0; l < m->L; l++) {
        const Layer &ly = m->layer[l];
        const int64_t n = (int64_t)ly.N * ly.K + ly.N;
        MCUDA(m, launch_adam(P<float>(m, m->p_w) + ly.poff, P<float>(m, m->p_m) + ly.poff,
                             P<float>(m, m->p_v) + ly.poff, P<float>(m, m->p_g) + ly.poff, n, 0.f, 1.f, 1.f, 1.f,
                             1.f, 1.f, ly.N, ly.K, ly.Kp, P<__nv_bfloat16>(m, ly.wb), P<__nv_bfloat16>(m, ly.wt),
                             m->stream));
    }
    return TLED_OK;
}

}  // namespace

extern "C" {

int tled_mlp_create(tled_mlp **out, int device, void *stream, int32_t n_layers, const int32_t *dims, int32_t max_batch) {
    if (!out || !dims || n_layers < 1 || n_layers > 16) return TLED_E_ARG;
    *out = nullptr;
    if (max_batch <= 0 || max_batch % 128) return TLED_E_ARG;
    for (int i = 0; i <= n_layers; i++)
        if (dims[i] <= 0) return TLED_E_ARG;
    for (int i = 1; i <= n_layers; i++)
        if (dims[i] % 128) return TLED_E_ARG;  // layer widths and outputs: multiples of 128
    tled_mlp *m = new tled_mlp();
    m->device = device;
    if (cudaDeviceGetAttribute(&m->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) m->n_sm = 148;
    m->stream = (cudaStream_t)stream;
    m->L = n_layers;
    m->Bmax = max_batch;
    m->layer.resize(n_layers);
    int64_t po = 0;
    for (int l = 0; l < n_layers; l++) {
        Layer &ly = m->layer[l];
        ly.K = dims[l];
        ly.Kp = (dims[l] + 63) / 64 * 64;
        ly.N = dims[l + 1];
        ly.poff = po;
        po += (int64_t)ly.N * ly.K + ly.N;
    }
    m->n_params = po;
    // workspace layout
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off = al256(off + std::max<size_t>(b, 1));
        return o;
    };
    const size_t np = (size_t)po, B = (size_t)max_batch;
    m->p_w = take(4 * np);
    m->p_m = take(4 * np);
    m->p_v = take(4 * np);
    m->p_g = take(4 * np);
    m->x_b = take(2 * B * m->layer[0].Kp);
    m->x_t = take(2 * B * m->layer[0].Kp);
    for (auto &ly : m->layer) {
        ly.wb = take(2 * (size_t)ly.N * ly.Kp);
        ly.wt = take(2 * (size_t)ly.N * ly.Kp);
        ly.G = take(4 * (size_t)ly.N * ly.Kp);
        ly.db = take(4 * (size_t)ly.N);
        ly.z = take(4 * B * ly.N);
        ly.a = take(2 * B * ly.N);
        ly.at = take(2 * B * ly.N);
        ly.dz = take(2 * B * ly.N);
        ly.dzt = take(2 * B * ly.N);
    }
    m->y = take(4 * B * m->layer.back().N);
    m->loss_part = take(8 * kLossBlocks);
    m->loss = take(8);
    m->status = take(16);
    m->in_shift = take(4 * (size_t)m->layer[0].K);
    m->in_scale = take(4 * (size_t)m->layer[0].K);
    m->total = off;
    *out = m;
    return TLED_OK;
}

int tled_mlp_destroy(tled_mlp *m) {
    delete m;
    return TLED_OK;
}

const char *tled_mlp_last_error(const tled_mlp *m) { return m ? m->err.c_str() : "null context"; }

int tled_mlp_num_params(tled_mlp *m, int64_t *n) {
    if (!m || !n) return TLED_E_ARG;
    *n = m->n_params;
    return TLED_OK;
}

int tled_mlp_workspace_size(tled_mlp *m, int64_t *bytes) {
    if (!m || !bytes) return TLED_E_ARG;
    *bytes = (int64_t)m->total;
    return TLED_OK;
}

int tled_mlp_init(tled_mlp *m, void *ws, int64_t bytes) {
    if (!m) return TLED_E_ARG;
    if (!ws || ((uintptr_t)ws & 255)) return fail(m, TLED_E_ARG, "workspace must be 256-byte aligned");
    if (bytes < (int64_t)m->total) return fail(m, TLED_E_NOMEM, "workspace smaller than tled_mlp_workspace_size()");
    MCUDA(m, cudaSetDevice(m->device));
    m->ws = (char *)ws;
    m->maps.clear();  // the maps point into the previous workspace
    MCUDA(m, cudaMemsetAsync(m->ws, 0, m->total, m->stream));
    MCUDA(m, cudaStreamSynchronize(m->stream));
    m->inited = true;
    m->adam_t = 0;
    m->has_scaling = false;
    return TLED_OK;
}

int tled_mlp_set_params(tled_mlp *m, const float *params) {
    if (!m || !params) return fail(m, TLED_E_ARG, "NULL parameters");
    if (!m->inited) return fail(m, TLED_E_STATE, "call tled_mlp_init first");
    MCUDA(m, cudaSetDevice(m->device));
    MCUDA(m, cudaMemcpyAsync(m->ws + m->p_w, params, 4 * m->n_params, cudaMemcpyHostToDevice, m->stream));
    MCUDA(m, cudaMemsetAsync(m->ws + m->p_m, 0, 4 * m->n_params, m->stream));
    MCUDA(m, cudaMemsetAsync(m->ws + m->p_v, 0, 4 * m->n_params, m->stream));
    m->adam_t = 0;
    if (int rc = refresh_bf16(m)) return rc;
    MCUDA(m, cudaStreamSynchronize(m->stream));
    return TLED_OK;
}

int tled_mlp_set_input_scaling(tled_mlp *m, const float *shift, const float *scale) {
    if (!m) return TLED_E_ARG;
    if (!m->inited) return fail(m, TLED_E_STATE, "call tled_mlp_init first");
    if (!shift != !scale) return fail(m, TLED_E_ARG, "give both shift and scale, or neither");
    MCUDA(m, cudaSetDevice(m->device));
    if (!shift) {
        m->has_scaling = false;
        return TLED_OK;
    }
    const int n = m->layer[0].K;
    for (int k = 0; k < n; k++)
        if (!std::isfinite(shift[k]) || !std::isfinite(scale[k])) return fail(m, TLED_E_ARG, "non-finite scaling");
    MCUDA(m, cudaMemcpyAsync(m->ws + m->in_shift, shift, 4 * (size_t)n, cudaMemcpyHostToDevice, m->stream));
    MCUDA(m, cudaMemcpyAsync(m->ws + m->in_scale, scale, 4 * (size_t)n, cudaMemcpyHostToDevice, m->stream));
    MCUDA(m, cudaStreamSynchronize(m->stream));  // the host arrays may go away
    m->has_scaling = true;
    return TLED_OK;
}

int tled_mlp_set_stream(tled_mlp *m, void *stream) {
    if (!m) return TLED_E_ARG;
    m->stream = (cudaStream_t)stream;
    return TLED_OK;
}

int tled_mlp_ensemble(int device, void *stream, int32_t n_members, const float *const *y, int32_t B, int32_t n_out,
                      const float *out_scale, const float *out_shift, const float *row_src, int32_t row_stride,
                      float row_mult, int32_t n_row_scaled, const float *out_offset, int32_t n_spread, float tol,
                      float *mean, float *std, float *spread, uint8_t *fallback) {
    if (n_out % 4 || ((uintptr_t)mean & 15) || ((uintptr_t)std & 15)) return TLED_E_ARG;  // float4 rows
    if (n_members < 1 || n_members > kMaxMembers || !y || B < 0 || n_out < 1 || n_spread < 0 || n_spread > n_out ||
        std::isnan(tol) || n_row_scaled < 0 || n_row_scaled > n_out || (row_src && row_stride < 1) ||
        !std::isfinite(row_mult))
        return TLED_E_ARG;
    EnsembleArgs e{};
    for (int k = 0; k < n_members; k++) {
        if (!y[k] || ((uintptr_t)y[k] & 15)) return TLED_E_ARG;
        e.y[k] = y[k];
    }
    e.n_members = n_members;
    e.n_out = n_out;
    e.n_spread = n_spread;
    e.scale = out_scale;
    e.shift = out_shift;
    e.row_src = row_src;
    e.row_stride = row_stride;
    e.row_mult = row_mult;
    e.n_row_scaled = row_src ? n_row_scaled : 0;
    e.offset = out_offset;
    e.tol = tol;
    e.mean = mean;
    e.std = std;
    e.spread = spread;
    e.fallback = fallback;
    if (cudaSetDevice(device) != cudaSuccess) return TLED_E_CUDA;
    return launch_ensemble(e, B, (cudaStream_t)stream) == cudaSuccess ? TLED_OK : TLED_E_CUDA;
}

int tled_mlp_get_params(tled_mlp *m, float *params) {
    if (!m || !params) return fail(m, TLED_E_ARG, "NULL parameters");
    if (!m->inited) return fail(m, TLED_E_STATE, "call tled_mlp_init first");
    MCUDA(m, cudaSetDevice(m->device));
    MCUDA(m, cudaMemcpyAsync(params, m->ws + m->p_w, 4 * m->n_params, cudaMemcpyDeviceToHost, m->stream));
    MCUDA(m, cudaStreamSynchronize(m->stream));
    return TLED_OK;
}

int tled_mlp_forward(tled_mlp *m, const float *x, int32_t B, float *y) {
    if (!m || !x || !y) return fail(m, TLED_E_ARG, "NULL argument");
    if (!m->inited) return fail(m, TLED_E_STATE, "call tled_mlp_init first");
    if (int rc = check_batch(m, B)) return rc;
    MCUDA(m, cudaSetDevice(m->device));
    return forward(m, x, nullptr, B, y);
}

int tled_mlp_gradients(tled_mlp *m, const float *x, const float *t, int32_t B, float *grad, float *loss) {
    if (!m || !x || !t) return fail(m, TLED_E_ARG, "NULL argument");
    if (!m->inited) return fail(m, TLED_E_STATE, "call tled_mlp_init first");
    if (int rc = check_batch(m, B)) return rc;
    MCUDA(m, cudaSetDevice(m->device));
    if (int rc = forward(m, x, nullptr, B, P<float>(m, m->y))) return rc;
    if (int rc = backward(m, t, nullptr, B, loss)) return rc;
    if (grad) MCUDA(m, cudaMemcpyAsync(grad, m->ws + m->p_g, 4 * m->n_params, cudaMemcpyDeviceToDevice, m->stream));
    return TLED_OK;
}

int tled_mlp_train_step(tled_mlp *m, const float *x, const float *t, int32_t B, float lr, float *loss) {
    return tled_mlp_train_step_rows(m, x, t, nullptr, B, lr, loss);
}

int tled_mlp_train_step_rows(tled_mlp *m, const float *x, const float *t, const int32_t *rows, int32_t B, float lr,
                             float *loss) {
    if (!m || !x || !t) return fail(m, TLED_E_ARG, "NULL argument");
    if (!m->inited) return fail(m, TLED_E_STATE, "call tled_mlp_init first");
    if (int rc = check_batch(m, B)) return rc;
    if (!(lr > 0) || !std::isfinite(lr)) return fail(m, TLED_E_ARG, "learning rate must be positive");
    MCUDA(m, cudaSetDevice(m->device));
    if (int rc = forward(m, x, rows, B, P<float>(m, m->y))) return rc;
    if (int rc = backward(m, t, rows, B, loss)) return rc;
    m->adam_t++;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)m->adam_t));
    const float bc2 = (float)(1.0 - std::pow(0.999, (double)m->adam_t));
    for (int l = 0; l < m->L; l++) {
        const Layer &ly = m->layer[l];
        const int64_t n = (int64_t)ly.N * ly.K + ly.N;
        MCUDA(m, launch_adam(P<float>(m, m->p_w) + ly.poff, P<float>(m, m->p_m) + ly.poff,
                             P<float>(m, m->p_v) + ly.poff, P<float>(m, m->p_g) + ly.poff, n, lr, b1, b2, eps, bc1,
                             bc2, ly.N, ly.K, ly.Kp, P<__nv_bfloat16>(m, ly.wb), P<__nv_bfloat16>(m, ly.wt),
                             m->stream));
    }
    return TLED_OK;
}

int tled_mlp_sync(tled_mlp *m) {
    if (!m) return TLED_E_ARG;
    if (!m->inited) return fail(m, TLED_E_STATE, "call tled_mlp_init first");
    MCUDA(m, cudaSetDevice(m->device));
    MCUDA(m, cudaStreamSynchronize(m->stream));
    unsigned st = 0;
    MCUDA(m, cudaMemcpy(&st, m->ws + m->status, 4, cudaMemcpyDeviceToHost));
    if (st) return fail(m, TLED_E_TIMEOUT, "a tensor-core pipeline wait timed out");
    return TLED_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// internal entries for the surrogate engine (sur_capi.cpp)
// ---------------------------------------------------------------------------
int tmlp_train_step_graphable(tled_mlp *m, cudaStream_t stream, const float *x, const float *t, const int32_t *rows,
                              int B, float lr, float lr_end, int64_t n_decay, float *loss, int64_t *t_dev,
                              float *bc_dev) {
    if (!m || !x || !t || !t_dev || !bc_dev) return fail(m, TLED_E_ARG, "NULL argument");
    if (!m->inited) return fail(m, TLED_E_STATE, "call tled_mlp_init first");
    if (int rc = check_batch(m, B)) return rc;
    cudaStream_t keep = m->stream;
    m->stream = stream;
    int rc = forward(m, x, rows, B, P<float>(m, m->y));
    if (!rc) rc = backward(m, t, rows, B, loss);
    if (!rc) {
        cudaError_t e = launch_adam_tick(t_dev, bc_dev, lr, lr_end, n_decay, stream);
        for (int l = 0; l < m->L && e == cudaSuccess; l++) {
            const Layer &ly = m->layer[l];
            const int64_t n = (int64_t)ly.N * ly.K + ly.N;
            e = launch_adam(P<float>(m, m->p_w) + ly.poff, P<float>(m, m->p_m) + ly.poff, P<float>(m, m->p_v) + ly.poff,
                            P<float>(m, m->p_g) + ly.poff, n, lr, 0.9f, 0.999f, 1e-8f, 1.f, 1.f, ly.N, ly.K, ly.Kp,
                            P<__nv_bfloat16>(m, ly.wb), P<__nv_bfloat16>(m, ly.wt), stream, bc_dev);
        }
        if (e != cudaSuccess) rc = fail(m, TLED_E_CUDA, std::string("adam: ") + cudaGetErrorString(e));
    }
    m->stream = keep;
    return rc;
}

int tmlp_forward_on(tled_mlp *m, cudaStream_t stream, const float *x, int B, float *y) {
    if (!m || !x || !y) return fail(m, TLED_E_ARG, "NULL argument");
    if (!m->inited) return fail(m, TLED_E_STATE, "call tled_mlp_init first");
    if (int rc = check_batch(m, B)) return rc;
    cudaStream_t keep = m->stream;
    m->stream = stream;
    const int rc = forward(m, x, nullptr, B, y);
    m->stream = keep;
    return rc;
}
