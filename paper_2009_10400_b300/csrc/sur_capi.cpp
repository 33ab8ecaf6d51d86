// C ABI of the learned surrogate (include/tled_mlp.h, tled_sur_*): an ensemble
// of MLPs (mlp_capi.cpp) that maps scenario parameters to temperature and damage
// at probe points, trained on solver data and answering with the ensemble mean,
// its spread, and a fallback flag where the spread exceeds a tolerance.
//
// The engine owns everything between raw data and answers: the input map to
// [-1, 1] and the sin / cos features of selected inputs (source position) at
// octave frequencies, the target transform (temperature rise per unit source
// power) and its standardisation
// (column statistics on the device in FP64, scales chosen here), the seeded He
// initialisation and per-epoch row permutations (a splitmix64 generator), the
// training loop -- each member on its own stream, one CUDA graph per member
// replaying a whole epoch of Adam steps, so the members train side by side --,
// the ensemble inference, and the calibration of the spread threshold.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tled_mlp.h"
#include "mlp_internal.h"

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// splitmix64 (Steele, Lea and Flood 2014): seeds, permutations and normal deviates
struct SplitMix {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0, 1)
    uint64_t below(uint64_t n) { return next() % n; }
    double normal() {  // Box-Muller
        double u1 = uniform();
        while (u1 <= 0.0) u1 = uniform();
        const double u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

}  // namespace

struct tled_sur {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int n_members = 0, n_in = 0, n_out = 0, n_T = 0, max_batch = 0, max_epochs = 0;
    int n_freq = 0, n_feat = 0;  // input encoding: octaves, features per row
    // symmetries of the scenario family (training data augmentation), host copies
    int n_sym = 0;
    std::vector<int32_t> sym_src, sym_perm;
    std::vector<float> sym_a, sym_b;
    unsigned enc_cols = 0;       // raw input columns that get sin / cos features
    int64_t max_rows = 0;
    std::vector<int32_t> dims;
    std::vector<tled_mlp *> net;
    std::vector<cudaStream_t> ms;
    std::vector<cudaEvent_t> ev;
    std::vector<cudaGraphExec_t> graph;  // per member: one epoch of Adam steps
    int graph_steps = 0, graph_batch = 0;
    int64_t graph_rows = 0;
    const float *graph_x = nullptr;
    float graph_lr = 0.f, graph_lr_end = 0.f;
    int64_t graph_decay = 0;
    // outputs: temperature rise per unit power for the first n_T outputs (power_col >= 0)
    int power_col = -1, norm = 0;
    float P_ref = 1.f, T_ref = 0.f;
    std::vector<float> in_lo, in_hi;
    // workspace
    char *ws = nullptr;
    bool inited = false, trained = false;
    std::vector<size_t> o_net;
    size_t o_targets = 0, o_scale = 0, o_shift = 0, o_offset = 0, o_rows = 0, o_perms = 0, o_steploss = 0, o_hist = 0, o_t = 0,
           o_bc = 0, o_ys = 0, o_feat = 0, o_feat_train = 0, o_in_shift = 0, o_in_scale = 0, o_err = 0, o_mean = 0,
           o_m2 = 0, o_spread = 0, o_cmean = 0, o_xaug = 0, o_sym_src = 0, o_sym_a = 0, o_sym_b = 0, o_sym_perm = 0,
           total = 0;
    int max_sym = 0;  // symmetries the workspace holds
    int max_steps = 0;
};

namespace {

int fail(tled_sur *s, int code, const std::string &m) {
    if (s) s->err = m;
    return code;
}
#define SCUDA(s, expr)                                                                                         \
    do {                                                                                                       \
        cudaError_t _e = (expr);                                                                               \
        if (_e != cudaSuccess) return fail(s, TLED_E_CUDA, std::string(#expr ": ") + cudaGetErrorString(_e)); \
    } while (0)
#define SMLP(s, k, expr)                                                                                   \
    do {                                                                                                   \
        int _r = (expr);                                                                                   \
        if (_r != TLED_OK) return fail(s, _r, std::string("member ") + std::to_string(k) + ": " +        \
                                                  tled_mlp_last_error(s->net[k]));                         \
    } while (0)

template <class T>
T *P(tled_sur *s, size_t off) {
    return reinterpret_cast<T *>(s->ws + off);
}

void drop_graphs(tled_sur *s) {
    for (auto &g : s->graph)
        if (g) cudaGraphExecDestroy(g);
    for (auto &g : s->graph) g = nullptr;
    s->graph_steps = 0;
}

// He-normal weights (std sqrt(2 / fan-in)), zero biases, in the MLP's parameter order
std::vector<float> he_init(const std::vector<int32_t> &dims, SplitMix &rng) {
    std::vector<float> p;
    for (size_t l = 0; l + 1 < dims.size(); l++) {
        const int K = dims[l], N = dims[l + 1];
        const double sd = std::sqrt(2.0 / K);
        for (int64_t i = 0; i < (int64_t)N * K; i++) p.push_back((float)(sd * rng.normal()));
        for (int i = 0; i < N; i++) p.push_back(0.f);
    }
    return p;
}

// The largest spread threshold tau (<= tol) such that the cases with spread <=
// tau -- a prefix of the cases sorted by spread -- have err <= tol in at least a
// `coverage` fraction; -1 if no prefix qualifies.  *frac: accepted fraction.
float spread_threshold(const std::vector<float> &spread, const std::vector<float> &err, float tol, float coverage,
                       float *frac) {
    const size_t n = spread.size();
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return spread[a] < spread[b]; });
    size_t good = 0, best = 0;
    for (size_t k = 0; k < n; k++) {
        good += err[order[k]] <= tol;
        if ((double)good >= coverage * (double)(k + 1)) best = k + 1;
    }
    if (best == 0) {
        *frac = 0.f;
        return -1.f;
    }
    float tau = spread[order[best - 1]];
    if (tau > tol) {  // never accept a spread above the tolerance itself
        best = 0;
        while (best < n && spread[order[best]] <= tol) best++;
        tau = tol;
    }
    *frac = (float)best / (float)n;
    return tau;
}

int check(tled_sur *s) {
    if (!s) return TLED_E_ARG;
    if (!s->inited) return fail(s, TLED_E_STATE, "call tled_sur_init first");
    return TLED_OK;
}

// members' forward passes of raw rows x [B][n_in] (B <= max_batch, any size) side by side:
// the input features of the rows (zero rows up to the tensor-core batch, a multiple of 128)
// on the main stream, then every member on its stream, joined back into the main stream
int forward_members(tled_sur *s, const float *x, int B) {
    const int Bp = (B + 127) / 128 * 128;
    float *feat = P<float>(s, s->o_feat);
    SCUDA(s, tmlp::launch_sur_encode(x, s->n_in, B, Bp, s->n_in, P<float>(s, s->o_in_shift), P<float>(s, s->o_in_scale),
                                     s->n_freq, s->enc_cols, s->n_feat, feat, s->stream));
    SCUDA(s, cudaEventRecord(s->ev[0], s->stream));
    for (int k = 0; k < s->n_members; k++) {
        SCUDA(s, cudaStreamWaitEvent(s->ms[k], s->ev[0], 0));
        SMLP(s, k, tmlp_forward_on(s->net[k], s->ms[k], feat, Bp,
                                   P<float>(s, s->o_ys) + (size_t)k * s->max_batch * s->n_out));
        SCUDA(s, cudaEventRecord(s->ev[1 + k], s->ms[k]));
        SCUDA(s, cudaStreamWaitEvent(s->stream, s->ev[1 + k], 0));
    }
    return TLED_OK;
}

int ensemble(tled_sur *s, const float *x, int B, int n_spread, float tol, float *mean, float *std, float *spread,
             uint8_t *fb) {
    std::vector<const float *> ys(s->n_members);
    for (int k = 0; k < s->n_members; k++) ys[k] = P<float>(s, s->o_ys) + (size_t)k * s->max_batch * s->n_out;
    const bool pp = s->power_col >= 0;
    return tled_mlp_ensemble(s->device, s->stream, s->n_members, ys.data(), B, s->n_out, P<float>(s, s->o_scale),
                             P<float>(s, s->o_shift), pp ? x + s->power_col : nullptr, s->n_in, 1.f / s->P_ref,
                             pp ? s->n_T : 0, P<float>(s, s->o_offset), n_spread, tol, mean, std, spread, fb);
}

}  // namespace

extern "C" {

int tled_sur_create(tled_sur **out, int device, void *stream, int32_t n_members, int32_t n_in, int32_t width,
                    int32_t depth, int32_t n_out, int32_t n_T, int32_t max_batch, int64_t max_rows,
                    int32_t max_epochs, int32_t n_freq, uint32_t enc_cols, int32_t max_sym) {
    if (!out) return TLED_E_ARG;
    *out = nullptr;
    if (n_members < 1 || n_members > tmlp::kMaxMembers || n_in < 1 || n_in > 32 || width < 128 || width % 128 ||
        depth < 2 || n_out < 128 || n_out % 128 || n_T < 0 || n_T > n_out || max_batch < 128 || max_batch % 128 ||
        max_rows < max_batch || max_epochs < 1 || n_freq < 0 || n_freq > 12 || (n_in < 32 && (enc_cols >> n_in)) ||
        max_sym < 0 || max_sym > 64)
        return TLED_E_ARG;
    tled_sur *s = new tled_sur;
    s->device = device;
    s->stream = static_cast<cudaStream_t>(stream);
    s->n_members = n_members;
    s->n_in = n_in;
    s->n_out = n_out;
    s->n_T = n_T;
    s->max_batch = max_batch;
    s->max_rows = max_rows;
    s->max_epochs = max_epochs;
    s->max_sym = max_sym;
    s->n_freq = n_freq;
    s->enc_cols = n_freq > 0 ? enc_cols : 0u;
    s->n_feat = n_in + 2 * n_freq * __builtin_popcount(s->enc_cols);
    s->dims.push_back(s->n_feat);
    for (int l = 0; l < depth - 1; l++) s->dims.push_back(width);
    s->dims.push_back(n_out);
    if (cudaSetDevice(device) != cudaSuccess) {
        delete s;
        return TLED_E_CUDA;
    }
    for (int k = 0; k < n_members; k++) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            tled_sur_destroy(s);
            return TLED_E_CUDA;
        }
        s->ms.push_back(st);
        tled_mlp *m = nullptr;
        const int rc = tled_mlp_create(&m, device, st, (int32_t)s->dims.size() - 1, s->dims.data(), max_batch);
        if (rc) {
            tled_sur_destroy(s);
            return rc;
        }
        s->net.push_back(m);
    }
    for (int k = 0; k <= n_members; k++) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            tled_sur_destroy(s);
            return TLED_E_CUDA;
        }
        s->ev.push_back(e);
    }
    s->graph.assign(n_members, nullptr);
    *out = s;
    return TLED_OK;
}

int tled_sur_destroy(tled_sur *s) {
    if (!s) return TLED_E_ARG;
    if (s->device >= 0) cudaSetDevice(s->device);
    drop_graphs(s);
    for (auto m : s->net) tled_mlp_destroy(m);
    for (auto st : s->ms) cudaStreamDestroy(st);
    for (auto e : s->ev) cudaEventDestroy(e);
    delete s;
    return TLED_OK;
}

const char *tled_sur_last_error(const tled_sur *s) { return s ? s->err.c_str() : "null surrogate"; }

int tled_sur_workspace_size(tled_sur *s, int64_t *bytes) {
    if (!s || !bytes) return fail(s, TLED_E_ARG, "NULL argument");
    size_t off = 0;
    auto take = [&](size_t n) {
        const size_t o = off;
        off += al256(n);
        return o;
    };
    s->o_net.clear();
    for (int k = 0; k < s->n_members; k++) {
        int64_t b = 0;
        if (int rc = tled_mlp_workspace_size(s->net[k], &b)) return fail(s, rc, tled_mlp_last_error(s->net[k]));
        s->o_net.push_back(take((size_t)b));
    }
    s->max_steps = (int)(s->max_rows / 128);  // the most Adam steps of one epoch (batch >= 128)
    const size_t no = (size_t)s->n_out, nm = (size_t)s->n_members;
    s->o_targets = take(4 * (size_t)s->max_rows * no);
    s->o_scale = take(4 * no);
    s->o_shift = take(4 * no);
    s->o_offset = take(4 * no);
    s->o_rows = take(4 * nm * (size_t)s->max_rows);                      // the epoch's rows, read by the graph
    s->o_perms = take(4 * nm * (size_t)s->max_epochs * s->max_rows);     // every epoch's permutation
    s->o_steploss = take(4 * nm * (size_t)s->max_steps);
    s->o_hist = take(4 * nm * (size_t)s->max_epochs);
    s->o_t = take(8 * nm);
    s->o_bc = take(16 * nm);  // per member: bias corrections and the step's learning rate
    s->o_ys = take(4 * nm * (size_t)s->max_batch * no);
    s->o_feat = take(4 * (size_t)s->max_batch * s->n_feat);
    s->o_feat_train = take(4 * (size_t)s->max_rows * s->n_feat);
    s->o_in_shift = take(4 * (size_t)s->n_in);
    s->o_in_scale = take(4 * (size_t)s->n_in);
    s->o_err = take(4 * (size_t)s->max_batch);
    s->o_spread = take(4 * (size_t)s->max_batch);
    s->o_cmean = take(4 * (size_t)s->max_batch * no);
    s->o_mean = take(8 * no);
    s->o_m2 = take(8 * no);
    s->o_xaug = take(4 * (size_t)s->max_rows * s->n_in);  // raw inputs of the (augmented) training set
    s->o_sym_src = take(4 * (size_t)s->max_sym * s->n_in);
    s->o_sym_a = take(4 * (size_t)s->max_sym * s->n_in);
    s->o_sym_b = take(4 * (size_t)s->max_sym * s->n_in);
    s->o_sym_perm = take(4 * (size_t)s->max_sym * no);
    s->total = off;
    *bytes = (int64_t)off;
    return TLED_OK;
}

int tled_sur_init(tled_sur *s, void *dev_workspace, int64_t bytes) {
    if (!s) return TLED_E_ARG;
    int64_t need = 0;
    if (int rc = tled_sur_workspace_size(s, &need)) return rc;
    if (!dev_workspace || ((uintptr_t)dev_workspace & 255)) return fail(s, TLED_E_ARG, "workspace must be 256-byte aligned");
    if (bytes < need) return fail(s, TLED_E_NOMEM, "workspace smaller than tled_sur_workspace_size()");
    SCUDA(s, cudaSetDevice(s->device));
    drop_graphs(s);
    s->ws = static_cast<char *>(dev_workspace);
    for (int k = 0; k < s->n_members; k++) {
        int64_t b = 0;
        tled_mlp_workspace_size(s->net[k], &b);
        SMLP(s, k, tled_mlp_init(s->net[k], s->ws + s->o_net[k], b));
    }
    // identity inputs and outputs until set / trained
    std::vector<float> one(std::max(s->n_out, s->n_in), 1.f), zero(std::max(s->n_out, s->n_in), 0.f);
    SCUDA(s, cudaMemcpy(s->ws + s->o_in_shift, zero.data(), 4 * (size_t)s->n_in, cudaMemcpyHostToDevice));
    SCUDA(s, cudaMemcpy(s->ws + s->o_in_scale, one.data(), 4 * (size_t)s->n_in, cudaMemcpyHostToDevice));
    SCUDA(s, cudaMemcpy(s->ws + s->o_scale, one.data(), 4 * (size_t)s->n_out, cudaMemcpyHostToDevice));
    SCUDA(s, cudaMemcpy(s->ws + s->o_shift, zero.data(), 4 * (size_t)s->n_out, cudaMemcpyHostToDevice));
    SCUDA(s, cudaMemcpy(s->ws + s->o_offset, zero.data(), 4 * (size_t)s->n_out, cudaMemcpyHostToDevice));
    s->inited = true;
    s->trained = false;
    if (s->n_sym > 0) {
        const int ns = s->n_sym;
        std::vector<int32_t> src(s->sym_src), perm(s->sym_perm);
        std::vector<float> a(s->sym_a), b(s->sym_b);
        if (int rc = tled_sur_set_symmetries(s, ns, src.data(), a.data(), b.data(), perm.data())) return rc;
    }
    if (!s->in_lo.empty()) return tled_sur_set_inputs(s, s->in_lo.data(), s->in_hi.data());
    return TLED_OK;
}

int tled_sur_set_inputs(tled_sur *s, const float *lo, const float *hi) {
    if (int rc = check(s)) return rc;
    if (!lo || !hi) return fail(s, TLED_E_ARG, "NULL input range");
    std::vector<float> shift(s->n_in), scale(s->n_in);
    for (int i = 0; i < s->n_in; i++) {
        if (!(hi[i] > lo[i]) || !std::isfinite(lo[i]) || !std::isfinite(hi[i]))
            return fail(s, TLED_E_ARG, "input range " + std::to_string(i) + " must have hi > lo");
        shift[i] = 0.5f * (lo[i] + hi[i]);
        scale[i] = 2.f / (hi[i] - lo[i]);
    }
    s->in_lo.assign(lo, lo + s->n_in);
    s->in_hi.assign(hi, hi + s->n_in);
    SCUDA(s, cudaSetDevice(s->device));
    SCUDA(s, cudaMemcpy(s->ws + s->o_in_shift, shift.data(), 4 * (size_t)s->n_in, cudaMemcpyHostToDevice));
    SCUDA(s, cudaMemcpy(s->ws + s->o_in_scale, scale.data(), 4 * (size_t)s->n_in, cudaMemcpyHostToDevice));
    return TLED_OK;
}

int tled_sur_set_symmetries(tled_sur *s, int32_t n_sym, const int32_t *in_src, const float *in_a, const float *in_b,
                            const int32_t *out_perm) {
    if (int rc = check(s)) return rc;
    if (n_sym < 0 || n_sym > s->max_sym) return fail(s, TLED_E_ARG, "0 <= n_sym <= max_sym");
    if (n_sym > 0 && (!in_src || !in_a || !in_b || !out_perm)) return fail(s, TLED_E_ARG, "NULL symmetry table");
    const size_t ni = (size_t)n_sym * s->n_in, no = (size_t)n_sym * s->n_out;
    for (size_t q = 0; q < ni; q++)
        if (in_src[q] < 0 || in_src[q] >= s->n_in || !std::isfinite(in_a[q]) || !std::isfinite(in_b[q]))
            return fail(s, TLED_E_ARG, "symmetry input map: source column out of range or a non-finite factor");
    for (size_t q = 0; q < no; q++)
        if (out_perm[q] < 0 || out_perm[q] >= s->n_out) return fail(s, TLED_E_ARG, "symmetry output index out of range");
    s->n_sym = n_sym;
    s->sym_src.assign(in_src, in_src + ni);
    s->sym_a.assign(in_a, in_a + ni);
    s->sym_b.assign(in_b, in_b + ni);
    s->sym_perm.assign(out_perm, out_perm + no);
    if (n_sym == 0) return TLED_OK;
    SCUDA(s, cudaSetDevice(s->device));
    SCUDA(s, cudaMemcpy(s->ws + s->o_sym_src, in_src, 4 * ni, cudaMemcpyHostToDevice));
    SCUDA(s, cudaMemcpy(s->ws + s->o_sym_a, in_a, 4 * ni, cudaMemcpyHostToDevice));
    SCUDA(s, cudaMemcpy(s->ws + s->o_sym_b, in_b, 4 * ni, cudaMemcpyHostToDevice));
    SCUDA(s, cudaMemcpy(s->ws + s->o_sym_perm, out_perm, 4 * no, cudaMemcpyHostToDevice));
    s->trained = false;
    return TLED_OK;
}

int tled_sur_set_outputs(tled_sur *s, int32_t power_col, float power_ref, float T_ref, int32_t norm) {
    if (!s) return TLED_E_ARG;
    if (power_col >= s->n_in || (power_col >= 0 && !(power_ref > 0)) || (norm != 0 && norm != 1))
        return fail(s, TLED_E_ARG, "power_col < n_in with power_ref > 0, norm 0 or 1");
    s->power_col = power_col < 0 ? -1 : power_col;
    s->P_ref = power_ref;
    s->T_ref = T_ref;
    s->norm = norm;
    s->trained = false;
    return TLED_OK;
}

int tled_sur_train(tled_sur *s, const float *x, const float *y, int64_t n, int32_t epochs, int32_t batch, float lr,
                   float lr_end, int32_t bootstrap, uint64_t seed, float *loss_history) {
    if (int rc = check(s)) return rc;
    if (!x || !y) return fail(s, TLED_E_ARG, "NULL data");
    if (batch < 128 || batch % 128 || batch > s->max_batch) return fail(s, TLED_E_ARG, "batch: a multiple of 128 <= max_batch");
    const int64_t n_data = n;
    if (s->n_sym > 0) n = n_data * s->n_sym;  // the augmented set
    if (n < batch || n > s->max_rows)
        return fail(s, TLED_E_ARG, "rows: batch <= n (x n_sym with symmetries) <= max_rows");
    if (epochs < 1 || epochs > s->max_epochs) return fail(s, TLED_E_ARG, "epochs: 1..max_epochs");
    if (!(lr > 0) || !std::isfinite(lr)) return fail(s, TLED_E_ARG, "learning rate must be positive");
    if (!(lr_end >= 0) || lr_end > lr) return fail(s, TLED_E_ARG, "0 <= lr_end <= lr");
    SCUDA(s, cudaSetDevice(s->device));
    const int no = s->n_out;
    // --- the training set (augmented by the symmetries, if set), then the targets:
    //     temperature rise per unit power, then standardised
    float *z = P<float>(s, s->o_targets);
    float *xr = P<float>(s, s->o_xaug);
    if (s->n_sym > 0) {
        SCUDA(s, tmlp::launch_sur_augment(x, y, n_data, s->n_in, no, s->n_sym, P<int32_t>(s, s->o_sym_src),
                                          P<float>(s, s->o_sym_a), P<float>(s, s->o_sym_b),
                                          P<int32_t>(s, s->o_sym_perm), xr, z, s->stream));
        y = z;  // transformed in place below (elementwise)
    } else {
        SCUDA(s, cudaMemcpyAsync(xr, x, 4 * (size_t)n * s->n_in, cudaMemcpyDeviceToDevice, s->stream));
    }
    x = xr;
    SCUDA(s, tmlp::launch_sur_transform(x, s->n_in, y, n, no, s->n_T, s->power_col, s->T_ref, 1.f / s->P_ref, z,
                                        s->stream));
    SCUDA(s, tmlp::launch_column_stats(z, n, no, P<double>(s, s->o_mean), P<double>(s, s->o_m2), s->stream));
    std::vector<double> mean(no), m2(no);
    SCUDA(s, cudaMemcpyAsync(mean.data(), s->ws + s->o_mean, 8 * (size_t)no, cudaMemcpyDeviceToHost, s->stream));
    SCUDA(s, cudaMemcpyAsync(m2.data(), s->ws + s->o_m2, 8 * (size_t)no, cudaMemcpyDeviceToHost, s->stream));
    SCUDA(s, cudaStreamSynchronize(s->stream));
    // pooled standard deviation of every target entry (the floor of a column's scale)
    double gm = 0.0, ss = 0.0;
    for (int j = 0; j < no; j++) gm += mean[j];
    gm /= no;
    for (int j = 0; j < no; j++) ss += m2[j] + (double)n * (mean[j] - gm) * (mean[j] - gm);
    const double sd_all = std::sqrt(ss / ((double)n * no));
    std::vector<float> scale(no), shift(no), offset(no, 0.f);
    // norm 1: one scale per output group (temperatures [0, n_T), the rest), the root mean
    // square of the group's column deviations, so that the loss weighs physical errors alike
    double g_var[2] = {0.0, 0.0};
    int g_n[2] = {0, 0};
    for (int j = 0; j < no; j++) {
        const int g = j < s->n_T ? 0 : 1;
        g_var[g] += m2[j] / (double)n;
        g_n[g]++;
    }
    for (int j = 0; j < no; j++) {
        const int g = j < s->n_T ? 0 : 1;
        const double sd = s->norm == 1 ? std::sqrt(g_var[g] / std::max(g_n[g], 1)) : std::sqrt(m2[j] / (double)n);
        scale[j] = (float)std::max(sd, 1e-3 * std::max(sd_all, 1e-12));
        shift[j] = (float)mean[j];
        if (s->power_col >= 0 && j < s->n_T) offset[j] = s->T_ref;
    }
    SCUDA(s, cudaMemcpyAsync(s->ws + s->o_scale, scale.data(), 4 * (size_t)no, cudaMemcpyHostToDevice, s->stream));
    SCUDA(s, cudaMemcpyAsync(s->ws + s->o_shift, shift.data(), 4 * (size_t)no, cudaMemcpyHostToDevice, s->stream));
    SCUDA(s, cudaMemcpyAsync(s->ws + s->o_offset, offset.data(), 4 * (size_t)no, cudaMemcpyHostToDevice, s->stream));
    SCUDA(s, tmlp::launch_standardize(z, n, no, P<float>(s, s->o_shift), P<float>(s, s->o_scale), s->stream));
    // the members learn from the rows' input features
    float *xf = P<float>(s, s->o_feat_train);
    SCUDA(s, tmlp::launch_sur_encode(x, s->n_in, n, n, s->n_in, P<float>(s, s->o_in_shift), P<float>(s, s->o_in_scale),
                                     s->n_freq, s->enc_cols, s->n_feat, xf, s->stream));
    SCUDA(s, cudaStreamSynchronize(s->stream));  // host copies consumed; data ready for the members' streams
    // --- members: seeded He initialisation; one epoch of Adam steps captured per member
    const int steps = (int)(n / batch);
    // cosine decay from lr to lr_end over the whole run (lr_end == lr: constant)
    const int64_t n_decay = lr_end < lr ? (int64_t)steps * epochs : 0;
    const bool same_graph = s->graph_steps == steps && s->graph_batch == batch && s->graph_x == x &&
                            s->graph_rows == n && s->graph_lr == lr && s->graph_lr_end == lr_end &&
                            s->graph_decay == n_decay;
    if (!same_graph) drop_graphs(s);
    SplitMix master{seed};
    std::vector<SplitMix> rng;
    for (int k = 0; k < s->n_members; k++) rng.push_back(SplitMix{master.next()});
    std::vector<int32_t> perm(n);
    for (int k = 0; k < s->n_members; k++) {
        int32_t *rows = P<int32_t>(s, s->o_rows) + (size_t)k * s->max_rows;
        float *sl = P<float>(s, s->o_steploss) + (size_t)k * s->max_steps;
        int64_t *tk = P<int64_t>(s, s->o_t) + k;
        float *bck = P<float>(s, s->o_bc) + 4 * k;
        if (!s->graph[k]) {
            // first use of every kernel outside capture (module loading, attributes): one step
            // on the first rows, undone by the initialisation below
            for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
            SCUDA(s, cudaMemcpyAsync(rows, perm.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s->ms[k]));
            SCUDA(s, cudaMemsetAsync(tk, 0, 8, s->ms[k]));
            SMLP(s, k, tmlp_train_step_graphable(s->net[k], s->ms[k], xf, z, rows, batch, lr, lr_end, n_decay, sl, tk,
                                                 bck));
            SCUDA(s, cudaStreamSynchronize(s->ms[k]));
            cudaGraph_t g = nullptr;
            SCUDA(s, cudaStreamBeginCapture(s->ms[k], cudaStreamCaptureModeThreadLocal));
            int rc = TLED_OK;
            for (int j = 0; j < steps && rc == TLED_OK; j++)
                rc = tmlp_train_step_graphable(s->net[k], s->ms[k], xf, z, rows + (size_t)j * batch, batch, lr, lr_end,
                                               n_decay, sl + j, tk, bck);
            const cudaError_t e = cudaStreamEndCapture(s->ms[k], &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return fail(s, rc, std::string("member ") + std::to_string(k) + ": " + tled_mlp_last_error(s->net[k]));
            }
            SCUDA(s, e);
            const cudaError_t ei = cudaGraphInstantiate(&s->graph[k], g, 0);
            cudaGraphDestroy(g);
            SCUDA(s, ei);
        }
        const std::vector<float> p = he_init(s->dims, rng[k]);
        SMLP(s, k, tled_mlp_set_params(s->net[k], p.data()));  // parameters, Adam moments reset
        SCUDA(s, cudaMemsetAsync(tk, 0, 8, s->ms[k]));
        SCUDA(s, cudaStreamSynchronize(s->ms[k]));
    }
    s->graph_steps = steps;
    s->graph_batch = batch;
    s->graph_x = x;
    s->graph_rows = n;
    s->graph_lr = lr;
    s->graph_lr_end = lr_end;
    s->graph_decay = n_decay;
    // --- every member's permutations of all epochs (Fisher-Yates), uploaded once; then the
    //     epochs: each member copies its epoch's rows on the device and replays its epoch
    //     graph, the members side by side on their streams
    //     (bootstrap: member k's rows are n draws with replacement, made once, and every epoch
    //     permutes that multiset, so the members see different samples of the data)
    std::vector<int32_t> perms((size_t)epochs * n), base(n);
    for (int k = 0; k < s->n_members; k++) {
        for (int64_t i = 0; i < n; i++) base[i] = bootstrap ? (int32_t)rng[k].below((uint64_t)n) : (int32_t)i;
        for (int e = 0; e < epochs; e++) {
            int32_t *pe = perms.data() + (size_t)e * n;
            std::copy(base.begin(), base.end(), pe);
            for (int64_t i = n - 1; i > 0; i--) std::swap(pe[i], pe[rng[k].below((uint64_t)i + 1)]);
        }
        int32_t *dst = P<int32_t>(s, s->o_perms) + (size_t)k * s->max_epochs * s->max_rows;
        for (int e = 0; e < epochs; e++)
            SCUDA(s, cudaMemcpyAsync(dst + (size_t)e * s->max_rows, perms.data() + (size_t)e * n, 4 * (size_t)n,
                                     cudaMemcpyHostToDevice, s->ms[k]));
    }
    for (int e = 0; e < epochs; e++) {
        for (int k = 0; k < s->n_members; k++) {
            int32_t *rows = P<int32_t>(s, s->o_rows) + (size_t)k * s->max_rows;
            const int32_t *pe = P<int32_t>(s, s->o_perms) + ((size_t)k * s->max_epochs + e) * s->max_rows;
            SCUDA(s, cudaMemcpyAsync(rows, pe, 4 * (size_t)steps * batch, cudaMemcpyDeviceToDevice, s->ms[k]));
            SCUDA(s, cudaGraphLaunch(s->graph[k], s->ms[k]));
            SCUDA(s, tmlp::launch_mean_losses(P<float>(s, s->o_steploss) + (size_t)k * s->max_steps, steps,
                                              P<float>(s, s->o_hist) + (size_t)k * s->max_epochs + e, s->ms[k]));
        }
    }
    for (int k = 0; k < s->n_members; k++) {
        SCUDA(s, cudaEventRecord(s->ev[1 + k], s->ms[k]));
        SCUDA(s, cudaStreamWaitEvent(s->stream, s->ev[1 + k], 0));
    }
    if (loss_history) {
        std::vector<float> h((size_t)s->n_members * s->max_epochs);
        SCUDA(s, cudaMemcpyAsync(h.data(), s->ws + s->o_hist, 4 * h.size(), cudaMemcpyDeviceToHost, s->stream));
        SCUDA(s, cudaStreamSynchronize(s->stream));
        for (int k = 0; k < s->n_members; k++)
            std::copy(h.begin() + (size_t)k * s->max_epochs, h.begin() + (size_t)k * s->max_epochs + epochs,
                      loss_history + (size_t)k * epochs);
    }
    s->trained = true;
    return TLED_OK;
}

int tled_sur_predict(tled_sur *s, const float *x, int32_t B, int32_t n_spread, float spread_tol_K, float *mean,
                     float *std, float *spread, uint8_t *fallback_mask) {
    if (int rc = check(s)) return rc;
    if (!x || B < 1 || B > s->max_batch) return fail(s, TLED_E_ARG, "1 <= B <= max_batch rows");
    if (n_spread < 0 || n_spread > s->n_out) return fail(s, TLED_E_ARG, "0 <= n_spread <= n_out");
    SCUDA(s, cudaSetDevice(s->device));
    if (int rc = forward_members(s, x, B)) return rc;
    if (int rc = ensemble(s, x, B, n_spread, spread_tol_K, mean, std, spread, fallback_mask))
        return fail(s, rc, "ensemble statistics");
    return TLED_OK;
}

int tled_sur_calibrate(tled_sur *s, const float *x, const float *y, int64_t n, int32_t n_spread, float tol_K,
                       float coverage, float *tau, float *accepted) {
    if (int rc = check(s)) return rc;
    if (!x || !y || !tau || n < 1) return fail(s, TLED_E_ARG, "NULL argument or no rows");
    if (n_spread < 1 || n_spread > s->n_out || !(coverage > 0 && coverage <= 1))
        return fail(s, TLED_E_ARG, "1 <= n_spread <= n_out, 0 < coverage <= 1");
    SCUDA(s, cudaSetDevice(s->device));
    std::vector<float> sp(n), er(n);
    for (int64_t b0 = 0; b0 < n; b0 += s->max_batch) {
        const int B = (int)std::min<int64_t>(s->max_batch, n - b0);
        const float *xb = x + (size_t)b0 * s->n_in;
        if (int rc = forward_members(s, xb, B)) return rc;
        float *cm = P<float>(s, s->o_cmean);
        if (int rc = ensemble(s, xb, B, n_spread, tol_K, cm, nullptr, P<float>(s, s->o_spread), nullptr))
            return fail(s, rc, "ensemble statistics");
        SCUDA(s, tmlp::launch_row_max_abs_diff(cm, y + (size_t)b0 * s->n_out, B, s->n_out, n_spread,
                                               P<float>(s, s->o_err), s->stream));
        SCUDA(s, cudaMemcpyAsync(sp.data() + b0, s->ws + s->o_spread, 4 * (size_t)B, cudaMemcpyDeviceToHost, s->stream));
        SCUDA(s, cudaMemcpyAsync(er.data() + b0, s->ws + s->o_err, 4 * (size_t)B, cudaMemcpyDeviceToHost, s->stream));
        SCUDA(s, cudaStreamSynchronize(s->stream));
    }
    float frac = 0.f;
    *tau = spread_threshold(sp, er, tol_K, coverage, &frac);
    if (accepted) *accepted = frac;
    return TLED_OK;
}

int tled_sur_spread_threshold(int64_t n, const float *spread, const float *err, float tol_K, float coverage,
                              float *tau, float *accepted) {
    if (n < 1 || !spread || !err || !tau || !(coverage > 0 && coverage <= 1)) return TLED_E_ARG;
    std::vector<float> sp(spread, spread + n), er(err, err + n);
    float frac = 0.f;
    *tau = spread_threshold(sp, er, tol_K, coverage, &frac);
    if (accepted) *accepted = frac;
    return TLED_OK;
}

int tled_sur_member(tled_sur *s, int32_t k, tled_mlp **member) {
    if (!s || !member || k < 0 || k >= s->n_members) return fail(s, TLED_E_ARG, "member index out of range");
    *member = s->net[k];
    return TLED_OK;
}

int tled_sur_sync(tled_sur *s) {
    if (int rc = check(s)) return rc;
    SCUDA(s, cudaSetDevice(s->device));
    SCUDA(s, cudaStreamSynchronize(s->stream));
    for (int k = 0; k < s->n_members; k++) {
        SCUDA(s, cudaStreamSynchronize(s->ms[k]));
        SMLP(s, k, tled_mlp_sync(s->net[k]));
    }
    return TLED_OK;
}

}  // extern "C"
