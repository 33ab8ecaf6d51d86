// C ABI of libtled (include/tled.h): context, set-up, workspace layout,
// CUDA-graph step loop, read-back, state I/O and checkpoints.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "tled_internal.h"

using tled::Plan;
using tled::StepArgs;

namespace {

constexpr int kGraphChunk = 32;  // steps per captured graph

struct Layout {
    size_t xu, lo, vel, X0, nodec, ubar, elem_rec, visc;
    size_t tile_info, tile_shared, part_pos, csr, partials, sh_rowptr;
    size_t src, nsrc, time_base, step_base, status, node_new, stat_part, stat_out, staging;
    size_t total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct tled_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only for graph capture
    std::string err;
    // inputs
    int npe = 0;
    int64_t nn = 0, ne = 0;
    std::vector<double> X;
    std::vector<int32_t> conn;
    bool have_mat = false;
    tled_material mat{};
    std::vector<double> mat6, fib;
    std::vector<uint8_t> mask;
    std::vector<double> ubar;
    double ramp = 0;
    std::vector<tled_source> src;
    tled_params prm{};
    // plan and device
    bool planned = false;
    Plan plan;
    Layout L{};
    char *ws = nullptr;
    bool inited = false;
    StepArgs A{};
    double dt = 0, dt_mech = 0, dt_th = 0;
    int64_t step = 0;
    double t = 0;
    uint64_t setup_hash = 0;
    std::map<int, cudaGraphExec_t> graphs;
    int tile_ctas = 1;  // persistent grid of the tile kernel
};

namespace {

int fail(tled_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(tled_ctx *c, cudaError_t e, const char *where) {
    return fail(c, TLED_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(c, expr)                                  \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return cuda_fail(c, _e, #expr); \
    } while (0)

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ULL) {
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < n; i++) {
        h ^= b[i];
        h *= 1099511628211ULL;
    }
    return h;
}

tled_params default_params() {
    tled_params p{};
    p.dt = 0.0;
    p.dt_safety = 0.8;
    p.gamma = 0.0;
    p.mass_scale = 1.0;
    p.kappa_hg = 0.1;
    p.kappa_hgT = 0.1;
    p.flags = TLED_EXPANSION | TLED_COMPENSATED;
    p.tile_elems = 0;
    return p;
}

int n_prony(const tled_ctx *c) { return c->mat.n_prony; }

// bytes of one tile's element record: local connectivity then the constant float components
size_t rec_bytes(const tled_ctx *c) {
    const int ncomp = 10 + (c->mat6.empty() ? 0 : 6) + (c->fib.empty() ? 0 : 3);
    return (size_t)tled::kTile * c->npe * 2 + (size_t)ncomp * tled::kTile * 4;
}
// Prony state index of element slot e, component q (tile-blocked [t][6 n_prony][kTile])
inline size_t visc_index(int np, int64_t e, int q) {
    return (size_t)(e / tled::kTile) * np * 6 * tled::kTile + (size_t)q * tled::kTile + (size_t)(e % tled::kTile);
}

Layout make_layout(const tled_ctx *c) {
    const Plan &p = c->plan;
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + std::max<size_t>(bytes, 1));
        return o;
    };
    const size_t nn = (size_t)c->nn, ne = (size_t)p.ne_pad;
    L.xu = take(16 * nn);
    L.lo = take(16 * nn);
    L.vel = take(16 * nn);
    L.X0 = take(16 * nn);
    L.nodec = take(16 * nn);
    L.ubar = take(c->ubar.empty() ? 0 : 16 * nn);
    L.elem_rec = take((size_t)p.n_tiles * rec_bytes(c));
    L.visc = take(4 * 6 * (size_t)std::max(n_prony(c), 0) * ne);
    L.tile_info = take(4 * p.tile_info.size());
    L.tile_shared = take(4 * p.tile_shared.size());
    L.csr = take(2 * p.csr.size());
    L.partials = take(16 * (size_t)p.n_partials);
    L.sh_rowptr = take(4 * p.sh_rowptr.size());
    L.part_pos = take(4 * p.part_pos.size());
    L.src = take(8 * 10 * tled::kMaxSources);
    L.nsrc = take(4);
    L.time_base = take(8);
    L.step_base = take(8);
    L.status = take(16);
    L.node_new = take(4 * nn);
    L.stat_part = take(8 * 8 * tled::kStatBlocks);
    L.stat_out = take(8 * 8);
    L.staging = take(8 * 3 * nn);
    L.total = off;
    return L;
}

int ensure_plan(tled_ctx *c) {
    if (c->planned) return TLED_OK;
    if (c->npe == 0) return fail(c, TLED_E_STATE, "tled_set_mesh has not been called");
    if (!c->have_mat) return fail(c, TLED_E_STATE, "tled_set_material has not been called");
    int rc = tled::build_plan(c->npe, c->nn, c->X.data(), c->ne, c->conn.data(), c->prm.tile_elems, c->plan, c->err);
    if (rc) return rc;
    c->L = make_layout(c);
    c->planned = true;
    return TLED_OK;
}

void invalidate(tled_ctx *c) {
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    c->planned = false;
    c->inited = false;
}

template <class T>
T *dptr(tled_ctx *c, size_t off) {
    return reinterpret_cast<T *>(c->ws + off);
}

int upload_sources(tled_ctx *c) {
    std::vector<double> s(10 * tled::kMaxSources, 0.0);
    for (size_t i = 0; i < c->src.size(); i++) {
        const tled_source &q = c->src[i];
        double *r = &s[10 * i];
        r[0] = q.c0[0]; r[1] = q.c0[1]; r[2] = q.c0[2];
        r[3] = q.vel[0]; r[4] = q.vel[1]; r[5] = q.vel[2];
        r[6] = q.sigma; r[7] = q.power; r[8] = q.t_on; r[9] = q.t_off;
    }
    int n = (int)c->src.size();
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.src, s.data(), s.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.nsrc, &n, 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // host staging buffers are on the stack
    return TLED_OK;
}

// Convert a float64 value into a float-float pair (hi = nearest float).
inline void split_ff(double x, float &hi, float &lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

int write_state(tled_ctx *c, const double *u, const double *v, const double *T, const double *Om, const double *visc) {
    const Plan &p = c->plan;
    const int64_t nn = c->nn;
    std::vector<float4> xu(nn), lo(nn), vel(nn);
    for (int64_t g = 0; g < nn; g++) {
        const int64_t i = p.node_old[g];
        float h[4], l[4];
        for (int d = 0; d < 3; d++) split_ff(u ? u[3 * i + d] : 0.0, h[d], l[d]);
        split_ff(T ? T[i] - c->mat.T0 : 0.0, h[3], l[3]);
        xu[g] = make_float4(h[0], h[1], h[2], h[3]);
        lo[g] = make_float4(l[0], l[1], l[2], l[3]);
        vel[g] = make_float4(v ? (float)v[3 * i] : 0.f, v ? (float)v[3 * i + 1] : 0.f, v ? (float)v[3 * i + 2] : 0.f,
                             Om ? (float)Om[i] : 0.f);
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.xu, xu.data(), 16 * nn, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.lo, lo.data(), 16 * nn, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.vel, vel.data(), 16 * nn, cudaMemcpyHostToDevice, c->stream));
    const int np = n_prony(c);
    const int64_t nep = p.ne_pad;
    std::vector<float> vs((size_t)np * 6 * nep, 0.f);
    if (visc)
        for (int64_t e = 0; e < nep; e++) {
            const int64_t eo = p.elem_old[e];
            if (eo < 0) continue;
            for (int q = 0; q < np * 6; q++) vs[visc_index(np, e, q)] = (float)visc[eo * np * 6 + q];
        }
    if (np) CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.visc, vs.data(), vs.size() * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return TLED_OK;
}

int set_clock(tled_ctx *c, double t, int64_t step) {
    c->t = t;
    c->step = step;
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.time_base, &c->t, 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.step_base, &c->step, 8, cudaMemcpyHostToDevice, c->stream));
    unsigned st[4] = {0u, 0xffffffffu, 0xffffffffu, 0u};
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.status, st, 16, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return TLED_OK;
}

int check_status(tled_ctx *c) {
    unsigned st[4];
    CUDA_TRY(c, cudaMemcpyAsync(st, c->ws + c->L.status, 16, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (st[0] & tled::kStatusInverted) {
        int64_t e = st[1] < (unsigned)c->plan.ne_pad ? c->plan.elem_old[st[1]] : -1;
        return fail(c, TLED_E_INVERTED, "element " + std::to_string(e) + " inverted (J <= 0)");
    }
    if (st[0] & tled::kStatusNaN) {
        int64_t i = st[2] < (unsigned)c->nn ? c->plan.node_old[st[2]] : -1;
        return fail(c, TLED_E_UNSTABLE, "non-finite state at node " + std::to_string(i));
    }
    if (st[0] & tled::kStatusTimeout) return fail(c, TLED_E_TIMEOUT, "device wait timed out");
    return TLED_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

int tled_version(void) { return TLED_VERSION; }

const char *tled_status_string(int code) {
    switch (code) {
        case TLED_OK: return "ok";
        case TLED_E_ARG: return "invalid argument";
        case TLED_E_MESH: return "invalid mesh";
        case TLED_E_STATE: return "call out of order";
        case TLED_E_CUDA: return "CUDA error";
        case TLED_E_UNSTABLE: return "unstable (non-finite state)";
        case TLED_E_INVERTED: return "element inverted";
        case TLED_E_TIMEOUT: return "device wait timed out";
        case TLED_E_NOMEM: return "workspace too small";
        case TLED_E_FORMAT: return "malformed checkpoint";
        default: return "unknown status";
    }
}

int tled_create(tled_ctx **out, int device, void *cuda_stream) {
    if (!out) return TLED_E_ARG;
    *out = nullptr;
    if (device == -1) {  // host-only: planning and validation without a GPU
        tled_ctx *c = new tled_ctx();
        c->device = -1;
        c->prm = default_params();
        *out = c;
        return TLED_OK;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return TLED_E_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return TLED_E_CUDA;
    tled_ctx *c = new tled_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->prm = default_params();
    if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return TLED_E_CUDA;
    }
    *out = c;
    return TLED_OK;
}

int tled_destroy(tled_ctx *c) {
    if (!c) return TLED_E_ARG;
    if (c->device < 0) {
        delete c;
        return TLED_OK;
    }
    cudaSetDevice(c->device);
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    if (c->cap) cudaStreamDestroy(c->cap);
    delete c;
    return TLED_OK;
}

const char *tled_last_error(const tled_ctx *c) { return c ? c->err.c_str() : "null context"; }

int tled_set_mesh(tled_ctx *c, int elem_type, int64_t n_nodes, const double *X0, int64_t n_elems,
                  const int32_t *conn) {
    if (!c) return TLED_E_ARG;
    if (elem_type != TLED_T4 && elem_type != TLED_H8) return fail(c, TLED_E_ARG, "elem_type must be 4 or 8");
    if (n_nodes <= 0 || n_elems <= 0 || !X0 || !conn) return fail(c, TLED_E_ARG, "empty mesh or NULL array");
    if (n_nodes > (int64_t)0x7fffffff || n_elems > (int64_t)0x7fffffff / 8)
        return fail(c, TLED_E_ARG, "mesh too large for 32-bit indices");
    for (int64_t i = 0; i < 3 * n_nodes; i++)
        if (!std::isfinite(X0[i])) return fail(c, TLED_E_ARG, "non-finite coordinate of node " + std::to_string(i / 3));
    for (int64_t e = 0; e < n_elems; e++)
        for (int a = 0; a < elem_type; a++) {
            int32_t v = conn[e * elem_type + a];
            if (v < 0 || v >= n_nodes)
                return fail(c, TLED_E_MESH, "element " + std::to_string(e) + " references node " + std::to_string(v) +
                                                " out of range");
        }
    for (int64_t e = 0; e < n_elems; e++) {
        double Ji[9], V;
        if (!tled::element_geometry(elem_type, X0, conn + e * elem_type, Ji, &V))
            return fail(c, TLED_E_MESH, "element " + std::to_string(e) + " has det J0 <= 0");
    }
    invalidate(c);
    c->npe = elem_type;
    c->nn = n_nodes;
    c->ne = n_elems;
    c->X.assign(X0, X0 + 3 * n_nodes);
    c->conn.assign(conn, conn + elem_type * n_elems);
    c->mask.assign(n_nodes, 0);
    c->ubar.clear();
    c->have_mat = false;
    c->mat6.clear();
    c->fib.clear();
    return TLED_OK;
}

int tled_set_material(tled_ctx *c, const tled_material *m, const double *per_elem, const double *fibre) {
    if (!c || !m) return fail(c, TLED_E_ARG, "NULL material");
    if (c->npe == 0) return fail(c, TLED_E_STATE, "set the mesh first");
    if (m->n_prony < 0 || m->n_prony > 4) return fail(c, TLED_E_ARG, "n_prony must be 0..4");
    const double vals[] = {m->rho, m->mu, m->kappa, m->k1, m->k2, m->alpha, m->k, m->c, m->wb_cb, m->T0, m->Ta, m->lnA, m->Ea};
    for (double v : vals)
        if (!std::isfinite(v)) return fail(c, TLED_E_ARG, "non-finite material value");
    if (!(m->rho > 0) || !(m->c > 0) || m->mu < 0 || m->kappa < 0 || m->k < 0 || m->k1 < 0 || m->k2 < 0)
        return fail(c, TLED_E_ARG, "material moduli must be non-negative and rho, c positive");
    double gsum = 0;
    for (int i = 0; i < m->n_prony; i++) {
        if (!(m->prony_tau[i] > 0) || m->prony_g[i] < 0) return fail(c, TLED_E_ARG, "Prony tau must be > 0, g >= 0");
        gsum += m->prony_g[i];
    }
    if (gsum >= 1.0) return fail(c, TLED_E_ARG, "sum of Prony g must be < 1");
    if (per_elem)
        for (int64_t i = 0; i < 6 * c->ne; i++)
            if (!std::isfinite(per_elem[i]) || (i % 6 != 5 && per_elem[i] < 0))
                return fail(c, TLED_E_ARG, "bad per-element material of element " + std::to_string(i / 6));
    if (fibre)
        for (int64_t e = 0; e < c->ne; e++) {
            const double *a = fibre + 3 * e;
            double n = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
            if (!(std::fabs(n - 1.0) < 1e-6)) return fail(c, TLED_E_ARG, "fibre of element " + std::to_string(e) + " is not a unit vector");
        }
    invalidate(c);
    c->mat = *m;
    c->mat6.assign(per_elem ? per_elem : nullptr, per_elem ? per_elem + 6 * c->ne : nullptr);
    c->fib.assign(fibre ? fibre : nullptr, fibre ? fibre + 3 * c->ne : nullptr);
    c->have_mat = true;
    return TLED_OK;
}

int tled_set_bcs(tled_ctx *c, const uint8_t *mask, const double *ubar, double ramp_time) {
    if (!c) return TLED_E_ARG;
    if (c->npe == 0) return fail(c, TLED_E_STATE, "set the mesh first");
    if (!mask) return fail(c, TLED_E_ARG, "NULL mask");
    if (!(ramp_time >= 0)) return fail(c, TLED_E_ARG, "ramp_time must be >= 0");
    invalidate(c);
    c->mask.assign(mask, mask + c->nn);
    c->ubar.assign(ubar ? ubar : nullptr, ubar ? ubar + 3 * c->nn : nullptr);
    c->ramp = ramp_time;
    return TLED_OK;
}

int tled_set_heat_sources(tled_ctx *c, int32_t n, const tled_source *s) {
    if (!c) return TLED_E_ARG;
    if (n < 0 || n > tled::kMaxSources || (n > 0 && !s)) return fail(c, TLED_E_ARG, "0 <= n <= 16 sources");
    for (int i = 0; i < n; i++)
        if (!(s[i].sigma > 0) || !std::isfinite(s[i].power)) return fail(c, TLED_E_ARG, "source sigma must be > 0");
    c->src.assign(s, s + n);
    if (c->inited) {
        cudaSetDevice(c->device);
        return upload_sources(c);
    }
    return TLED_OK;
}

int tled_set_params(tled_ctx *c, const tled_params *p) {
    if (!c) return TLED_E_ARG;
    tled_params q = p ? *p : default_params();
    if (q.dt < 0 || !(q.dt_safety > 0) || q.gamma < 0 || !(q.mass_scale >= 1.0) || q.kappa_hg < 0 || q.kappa_hgT < 0 ||
        q.tile_elems < 0)
        return fail(c, TLED_E_ARG, "invalid solver parameters");
    invalidate(c);
    c->prm = q;
    return TLED_OK;
}

int tled_workspace_size(tled_ctx *c, int64_t *bytes) {
    if (!c || !bytes) return TLED_E_ARG;
    int rc = ensure_plan(c);
    if (rc) return rc;
    *bytes = (int64_t)c->L.total;
    return TLED_OK;
}

int tled_init(tled_ctx *c, void *dev_workspace, int64_t bytes) {
    if (!c) return TLED_E_ARG;
    if (c->device < 0) return fail(c, TLED_E_STATE, "host-only context (device -1) cannot be initialised");
    int rc = ensure_plan(c);
    if (rc) return rc;
    if (!dev_workspace || ((uintptr_t)dev_workspace & 255)) return fail(c, TLED_E_ARG, "workspace must be 256-byte aligned");
    if (bytes < (int64_t)c->L.total) return fail(c, TLED_E_NOMEM, "workspace smaller than tled_workspace_size()");
    CUDA_TRY(c, cudaSetDevice(c->device));
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    c->ws = (char *)dev_workspace;
    const Plan &p = c->plan;
    const int npe = c->npe;
    const int64_t nn = c->nn, ne = c->ne;
    const tled_material &m = c->mat;
    // --- element geometry (new order), lumped masses
    const int64_t nep = p.ne_pad;
    const size_t rb = rec_bytes(c);
    const int kT = tled::kTile;
    std::vector<char> rec((size_t)p.n_tiles * rb, 0);
    std::vector<double> Mn(nn, 0.0), Cn(nn, 0.0), Vn(nn, 0.0);
    for (int64_t e = 0; e < nep; e++) {
        const int64_t eo = p.elem_old[e];
        if (eo < 0) continue;  // padding slot
        double Ji[9], V;
        tled::element_geometry(npe, c->X.data(), c->conn.data() + eo * npe, Ji, &V);
        char *r = rec.data() + (size_t)(e / kT) * rb;
        const int ei = (int)(e % kT);
        std::memcpy(r + (size_t)ei * npe * 2, &p.conn_local[(size_t)e * npe], (size_t)npe * 2);
        float *cf = reinterpret_cast<float *>(r + (size_t)kT * npe * 2) + ei;
        int q = 0;
        for (int j = 0; j < 9; j++) cf[(q++) * kT] = (float)Ji[j];
        cf[(q++) * kT] = (float)V;
        if (!c->mat6.empty())
            for (int j = 0; j < 6; j++) cf[(q++) * kT] = (float)c->mat6[6 * eo + j];
        if (!c->fib.empty())
            for (int j = 0; j < 3; j++) cf[(q++) * kT] = (float)c->fib[3 * eo + j];
        for (int a = 0; a < npe; a++) {
            const int64_t i = c->conn[eo * npe + a];
            Mn[i] += c->prm.mass_scale * m.rho * V / npe;
            Cn[i] += m.rho * m.c * V / npe;
            Vn[i] += V / npe;
        }
    }
    std::vector<float4> X0(nn), nodec(nn), ub(c->ubar.empty() ? 0 : nn);
    std::vector<int32_t> node_new(p.node_new.begin(), p.node_new.end());
    for (int64_t g = 0; g < nn; g++) {
        const int64_t i = p.node_old[g];
        X0[g] = make_float4((float)c->X[3 * i], (float)c->X[3 * i + 1], (float)c->X[3 * i + 2], (float)Vn[i]);
        unsigned mk = c->mask[i] & 15u;
        float mkf;
        std::memcpy(&mkf, &mk, 4);
        nodec[g] = make_float4((float)(1.0 / Mn[i]), (float)(1.0 / Cn[i]), mkf, 0.f);
        if (!c->ubar.empty())
            ub[g] = make_float4((float)c->ubar[3 * i], (float)c->ubar[3 * i + 1], (float)c->ubar[3 * i + 2], 0.f);
    }
    // --- time step
    tled::stable_dt(npe, nn, c->X.data(), ne, c->conn.data(), m, c->mat6.empty() ? nullptr : c->mat6.data(), c->prm,
                    &c->dt_mech, &c->dt_th);
    c->dt = c->prm.dt > 0 ? c->prm.dt : c->prm.dt_safety * std::min(c->dt_mech, c->dt_th);
    // --- upload
    auto up = [&](size_t off, const void *src, size_t n) -> cudaError_t {
        if (n == 0) return cudaSuccess;
        return cudaMemcpyAsync(c->ws + off, src, n, cudaMemcpyHostToDevice, c->stream);
    };
    const Layout &L = c->L;
    CUDA_TRY(c, up(L.X0, X0.data(), 16 * nn));
    CUDA_TRY(c, up(L.nodec, nodec.data(), 16 * nn));
    CUDA_TRY(c, up(L.ubar, ub.data(), 16 * ub.size()));
    CUDA_TRY(c, up(L.elem_rec, rec.data(), rec.size()));
    CUDA_TRY(c, up(L.tile_info, p.tile_info.data(), 4 * p.tile_info.size()));
    CUDA_TRY(c, up(L.tile_shared, p.tile_shared.data(), 4 * p.tile_shared.size()));
    CUDA_TRY(c, up(L.csr, p.csr.data(), 2 * p.csr.size()));
    CUDA_TRY(c, up(L.sh_rowptr, p.sh_rowptr.data(), 4 * p.sh_rowptr.size()));
    CUDA_TRY(c, up(L.part_pos, p.part_pos.data(), 4 * p.part_pos.size()));
    CUDA_TRY(c, up(L.node_new, node_new.data(), 4 * nn));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->inited = true;  // buffers placed; the rest uses the regular paths
    int r2 = upload_sources(c);
    if (r2) return r2;
    r2 = write_state(c, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (r2) return r2;
    r2 = set_clock(c, 0.0, 0);
    if (r2) return r2;
    // --- kernel arguments
    StepArgs &A = c->A;
    A = StepArgs{};
    A.xu = dptr<float4>(c, L.xu);
    A.lo = dptr<float4>(c, L.lo);
    A.vel = dptr<float4>(c, L.vel);
    A.X0 = dptr<float4>(c, L.X0);
    A.nodec = dptr<float4>(c, L.nodec);
    A.ubar = c->ubar.empty() ? nullptr : dptr<float4>(c, L.ubar);
    A.elem_rec = dptr<char>(c, L.elem_rec);
    A.rec_bytes = (int64_t)rb;
    A.has_mat = !c->mat6.empty();
    A.has_fib = !c->fib.empty();
    A.visc = dptr<float>(c, L.visc);
    A.ne = nep;
    A.tile_info = dptr<int>(c, L.tile_info);
    A.tile_shared = dptr<int>(c, L.tile_shared);
    A.csr = dptr<uint16_t>(c, L.csr);
    A.partials = dptr<float4>(c, L.partials);
    A.part_pos = dptr<int>(c, L.part_pos);
    A.sh_rowptr = dptr<int>(c, L.sh_rowptr);
    A.n_interior = p.n_interior;
    A.n_shared = p.n_shared;
    A.src = dptr<double>(c, L.src);
    A.n_src = dptr<int>(c, L.nsrc);
    A.time_base = dptr<double>(c, L.time_base);
    A.step_base = dptr<int64_t>(c, L.step_base);
    A.status = dptr<unsigned>(c, L.status);
    const double dt = c->dt, g = c->prm.gamma;
    A.dt = dt;
    A.dtf = (float)dt;
    A.inv_dt = (float)(1.0 / dt);
    A.damp_a = (float)((1.0 - 0.5 * g * dt) / (1.0 + 0.5 * g * dt));
    A.damp_b = (float)(dt / (1.0 + 0.5 * g * dt));
    A.mu = (float)m.mu; A.kappa = (float)m.kappa; A.k1 = (float)m.k1; A.k2 = (float)m.k2;
    A.kc = (float)m.k; A.alpha = (float)m.alpha;
    A.a0x = (float)m.a0[0]; A.a0y = (float)m.a0[1]; A.a0z = (float)m.a0[2];
    A.n_prony = m.n_prony;
    for (int i = 0; i < 4; i++) {
        if (i < m.n_prony) {
            A.pr_a[i] = (float)(dt * m.prony_g[i] / (dt + m.prony_tau[i]));
            A.pr_b[i] = (float)(m.prony_tau[i] / (dt + m.prony_tau[i]));
        } else {
            A.pr_a[i] = A.pr_b[i] = 0.f;
        }
    }
    A.flags = c->prm.flags;
    A.beta_c = (float)m.beta_c;
    A.beta_k = (float)m.beta_k;
    A.Tref_m_T0 = (float)(m.T_ref - m.T0);
    A.theta_a = (float)(m.Ta - m.T0);
    A.wbcb = (float)m.wb_cb;
    A.Qm = (float)m.Qm;
    A.lnA = (float)m.lnA;
    A.Ea_R = (float)(m.Ea / 8.314);
    A.T0_K = (float)(m.T0 + 273.15);
    A.khg = (float)c->prm.kappa_hg;
    A.khgT = (float)c->prm.kappa_hgT;
    A.ramp_time = c->ramp;
    A.n_tiles = p.n_tiles;
    tled::tile_smem_layout(A, npe);
    CUDA_TRY(c, tled::tile_kernel_setup(A, npe));
    int n_sm = 0;
    CUDA_TRY(c, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device));
    c->tile_ctas = tled::tile_grid(A, npe, n_sm);
    // set-up hash for checkpoints
    uint64_t h = fnv1a(c->X.data(), 8 * c->X.size());
    h = fnv1a(c->conn.data(), 4 * c->conn.size(), h);
    h = fnv1a(&c->mat, sizeof(tled_material), h);
    h = fnv1a(&c->prm, sizeof(tled_params), h);
    h = fnv1a(&c->dt, 8, h);
    c->setup_hash = h;
    return TLED_OK;
}

int tled_get_dt(tled_ctx *c, double *dt, double *dt_mech, double *dt_thermal) {
    if (!c) return TLED_E_ARG;
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (dt) *dt = c->dt;
    if (dt_mech) *dt_mech = c->dt_mech;
    if (dt_thermal) *dt_thermal = c->dt_th;
    return TLED_OK;
}

static int get_graph(tled_ctx *c, int K, cudaGraphExec_t *out) {
    auto it = c->graphs.find(K);
    if (it != c->graphs.end()) {
        *out = it->second;
        return TLED_OK;
    }
    CUDA_TRY(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < K && e == cudaSuccess; k++) {
        e = tled::launch_tile_step(c->A, c->tile_ctas, c->npe, k, c->cap);
        if (e == cudaSuccess) e = tled::launch_shared_step(c->A, k, c->cap);
    }
    if (e == cudaSuccess)
        e = tled::launch_bump(dptr<double>(c, c->L.time_base), dptr<int64_t>(c, c->L.step_base), K, c->dt, c->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->cap, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(c, e, "capture step kernels");
    }
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    c->graphs[K] = exec;
    *out = exec;
    return TLED_OK;
}

int tled_step(tled_ctx *c, int64_t n) {
    if (!c) return TLED_E_ARG;
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (n < 0) return fail(c, TLED_E_ARG, "n must be >= 0");
    CUDA_TRY(c, cudaSetDevice(c->device));
    while (n > 0) {
        const int K = (int)std::min<int64_t>(n, kGraphChunk);
        cudaGraphExec_t g;
        int rc = get_graph(c, K, &g);
        if (rc) return rc;
        CUDA_TRY(c, cudaGraphLaunch(g, c->stream));
        n -= K;
        c->step += K;
        c->t += K * c->dt;
    }
    return TLED_OK;
}

int tled_sync(tled_ctx *c) {
    if (!c) return TLED_E_ARG;
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return check_status(c);
}

static int readback(tled_ctx *c, double *out, int where, int mode) {
    if (!c || !out) return fail(c, TLED_E_ARG, "NULL output");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (where != TLED_HOST && where != TLED_DEVICE) return fail(c, TLED_E_ARG, "where must be TLED_HOST or TLED_DEVICE");
    CUDA_TRY(c, cudaSetDevice(c->device));
    double *dst = where == TLED_DEVICE ? out : dptr<double>(c, c->L.staging);
    CUDA_TRY(c, tled::launch_readback(c->A, dptr<int32_t>(c, c->L.node_new), c->nn, c->mat.T0, mode, dst, c->stream));
    if (where == TLED_HOST) {
        const size_t n = (size_t)c->nn * (mode == 0 ? 3 : 1);
        CUDA_TRY(c, cudaMemcpyAsync(out, dst, 8 * n, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    return TLED_OK;
}

int tled_get_displacement(tled_ctx *c, double *out, int where) { return readback(c, out, where, 0); }
int tled_get_temperature(tled_ctx *c, double *out, int where) { return readback(c, out, where, 1); }
int tled_get_damage(tled_ctx *c, double *out, int where) { return readback(c, out, where, 2); }

int tled_set_state(tled_ctx *c, const double *u, const double *v, const double *T, const double *Omega,
                   const double *visc, double t, int64_t step) {
    if (!c) return TLED_E_ARG;
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (!u || !v || !T || !Omega) return fail(c, TLED_E_ARG, "u, v, T and Omega are required");
    if (!std::isfinite(t) || step < 0) return fail(c, TLED_E_ARG, "bad time or step");
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    int rc = write_state(c, u, v, T, Omega, visc);
    if (rc) return rc;
    return set_clock(c, t, step);
}

int tled_get_state(tled_ctx *c, double *u, double *v, double *T, double *Omega, double *visc, double *t,
                   int64_t *step) {
    if (!c) return TLED_E_ARG;
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int64_t nn = c->nn, ne = c->ne;
    const Plan &p = c->plan;
    std::vector<float4> xu(nn), lo(nn), vel(nn);
    CUDA_TRY(c, cudaMemcpyAsync(xu.data(), c->ws + c->L.xu, 16 * nn, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(lo.data(), c->ws + c->L.lo, 16 * nn, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(vel.data(), c->ws + c->L.vel, 16 * nn, cudaMemcpyDeviceToHost, c->stream));
    const int np = n_prony(c);
    const int64_t nep = p.ne_pad;
    std::vector<float> vs((size_t)np * 6 * nep);
    if (np && visc)
        CUDA_TRY(c, cudaMemcpyAsync(vs.data(), c->ws + c->L.visc, 4 * vs.size(), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int64_t g = 0; g < nn; g++) {
        const int64_t i = p.node_old[g];
        if (u) {
            u[3 * i] = (double)xu[g].x + lo[g].x;
            u[3 * i + 1] = (double)xu[g].y + lo[g].y;
            u[3 * i + 2] = (double)xu[g].z + lo[g].z;
        }
        if (v) {
            v[3 * i] = vel[g].x;
            v[3 * i + 1] = vel[g].y;
            v[3 * i + 2] = vel[g].z;
        }
        if (T) T[i] = c->mat.T0 + ((double)xu[g].w + lo[g].w);
        if (Omega) Omega[i] = vel[g].w;
    }
    if (visc && np)
        for (int64_t e = 0; e < nep; e++) {
            const int64_t eo = p.elem_old[e];
            if (eo < 0) continue;
            for (int q = 0; q < np * 6; q++) visc[eo * np * 6 + q] = vs[visc_index(np, e, q)];
        }
    if (t) *t = c->t;
    if (step) *step = c->step;
    return TLED_OK;
}

int tled_step_timed(tled_ctx *c, int64_t n, double *ms) {
    if (!c || !ms) return fail(c, TLED_E_ARG, "NULL ms");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (n <= 0 || n > 100000) return fail(c, TLED_E_ARG, "1 <= n <= 100000");
    CUDA_TRY(c, cudaSetDevice(c->device));
    std::vector<cudaEvent_t> ev(3 * (size_t)n, nullptr);
    for (auto &e : ev) CUDA_TRY(c, cudaEventCreate(&e));
    cudaError_t err = cudaSuccess;
    for (int64_t i = 0; i < n && err == cudaSuccess; i++) {
        cudaEventRecord(ev[3 * i], c->stream);
        err = tled::launch_tile_step(c->A, c->tile_ctas, c->npe, 0, c->stream);
        cudaEventRecord(ev[3 * i + 1], c->stream);
        if (err == cudaSuccess) err = tled::launch_shared_step(c->A, 0, c->stream);
        cudaEventRecord(ev[3 * i + 2], c->stream);
        if (err == cudaSuccess)
            err = tled::launch_bump(dptr<double>(c, c->L.time_base), dptr<int64_t>(c, c->L.step_base), 1, c->dt,
                                    c->stream);
    }
    cudaError_t se = cudaStreamSynchronize(c->stream);
    double a = 0, b = 0;
    for (int64_t i = 0; i < n && err == cudaSuccess && se == cudaSuccess; i++) {
        float x = 0, y = 0;
        cudaEventElapsedTime(&x, ev[3 * i], ev[3 * i + 1]);
        cudaEventElapsedTime(&y, ev[3 * i + 1], ev[3 * i + 2]);
        a += x;
        b += y;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (err != cudaSuccess) return cuda_fail(c, err, "tled_step_timed launch");
    if (se != cudaSuccess) return cuda_fail(c, se, "tled_step_timed sync");
    c->step += n;
    c->t += n * c->dt;
    ms[0] = a;
    ms[1] = b;
    return check_status(c);
}

int tled_plan_info(tled_ctx *c, int64_t *info) {
    if (!c || !info) return fail(c, TLED_E_ARG, "NULL info");
    int rc = ensure_plan(c);
    if (rc) return rc;
    info[0] = c->plan.n_tiles;
    info[1] = c->plan.n_interior;
    info[2] = c->plan.n_shared;
    info[3] = c->plan.n_partials;
    info[4] = (int64_t)c->L.total;
    info[5] = c->npe;
    return TLED_OK;
}

int tled_get_stats(tled_ctx *c, tled_stats *s) {
    if (!c || !s) return fail(c, TLED_E_ARG, "NULL stats");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, tled::launch_stats(c->A, c->nn, dptr<double>(c, c->L.stat_part), dptr<double>(c, c->L.stat_out),
                                   c->stream));
    double o[8];
    unsigned st[4];
    CUDA_TRY(c, cudaMemcpyAsync(o, c->ws + c->L.stat_out, 64, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(st, c->ws + c->L.status, 16, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::memset(s, 0, sizeof(*s));
    s->step = c->step;
    s->t = c->t;
    s->dt = c->dt;
    s->kinetic_energy = o[0];
    s->heat_content = o[1];
    s->T_max = c->mat.T0 + o[2];
    s->T_min = c->mat.T0 + o[3];
    s->u_max = std::sqrt(o[4]);
    s->damage_volume = o[5];
    s->status = st[0];
    return TLED_OK;
}

int tled_get_stats_noalloc(tled_ctx *c, int32_t n_blocks, double *out) {
    if (!c || !out) return fail(c, TLED_E_ARG, "NULL context or output");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (n_blocks == 0) n_blocks = tled::kNoAllocMaxBlocks;
    if (n_blocks < 0 || n_blocks > tled::kNoAllocMaxBlocks)
        return fail(c, TLED_E_ARG, "n_blocks must be 1.." + std::to_string(tled::kNoAllocMaxBlocks) +
                                       " (size of the static scratch array), got " + std::to_string(n_blocks));
    CUDA_TRY(c, cudaSetDevice(c->device));
    double *scratch = nullptr;
    CUDA_TRY(c, tled::noalloc_scratch(c->device, &scratch));
    CUDA_TRY(c, tled::launch_stats_blocks(c->A, c->nn, n_blocks, scratch, out, c->stream));
    return TLED_OK;
}

// --- checkpoints -----------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];
    uint32_t version, npe;
    int64_t nn, ne;
    int32_t n_prony, pad;
    uint64_t setup_hash;
    int64_t step;
    double t;
    int64_t payload;
    uint64_t checksum;
};
}  // namespace

int tled_save_state(tled_ctx *c, void *buf, int64_t *bytes) {
    if (!c || !bytes) return fail(c, TLED_E_ARG, "NULL size pointer");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    const size_t nn = c->nn, nv = (size_t)n_prony(c) * 6 * c->plan.ne_pad;
    const int64_t payload = (int64_t)(3 * 16 * nn + 4 * nv);
    const int64_t need = (int64_t)sizeof(CkptHeader) + payload;
    if (!buf) {
        *bytes = need;
        return TLED_OK;
    }
    if (*bytes < need) return fail(c, TLED_E_ARG, "checkpoint buffer too small");
    CUDA_TRY(c, cudaSetDevice(c->device));
    char *p = (char *)buf + sizeof(CkptHeader);
    CUDA_TRY(c, cudaMemcpyAsync(p, c->ws + c->L.xu, 16 * nn, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(p + 16 * nn, c->ws + c->L.lo, 16 * nn, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(p + 32 * nn, c->ws + c->L.vel, 16 * nn, cudaMemcpyDeviceToHost, c->stream));
    if (nv) CUDA_TRY(c, cudaMemcpyAsync(p + 48 * nn, c->ws + c->L.visc, 4 * nv, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CkptHeader h{};
    std::memcpy(h.magic, "TLEDCKP1", 8);
    h.version = TLED_VERSION;
    h.npe = c->npe;
    h.nn = c->nn;
    h.ne = c->ne;
    h.n_prony = n_prony(c);
    h.setup_hash = c->setup_hash;
    h.step = c->step;
    h.t = c->t;
    h.payload = payload;
    h.checksum = fnv1a(p, payload);
    std::memcpy(buf, &h, sizeof(h));
    *bytes = need;
    return TLED_OK;
}

int tled_load_state(tled_ctx *c, const void *buf, int64_t bytes) {
    if (!c || !buf) return fail(c, TLED_E_ARG, "NULL checkpoint");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (bytes < (int64_t)sizeof(CkptHeader)) return fail(c, TLED_E_FORMAT, "checkpoint shorter than its header");
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, "TLEDCKP1", 8) != 0) return fail(c, TLED_E_FORMAT, "bad checkpoint magic");
    const size_t nn = c->nn, nv = (size_t)n_prony(c) * 6 * c->plan.ne_pad;
    const int64_t payload = (int64_t)(3 * 16 * nn + 4 * nv);
    if (h.version != TLED_VERSION || h.npe != (uint32_t)c->npe || h.nn != c->nn || h.ne != c->ne ||
        h.n_prony != n_prony(c) || h.payload != payload || bytes < (int64_t)sizeof(h) + payload)
        return fail(c, TLED_E_FORMAT, "checkpoint does not match this problem's sizes");
    if (h.setup_hash != c->setup_hash) return fail(c, TLED_E_FORMAT, "checkpoint was written for a different set-up");
    const char *p = (const char *)buf + sizeof(CkptHeader);
    if (fnv1a(p, payload) != h.checksum) return fail(c, TLED_E_FORMAT, "checkpoint checksum mismatch");
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.xu, p, 16 * nn, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.lo, p + 16 * nn, 16 * nn, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.vel, p + 32 * nn, 16 * nn, cudaMemcpyHostToDevice, c->stream));
    if (nv) CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.visc, p + 48 * nn, 4 * nv, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return set_clock(c, h.t, h.step);
}

}  // extern "C"
