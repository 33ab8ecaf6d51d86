// C ABI of libtled (include/tled.h): contexts of one or many scenarios,
// set-up, workspace layout, CUDA-graph step loop, read-back, probes, state I/O,
// checkpoints and the autotuner.
//
// A context holds one or more independent scenarios (meshes, materials, heat
// sources, step sizes).  Their meshes are concatenated (caller numbering:
// scenario 0's nodes and elements first, then scenario 1's, ...), tiled so
// that no tile spans two scenarios, and advanced together: one launch of the
// tile kernel and one of the shared-node kernel per step for all scenarios.
// Tiles are ordered by decreasing scenario length, so the tiles of unfinished
// scenarios always form a prefix; the step loop splits at the steps where a
// scenario finishes and the kernels read the prefix lengths from device
// memory.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "tled_internal.h"

using tled::Plan;
using tled::ScenDev;
using tled::StepArgs;

namespace {

constexpr int kGraphChunk = 32;  // steps per captured graph
constexpr double kL2PersistShare = 0.4;  // largest share of L2 the persisting window may set aside
constexpr int kCoopTilesMax = 512;  // tiles of a grid-resident candidate (its partial sums are double-buffered)
constexpr int kSingleSources = tled::kMaxSources;

struct Layout {
    size_t xu, lo, vel, X0, nodec, ubar, elem_rec, visc;
    size_t tile_info, tile_shared, part_pos, pattern, partials, sh_rowptr;
    size_t scn, src, scn_time, scn_step, tile_scn, shared_scn, n_active, status, res, gbar;
    size_t node_new, probe_node, probe_w, probe_out, stat_part, stat_out, staging, cem;
    size_t total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Scenario {
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
    std::vector<double> probes;  // [n][3]
    int64_t n_steps = INT64_MAX;
    // derived at init (the stable-step bounds once per set-up: dt_valid)
    double dt = 0, dt_mech = 0, dt_th = 0;
    double mass_scale = 1.0;  // mechanical mass multiplier in use (prm.mass_scale, or the automatic choice)
    double dt_thermal = 0;    // the thermal step (dt with n_sub = 1; n_sub dt with mechanical subcycling)
    bool dt_valid = false;
    int64_t node_off = 0, elem_off = 0, probe_off = 0;
    int src_off = 0;
};

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
    p.n_sub = 1;
    return p;
}

}  // namespace

struct tled_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only for graph capture
    bool l2_set = false;         // this context raised the persisting-L2 set-aside (restored on destroy)
    size_t l2_prev = 0;          // ... from this value
    std::string err;
    bool batch = false;
    std::vector<Scenario> sc;
    // combined problem; npe = 0 when a batch mixes T4 and H8 scenarios
    int npe = 0, npe_max = 0;
    int64_t nn = 0, ne = 0, n_probes = 0;
    bool has_mat = false, has_fib = false;
    std::vector<int> rank_of;      // scenario -> rank (order of decreasing n_steps)
    std::vector<int> scn_of_rank;  // rank -> scenario
    std::vector<int64_t> tiles_upto, shared_upto;  // [rank + 1]: tiles / shared nodes of ranks < r
    std::vector<int32_t> probe_node;               // [n_probes][8] new node ids
    std::vector<float> probe_w;                    // [n_probes][8]
    int tile_override = 0, grid_override = 0;      // set by the autotuner
    int mode_override = 0;  // autotuner: 1 streamed, 2 resident, 3 grid-resident (if it fits), 0 default
    // plan and device
    bool planned = false;
    Plan plan;
    Layout L{};
    char *ws = nullptr;
    bool inited = false;
    StepArgs A{};
    int64_t step = 0;              // steps taken since init / set_state / load
    double t0 = 0;                 // time at step 0 (single scenario)
    uint64_t setup_hash = 0;
    std::map<int, cudaGraphExec_t> graphs;
    int tile_ctas = 1;
    int shared_blocks = 1;         // persistent grid of the shared-node kernel
    int active_host[2] = {0, 0};   // last uploaded active prefix lengths
    bool res_ok = false;           // every scenario fits one CTA's shared memory (resident mode possible)
    bool resident = false;         // steps run by the resident kernel
    bool coop_ok = false;          // a single problem whose tiles fit co-resident CTAs (grid-resident mode)
    bool coop = false;             // steps run by the grid-resident (cooperative) kernel
};

namespace {

int fail(tled_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(tled_ctx *c, cudaError_t e, const char *where) {
    return fail(c, TLED_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(c, expr)                                      \
    do {                                                       \
        cudaError_t _e = (expr);                               \
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

Scenario &single(tled_ctx *c) { return c->sc[0]; }
int n_prony(const tled_ctx *c) { return c->sc.empty() ? 0 : c->sc[0].mat.n_prony; }

// element record bytes of a tile (float components; the connectivity is in the structure record)
size_t rec_bytes(const tled_ctx *c) {
    const int ncomp = 10 + (c->has_mat ? 6 : 0) + (c->has_fib ? 3 : 0);
    return (size_t)ncomp * tled::kTile * 4;
}
// Prony state index of element slot e, component q (tile-blocked [t][6 n_prony][kTile])
inline size_t visc_index(int np, int64_t e, int q) {
    return (size_t)(e / tled::kTile) * np * 6 * tled::kTile + (size_t)q * tled::kTile + (size_t)(e % tled::kTile);
}

// total source-table capacity (a single problem may change its sources after init)
int source_capacity(const tled_ctx *c) {
    if (!c->batch) return kSingleSources;
    int n = 0;
    for (auto &s : c->sc) n += (int)s.src.size();
    return std::max(n, 1);
}

// fibre / transverse ratio of the anisotropic thermal physics (0 means 1: isotropic)
double fibre_ratio(double r) { return r == 0.0 ? 1.0 : r; }

// CEM43 dose tracked (single problems that ask for it)
bool cem_on(const tled_ctx *c) { return !c->batch && !c->sc.empty() && (c->sc[0].prm.flags & TLED_CEM43); }

Layout make_layout(const tled_ctx *c) {
    const Plan &p = c->plan;
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + std::max<size_t>(bytes, 1));
        return o;
    };
    const size_t nn = (size_t)c->nn, ne = (size_t)p.ne_pad, ns = c->sc.size();
    bool any_ubar = false;
    for (auto &s : c->sc) any_ubar |= !s.ubar.empty();
    L.xu = take(16 * nn);
    // the partial sums directly after (u, theta): with the shared nodes' entries, which sit at
    // the end of xu, they form one range for the L2 persistence window (tled_init)
    // small problems (grid-resident candidates) get a second buffer of partial sums
    L.partials = take(16 * (size_t)p.n_partials * (p.n_tiles <= kCoopTilesMax ? 2 : 1));
    L.lo = take(16 * nn);
    L.vel = take(16 * nn);
    L.X0 = take(16 * nn);
    L.nodec = take(16 * nn);
    L.ubar = take(any_ubar ? 16 * nn : 0);
    L.elem_rec = take((size_t)p.n_tiles * rec_bytes(c));
    L.visc = take(4 * 6 * (size_t)std::max(n_prony(c), 0) * ne);
    L.tile_info = take(4 * p.tile_info.size());
    L.tile_shared = take(4 * p.tile_shared.size());
    L.pattern = take(2 * p.patterns.size());
    L.sh_rowptr = take(4 * p.sh_rowptr.size());
    L.part_pos = take(4 * p.part_pos.size());
    L.scn = take(sizeof(ScenDev) * ns);
    L.src = take(8 * tled::kSrcRow * (size_t)source_capacity(c));
    L.scn_time = take(8 * ns);
    L.scn_step = take(8 * ns);
    L.tile_scn = take(4 * (size_t)p.n_tiles);
    L.shared_scn = take(4 * (size_t)p.n_shared);
    L.n_active = take(8);
    L.res = take(sizeof(tled::ResDesc) * ns);
    L.gbar = take(8);
    L.status = take(16);
    L.node_new = take(4 * nn);
    L.probe_node = take(4 * 8 * (size_t)c->n_probes);
    L.probe_w = take(4 * 8 * (size_t)c->n_probes);
    L.probe_out = take(8 * 2 * (size_t)c->n_probes);
    L.stat_part = take(8 * 8 * tled::kStatBlocks);
    L.stat_out = take(8 * 8);
    L.staging = take(8 * std::max<size_t>(3 * nn, 2 * (size_t)c->n_probes));
    L.cem = take(cem_on(c) ? 8 * nn : 0);
    L.total = off;
    return L;
}

template <class T>
T *dptr(tled_ctx *c, size_t off) {
    return reinterpret_cast<T *>(c->ws + off);
}

// ---------------------------------------------------------------------------
// probes: locate points in a scenario's mesh; weights are the shape functions
// ---------------------------------------------------------------------------
const double kH8S[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                           {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

bool invert3(const double J[9], double Ji[9]) {
    double c00 = J[4] * J[8] - J[5] * J[7], c01 = J[5] * J[6] - J[3] * J[8], c02 = J[3] * J[7] - J[4] * J[6];
    double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
    if (!(std::fabs(det) > 0)) return false;
    double id = 1.0 / det;
    Ji[0] = c00 * id; Ji[1] = (J[2] * J[7] - J[1] * J[8]) * id; Ji[2] = (J[1] * J[5] - J[2] * J[4]) * id;
    Ji[3] = c01 * id; Ji[4] = (J[0] * J[8] - J[2] * J[6]) * id; Ji[5] = (J[2] * J[3] - J[0] * J[5]) * id;
    Ji[6] = c02 * id; Ji[7] = (J[1] * J[6] - J[0] * J[7]) * id; Ji[8] = (J[0] * J[4] - J[1] * J[3]) * id;
    return true;
}

// natural coordinates of x in element e; returns true if inside (with tolerance)
bool locate_in(const Scenario &s, int64_t e, const double *x, double w[8]) {
    const int32_t *cn = s.conn.data() + e * s.npe;
    const double tol = 1e-9;
    if (s.npe == 4) {
        const double *p0 = &s.X[3 * (int64_t)cn[0]];
        double J[9], Ji[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) J[3 * i + j] = s.X[3 * (int64_t)cn[j + 1] + i] - p0[i];
        if (!invert3(J, Ji)) return false;
        double xi[3];
        for (int i = 0; i < 3; i++)
            xi[i] = Ji[3 * i] * (x[0] - p0[0]) + Ji[3 * i + 1] * (x[1] - p0[1]) + Ji[3 * i + 2] * (x[2] - p0[2]);
        const double l0 = 1.0 - xi[0] - xi[1] - xi[2];
        if (xi[0] < -tol || xi[1] < -tol || xi[2] < -tol || l0 < -tol) return false;
        w[0] = l0; w[1] = xi[0]; w[2] = xi[1]; w[3] = xi[2];
        for (int a = 4; a < 8; a++) w[a] = 0;
        return true;
    }
    double xi[3] = {0, 0, 0};
    for (int it = 0; it < 30; it++) {
        double r[3] = {-x[0], -x[1], -x[2]}, J[9] = {0};
        for (int a = 0; a < 8; a++) {
            const double N = 0.125 * (1 + kH8S[a][0] * xi[0]) * (1 + kH8S[a][1] * xi[1]) * (1 + kH8S[a][2] * xi[2]);
            const double dN[3] = {0.125 * kH8S[a][0] * (1 + kH8S[a][1] * xi[1]) * (1 + kH8S[a][2] * xi[2]),
                                  0.125 * kH8S[a][1] * (1 + kH8S[a][0] * xi[0]) * (1 + kH8S[a][2] * xi[2]),
                                  0.125 * kH8S[a][2] * (1 + kH8S[a][0] * xi[0]) * (1 + kH8S[a][1] * xi[1])};
            for (int i = 0; i < 3; i++) {
                const double Xi = s.X[3 * (int64_t)cn[a] + i];
                r[i] += N * Xi;
                for (int j = 0; j < 3; j++) J[3 * i + j] += Xi * dN[j];
            }
        }
        double Ji[9];
        if (!invert3(J, Ji)) return false;
        double d[3];
        for (int i = 0; i < 3; i++) d[i] = Ji[3 * i] * r[0] + Ji[3 * i + 1] * r[1] + Ji[3 * i + 2] * r[2];
        for (int i = 0; i < 3; i++) xi[i] -= d[i];
        if (std::fabs(d[0]) + std::fabs(d[1]) + std::fabs(d[2]) < 1e-14) break;
        if (std::fabs(xi[0]) > 3 || std::fabs(xi[1]) > 3 || std::fabs(xi[2]) > 3) return false;
    }
    if (std::fabs(xi[0]) > 1 + 1e-7 || std::fabs(xi[1]) > 1 + 1e-7 || std::fabs(xi[2]) > 1 + 1e-7) return false;
    for (int a = 0; a < 8; a++)
        w[a] = 0.125 * (1 + kH8S[a][0] * xi[0]) * (1 + kH8S[a][1] * xi[1]) * (1 + kH8S[a][2] * xi[2]);
    return true;
}

// probe weights for scenario s: nodes [n][8] (scenario-local caller ids), w [n][8]
int locate_probes(tled_ctx *c, const Scenario &s, std::vector<int32_t> &nodes, std::vector<double> &w) {
    const int64_t n = (int64_t)s.probes.size() / 3;
    nodes.assign(8 * n, 0);
    w.assign(8 * n, 0.0);
    if (n == 0) return TLED_OK;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < s.nn; i++)
        for (int j = 0; j < 3; j++) {
            lo[j] = std::min(lo[j], s.X[3 * i + j]);
            hi[j] = std::max(hi[j], s.X[3 * i + j]);
        }
    const int G = std::max(1, (int)std::cbrt((double)s.ne / 2.0));
    auto cell = [&](double v, int j) {
        const double ext = hi[j] - lo[j];
        int q = ext > 0 ? (int)((v - lo[j]) / ext * G) : 0;
        return std::min(std::max(q, 0), G - 1);
    };
    std::vector<std::vector<int32_t>> grid((size_t)G * G * G);
    for (int64_t e = 0; e < s.ne; e++) {
        double bl[3] = {INFINITY, INFINITY, INFINITY}, bh[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int a = 0; a < s.npe; a++)
            for (int j = 0; j < 3; j++) {
                const double v = s.X[3 * (int64_t)s.conn[e * s.npe + a] + j];
                bl[j] = std::min(bl[j], v);
                bh[j] = std::max(bh[j], v);
            }
        for (int i = cell(bl[0], 0); i <= cell(bh[0], 0); i++)
            for (int j = cell(bl[1], 1); j <= cell(bh[1], 1); j++)
                for (int k = cell(bl[2], 2); k <= cell(bh[2], 2); k++) grid[((size_t)k * G + j) * G + i].push_back((int32_t)e);
    }
    for (int64_t q = 0; q < n; q++) {
        const double *x = &s.probes[3 * q];
        const auto &cand = grid[((size_t)cell(x[2], 2) * G + cell(x[1], 1)) * G + cell(x[0], 0)];
        bool found = false;
        for (int32_t e : cand) {
            double ww[8];
            if (locate_in(s, e, x, ww)) {
                for (int a = 0; a < 8; a++) {
                    nodes[8 * q + a] = a < s.npe ? s.conn[(int64_t)e * s.npe + a] : s.conn[(int64_t)e * s.npe];
                    w[8 * q + a] = a < s.npe ? ww[a] : 0.0;
                }
                found = true;
                break;
            }
        }
        if (!found) return fail(c, TLED_E_ARG, "probe " + std::to_string(q) + " lies outside the mesh");
    }
    return TLED_OK;
}

// ---------------------------------------------------------------------------
// plan: concatenate scenarios, order by decreasing length, tile
// ---------------------------------------------------------------------------
int ensure_plan(tled_ctx *c) {
    if (c->planned) return TLED_OK;
    if (c->sc.empty()) return fail(c, TLED_E_STATE, "the batch has no scenarios");
    for (auto &s : c->sc) {
        if (s.npe == 0) return fail(c, TLED_E_STATE, "tled_set_mesh has not been called");
        if (!s.have_mat) return fail(c, TLED_E_STATE, "tled_set_material has not been called");
    }
    const int ns = (int)c->sc.size();
    c->npe = c->npe_max = c->sc[0].npe;
    for (auto &s : c->sc) {
        if (s.npe != c->npe) c->npe = 0;
        c->npe_max = std::max(c->npe_max, s.npe);
    }
    c->nn = c->ne = c->n_probes = 0;
    c->has_mat = c->has_fib = false;
    const tled_material &m0 = c->sc[0].mat;
    for (auto &s : c->sc) {
        s.node_off = c->nn;
        s.elem_off = c->ne;
        s.probe_off = c->n_probes;
        c->nn += s.nn;
        c->ne += s.ne;
        c->n_probes += (int64_t)s.probes.size() / 3;
        c->has_mat |= !s.mat6.empty() || (ns > 1 && (s.mat.mu != m0.mu || s.mat.kappa != m0.kappa || s.mat.k1 != m0.k1 ||
                                                     s.mat.k2 != m0.k2 || s.mat.k != m0.k || s.mat.alpha != m0.alpha));
        c->has_fib |= !s.fib.empty() ||
                      (ns > 1 && (s.mat.a0[0] != m0.a0[0] || s.mat.a0[1] != m0.a0[1] || s.mat.a0[2] != m0.a0[2]));
    }
    if (c->nn > (int64_t)0x7fffffff || c->ne > (int64_t)0x7fffffff / 8)
        return fail(c, TLED_E_ARG, "combined mesh too large for 32-bit indices");
    // scenario ranks: decreasing n_steps (stable)
    c->scn_of_rank.resize(ns);
    std::iota(c->scn_of_rank.begin(), c->scn_of_rank.end(), 0);
    std::stable_sort(c->scn_of_rank.begin(), c->scn_of_rank.end(),
                     [&](int a, int b) { return c->sc[a].n_steps > c->sc[b].n_steps; });
    c->rank_of.assign(ns, 0);
    for (int r = 0; r < ns; r++) c->rank_of[c->scn_of_rank[r]] = r;
    // concatenated mesh (connectivity stride npe_max; per-element type when mixed)
    const int cs = c->npe_max;
    std::vector<double> X(3 * c->nn);
    std::vector<int32_t> conn((size_t)cs * c->ne, 0), group(c->ne);
    std::vector<int8_t> etype(c->npe ? 0 : c->ne);
    for (int si = 0; si < ns; si++) {
        const Scenario &s = c->sc[si];
        std::copy(s.X.begin(), s.X.end(), X.begin() + 3 * s.node_off);
        for (int64_t e = 0; e < s.ne; e++)
            for (int a = 0; a < s.npe; a++)
                conn[(size_t)cs * (s.elem_off + e) + a] = s.conn[(size_t)s.npe * e + a] + (int32_t)s.node_off;
        if (!etype.empty()) std::fill(etype.begin() + s.elem_off, etype.begin() + s.elem_off + s.ne, (int8_t)s.npe);
        std::fill(group.begin() + s.elem_off, group.begin() + s.elem_off + s.ne, c->rank_of[si]);
    }
    const int te = c->tile_override ? c->tile_override : c->sc[0].prm.tile_elems;
    int rc = tled::build_plan(cs, c->nn, X.data(), c->ne, conn.data(), etype.empty() ? nullptr : etype.data(),
                              ns > 1 ? group.data() : nullptr, te, c->plan, c->err);
    if (rc) return rc;
    // active prefixes per rank
    const Plan &p = c->plan;
    c->tiles_upto.assign(ns + 1, 0);
    c->shared_upto.assign(ns + 1, 0);
    std::vector<int32_t> scn_of_node(c->nn);
    for (int si = 0; si < ns; si++)
        std::fill(scn_of_node.begin() + c->sc[si].node_off, scn_of_node.begin() + c->sc[si].node_off + c->sc[si].nn, si);
    for (int t = 0; t < p.n_tiles; t++) {
        const int32_t eo = p.elem_old[(size_t)t * tled::kTile];
        c->tiles_upto[group[eo] + 1]++;
    }
    for (int64_t sidx = 0; sidx < p.n_shared; sidx++)
        c->shared_upto[c->rank_of[scn_of_node[p.node_old[p.n_interior + sidx]]] + 1]++;
    for (int r = 0; r < ns; r++) {
        c->tiles_upto[r + 1] += c->tiles_upto[r];
        c->shared_upto[r + 1] += c->shared_upto[r];
    }
    // probes
    c->probe_node.assign(8 * c->n_probes, 0);
    c->probe_w.assign(8 * c->n_probes, 0.f);
    for (auto &s : c->sc) {
        std::vector<int32_t> pn;
        std::vector<double> pw;
        rc = locate_probes(c, s, pn, pw);
        if (rc) return rc;
        for (size_t i = 0; i < pn.size(); i++) {
            c->probe_node[8 * s.probe_off + i] = p.node_new[pn[i] + s.node_off];
            c->probe_w[8 * s.probe_off + i] = (float)pw[i];
        }
    }
    c->L = make_layout(c);
    c->planned = true;
    return TLED_OK;
}

void drop_graphs(tled_ctx *c) {
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
}

void invalidate(tled_ctx *c) {
    drop_graphs(c);
    c->planned = false;
    c->inited = false;
}

ScenDev scen_dev(const Scenario &s) {
    ScenDev d{};
    const double dt = s.dt, g = s.prm.gamma;
    d.dt = dt;
    d.dtf = (float)dt;
    d.inv_dt = (float)(1.0 / dt);
    d.damp_a = (float)((1.0 - 0.5 * g * dt) / (1.0 + 0.5 * g * dt));
    d.damp_b = (float)(dt / (1.0 + 0.5 * g * dt));
    for (int i = 0; i < 4; i++) {
        if (i < s.mat.n_prony) {
            d.pr_a[i] = (float)(dt * s.mat.prony_g[i] / (dt + s.mat.prony_tau[i]));
            d.pr_b[i] = (float)(s.mat.prony_tau[i] / (dt + s.mat.prony_tau[i]));
        }
    }
    d.Qm = (float)s.mat.Qm;
    d.src_off = s.src_off;
    d.n_src = (int)s.src.size();
    d.n_sub = s.prm.n_sub;
    d.dt_th = s.prm.n_sub == 1 ? dt : s.dt_thermal;
    d.dtf_th = (float)d.dt_th;
    return d;
}

int upload_scenarios(tled_ctx *c) {
    std::vector<ScenDev> d(c->sc.size());
    std::vector<double> src(tled::kSrcRow * (size_t)source_capacity(c), 0.0);
    for (size_t i = 0; i < c->sc.size(); i++) {
        d[i] = scen_dev(c->sc[i]);
        for (size_t q = 0; q < c->sc[i].src.size(); q++) {
            const tled_source &s = c->sc[i].src[q];
            double *r = &src[tled::kSrcRow * (c->sc[i].src_off + q)];
            r[0] = s.c0[0]; r[1] = s.c0[1]; r[2] = s.c0[2];
            r[3] = s.vel[0]; r[4] = s.vel[1]; r[5] = s.vel[2];
            r[6] = s.sigma; r[7] = s.power; r[8] = s.t_on; r[9] = s.t_off; r[10] = (double)s.shape;
        }
    }
    // stream-ordered after the steps already enqueued, without a host wait: a single
    // problem's tables travel as the parameters of a one-block kernel; a batch's (larger)
    // tables are pageable host memory, which the runtime stages before the copies return
    if (!c->batch && src.size() == (size_t)tled::kMaxSources * tled::kSrcRow) {
        tled::SingleScenUpload u{};
        u.d = d[0];
        std::copy(src.begin(), src.end(), u.src);
        CUDA_TRY(c, tled::launch_single_upload(u, dptr<ScenDev>(c, c->L.scn), dptr<double>(c, c->L.src), c->stream));
        return TLED_OK;
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.scn, d.data(), sizeof(ScenDev) * d.size(), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.src, src.data(), 8 * src.size(), cudaMemcpyHostToDevice, c->stream));
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
    const double T0 = c->sc[0].mat.T0;
    std::vector<float4> xu(nn), lo(nn), vel(nn);
    for (int64_t g = 0; g < nn; g++) {
        const int64_t i = p.node_old[g];
        float h[4], l[4];
        for (int d = 0; d < 3; d++) split_ff(u ? u[3 * i + d] : 0.0, h[d], l[d]);
        split_ff(T ? T[i] - T0 : 0.0, h[3], l[3]);
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
    if (cem_on(c)) CUDA_TRY(c, cudaMemsetAsync(c->ws + c->L.cem, 0, 8 * (size_t)nn, c->stream));  // dose restarts
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return TLED_OK;
}

// every scenario's clock: `step` steps taken, time t0 + step dt (t0 = 0 for batches)
int upload_clock(tled_ctx *c, int64_t step, double t0) {
    const size_t ns = c->sc.size();
    std::vector<double> tb(ns, c->batch ? 0.0 : t0);
    std::vector<int64_t> sb(ns, step);
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.scn_time, tb.data(), 8 * ns, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.scn_step, sb.data(), 8 * ns, cudaMemcpyHostToDevice, c->stream));
    unsigned st[4] = {0u, 0xffffffffu, 0xffffffffu, 0u};
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.status, st, 16, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->step = step;
    c->t0 = t0;
    c->active_host[0] = c->active_host[1] = -1;
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

// number of scenarios still running at step `step`
int active_ranks(const tled_ctx *c, int64_t step) {
    int r = 0;
    while (r < (int)c->sc.size() && c->sc[c->scn_of_rank[r]].n_steps > step) r++;
    return r;
}

int set_active(tled_ctx *c, int ranks) {
    const int na[2] = {(int)c->tiles_upto[ranks], (int)c->shared_upto[ranks]};
    if (na[0] == c->active_host[0] && na[1] == c->active_host[1]) return TLED_OK;
    c->active_host[0] = na[0];
    c->active_host[1] = na[1];
    // stream-ordered copy from the context's own host array (kept alive with the context)
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.n_active, c->active_host, 8, cudaMemcpyHostToDevice, c->stream));
    return TLED_OK;
}

int validate_material(tled_ctx *c, const tled_material *m, int64_t ne, const double *per_elem, const double *fibre) {
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
    if (!(m->alpha_fibre_ratio >= 0) || !(m->k_fibre_ratio >= 0) || !std::isfinite(m->alpha_fibre_ratio) ||
        !std::isfinite(m->k_fibre_ratio))
        return fail(c, TLED_E_ARG, "fibre ratios must be finite and >= 0 (0 or 1: isotropic)");
    if (per_elem)
        for (int64_t i = 0; i < 6 * ne; i++)
            if (!std::isfinite(per_elem[i]) || (i % 6 != 5 && per_elem[i] < 0))
                return fail(c, TLED_E_ARG, "bad per-element material of element " + std::to_string(i / 6));
    if (fibre)
        for (int64_t e = 0; e < ne; e++) {
            const double *a = fibre + 3 * e;
            double n = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
            if (!(std::fabs(n - 1.0) < 1e-6))
                return fail(c, TLED_E_ARG, "fibre of element " + std::to_string(e) + " is not a unit vector");
        }
    return TLED_OK;
}

int require_single(tled_ctx *c) {
    if (c->batch) return fail(c, TLED_E_STATE, "set-up calls apply to single-scenario contexts; use tled_batch_add");
    return TLED_OK;
}

// The two stable-step bounds of a scenario (R16) and the mass scale in use.  With
// mass_scale < 0 (automatic, R17) the mechanical mass is scaled by
// s_m = max(1, (dt / (dt_safety dt_mech))^2), dt_mech the CFL bound of the unscaled
// mesh, which makes the fixed dt the safe mechanical step; the scaled mesh's bound
// is then dt_mech sqrt(s_m).  E_ARG if dt exceeds the thermal step's safe fraction.
int resolve_bounds(tled_ctx *c, Scenario &s) {
    if (s.dt_valid) return TLED_OK;  // mesh, material and parameters unchanged since: the bounds stand
    tled_params q = s.prm;
    const bool automatic = q.mass_scale < 0;
    if (automatic) q.mass_scale = 1.0;
    tled::stable_dt(s.npe, s.nn, s.X.data(), s.ne, s.conn.data(), s.mat, s.mat6.empty() ? nullptr : s.mat6.data(),
                    s.fib.empty() ? nullptr : s.fib.data(), q, &s.dt_mech, &s.dt_th);
    s.mass_scale = q.mass_scale;
    if (automatic) {
        if (s.prm.dt > s.prm.dt_safety * s.dt_th)
            return fail(c, TLED_E_ARG, "dt " + std::to_string(s.prm.dt) + " exceeds the thermal stable step " +
                                           std::to_string(s.prm.dt_safety * s.dt_th));
        const double r = s.prm.dt / s.prm.n_sub / (s.prm.dt_safety * s.dt_mech);  // the mechanical step
        s.mass_scale = std::max(1.0, r * r);
        s.dt_mech *= std::sqrt(s.mass_scale);
    }
    s.dt_valid = true;
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

// Persisting-L2 window of the streamed step: the shared nodes' (u, theta) and the partial sums,
// which the tile kernel writes and the shared-node kernel reads back within the step, and which
// the tiles around a shared node read several times (the rest of the step streams ~10x more
// bytes through L2 and would evict them).  The set-aside is this process's CUDA context limit;
// the previous value comes back when the context is destroyed.
void release_l2(tled_ctx *c) {
    if (!c->l2_set) return;
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, c->l2_prev);
    c->l2_set = false;
}
void setup_l2(tled_ctx *c, tled::StepArgs &A) {
    A.l2_base = nullptr;
    A.l2_bytes = 0;
    A.l2_hit = 0.f;
    const Plan &p = c->plan;
    if (p.n_shared <= 0) return;
    int max_set = 0, max_win = 0, l2 = 0;
    if (cudaDeviceGetAttribute(&max_set, cudaDevAttrMaxPersistingL2CacheSize, c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device) != cudaSuccess || max_set <= 0 ||
        max_win <= 0 || l2 <= 0)
        return;
    char *lo = c->ws + c->L.xu + 16 * (size_t)p.n_interior;
    char *hi = c->ws + c->L.partials + 16 * (size_t)p.n_partials;
    const size_t win = std::min<size_t>((size_t)(hi - lo), (size_t)max_win);
    // at most kL2PersistShare of L2 is set aside: the rest of the step streams through the
    // remainder (a 256-scenario batch whose window would take the device maximum, 63 % of L2,
    // ran 16.0 -> 13.9 scenario-solves/s)
    const size_t cap = (size_t)(kL2PersistShare * (double)l2);
    const size_t set = std::min<size_t>({win, (size_t)max_set, cap});
    size_t prev = 0;
    if (cudaDeviceGetLimit(&prev, cudaLimitPersistingL2CacheSize) != cudaSuccess) return;
    if (set > prev) {
        if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, set) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        if (!c->l2_set) c->l2_prev = prev;
        c->l2_set = true;
    }
    A.l2_base = lo;
    A.l2_bytes = win;
    A.l2_hit = (float)std::min(1.0, (double)set / (double)win);
}

static int create_ctx(tled_ctx **out, int device, void *cuda_stream, bool batch) {
    if (!out) return TLED_E_ARG;
    *out = nullptr;
    tled_ctx *c = new tled_ctx();
    c->batch = batch;
    if (!batch) {
        c->sc.resize(1);
        c->sc[0].prm = default_params();
    }
    if (device == -1) {  // host-only: planning and validation without a GPU
        c->device = -1;
        *out = c;
        return TLED_OK;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev || cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return TLED_E_CUDA;
    }
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return TLED_E_CUDA;
    }
    *out = c;
    return TLED_OK;
}

int tled_create(tled_ctx **out, int device, void *cuda_stream) { return create_ctx(out, device, cuda_stream, false); }

int tled_batch_create(tled_ctx **out, int device, void *cuda_stream) {
    return create_ctx(out, device, cuda_stream, true);
}

int tled_destroy(tled_ctx *c) {
    if (!c) return TLED_E_ARG;
    if (c->device >= 0) {
        cudaSetDevice(c->device);
        drop_graphs(c);
        if (c->cap) cudaStreamDestroy(c->cap);
        release_l2(c);
    }
    delete c;
    return TLED_OK;
}

const char *tled_last_error(const tled_ctx *c) { return c ? c->err.c_str() : "null context"; }

int tled_set_mesh(tled_ctx *c, int elem_type, int64_t n_nodes, const double *X0, int64_t n_elems,
                  const int32_t *conn) {
    if (!c) return TLED_E_ARG;
    if (int rc = require_single(c)) return rc;
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
    Scenario &s = single(c);
    s.npe = elem_type;
    s.nn = n_nodes;
    s.ne = n_elems;
    s.X.assign(X0, X0 + 3 * n_nodes);
    s.conn.assign(conn, conn + elem_type * n_elems);
    s.mask.assign(n_nodes, 0);
    s.ubar.clear();
    s.have_mat = false;
    s.mat6.clear();
    s.fib.clear();
    s.probes.clear();
    s.dt_valid = false;
    return TLED_OK;
}

int tled_set_material(tled_ctx *c, const tled_material *m, const double *per_elem, const double *fibre) {
    if (!c || !m) return fail(c, TLED_E_ARG, "NULL material");
    if (int rc = require_single(c)) return rc;
    Scenario &s = single(c);
    if (s.npe == 0) return fail(c, TLED_E_STATE, "set the mesh first");
    if (int rc = validate_material(c, m, s.ne, per_elem, fibre)) return rc;
    invalidate(c);
    s.mat = *m;
    s.mat6.assign(per_elem ? per_elem : nullptr, per_elem ? per_elem + 6 * s.ne : nullptr);
    s.fib.assign(fibre ? fibre : nullptr, fibre ? fibre + 3 * s.ne : nullptr);
    s.have_mat = true;
    s.dt_valid = false;
    return TLED_OK;
}

int tled_set_bcs(tled_ctx *c, const uint8_t *mask, const double *ubar, double ramp_time) {
    if (!c) return TLED_E_ARG;
    if (int rc = require_single(c)) return rc;
    Scenario &s = single(c);
    if (s.npe == 0) return fail(c, TLED_E_STATE, "set the mesh first");
    if (!mask) return fail(c, TLED_E_ARG, "NULL mask");
    if (!(ramp_time >= 0)) return fail(c, TLED_E_ARG, "ramp_time must be >= 0");
    invalidate(c);
    s.mask.assign(mask, mask + s.nn);
    s.ubar.assign(ubar ? ubar : nullptr, ubar ? ubar + 3 * s.nn : nullptr);
    s.ramp = ramp_time;
    return TLED_OK;
}

int tled_set_heat_sources(tled_ctx *c, int32_t n, const tled_source *src) {
    if (!c) return TLED_E_ARG;
    if (int rc = require_single(c)) return rc;
    if (n < 0 || n > tled::kMaxSources || (n > 0 && !src)) return fail(c, TLED_E_ARG, "0 <= n <= 16 sources");
    for (int i = 0; i < n; i++)
        if (!(src[i].sigma > 0) || !std::isfinite(src[i].power) ||
            (src[i].shape != TLED_SRC_GAUSSIAN && src[i].shape != TLED_SRC_SPHERE))
            return fail(c, TLED_E_ARG, "source sigma must be > 0 and its shape TLED_SRC_GAUSSIAN or TLED_SRC_SPHERE");
    single(c).src.assign(src, src + n);
    if (c->inited) {
        cudaSetDevice(c->device);
        return upload_scenarios(c);
    }
    return TLED_OK;
}

int tled_set_params(tled_ctx *c, const tled_params *p) {
    if (!c) return TLED_E_ARG;
    if (int rc = require_single(c)) return rc;
    tled_params q = p ? *p : default_params();
    if (q.dt < 0 || !(q.dt_safety > 0) || q.gamma < 0 || q.kappa_hg < 0 || q.kappa_hgT < 0 || q.tile_elems < 0)
        return fail(c, TLED_E_ARG, "invalid solver parameters");
    if (q.mass_scale < 0 ? !(q.dt > 0) : !(q.mass_scale >= 1.0))
        return fail(c, TLED_E_ARG, "mass_scale must be >= 1, or < 0 (automatic) with a fixed dt > 0");
    if (q.n_sub == 0) q.n_sub = 1;
    if (q.n_sub < 1 || q.n_sub > 1000000) return fail(c, TLED_E_ARG, "n_sub must be 1..1000000 (0 = 1)");
    invalidate(c);
    single(c).prm = q;
    single(c).dt_valid = false;
    return TLED_OK;
}

int tled_set_probes(tled_ctx *c, int64_t n, const double *xyz) {
    if (!c) return TLED_E_ARG;
    if (int rc = require_single(c)) return rc;
    if (single(c).npe == 0) return fail(c, TLED_E_STATE, "set the mesh first");
    if (n < 0 || (n > 0 && !xyz)) return fail(c, TLED_E_ARG, "bad probe list");
    for (int64_t i = 0; i < 3 * n; i++)
        if (!std::isfinite(xyz[i])) return fail(c, TLED_E_ARG, "non-finite probe coordinate");
    invalidate(c);
    single(c).probes.assign(xyz, xyz + 3 * n);
    return TLED_OK;
}

int tled_batch_add(tled_ctx *b, const tled_ctx *scenario, int64_t n_steps, int32_t *index) {
    if (!b || !scenario) return fail(b, TLED_E_ARG, "NULL context");
    if (!b->batch) return fail(b, TLED_E_STATE, "not a batch context (use tled_batch_create)");
    if (scenario->batch) return fail(b, TLED_E_ARG, "a batch cannot be added to a batch");
    if (n_steps <= 0) return fail(b, TLED_E_ARG, "n_steps must be > 0");
    const Scenario &s = scenario->sc[0];
    if (s.npe == 0 || !s.have_mat) return fail(b, TLED_E_STATE, "the scenario needs a mesh and a material");
    if (s.prm.flags & TLED_CEM43) return fail(b, TLED_E_ARG, "CEM43 is tracked for single problems only");
    if (!b->sc.empty()) {
        const Scenario &f = b->sc[0];
        const tled_material &a = f.mat, &m = s.mat;
        bool same = a.n_prony == m.n_prony && a.T0 == m.T0 && a.Ta == m.Ta && a.lnA == m.lnA && a.Ea == m.Ea &&
                    fibre_ratio(a.alpha_fibre_ratio) == fibre_ratio(m.alpha_fibre_ratio) &&
                    fibre_ratio(a.k_fibre_ratio) == fibre_ratio(m.k_fibre_ratio) &&
                    a.beta_c == m.beta_c && a.beta_k == m.beta_k && a.T_ref == m.T_ref &&
                    f.prm.flags == s.prm.flags && f.prm.kappa_hg == s.prm.kappa_hg &&
                    f.prm.kappa_hgT == s.prm.kappa_hgT && f.ramp == s.ramp;
        if (!same)
            return fail(b, TLED_E_ARG,
                        "scenarios of a batch must share n_prony, T0, Ta, Arrhenius constants, c/k slopes, fibre ratios, flags, "
                        "hourglass coefficients and ramp time");
    }
    invalidate(b);
    b->sc.push_back(s);
    b->sc.back().n_steps = n_steps;
    if (index) *index = (int32_t)b->sc.size() - 1;
    return TLED_OK;
}

int tled_scenario_info(tled_ctx *c, int32_t idx, int64_t *info) {
    if (!c || !info) return fail(c, TLED_E_ARG, "NULL info");
    if (idx < 0 || idx >= (int32_t)c->sc.size()) return fail(c, TLED_E_ARG, "scenario index out of range");
    if (int rc = ensure_plan(c)) return rc;
    const Scenario &s = c->sc[idx];
    info[0] = s.node_off;
    info[1] = s.nn;
    info[2] = s.elem_off;
    info[3] = s.ne;
    info[4] = s.n_steps == INT64_MAX ? -1 : s.n_steps;
    info[5] = std::min<int64_t>(c->step, s.n_steps);
    info[6] = s.probe_off;
    info[7] = (int64_t)s.probes.size() / 3;
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
    drop_graphs(c);
    c->inited = false;
    c->ws = (char *)dev_workspace;
    const Plan &p = c->plan;
    const int npe = c->npe;  // 0 for a mixed batch
    const int64_t nn = c->nn;
    const int ns = (int)c->sc.size();
    // --- per-scenario time steps and source offsets
    int src_off = 0;
    for (auto &s : c->sc) {
        if ((rc = resolve_bounds(c, s))) return rc;
        // the step is the mechanical (sub)step; the thermal step is n_sub of them
        const int ns_ = s.prm.n_sub;
        const double dt_thermal = s.prm.dt > 0 ? s.prm.dt : s.prm.dt_safety * std::min(ns_ * s.dt_mech, s.dt_th);
        s.dt = ns_ == 1 ? dt_thermal : dt_thermal / ns_;
        s.dt_thermal = dt_thermal;
        s.src_off = src_off;
        src_off += c->batch ? (int)s.src.size() : kSingleSources;
    }
    // --- element records (tile-blocked), lumped masses, nodal constants
    const int64_t nep = p.ne_pad;
    const size_t rb = rec_bytes(c);  // tile stride
    const int kT = tled::kTile;
    std::vector<int32_t> scn_of_elem(c->ne);
    for (int si = 0; si < ns; si++)
        std::fill(scn_of_elem.begin() + c->sc[si].elem_off, scn_of_elem.begin() + c->sc[si].elem_off + c->sc[si].ne, si);
    std::vector<char> rec((size_t)p.n_tiles * rb, 0);
    std::vector<double> Mn(nn, 0.0), Cn(nn, 0.0), Vn(nn, 0.0), Kb(nn, 0.0);
    // every element an H8 axis-aligned box: the brick instance, whose records hold the
    // diagonal of J0^-1 only
    bool brick = !(c->sc[0].prm.flags & TLED_GENERAL_H8);
    for (int64_t e = 0; e < nep && brick; e++) {
        const int64_t eo = p.elem_old[e];
        if (eo < 0) continue;
        const Scenario &s = c->sc[scn_of_elem[eo]];
        brick = s.npe == 8 && tled::brick_element(s.X.data(), s.conn.data() + (eo - s.elem_off) * 8);
    }
    for (int64_t e = 0; e < nep; e++) {
        const int64_t eo = p.elem_old[e];
        if (eo < 0) continue;  // padding slot
        const Scenario &s = c->sc[scn_of_elem[eo]];
        const int64_t el = eo - s.elem_off;
        const int ke = s.npe;  // this element's (and its tile's) type
        const int32_t *cn = s.conn.data() + el * ke;
        double Ji[9], V;
        tled::element_geometry(ke, s.X.data(), cn, Ji, &V);
        char *r = rec.data() + (size_t)(e / kT) * rb;
        const int ei = (int)(e % kT);
        float *cf = reinterpret_cast<float *>(r) + ei;
        int q = 0;
        for (int j = 0; j < 9; j += brick ? 4 : 1) cf[(q++) * kT] = (float)Ji[j];
        cf[(q++) * kT] = (float)V;
        if (c->has_mat) {
            if (!s.mat6.empty()) {
                for (int j = 0; j < 6; j++) cf[(q++) * kT] = (float)s.mat6[6 * el + j];
            } else {
                const double u[6] = {s.mat.mu, s.mat.kappa, s.mat.k1, s.mat.k2, s.mat.k, s.mat.alpha};
                for (int j = 0; j < 6; j++) cf[(q++) * kT] = (float)u[j];
            }
        }
        if (c->has_fib)
            for (int j = 0; j < 3; j++) cf[(q++) * kT] = (float)(s.fib.empty() ? s.mat.a0[j] : s.fib[3 * el + j]);
        for (int a = 0; a < ke; a++) {
            const int64_t i = cn[a] + s.node_off;
            Mn[i] += s.mass_scale * s.mat.rho * V / ke;
            Cn[i] += s.mat.rho * s.mat.c * V / ke;
            Vn[i] += V / ke;
            Kb[i] += s.mat.wb_cb * V / ke;
        }
    }
    std::vector<float4> X0(nn), nodec(nn), ub;
    bool any_ubar = false;
    for (auto &s : c->sc) any_ubar |= !s.ubar.empty();
    if (any_ubar) ub.assign(nn, make_float4(0.f, 0.f, 0.f, 0.f));
    std::vector<int32_t> node_new(p.node_new.begin(), p.node_new.end());
    std::vector<int32_t> scn_of_node(nn);
    for (int si = 0; si < ns; si++)
        std::fill(scn_of_node.begin() + c->sc[si].node_off, scn_of_node.begin() + c->sc[si].node_off + c->sc[si].nn, si);
    for (int64_t g = 0; g < nn; g++) {
        const int64_t i = p.node_old[g];
        const Scenario &s = c->sc[scn_of_node[i]];
        const int64_t li = i - s.node_off;
        X0[g] = make_float4((float)s.X[3 * li], (float)s.X[3 * li + 1], (float)s.X[3 * li + 2], (float)Vn[i]);
        unsigned mk = s.mask[li] & 15u;
        float mkf;
        std::memcpy(&mkf, &mk, 4);
        nodec[g] = make_float4((float)(1.0 / Mn[i]), (float)(1.0 / Cn[i]), mkf, (float)Kb[i]);
        if (!s.ubar.empty())
            ub[g] = make_float4((float)s.ubar[3 * li], (float)s.ubar[3 * li + 1], (float)s.ubar[3 * li + 2], 0.f);
    }
    std::vector<int32_t> tile_scn(p.n_tiles), shared_scn(p.n_shared);
    for (int t = 0; t < p.n_tiles; t++) tile_scn[t] = scn_of_elem[p.elem_old[(size_t)t * kT]];
    for (int64_t sidx = 0; sidx < p.n_shared; sidx++) shared_scn[sidx] = scn_of_node[p.node_old[p.n_interior + sidx]];
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
    CUDA_TRY(c, up(L.pattern, p.patterns.data(), 2 * p.patterns.size()));
    CUDA_TRY(c, up(L.sh_rowptr, p.sh_rowptr.data(), 4 * p.sh_rowptr.size()));
    CUDA_TRY(c, up(L.part_pos, p.part_pos.data(), 4 * p.part_pos.size()));
    CUDA_TRY(c, up(L.node_new, node_new.data(), 4 * nn));
    CUDA_TRY(c, up(L.tile_scn, tile_scn.data(), 4 * tile_scn.size()));
    CUDA_TRY(c, up(L.shared_scn, shared_scn.data(), 4 * shared_scn.size()));
    CUDA_TRY(c, up(L.probe_node, c->probe_node.data(), 4 * c->probe_node.size()));
    CUDA_TRY(c, up(L.probe_w, c->probe_w.data(), 4 * c->probe_w.size()));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->inited = true;  // buffers placed; the rest uses the regular paths
    if ((rc = upload_scenarios(c))) return rc;
    if ((rc = write_state(c, nullptr, nullptr, nullptr, nullptr, nullptr))) return rc;
    if ((rc = upload_clock(c, 0, 0.0))) return rc;
    {  // the active prefixes on the device from the start (every launch reads them)
        const int ranks = active_ranks(c, 0);
        if (ranks > 0 && (rc = set_active(c, ranks))) return rc;
    }
    // --- kernel arguments
    const Scenario &s0 = c->sc[0];
    const tled_material &m = s0.mat;
    StepArgs &A = c->A;
    A = StepArgs{};
    A.xu = dptr<float4>(c, L.xu);
    A.lo = dptr<float4>(c, L.lo);
    A.vel = dptr<float4>(c, L.vel);
    A.X0 = dptr<float4>(c, L.X0);
    A.nodec = dptr<float4>(c, L.nodec);
    A.ubar = any_ubar ? dptr<float4>(c, L.ubar) : nullptr;
    A.elem_rec = dptr<char>(c, L.elem_rec);
    A.rec_bytes = (int64_t)rb;
    A.has_mat = c->has_mat;
    A.has_fib = c->has_fib;
    A.visc = dptr<float>(c, L.visc);
    A.ne = nep;
    A.tile_info = dptr<int>(c, L.tile_info);
    A.tile_shared = dptr<int>(c, L.tile_shared);
    A.pattern = dptr<uint16_t>(c, L.pattern);
    A.partials = dptr<float4>(c, L.partials);
    A.n_partials = p.n_partials;
    A.part_pos = dptr<int>(c, L.part_pos);
    A.sh_rowptr = dptr<int>(c, L.sh_rowptr);
    A.n_interior = p.n_interior;
    A.n_shared = p.n_shared;
    A.scn = dptr<ScenDev>(c, L.scn);
    A.src = dptr<double>(c, L.src);
    A.scn_time = dptr<double>(c, L.scn_time);
    A.scn_step = dptr<int64_t>(c, L.scn_step);
    A.tile_scn = dptr<int>(c, L.tile_scn);
    A.shared_scn = dptr<int>(c, L.shared_scn);
    A.n_active = dptr<int>(c, L.n_active);
    A.n_scn = ns;
    A.status = dptr<unsigned>(c, L.status);
    A.mu = (float)m.mu; A.kappa = (float)m.kappa; A.k1 = (float)m.k1; A.k2 = (float)m.k2;
    A.kc = (float)m.k; A.alpha = (float)m.alpha;
    A.a0x = (float)m.a0[0]; A.a0y = (float)m.a0[1]; A.a0z = (float)m.a0[2];
    A.n_prony = m.n_prony;
    A.flags = s0.prm.flags;
    A.beta_c = (float)m.beta_c;
    A.beta_k = (float)m.beta_k;
    A.Tref_m_T0 = (float)(m.T_ref - m.T0);
    A.theta_a = (float)(m.Ta - m.T0);
    A.lnA = (float)m.lnA;
    A.Ea_R = (float)(m.Ea / 8.314);
    A.T0_K = (float)(m.T0 + 273.15);
    A.khg = (float)s0.prm.kappa_hg;
    A.khgT = (float)s0.prm.kappa_hgT;
    A.ramp_time = s0.ramp;
    A.cem = cem_on(c) ? dptr<double>(c, L.cem) : nullptr;
    A.ani_alpha = (float)fibre_ratio(m.alpha_fibre_ratio);
    A.ani_k = (float)fibre_ratio(m.k_fibre_ratio);
    A.ani = fibre_ratio(m.alpha_fibre_ratio) != 1.0 || fibre_ratio(m.k_fibre_ratio) != 1.0;
    A.brick = brick;  // (TLED_GENERAL_H8 excluded above)
    A.T0 = m.T0;
    A.n_tiles = p.n_tiles;
    A.pat_stride = p.pat_stride;
    int n_sm = 0;
    CUDA_TRY(c, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device));
    A.wide = npe == 4 && p.n_tiles > tled::kTileCtasPerSm * n_sm;
    tled::tile_smem_layout(A, npe);
    CUDA_TRY(c, tled::tile_kernel_setup(A, npe));
    setup_l2(c, A);
    c->tile_ctas = tled::tile_grid(A, npe, n_sm);
    c->shared_blocks = tled::shared_grid(A, n_sm);
    if (c->grid_override > 0) c->tile_ctas = std::min(c->tile_ctas, c->grid_override);
    // resident mode: possible when every scenario (one element type) fits one
    // CTA's shared memory; one descriptor per rank (CTA b runs the scenario of rank b)
    c->res_ok = c->resident = false;
    if (npe != 0) {
        std::vector<tled::ResDesc> rd(ns);
        int nn_max = 0, nt_max = 0, np_max = 0, nsh_max = 0;
        for (int r = 0; r < ns; r++) {
            tled::ResDesc d{};
            d.scn = c->scn_of_rank[r];
            d.t0 = (int)c->tiles_upto[r];
            d.n_t = (int)(c->tiles_upto[r + 1] - c->tiles_upto[r]);
            d.i0 = d.n_t ? p.tile_info[(size_t)d.t0 * tled::kTileInfo + 2] : 0;
            for (int t = d.t0; t < d.t0 + d.n_t; t++) d.n_int += p.tile_info[(size_t)t * tled::kTileInfo + 3];
            d.s0 = (int)c->shared_upto[r];
            d.n_sh = (int)(c->shared_upto[r + 1] - c->shared_upto[r]);
            d.p0 = p.sh_rowptr[d.s0];
            d.n_part = p.sh_rowptr[d.s0 + d.n_sh] - d.p0;
            rd[r] = d;
            nn_max = std::max(nn_max, d.n_int + d.n_sh);
            nt_max = std::max(nt_max, d.n_t);
            np_max = std::max(np_max, d.n_part);
            nsh_max = std::max(nsh_max, d.n_sh);
        }
        const int need = tled::resident_smem_layout(A, npe, nn_max, nt_max, np_max, nsh_max);
        if (need <= tled::resident_smem_limit() && nn_max < 65536) {
            CUDA_TRY(c, cudaMemcpyAsync(c->ws + L.res, rd.data(), sizeof(tled::ResDesc) * ns, cudaMemcpyHostToDevice,
                                        c->stream));
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
            A.res = dptr<tled::ResDesc>(c, L.res);
            CUDA_TRY(c, tled::resident_kernel_setup(A, npe));
            c->res_ok = true;
            c->resident = c->mode_override == 2 || (c->mode_override == 0 && !(s0.prm.flags & TLED_STREAMED));
        }
    }
    // grid-resident mode: a single problem whose tiles (one CTA each) all fit co-resident CTAs of
    // a cooperative launch
    c->coop_ok = c->coop = false;
    int coop_dev = 0;
    CUDA_TRY(c, cudaDeviceGetAttribute(&coop_dev, cudaDevAttrCooperativeLaunch, c->device));
    if (npe != 0 && ns == 1 && !c->resident && coop_dev && p.n_tiles > 0) {
        tled::coop_smem_layout(A, npe);
        if (A.cs_total <= tled::resident_smem_limit() && p.n_tiles <= kCoopTilesMax) {
            CUDA_TRY(c, tled::coop_kernel_setup(A, npe));
            const int per_sm = tled::coop_ctas_per_sm(A, npe);
            if ((int64_t)per_sm * n_sm >= p.n_tiles) {
                c->coop_ok = true;
                A.gbar = dptr<unsigned>(c, L.gbar);
                c->coop = c->mode_override == 3 || (c->mode_override == 0 && !(s0.prm.flags & TLED_STREAMED));
            }
        }
    }
    // set-up hash for checkpoints
    uint64_t h = 1469598103934665603ULL;
    for (auto &s : c->sc) {
        h = fnv1a(s.X.data(), 8 * s.X.size(), h);
        h = fnv1a(s.conn.data(), 4 * s.conn.size(), h);
        h = fnv1a(&s.mat, sizeof(tled_material), h);
        h = fnv1a(&s.prm, sizeof(tled_params), h);
        h = fnv1a(&s.dt, 8, h);
        h = fnv1a(&s.prm.n_sub, 4, h);
    }
    c->setup_hash = h;
    return TLED_OK;
}

int tled_get_dt(tled_ctx *c, double *dt, double *dt_mech, double *dt_thermal) {
    if (!c) return TLED_E_ARG;
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (dt) *dt = c->sc[0].dt;
    if (dt_mech) *dt_mech = c->sc[0].dt_mech;
    if (dt_thermal) *dt_thermal = c->sc[0].dt_th;
    return TLED_OK;
}

int tled_stable_dt(tled_ctx *c, double *dt_mech, double *dt_thermal) {
    if (!c || !dt_mech || !dt_thermal) return fail(c, TLED_E_ARG, "NULL argument");
    if (int rc = require_single(c)) return rc;
    Scenario &s = single(c);
    if (s.npe == 0 || !s.have_mat) return fail(c, TLED_E_STATE, "set the mesh and the material first");
    if (int rc = resolve_bounds(c, s)) return rc;
    *dt_mech = s.dt_mech;
    *dt_thermal = s.dt_th;
    return TLED_OK;
}

int tled_get_mass_scale(tled_ctx *c, int32_t idx, double *mass_scale) {
    if (!c || !mass_scale) return fail(c, TLED_E_ARG, "NULL argument");
    if (idx < 0 || idx >= (int32_t)c->sc.size()) return fail(c, TLED_E_ARG, "scenario index out of range");
    Scenario &s = c->sc[idx];
    if (s.npe == 0 || !s.have_mat) return fail(c, TLED_E_STATE, "set the mesh and the material first");
    if (int rc = resolve_bounds(c, s)) return rc;
    *mass_scale = s.mass_scale;
    return TLED_OK;
}

int tled_scenario_dt(tled_ctx *c, int32_t idx, double *dt) {
    if (!c || !dt) return fail(c, TLED_E_ARG, "NULL argument");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (idx < 0 || idx >= (int32_t)c->sc.size()) return fail(c, TLED_E_ARG, "scenario index out of range");
    *dt = c->sc[idx].dt;
    return TLED_OK;
}

static int capture_graph(tled_ctx *c, int K, cudaGraphExec_t *out);
// the step graphs of 1, 2, 4, ..., kGraphChunk steps
static int capture_graphs(tled_ctx *c) {
    for (int k = 1; k <= kGraphChunk; k *= 2) {
        cudaGraphExec_t g;
        if (int rc = capture_graph(c, k, &g)) return rc;
    }
    return TLED_OK;
}
// The step graph of K steps, K a power of two up to kGraphChunk.  The first request captures
// (and uploads) all of them, so that every later call, of any step count, replays cached
// graphs only: n steps run as the graphs of n's binary digits.  Should the grid-resident
// launch be refused (a cooperative launch needs every CTA placed at once), the context falls
// back to the streamed kernels, which compute the same numbers.
static int get_graph(tled_ctx *c, int K, cudaGraphExec_t *out) {
    auto it = c->graphs.find(K);
    if (it == c->graphs.end()) {
        int rc = capture_graphs(c);
        if (rc && c->coop) {
            cudaGetLastError();  // clear the refused launch's error
            drop_graphs(c);
            c->coop = false;
            c->coop_ok = false;
            rc = capture_graphs(c);
        }
        if (rc) return rc;
        it = c->graphs.find(K);
        if (it == c->graphs.end()) return fail(c, TLED_E_STATE, "no step graph for this chunk size");
    }
    *out = it->second;
    return TLED_OK;
}
static int capture_graph(tled_ctx *c, int K, cudaGraphExec_t *out) {
    auto it = c->graphs.find(K);
    if (it != c->graphs.end()) {
        *out = it->second;
        return TLED_OK;
    }
    CUDA_TRY(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    if (c->resident) {  // K steps in one launch, one CTA per scenario (finished ones return at once)
        e = tled::launch_resident_step(c->A, (int)c->sc.size(), c->npe, K, c->cap);
    } else if (c->coop) {  // K steps in one cooperative launch, one CTA per tile
        e = tled::launch_coop_step(c->A, c->npe, K, c->cap);
    } else {
        for (int k = 0; k < K && e == cudaSuccess; k++) {
            e = tled::launch_tile_step(c->A, c->tile_ctas, c->npe, k, c->cap);
            if (e == cudaSuccess) e = tled::launch_shared_step(c->A, c->shared_blocks, k, c->cap);
        }
    }
    if (e == cudaSuccess) e = tled::launch_bump(c->A, K, c->cap);
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
    e = cudaGraphUpload(exec, c->stream);  // the first replay then starts at once
    if (e != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return cuda_fail(c, e, "cudaGraphUpload");
    }
    c->graphs[K] = exec;
    *out = exec;
    return TLED_OK;
}

// Run up to n steps; scenarios stop at their own step counts.  *done = steps run.
static int run_steps(tled_ctx *c, int64_t n, int64_t *done) {
    int64_t ran = 0;
    while (ran < n) {
        const int ranks = active_ranks(c, c->step);
        if (ranks == 0) break;
        // the shortest running scenario bounds this segment
        const int64_t end = c->sc[c->scn_of_rank[ranks - 1]].n_steps;
        int64_t seg = std::min<int64_t>(n - ran, end == INT64_MAX ? INT64_MAX : end - c->step);
        if (int rc = set_active(c, ranks)) return rc;
        while (seg > 0) {
            int K = kGraphChunk;  // the largest cached chunk that fits
            while (K > seg) K >>= 1;
            cudaGraphExec_t g;
            if (int rc = get_graph(c, K, &g)) return rc;
            CUDA_TRY(c, cudaGraphLaunch(g, c->stream));
            seg -= K;
            ran += K;
            c->step += K;
        }
    }
    if (done) *done = ran;
    return TLED_OK;
}

int tled_step(tled_ctx *c, int64_t n) {
    if (!c) return TLED_E_ARG;
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (n < 0) return fail(c, TLED_E_ARG, "n must be >= 0");
    CUDA_TRY(c, cudaSetDevice(c->device));
    return run_steps(c, n, nullptr);
}

int tled_batch_run(tled_ctx *c, int64_t *steps) {
    if (!c) return TLED_E_ARG;
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (!c->batch) return fail(c, TLED_E_STATE, "tled_batch_run needs a batch context");
    CUDA_TRY(c, cudaSetDevice(c->device));
    return run_steps(c, INT64_MAX, steps);
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
    CUDA_TRY(c, tled::launch_readback(c->A, dptr<int32_t>(c, c->L.node_new), c->nn, c->sc[0].mat.T0, mode, dst,
                                      c->stream));
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
int tled_get_cem43(tled_ctx *c, double *out, int where) {
    if (c && c->inited && !c->A.cem) return fail(c, TLED_E_STATE, "CEM43 is tracked only with the TLED_CEM43 flag");
    return readback(c, out, where, 3);
}

int tled_get_isotherm_volume(tled_ctx *c, double T_iso, double *volume) {
    if (!c || !volume || !std::isfinite(T_iso)) return fail(c, TLED_E_ARG, "NULL volume or non-finite temperature");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, tled::launch_isotherm(c->A, c->nn, T_iso - c->sc[0].mat.T0, dptr<double>(c, c->L.stat_part),
                                      dptr<double>(c, c->L.stat_out), c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(volume, c->ws + c->L.stat_out, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return TLED_OK;
}

int tled_get_probes(tled_ctx *c, double *out, int where) {
    if (!c || !out) return fail(c, TLED_E_ARG, "NULL output");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (where != TLED_HOST && where != TLED_DEVICE) return fail(c, TLED_E_ARG, "where must be TLED_HOST or TLED_DEVICE");
    if (c->n_probes == 0) return TLED_OK;
    CUDA_TRY(c, cudaSetDevice(c->device));
    double *dst = where == TLED_DEVICE ? out : dptr<double>(c, c->L.staging);
    CUDA_TRY(c, tled::launch_probes(c->A, dptr<int32_t>(c, c->L.probe_node), dptr<float>(c, c->L.probe_w),
                                    c->n_probes, c->sc[0].mat.T0, dst, c->stream));
    if (where == TLED_HOST) {
        CUDA_TRY(c, cudaMemcpyAsync(out, dst, 16 * (size_t)c->n_probes, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    return TLED_OK;
}

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
    return upload_clock(c, step, t - step * c->sc[0].dt);
}

int tled_get_state(tled_ctx *c, double *u, double *v, double *T, double *Omega, double *visc, double *t,
                   int64_t *step) {
    if (!c) return TLED_E_ARG;
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int64_t nn = c->nn;
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
    const double T0 = c->sc[0].mat.T0;
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
        if (T) T[i] = T0 + ((double)xu[g].w + lo[g].w);
        if (Omega) Omega[i] = vel[g].w;
    }
    if (visc && np)
        for (int64_t e = 0; e < nep; e++) {
            const int64_t eo = p.elem_old[e];
            if (eo < 0) continue;
            for (int q = 0; q < np * 6; q++) visc[eo * np * 6 + q] = vs[visc_index(np, e, q)];
        }
    if (t) *t = c->t0 + c->step * c->sc[0].dt;
    if (step) *step = c->step;
    return TLED_OK;
}

int tled_step_timed(tled_ctx *c, int64_t n, double *ms) {
    if (!c || !ms) return fail(c, TLED_E_ARG, "NULL ms");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (n <= 0 || n > 100000) return fail(c, TLED_E_ARG, "1 <= n <= 100000");
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int ranks = active_ranks(c, c->step);
    if (ranks == 0) return fail(c, TLED_E_STATE, "every scenario has finished");
    const int64_t end = c->sc[c->scn_of_rank[ranks - 1]].n_steps;
    if (end != INT64_MAX && c->step + n > end) return fail(c, TLED_E_ARG, "n crosses the end of a scenario");
    if (int rc = set_active(c, ranks)) return rc;
    std::vector<cudaEvent_t> ev(3 * (size_t)n, nullptr);
    for (auto &e : ev) CUDA_TRY(c, cudaEventCreate(&e));
    cudaError_t err = cudaSuccess;
    for (int64_t i = 0; i < n && err == cudaSuccess; i++) {
        cudaEventRecord(ev[3 * i], c->stream);
        if (err == cudaSuccess)
            err = c->resident ? tled::launch_resident_step(c->A, (int)c->sc.size(), c->npe, 1, c->stream)
                : c->coop     ? tled::launch_coop_step(c->A, c->npe, 1, c->stream)
                              : tled::launch_tile_step(c->A, c->tile_ctas, c->npe, 0, c->stream);
        cudaEventRecord(ev[3 * i + 1], c->stream);
        if (err == cudaSuccess && !c->resident && !c->coop)
            err = tled::launch_shared_step(c->A, c->shared_blocks, 0, c->stream);
        cudaEventRecord(ev[3 * i + 2], c->stream);
        if (err == cudaSuccess) err = tled::launch_bump(c->A, 1, c->stream);
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
    info[6] = (int64_t)c->sc.size();
    info[7] = c->tile_ctas;
    return TLED_OK;
}

int tled_l2_window(tled_ctx *c, int64_t *out) {
    if (!c || !out) return fail(c, TLED_E_ARG, "NULL out");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    size_t set = 0;
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaDeviceGetLimit(&set, cudaLimitPersistingL2CacheSize));
    out[0] = (int64_t)c->A.l2_bytes;
    out[1] = (int64_t)set;
    out[2] = (int64_t)std::llround(1e6 * (double)c->A.l2_hit);
    return TLED_OK;
}

int tled_get_stats(tled_ctx *c, tled_stats *s) {
    if (!c || !s) return fail(c, TLED_E_ARG, "NULL stats");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, tled::launch_stats(c->A, c->npe, c->nn, dptr<double>(c, c->L.stat_part),
                                   dptr<double>(c, c->L.stat_out), c->stream));
    double o[8];
    unsigned st[4];
    CUDA_TRY(c, cudaMemcpyAsync(o, c->ws + c->L.stat_out, 64, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(st, c->ws + c->L.status, 16, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::memset(s, 0, sizeof(*s));
    s->step = c->step;
    s->t = c->t0 + c->step * c->sc[0].dt;
    s->dt = c->sc[0].dt;
    s->kinetic_energy = o[0];
    s->strain_energy = o[6];
    s->hourglass_energy = o[7];
    s->heat_content = o[1];
    s->T_max = c->sc[0].mat.T0 + o[2];
    s->T_min = c->sc[0].mat.T0 + o[3];
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
    cudaPointerAttributes pa{};  // a query: allocates nothing
    if (cudaPointerGetAttributes(&pa, out) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, TLED_E_ARG, "out is not a device pointer");
    }
    if (!((pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) && pa.device == c->device))
        return fail(c, TLED_E_ARG, "out must be device (or managed) memory of the context's device");
    double *scratch = nullptr;
    CUDA_TRY(c, tled::noalloc_scratch(c->device, &scratch));
    CUDA_TRY(c, tled::launch_stats_blocks(c->A, c->nn, n_blocks, scratch, out, c->stream));
    return TLED_OK;
}

// --- autotuner ---------------------------------------------------------------
// Candidates: elements per tile x persistent grid size.  Each is planned,
// initialised in the caller's workspace and timed over `trial_steps` steps;
// the fastest is kept (and cached for this element type, size bucket and
// layout), and the context is left initialised with it at t = 0.
namespace {
std::mutex g_tune_mu;
struct TuneChoice {
    int tile_elems, grid, mode;  // mode: 1 streamed, 2 resident
};
std::map<uint64_t, TuneChoice> g_tune_cache;
}  // namespace

int tled_autotune(tled_ctx *c, void *dev_workspace, int64_t bytes, int32_t trial_steps, int32_t *choice) {
    if (!c || !dev_workspace) return fail(c, TLED_E_ARG, "NULL argument");
    if (c->device < 0) return fail(c, TLED_E_STATE, "host-only context");
    if (trial_steps <= 0 || trial_steps > 10000) return fail(c, TLED_E_ARG, "1 <= trial_steps <= 10000");
    if (int rc = ensure_plan(c)) return rc;
    int64_t ne = 0;
    for (auto &s : c->sc) ne += s.ne;
    const int bucket = (int)std::floor(std::log2((double)std::max<int64_t>(ne, 1)));
    const uint64_t key = ((uint64_t)c->npe << 56) ^ ((uint64_t)bucket << 40) ^ ((uint64_t)c->has_mat << 36) ^
                         ((uint64_t)c->has_fib << 35) ^ ((uint64_t)n_prony(c) << 32) ^ (uint64_t)c->sc.size();
    TuneChoice best{0, 0, 1};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        double best_ms = INFINITY;
        int n_sm = 0;
        CUDA_TRY(c, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device));
        // candidates: (elements per tile, grid scale, mode); candidates of one tile size share
        // the plan (only the set-up is redone), and the resident modes are tried only when the
        // streamed set-up of that plan found the problem fits them
        struct Cand {
            int te, gscale, mode;
        };
        const Cand cands[] = {{256, 0, 1}, {256, 0, 2}, {256, 0, 3}, {256, 1, 1}, {192, 0, 1}, {192, 1, 1}, {128, 0, 1},
                              {128, 1, 1}};
        bool res_ok = false, coop_ok = false;
        for (const Cand &cd : cands) {
            const int te = cd.te;
            {
                if ((cd.mode == 2 && !res_ok) || (cd.mode == 3 && !coop_ok)) continue;  // mode not available
                if (!c->planned || c->tile_override != te) {
                    invalidate(c);
                    c->tile_override = te;
                } else {
                    drop_graphs(c);
                    c->inited = false;
                }
                c->grid_override = cd.gscale == 1 ? n_sm : 0;
                c->mode_override = cd.mode;
                if (int rc = ensure_plan(c)) return rc;
                if ((int64_t)c->L.total > bytes) continue;  // does not fit the caller's workspace
                if (int rc = tled_init(c, dev_workspace, bytes)) return rc;
                if (cd.mode == 1) {
                    res_ok = c->res_ok;
                    coop_ok = c->coop_ok;
                }
                if (int rc = run_steps(c, 3, nullptr)) return rc;  // graphs captured, caches warm
                cudaEvent_t e0, e1;
                CUDA_TRY(c, cudaEventCreate(&e0));
                CUDA_TRY(c, cudaEventCreate(&e1));
                CUDA_TRY(c, cudaEventRecord(e0, c->stream));
                int rc = run_steps(c, trial_steps, nullptr);
                CUDA_TRY(c, cudaEventRecord(e1, c->stream));
                CUDA_TRY(c, cudaEventSynchronize(e1));
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (rc) return rc;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = {te, c->grid_override, cd.mode};
                }
            }
        }
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
    }
    if (!c->planned || c->tile_override != best.tile_elems) {
        invalidate(c);
        c->tile_override = best.tile_elems;
    } else {
        drop_graphs(c);
        c->inited = false;
    }
    c->grid_override = best.grid;
    c->mode_override = best.mode;
    if (int rc = ensure_plan(c)) return rc;
    if ((int64_t)c->L.total > bytes) return fail(c, TLED_E_NOMEM, "workspace too small for the tuned plan");
    if (int rc = tled_init(c, dev_workspace, bytes)) return rc;
    if (choice) {
        choice[0] = best.tile_elems;
        choice[1] = c->tile_ctas;
        choice[2] = cached;
    }
    return TLED_OK;
}

int tled_selftest_wait(tled_ctx *c, int32_t which) {
    if (!c) return TLED_E_ARG;
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    if (which < 0 || which > 2)
        return fail(c, TLED_E_ARG, "which must be 0 (mbarrier), 1 (grid barrier) or 2 (tile kernel)");
    if (which == 2 && (c->resident || c->coop))
        return fail(c, TLED_E_STATE, "the tile-kernel self-test needs the streamed step mode (TLED_STREAMED)");
    CUDA_TRY(c, cudaSetDevice(c->device));
    if (int rc = check_status(c)) return rc;  // start from a clean status
    tled::StepArgs a = c->A;
    a.gbar = dptr<unsigned>(c, c->L.gbar);
    CUDA_TRY(c, cudaMemsetAsync(a.gbar, 0, 4, c->stream));
    if (which == 2) {  // the step's own tile kernel, with tile 0's node staging left out
        const int ranks = active_ranks(c, c->step);
        if (ranks == 0) return fail(c, TLED_E_STATE, "every scenario has finished");
        if (int rc = set_active(c, ranks)) return rc;  // the active-tile count the kernel reads
        a.stage_skip = 1;
        CUDA_TRY(c, tled::launch_tile_step(a, c->tile_ctas, c->npe, 0, c->stream));
    } else {
        CUDA_TRY(c, tled::launch_wait_selftest(a, which, c->stream));
    }
    const int rc = check_status(c);  // the timed-out wait's status, as a step would report it
    // clear it again: the context stays usable
    const unsigned st[4] = {0u, 0xffffffffu, 0xffffffffu, 0u};
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.status, st, 16, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(a.gbar, 0, 4, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return rc;
}

int tled_get_mode(tled_ctx *c, int32_t *mode) {
    if (!c || !mode) return fail(c, TLED_E_ARG, "NULL argument");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    *mode = (c->resident ? TLED_MODE_RESIDENT : 0) | (c->A.brick ? TLED_MODE_BRICK : 0) | (c->coop ? TLED_MODE_GRID : 0);
    return TLED_OK;
}

// --- checkpoints -----------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];
    uint32_t version, npe;
    int64_t nn, ne;
    int32_t n_prony, n_scn;
    uint64_t setup_hash;
    int64_t step;
    double t0;
    int64_t payload;
    uint64_t checksum;
};
}  // namespace

int tled_save_state(tled_ctx *c, void *buf, int64_t *bytes) {
    if (!c || !bytes) return fail(c, TLED_E_ARG, "NULL size pointer");
    if (!c->inited) return fail(c, TLED_E_STATE, "call tled_init first");
    const size_t nn = c->nn, nv = (size_t)n_prony(c) * 6 * c->plan.ne_pad, nc = c->A.cem ? nn : 0;
    const int64_t payload = (int64_t)(3 * 16 * nn + 4 * nv + 8 * nc);
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
    if (nc) CUDA_TRY(c, cudaMemcpyAsync(p + 48 * nn + 4 * nv, c->ws + c->L.cem, 8 * nc, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CkptHeader h{};
    std::memcpy(h.magic, "TLEDCKP2", 8);
    h.version = TLED_VERSION;
    h.npe = c->npe;
    h.nn = c->nn;
    h.ne = c->ne;
    h.n_prony = n_prony(c);
    h.n_scn = (int32_t)c->sc.size();
    h.setup_hash = c->setup_hash;
    h.step = c->step;
    h.t0 = c->t0;
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
    if (std::memcmp(h.magic, "TLEDCKP2", 8) != 0) return fail(c, TLED_E_FORMAT, "bad checkpoint magic");
    const size_t nn = c->nn, nv = (size_t)n_prony(c) * 6 * c->plan.ne_pad, nc = c->A.cem ? nn : 0;
    const int64_t payload = (int64_t)(3 * 16 * nn + 4 * nv + 8 * nc);
    if (h.version != TLED_VERSION || h.npe != (uint32_t)c->npe || h.nn != c->nn || h.ne != c->ne ||
        h.n_prony != n_prony(c) || h.n_scn != (int32_t)c->sc.size() || h.payload != payload ||
        bytes < (int64_t)sizeof(h) + payload)
        return fail(c, TLED_E_FORMAT, "checkpoint does not match this problem's sizes");
    if (h.setup_hash != c->setup_hash) return fail(c, TLED_E_FORMAT, "checkpoint was written for a different set-up");
    const char *p = (const char *)buf + sizeof(CkptHeader);
    if (fnv1a(p, payload) != h.checksum) return fail(c, TLED_E_FORMAT, "checkpoint checksum mismatch");
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.xu, p, 16 * nn, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.lo, p + 16 * nn, 16 * nn, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.vel, p + 32 * nn, 16 * nn, cudaMemcpyHostToDevice, c->stream));
    if (nv) CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.visc, p + 48 * nn, 4 * nv, cudaMemcpyHostToDevice, c->stream));
    if (nc) CUDA_TRY(c, cudaMemcpyAsync(c->ws + c->L.cem, p + 48 * nn + 4 * nv, 8 * nc, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return upload_clock(c, h.step, h.t0);  // exact clocks: the same per-scenario times as the writer's
}

}  // extern "C"
