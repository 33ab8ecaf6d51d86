// Host-side set-up of libtled: reference geometry, lumped masses, the stable
// time step, and the tiling/renumbering plan that lets one CTA gather element
// contributions into nodes in a fixed order without float atomics.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_map>

#include "tled_internal.h"

namespace tled {

// Natural-coordinate derivatives of the shape functions at the single
// integration point.  H8 (VTK order): dN_a/dxi = s_a / 8 at the centroid with
// corner signs s_a (Eqs. 18, 25: one-point rule).  T4: N = (1-xi-eta-zeta,
// xi, eta, zeta), constant derivatives (Eqs. 19, 26).
static const double kH8Sign[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                     {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
static const double kT4Deriv[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

static inline double nat_deriv(int npe, int a, int k) {
    return npe == 8 ? kH8Sign[a][k] * 0.125 : kT4Deriv[a][k];
}

// True for an axis-aligned box: the H8 element's reference corner coordinates,
// rounded to float and transformed in the tile kernel's butterfly order, have
// exactly zero hourglass projections (the Walsh-Hadamard coefficients xi eta,
// eta zeta, xi zeta and xi eta zeta), and each coordinate has zero first-order
// coefficients along the other two reference directions (J0 diagonal) -- voxel
// and block meshes.  The kernel then drops every term these coefficients multiply
// and stores only the diagonal of J0^-1 (the off-diagonal entries computed in
// double are round-off, some 1e-14 of the diagonal).
bool brick_element(const double *X, const int32_t *cn) {
    for (int d = 0; d < 3; d++) {
        float w[8];
        for (int i = 0; i < 8; i++) {
            const int a = i == 2 ? 3 : i == 3 ? 2 : i == 6 ? 7 : i == 7 ? 6 : i;  // transform index -> VTK corner
            w[i] = (float)X[3 * (int64_t)cn[a] + d];
        }
        for (int h = 1; h < 8; h <<= 1)
            for (int i = 0; i < 8; i++)
                if ((i & h) == 0) {
                    const float x = w[i], y = w[i + h];
                    w[i] = x + y;
                    w[i + h] = x - y;
                }
        if (w[3] != 0.f || w[5] != 0.f || w[6] != 0.f || w[7] != 0.f) return false;
        for (int j = 0; j < 3; j++)  // first-order coefficients: xi (1), eta (2), zeta (4)
            if (j != d && w[1 << j] != 0.f) return false;
    }
    return true;
}

// Reference Jacobian J0 = sum_a X_a (x) dN_a/dxi, its inverse, and the element
// volume (8 det J0 for H8, det J0 / 6 for T4).  Returns false if det J0 <= 0.
bool element_geometry(int npe, const double *X, const int32_t *cn, double Jinv[9], double *V) {
    double J[9] = {0};
    for (int a = 0; a < npe; a++)
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) J[3 * i + j] += X[3 * (int64_t)cn[a] + i] * nat_deriv(npe, a, j);
    double c00 = J[4] * J[8] - J[5] * J[7];
    double c01 = J[5] * J[6] - J[3] * J[8];
    double c02 = J[3] * J[7] - J[4] * J[6];
    double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
    if (!(det > 0.0)) return false;
    double id = 1.0 / det;
    Jinv[0] = c00 * id;
    Jinv[1] = (J[2] * J[7] - J[1] * J[8]) * id;
    Jinv[2] = (J[1] * J[5] - J[2] * J[4]) * id;
    Jinv[3] = c01 * id;
    Jinv[4] = (J[0] * J[8] - J[2] * J[6]) * id;
    Jinv[5] = (J[2] * J[3] - J[0] * J[5]) * id;
    Jinv[6] = c02 * id;
    Jinv[7] = (J[1] * J[6] - J[0] * J[7]) * id;
    Jinv[8] = (J[0] * J[4] - J[1] * J[3]) * id;
    *V = npe == 8 ? 8.0 * det : det / 6.0;
    return true;
}

// dh_a/dX_j = sum_k dN_a/dxi_k (J0^-1)_kj
static void shape_gradients(int npe, const double Jinv[9], double B[8][3]) {
    for (int a = 0; a < npe; a++)
        for (int j = 0; j < 3; j++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += nat_deriv(npe, a, k) * Jinv[3 * k + j];
            B[a][j] = s;
        }
}

// H8 hourglass base vectors at the corners: xi eta, eta zeta, xi zeta, xi eta zeta
static inline double hg_h(int a, int al) {
    const double *s = kH8Sign[a];
    return al == 0 ? s[0] * s[1] : al == 1 ? s[1] * s[2] : al == 2 ? s[0] * s[2] : s[0] * s[1] * s[2];
}

static double cross_norm_half(const double *d1, const double *d2) {
    double c0 = d1[1] * d2[2] - d1[2] * d2[1];
    double c1 = d1[2] * d2[0] - d1[0] * d2[2];
    double c2 = d1[0] * d2[1] - d1[1] * d2[0];
    return 0.5 * std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
}

// Stable-step reading: dt_mech = min_e L_e / c_d with L_e = V / A_max (H8) or
// the minimum altitude 3 V / A_max (T4), c_d = sqrt((kappa + 4 mu / 3 + 4 k1) /
// (rho * mass_scale)); dt_th = min_i 2 C_i / (sum over incident elements of
// the absolute row sums of the element conduction matrix at k_max, plus the
// perfusion conductance).  Per-element moduli come from `mat6` ([ne][6], caller
// order) when given.
void stable_dt(int npe, int64_t nn, const double *X, int64_t ne, const int32_t *conn, const tled_material &m,
               const double *mat6, const double *fib, const tled_params &p, double *dt_mech, double *dt_th) {
    const double rk = m.k_fibre_ratio == 0.0 ? 1.0 : m.k_fibre_ratio;  // conductivity along the fibre / transverse
    static const int HF[6][4] = {{0, 1, 2, 3}, {4, 5, 6, 7}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}};
    static const int TF[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
    const bool td = (p.flags & TLED_TEMP_DEP) != 0;
    const double kfac = td ? std::max(1.0, 1.0 + m.beta_k * (90.0 - m.T_ref)) : 1.0;
    const double cfac = td ? std::min(1.0, 1.0 + m.beta_c * (90.0 - m.T_ref)) : 1.0;
    std::vector<double> row(nn, 0.0), Vn(nn, 0.0);
    double dtm = INFINITY;
    for (int64_t e = 0; e < ne; e++) {
        const int32_t *cn = conn + e * npe;
        double Jinv[9], V;
        element_geometry(npe, X, cn, Jinv, &V);
        double B[8][3];
        shape_gradients(npe, Jinv, B);
        const double *P[8];
        for (int a = 0; a < npe; a++) P[a] = X + 3 * (int64_t)cn[a];
        double Amax = 0;
        if (npe == 8) {
            for (auto &f : HF) {
                double d1[3], d2[3];
                for (int j = 0; j < 3; j++) {
                    d1[j] = P[f[2]][j] - P[f[0]][j];
                    d2[j] = P[f[3]][j] - P[f[1]][j];
                }
                Amax = std::max(Amax, cross_norm_half(d1, d2));
            }
        } else {
            for (auto &f : TF) {
                double d1[3], d2[3];
                for (int j = 0; j < 3; j++) {
                    d1[j] = P[f[1]][j] - P[f[0]][j];
                    d2[j] = P[f[2]][j] - P[f[0]][j];
                }
                Amax = std::max(Amax, cross_norm_half(d1, d2));
            }
        }
        const double mu = mat6 ? mat6[6 * e + 0] : m.mu;
        const double kap = mat6 ? mat6[6 * e + 1] : m.kappa;
        const double k1 = mat6 ? mat6[6 * e + 2] : m.k1;
        const double kc = mat6 ? mat6[6 * e + 4] : m.k;
        const double L = (npe == 8 ? 1.0 : 3.0) * V / Amax;
        const double cd = std::sqrt((kap + 4.0 * mu / 3.0 + 4.0 * k1) / (m.rho * p.mass_scale));
        dtm = std::min(dtm, L / cd);
        // element conduction matrix at F = I, k_max, plus the thermal hourglass term
        const double kmax = kc * kfac;
        double G[8][4] = {{0}};
        double BB = 0;
        if (npe == 8) {
            for (int a = 0; a < 8; a++)
                for (int j = 0; j < 3; j++) BB += B[a][j] * B[a][j];
            for (int al = 0; al < 4; al++) {
                double c[3] = {0, 0, 0};
                for (int b = 0; b < 8; b++)
                    for (int j = 0; j < 3; j++) c[j] += hg_h(b, al) * P[b][j];
                for (int a = 0; a < 8; a++) G[a][al] = hg_h(a, al) - (c[0] * B[a][0] + c[1] * B[a][1] + c[2] * B[a][2]);
            }
        }
        const double khgT = p.kappa_hgT * V * BB / 8.0;
        const double *af = fib ? fib + 3 * e : m.a0;
        double Bm[8];  // dh_a/dX . a0 for the anisotropic conduction D = k (I + (rk - 1) a0 a0) at F = I
        for (int a = 0; a < npe; a++) Bm[a] = B[a][0] * af[0] + B[a][1] * af[1] + B[a][2] * af[2];
        for (int a = 0; a < npe; a++) {
            double rs = 0;
            for (int b = 0; b < npe; b++) {
                double K = V * kmax * (B[a][0] * B[b][0] + B[a][1] * B[b][1] + B[a][2] * B[b][2] +
                                       (rk - 1.0) * Bm[a] * Bm[b]);
                if (npe == 8)
                    K += kmax * khgT * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2] + G[a][3] * G[b][3]);
                rs += std::fabs(K);
            }
            row[cn[a]] += rs;
            Vn[cn[a]] += V / npe;
        }
    }
    double dtt = INFINITY;
    for (int64_t i = 0; i < nn; i++) {
        const double r = row[i] + m.wb_cb * Vn[i];
        const double C = m.rho * m.c * Vn[i] * cfac;
        if (r > 0) dtt = std::min(dtt, 2.0 * C / r);
    }
    *dt_mech = dtm;
    *dt_th = dtt;
}

// ---------------------------------------------------------------------------
// tiling plan
// ---------------------------------------------------------------------------
static inline uint64_t spread3(uint64_t v) {  // 21 bits -> every third bit
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}

int build_plan(int npe, int64_t nn, const double *X, int64_t ne, const int32_t *conn, const int8_t *etype,
               const int32_t *group, int tile_elems, Plan &p, std::string &err) {
    p = Plan();
    // element e has nc(e) corners: etype[e] (4 or 8) in a mixed mesh, else npe; conn stride npe
    auto nc = [&](int64_t e) { return etype ? (int)etype[e] : npe; };
    p.npe = npe;
    p.nn = nn;
    p.ne = ne;
    if (tile_elems <= 0) tile_elems = kTile;
    tile_elems = std::min(tile_elems, kTile);
    // --- Morton order of element centroids
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nn; i++)
        for (int j = 0; j < 3; j++) {
            lo[j] = std::min(lo[j], X[3 * i + j]);
            hi[j] = std::max(hi[j], X[3 * i + j]);
        }
    double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
    std::vector<uint64_t> key(ne);
    std::vector<double> cen(3 * (size_t)ne);  // element centroids
    for (int64_t e = 0; e < ne; e++) {
        double c[3] = {0, 0, 0};
        const int ke = nc(e);
        for (int a = 0; a < ke; a++)
            for (int j = 0; j < 3; j++) c[j] += X[3 * (int64_t)conn[e * npe + a] + j];
        for (int j = 0; j < 3; j++) cen[3 * e + j] = c[j] / ke;
        uint64_t k = 0;
        for (int j = 0; j < 3; j++) {
            double q = (c[j] / ke - lo[j]) / ext;
            uint64_t iq = (uint64_t)std::min(std::max(q, 0.0) * 2097151.0, 2097151.0);
            k |= spread3(iq) << j;
        }
        key[e] = k;
    }
    p.elem_old.resize(ne);
    std::iota(p.elem_old.begin(), p.elem_old.end(), 0);
    // elements ordered by group (scenario rank), then along the Morton curve
    std::stable_sort(p.elem_old.begin(), p.elem_old.end(), [&](int32_t a, int32_t b) {
        const int32_t ga = group ? group[a] : 0, gb = group ? group[b] : 0;
        return ga != gb ? ga < gb : key[a] < key[b];
    });

    // --- cut tiles: at most tile_elems elements and cap distinct nodes; a tile
    //     holds one group and one element type
    const int cap = etype ? kMaxLocal : max_local(npe);  // local nodes per tile (the kernel's layout)
    std::vector<int32_t> mark(nn, -1);
    std::vector<int32_t> tile_begin;
    int n_local = 0, n_in = 0, t = -1;
    int32_t prev_group = -1;
    int prev_type = -1;
    for (int64_t i = 0; i < ne; i++) {
        const int32_t *cn = conn + (int64_t)p.elem_old[i] * npe;
        const int32_t gi = group ? group[p.elem_old[i]] : 0;
        const int ki = nc(p.elem_old[i]);
        int fresh = 0;
        if (t >= 0)
            for (int a = 0; a < ki; a++) fresh += (mark[cn[a]] != t);
        if (t < 0 || n_in == tile_elems || n_local + fresh > cap || gi != prev_group || ki != prev_type) {
            prev_group = gi;
            prev_type = ki;
            t++;
            tile_begin.push_back((int32_t)i);
            n_local = 0;
            n_in = 0;
        }
        for (int a = 0; a < ki; a++)
            if (mark[cn[a]] != t) {
                mark[cn[a]] = t;
                n_local++;
            }
        n_in++;
    }
    p.n_tiles = (int)tile_begin.size();
    tile_begin.push_back((int32_t)ne);
    // inside a tile, elements in (z, y, x) order of their centroids and (below) nodes in
    // (z, y, x) order of their coordinates: in a block of bricks, eight consecutive
    // elements are then a row, and the corner nodes they read, like the element slots a
    // row of nodes reads, sit at consecutive local positions -- distinct shared-memory
    // banks for the eight threads a 16-byte load serves at a time
    auto zyx_less = [](const double *a, const double *b) {
        return a[2] != b[2] ? a[2] < b[2] : a[1] != b[1] ? a[1] < b[1] : a[0] < b[0];
    };
    for (int tt = 0; tt < p.n_tiles; tt++)
        std::stable_sort(p.elem_old.begin() + tile_begin[tt], p.elem_old.begin() + tile_begin[tt + 1],
                         [&](int32_t a, int32_t b) { return zyx_less(&cen[3 * (size_t)a], &cen[3 * (size_t)b]); });
    auto node_less = [&](int32_t a, int32_t b) { return zyx_less(X + 3 * (int64_t)a, X + 3 * (int64_t)b); };

    // --- how many tiles touch each node
    std::vector<int32_t> ntouch(nn, 0), last(nn, -1);
    for (int tt = 0; tt < p.n_tiles; tt++)
        for (int64_t i = tile_begin[tt]; i < tile_begin[tt + 1]; i++) {
            const int32_t *cn = conn + (int64_t)p.elem_old[i] * npe;
            for (int a = 0, ka = nc(p.elem_old[i]); a < ka; a++)
                if (last[cn[a]] != tt) {
                    last[cn[a]] = tt;
                    ntouch[cn[a]]++;
                }
        }
    for (int64_t i = 0; i < nn; i++)
        if (ntouch[i] == 0) {
            err = "node " + std::to_string(i) + " belongs to no element";
            return TLED_E_MESH;
        }

    // --- numbering: interior nodes tile by tile, then shared nodes by first tile.
    // Every tile owns kTile element slots (tile-blocked device records).
    p.node_new.assign(nn, -1);
    p.tile_info.assign((size_t)p.n_tiles * kTileInfo, 0);
    std::vector<int64_t> tile_pad(p.n_tiles + 1, 0);
    for (int tt = 0; tt < p.n_tiles; tt++) tile_pad[tt + 1] = tile_pad[tt] + kTile;
    p.ne_pad = tile_pad[p.n_tiles];
    if (p.ne_pad > 0x7fffffff) {
        err = "mesh too large";
        return TLED_E_MESH;
    }
    int32_t next = 0;
    std::vector<int32_t> own;
    for (int tt = 0; tt < p.n_tiles; tt++) {
        int32_t *ti = &p.tile_info[(size_t)tt * kTileInfo];
        ti[0] = (int32_t)tile_pad[tt];
        ti[1] = tile_begin[tt + 1] - tile_begin[tt];
        ti[2] = next;
        own.clear();
        for (int64_t i = tile_begin[tt]; i < tile_begin[tt + 1]; i++) {
            const int32_t *cn = conn + (int64_t)p.elem_old[i] * npe;
            for (int a = 0, ka = nc(p.elem_old[i]); a < ka; a++)
                if (ntouch[cn[a]] == 1 && p.node_new[cn[a]] < 0) {
                    p.node_new[cn[a]] = 0;  // collected; numbered below, in coordinate order
                    own.push_back(cn[a]);
                }
        }
        std::stable_sort(own.begin(), own.end(), node_less);
        for (int32_t n : own) p.node_new[n] = next++;
        ti[3] = next - ti[2];
    }
    p.n_interior = next;
    for (int tt = 0; tt < p.n_tiles; tt++)
        for (int64_t i = tile_begin[tt]; i < tile_begin[tt + 1]; i++) {
            const int32_t *cn = conn + (int64_t)p.elem_old[i] * npe;
            for (int a = 0, ka = nc(p.elem_old[i]); a < ka; a++)
                if (p.node_new[cn[a]] < 0) p.node_new[cn[a]] = next++;
        }
    p.n_shared = next - p.n_interior;
    p.node_old.assign(nn, 0);
    for (int64_t i = 0; i < nn; i++) p.node_old[p.node_new[i]] = (int32_t)i;

    // --- per tile: local node lists, local connectivity, gather CSR, partial slots
    std::vector<int32_t> sorted_old(p.elem_old);
    p.elem_old.assign(p.ne_pad, -1);
    for (int tt = 0; tt < p.n_tiles; tt++)
        for (int64_t i = tile_begin[tt]; i < tile_begin[tt + 1]; i++) p.elem_old[tile_pad[tt] + (i - tile_begin[tt])] = sorted_old[i];
    std::vector<uint16_t> conn_local((size_t)p.ne_pad * npe, 0);  // [slot][npe] tile-local node index
    p.pat_stride = pattern_u16(npe);
    p.patterns.clear();
    std::unordered_map<uint64_t, std::vector<int32_t>> pat_by_hash;  // content hash -> pattern ids
    std::vector<uint16_t> pat(p.pat_stride);
    std::vector<int> pat_type;  // element type of each distinct record
    std::vector<int32_t> local(nn, -1);
    std::vector<int32_t> sh_n(p.n_shared, 0);  // tiles touching each shared node so far
    int64_t part = 0;
    for (int tt = 0; tt < p.n_tiles; tt++) {
        int32_t *ti = &p.tile_info[(size_t)tt * kTileInfo];
        const int32_t e0 = ti[0], ne_t = ti[1], int_begin = ti[2], n_int = ti[3];
        std::vector<int32_t> shared;
        for (int64_t i = e0; i < e0 + ne_t; i++) {
            const int32_t *cn = conn + (int64_t)p.elem_old[i] * npe;
            for (int a = 0, ka = nc(p.elem_old[i]); a < ka; a++) {
                int32_t g = p.node_new[cn[a]];
                if (g >= p.n_interior && local[g] != -2 - tt) {
                    local[g] = -2 - tt;  // seen in this tile
                    shared.push_back(g);
                }
            }
        }
        // shared nodes in (z, y, x) order inside the tile (tiles of the same shape and
        // position class get identical local structures)
        std::stable_sort(shared.begin(), shared.end(),
                         [&](int32_t a, int32_t b) { return node_less(p.node_old[a], p.node_old[b]); });
        const int nl = n_int + (int)shared.size();
        if (nl > cap) {
            err = "internal: tile exceeds the local node limit";
            return TLED_E_MESH;
        }
        ti[4] = nl;
        // each tile's shared-node lists start on a 16-byte boundary (bulk-copied to shared memory)
        while (p.tile_shared.size() % 4) {
            p.tile_shared.push_back(-1);
            p.part_pos.push_back(0);
        }
        ti[5] = (int32_t)p.tile_shared.size();
        const int kt = nc(p.elem_old[e0]);
        ti[7] = kt;  // element type of the tile (4 or 8)
        for (size_t j = 0; j < shared.size(); j++) {
            p.tile_shared.push_back(shared[j]);
            p.part_pos.push_back(sh_n[shared[j] - p.n_interior]++);  // rank; made absolute below
        }
        part += (int64_t)shared.size();
        for (size_t j = 0; j < shared.size(); j++) local[shared[j]] = n_int + (int32_t)j;
        // local index of every node of the tile
        for (int64_t i = e0; i < e0 + ne_t; i++) {
            const int32_t *cn = conn + (int64_t)p.elem_old[i] * npe;
            for (int a = 0, ka = nc(p.elem_old[i]); a < ka; a++) {
                const int32_t g = p.node_new[cn[a]];
                conn_local[(size_t)i * npe + a] = (uint16_t)(g < p.n_interior ? g - int_begin : local[g]);
            }
        }
        // the tile's structure record: local connectivity [kTile][kt], then the gather
        // list -- for every local node the slot offsets slot_pos(element, corner) of its
        // incident corners, ascending corner then element -- and the nl + 1 row offsets
        std::fill(pat.begin(), pat.end(), (uint16_t)0);
        uint16_t *rec_conn = pat.data();
        uint16_t *rec_codes = rec_conn + kTile * kt;
        uint16_t *rec_row = rec_codes + kTile * kt;
        for (int64_t i = e0; i < e0 + ne_t; i++)
            for (int a = 0; a < kt; a++) rec_conn[(i - e0) * kt + a] = conn_local[(size_t)i * npe + a];
        std::vector<int32_t> cnt(nl + 1, 0);
        for (int64_t i = e0; i < e0 + ne_t; i++)
            for (int a = 0; a < kt; a++) cnt[conn_local[(size_t)i * npe + a] + 1]++;
        for (int l = 0; l < nl; l++) cnt[l + 1] += cnt[l];
        for (int l = 0; l <= nl; l++) rec_row[l] = (uint16_t)cnt[l];
        std::vector<int32_t> cur(cnt.begin(), cnt.end() - 1);
        for (int a = 0; a < kt; a++)
            for (int64_t i = e0; i < e0 + ne_t; i++) {
                int l = conn_local[(size_t)i * npe + a];
                rec_codes[cur[l]++] = (uint16_t)slot_pos((int)(i - e0), a);
            }
        // tiles with the same element type and structure share one record (FNV-1a hash,
        // then a full compare)
        uint64_t h = 1469598103934665603ull ^ (uint64_t)kt;
        for (uint16_t v : pat) h = (h ^ v) * 1099511628211ull;
        int32_t id = -1;
        auto &cand = pat_by_hash[h];
        for (int32_t c : cand)
            if (pat_type[c] == kt && std::equal(pat.begin(), pat.end(), p.patterns.begin() + (size_t)c * p.pat_stride)) {
                id = c;
                break;
            }
        if (id < 0) {
            id = (int32_t)pat_type.size();
            p.patterns.insert(p.patterns.end(), pat.begin(), pat.end());
            pat_type.push_back(kt);
            cand.push_back(id);
        }
        ti[6] = id;
    }
    while (p.tile_shared.size() % 4) {  // the last tile's padded copy stays inside the arrays
        p.tile_shared.push_back(-1);
        p.part_pos.push_back(0);
    }
    p.n_partials = part;
    p.sh_rowptr.assign(p.n_shared + 1, 0);
    for (int64_t s = 0; s < p.n_shared; s++) p.sh_rowptr[s + 1] = p.sh_rowptr[s] + sh_n[s];
    for (size_t j = 0; j < p.tile_shared.size(); j++)
        if (p.tile_shared[j] >= 0) p.part_pos[j] += p.sh_rowptr[p.tile_shared[j] - p.n_interior];
    return TLED_OK;
}

}  // namespace tled
