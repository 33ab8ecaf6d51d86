// Internal declarations of libtled: device data layout, kernel arguments,
// host-side plan.  Not part of the public C ABI (include/tled.h).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tled.h"

namespace tled {

constexpr int kBlock = 256;        // threads per CTA of the tile kernel
constexpr int kTile = 256;         // elements per tile (one per thread); every tile owns kTile element slots
constexpr int kTileCtasPerSm = 3; // tile kernel CTAs resident per SM (register budget 85 per thread)
constexpr int kMaxLocal = 448;     // max nodes touched by one tile (shared memory)
constexpr int kMaxLocalT4 = 256;   // ... by a tile of a T4-only problem (smaller layout: fits 4 CTAs per SM)
constexpr int max_local(int npe) { return npe == 4 ? kMaxLocalT4 : kMaxLocal; }
constexpr int kTileCtasPerSmT4 = 4; // T4 problems with more tiles than 3 CTAs per SM cover (64 registers)
constexpr int kNsMax = 256;        // interior nodes whose state is staged in shared memory
constexpr int kResLanes = 2;       // resident mode: tiles processed side by side in one CTA
constexpr int kResBlock = kResLanes * kBlock;
// per-tile structure record (uint16): local connectivity [kTile * npe], gather slot
// offsets [kTile * npe], row offsets [kMaxLocal + 8]; tiles of equal structure share one
constexpr int pattern_u16(int npe) { return 2 * kTile * npe + kMaxLocal + 8; }
// Position of element e's corner c in a tile's corner-slot buffer ([corner][kTile] float4).
// The low three bits of e are XOR-ed with a linear function of bits 3-5 of e and of c: for
// a fixed corner this permutes each aligned group of 8 elements (the element pass's stores
// stay conflict-free), and a warp gathering one node per thread, entry by entry in corner
// order, spreads its reads over more shared-memory banks (on 8x8x4 Morton blocks of bricks
// about 30 % fewer excess wavefronts than the plain [corner][element] layout, by a model of
// 128-bit loads served eight threads at a time that matches the profiler's counts).
constexpr int slot_swz_e(int h) { return ((h >> 1 ^ h >> 2) & 1) | ((h ^ h >> 2) & 1) << 1 | (h & 1) << 2; }
constexpr int slot_swz_c(int c) { return (c & 1) << 1 | ((c ^ c >> 1 ^ c >> 2) & 1) << 2; }
constexpr int slot_pos(int e, int c) { return c * kTile + (e ^ slot_swz_e((e >> 3) & 7) ^ slot_swz_c(c)); }
constexpr int kMaxSources = 16;
constexpr int kSrcRow = 11;        // doubles per source in the device table: c0, vel, sigma, P, t_on, t_off, shape
constexpr int kTileInfo = 8;       // ints per tile record

// device status word bits
constexpr uint32_t kStatusInverted = 1u;
constexpr uint32_t kStatusNaN = 2u;
constexpr uint32_t kStatusTimeout = 4u;

// Host-side plan: element/node renumbering and tiling.  Elements are sorted
// along a Morton curve and cut into tiles; a node touched by exactly one tile
// is "interior" (updated by that tile's CTA), otherwise "shared" (its partial
// sums go through a fixed-order second pass).
struct Plan {
    int npe = 0;
    int64_t nn = 0, ne = 0;
    int64_t ne_pad = 0;                 // n_tiles * kTile element slots
    std::vector<int32_t> elem_old;      // element slot (tile * kTile + i) -> caller element (-1 = padding)
    std::vector<int32_t> node_new;      // caller node -> new node
    std::vector<int32_t> node_old;      // new node -> caller node
    int64_t n_interior = 0, n_shared = 0;
    int n_tiles = 0;
    std::vector<int32_t> tile_info;     // [n_tiles][8]: e0 (= tile * kTile), ne, int_begin, n_int,
                                        //   n_local, sh_off, structure record id, element type (4 or 8)
    std::vector<int32_t> tile_shared;   // per tile (from a multiple of 4, -1 padded): new ids of its shared nodes (ascending)
    std::vector<uint16_t> patterns;     // [n_patterns][pat_stride] distinct structure records: local connectivity
                                        //   [kTile][npe], slot offsets slot_pos(element, corner) grouped by local
                                        //   node (ascending corner, element), then the n_local + 1 row offsets
    int pat_stride = 0;                 // pattern_u16(npe)
    std::vector<int32_t> sh_rowptr;     // [n_shared + 1]: node-major partial positions, tile order within a node
    std::vector<int32_t> part_pos;      // parallel to tile_shared: partial position of that (tile, node)
    int64_t n_partials = 0;
};

// Resident mode: one CTA holds a whole scenario (its tiles' element data, structure
// records, node state and partial sums) in shared memory and runs many steps in one
// launch, one block barrier between phases instead of a kernel boundary.  One
// descriptor per CTA, in rank order.
struct ResDesc {
    int scn;          // scenario
    int t0, n_t;      // tiles [t0, t0 + n_t)
    int i0, n_int;    // interior nodes [i0, i0 + n_int)
    int s0, n_sh;     // shared nodes [n_interior + s0, n_interior + s0 + n_sh)
    int p0, n_part;   // their node-major partial sums [p0, p0 + n_part)
    int pad[3];
};

// Constant per-scenario parameters (device table).
struct ScenDev {
    double dt;             // the step: the mechanical (sub)step
    double dt_th;          // the thermal step, n_sub dt
    float dtf, inv_dt;
    float dtf_th;          // (float) dt_th
    float damp_a, damp_b;  // v+ = damp_a v - damp_b f / m: (1 - g dt/2)/(1 + g dt/2), dt/(1 + g dt/2)
    float pr_a[4], pr_b[4];  // Prony: dt phi/(dt + tau), tau/(dt + tau)
    float Qm;              // metabolic heat W/m^3
    int src_off, n_src;    // sources [src_off, src_off + n_src) of the global table
    int n_sub;             // mechanical substeps per thermal step (1: every step is a coupled step)
};

// A single problem's scenario table and source rows, passed by value to a one-block
// upload kernel so that a source change is stream-ordered without a host wait.
struct SingleScenUpload {
    ScenDev d;
    double src[kMaxSources * kSrcRow];
};

// Arguments of the step kernels (passed by value).
struct StepArgs {
    // node arrays (new numbering)
    float4 *xu;            // u_hi.xyz, theta_hi
    float4 *lo;            // u_lo.xyz, theta_lo
    float4 *vel;           // v.xyz, Omega
    const float4 *X0;      // X.xyz, lumped volume V_i
    const float4 *nodec;   // m_i, Cth_i, mask bits (as float bits), 0
    const float4 *ubar;    // prescribed displacement or nullptr
    // element data, tile-blocked: tile t's record at elem_rec + t * rec_bytes holds float
    // components [q][kTile]: J0^-1 (9; bricks: its diagonal, 3), V0, [mu kappa k1 k2 k alpha],
    // [fibre xyz] (rec_bytes is sized for 9); the Prony
    // state lives in visc [t][6 n_prony][kTile]; the local connectivity is in the tile's
    // structure record (pattern).
    const char *elem_rec;
    int64_t rec_bytes;
    int has_mat, has_fib;
    float *visc;
    int64_t ne;            // element slots (n_tiles * kTile)
    // tiles
    const int *tile_info;
    const int *tile_shared;
    const uint16_t *pattern;  // [n_patterns][pat_stride]: pattern_u16(npe of the tile) entries used
    float4 *partials;      // node-major: shared node s owns [sh_rowptr[s], sh_rowptr[s+1]), one per touching tile
    const int *part_pos;   // per (tile, shared node) entry of tile_shared: its partial's position
    const int *sh_rowptr;
    int64_t n_interior, n_shared;
    // scenarios (a single problem is one scenario)
    const struct ScenDev *scn;  // [n_scn] constant per-scenario parameters
    const double *src;     // [total sources][kSrcRow]: c0 xyz, velocity xyz, sigma/radius, peak, t_on, t_off, shape
    double *cem;           // [nn] CEM43 dose (minutes), or nullptr
    double T0;             // initial temperature, C (theta = T - T0)
    double *scn_time;      // [n_scn] time t0 at step 0; step n is at t0 + n dt
    int64_t *scn_step;     // [n_scn] steps taken at the start of the current graph chunk
    const int *tile_scn;   // [n_tiles] scenario of each tile
    const int *shared_scn; // [n_shared] scenario of each shared node
    const int *n_active;   // device [2]: active tiles, active shared nodes (prefixes of the orders)
    int n_scn;
    unsigned int *status;  // [4]: bits, first bad element (slot), first bad node (new id), spare
    // dynamic shared-memory layout of the tile kernel (bytes)
    int sm_in;             // bytes of a tile's staged element inputs (record + Prony state)
    int sm_buf;            // max(sm_in, slot buffer bytes), 128-aligned; two such buffers
    int sm_ns, sm_pat, sm_sh, sm_xu, sm_X, sm_bar, sm_total;  // sm_pat: structure record, sm_sh: shared-node lists
    int n_tiles;
    int pat_stride;        // uint16 entries between consecutive structure records
    int n_comp;            // staged float components per element (J0^-1 9 or, bricks, its diagonal 3, V0,
                           //   [mat 6], [fibre 3], Prony 6 n)
    // batch-wide scalars
    float mu, kappa, k1, k2, kc, alpha;   // uniform material (used when has_mat == 0)
    float a0x, a0y, a0z;                  // uniform fibre (used when has_fib == 0)
    int n_prony;
    unsigned int flags;
    float beta_c, beta_k, Tref_m_T0;      // T_ref - T0
    float theta_a;                        // Ta - T0
    float lnA, Ea_R, T0_K;                // T0 + 273.15
    float khg, khgT;                      // kappa_hg, kappa_hgT
    int ani;                              // anisotropic thermal physics (the ratios below differ from 1)
    int brick;                            // every element an axis-aligned H8 box (no reference hourglass
                                          //   projections, diagonal J0^-1; records hold its diagonal)
    int wide;                             // T4 problem with more tiles than 3 CTAs per SM: the 4-CTA instance
    float ani_alpha, ani_k;               // fibre / transverse expansion and conductivity
    double ramp_time;
    // resident mode (shared-memory byte offsets; rs_tile is the per-tile block stride and
    // rt_* are offsets inside a tile block)
    const ResDesc *res;
    int rs_xu, rs_lo, rs_vel, rs_X, rs_nc, rs_rowptr, rs_part, rs_slot, rs_tiles, rs_tile, rs_total;
    int rt_conn, rt_codes, rt_ppos, rt_info;
    // grid-resident mode (cooperative launch, one CTA per tile): shared-memory offsets, and
    // the grid barrier's arrival count
    int cs_rec, cs_pat, cs_sh, cs_xu, cs_X, cs_lo, cs_vo, cs_nc, cs_slot, cs_total;
    int64_t n_partials;     // partial sums per buffer (the grid-resident mode double-buffers them)
    unsigned int *gbar;
    // persisting-L2 access window of the streamed step kernels (l2_bytes 0: none)
    void *l2_base;
    size_t l2_bytes;
    float l2_hit;
    // self-test of the tile kernel's own bounded wait: 1 + the tile whose node staging the
    // kernel leaves out (so that the wait for it runs out); 0 = none (every normal launch)
    int stage_skip;
};

// kernel launchers (tled_kernels.cu); npe 4 or 8, or 0 for a batch mixing both element types
cudaError_t launch_tile_step(const StepArgs &a, int n_ctas, int npe, int k, cudaStream_t s);
int tile_grid(const StepArgs &a, int npe, int n_sm);  // persistent grid size
int shared_grid(const StepArgs &a, int n_sm);  // persistent grid of the shared-node kernel
// CEM43 dose += dt R^(43 - T) / 60 at every node (single problems; before the step's update)
// sum of the lumped volumes of the nodes with theta >= theta_iso, FP64, fixed order: out[0]
cudaError_t launch_isotherm(const StepArgs &a, int64_t nn, double theta_iso, double *partials, double *out,
                            cudaStream_t s);
cudaError_t launch_shared_step(const StepArgs &a, int n_blocks, int k, cudaStream_t s);
cudaError_t launch_bump(const StepArgs &a, int K, cudaStream_t s);
// temperature and damage at probe points: out [2][n]
cudaError_t launch_probes(const StepArgs &a, const int32_t *node, const float *w, int64_t n, double T0, double *out,
                          cudaStream_t s);
// read-back in caller order: mode 0 displacement [nn][3], 1 temperature, 2 damage fraction, 3 CEM43
cudaError_t launch_readback(const StepArgs &a, const int32_t *node_new, int64_t nn, double T0, int mode, double *out,
                            cudaStream_t s);
void tile_smem_layout(StepArgs &a, int npe);  // fills the sm_* fields and pat_stride
cudaError_t tile_kernel_setup(const StepArgs &a, int npe);
// resident mode: shared-memory layout for the largest scenario (returns the bytes), the
// kernel's attribute set-up, and a launch of K steps for the first n_ctas descriptors
int resident_smem_layout(StepArgs &a, int npe, int nn_max, int nt_max, int npart_max, int nsh_max);
int resident_smem_limit();
cudaError_t resident_kernel_setup(const StepArgs &a, int npe);
cudaError_t launch_resident_step(const StepArgs &a, int n_ctas, int npe, int K, cudaStream_t s);
// grid-resident mode: layout (returns the bytes), co-resident CTAs per SM for it, set-up,
// and a cooperative launch of K steps (one CTA per tile)
int coop_smem_layout(StepArgs &a, int npe);
int coop_ctas_per_sm(const StepArgs &a, int npe);
cudaError_t coop_kernel_setup(const StepArgs &a, int npe);
cudaError_t launch_coop_step(const StepArgs &a, int npe, int K, cudaStream_t s);
cudaError_t launch_wait_selftest(const StepArgs &a, int which, cudaStream_t s);
cudaError_t launch_single_upload(const SingleScenUpload &u, ScenDev *scn, double *src, cudaStream_t s);
// FP64 diagnostics: out[0..5] = kinetic energy, heat content, T max (rel), T min (rel), max |u|^2,
// damaged volume, out[6..7] = stored (hyperelastic) energy and hourglass energy; deterministic
// two-stage reduction through `partials` [kStatBlocks][8].
constexpr int kStatBlocks = 296;
cudaError_t launch_stats(const StepArgs &a, int npe, int64_t nn, double *partials, double *out, cudaStream_t s);
// the nodal part (out[0..5]) over a caller-chosen number of blocks (partials [n_blocks][8])
cudaError_t launch_stats_blocks(const StepArgs &a, int64_t nn, int n_blocks, double *partials, double *out,
                                cudaStream_t s);
// allocation-free variant: block partials in a static device array (tled_noalloc.cu)
constexpr int kNoAllocMaxBlocks = 296;
cudaError_t noalloc_scratch(int device, double **ptr);

// host geometry and planning (tled_host.cpp)
bool element_geometry(int npe, const double *X, const int32_t *cn, double Jinv[9], double *V);
bool brick_element(const double *X, const int32_t *cn);  // H8 axis-aligned box test
// fib: per-element fibres [ne][3] or NULL (m.a0); the conduction bound uses the anisotropic
// conductivity at F = I when m.k_fibre_ratio is not 0 or 1
void stable_dt(int npe, int64_t nn, const double *X, int64_t ne, const int32_t *conn, const tled_material &m,
               const double *mat6, const double *fib, const tled_params &p, double *dt_mech, double *dt_th);
// group: optional [ne] group id per element (scenario rank); tiles never span groups and
// follow ascending group order.
int build_plan(int npe, int64_t nn, const double *X, int64_t ne, const int32_t *conn, const int8_t *etype,
               const int32_t *group,
               int tile_elems, Plan &p, std::string &err);

}  // namespace tled
