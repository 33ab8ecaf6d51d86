/*
 * libtled -- coupled thermo-visco-hyperelastic total Lagrangian explicit
 * dynamics (TLED) for soft tissue under thermal ablation, on one NVIDIA B300
 * (sm_103a).  The method is that of Zhang, Lay, Roberts and Chauhan,
 * arXiv 2009.10400: bioheat transfer (Pennes, Eq. 1) computed on the deformed
 * configuration (Eqs. 5-6), thermal expansion through the multiplicative
 * split F = F_elas F_ther (Eqs. 7-11), a transversely isotropic
 * visco-hyperelastic law (Table 5, Prony recurrence of Section 4.3), explicit
 * Euler for temperature (Eq. 20) and central differences for displacement
 * (Eq. 27), on one-point hexahedra (H8, Eqs. 18, 25) or linear tetrahedra
 * (T4, Eqs. 19, 26), plus an Arrhenius damage integral (Section 7).
 *
 * Conventions
 *  - Every call returns an int status: TLED_OK (0) or a negative TLED_E_*
 *    code.  Nothing throws across this boundary.  tled_last_error() gives a
 *    one-line detail (offending element / node ids are 0-based, in the
 *    caller's numbering).
 *  - SI units; temperatures in degrees C; indices int32; floating inputs are
 *    float64 and are copied at call time (the library keeps no caller
 *    pointer).  The device computes in FP32 with compensated (float-float)
 *    accumulation of nodal displacement and temperature.
 *  - Device memory: the library never allocates device memory.  After the
 *    set-up calls, tled_workspace_size() reports how many bytes it needs; the
 *    caller passes a device buffer of at least that size (256-byte aligned)
 *    to tled_init() and keeps it alive until tled_destroy().
 *  - Streams: all device work is enqueued on the stream given to
 *    tled_create() (NULL = the legacy default stream).  Calls that return
 *    host data synchronise that stream.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - Step modes (chosen at init, reported by tled_get_mode, all computing the
 *    same numbers): streamed (a tile kernel and a shared-node kernel per step,
 *    captured in CUDA graphs of 32 steps), resident (a problem -- or each
 *    scenario of a batch -- that fits one CTA's shared memory runs 32 steps
 *    per launch in one CTA) and grid-resident (a single problem whose tiles fit
 *    co-resident CTAs runs 32 steps per cooperative launch).
 *
 * Call order:  create -> set_mesh -> set_material -> [set_bcs] ->
 *   [set_heat_sources] -> [set_params] -> workspace_size -> init ->
 *   { step, sync, get_*, set_state, set_heat_sources, save/load } -> destroy.
 */
#ifndef TLED_H
#define TLED_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TLED_VERSION 5

/* status codes */
#define TLED_OK 0
#define TLED_E_ARG (-1)      /* bad argument: NULL pointer, size or value out of range */
#define TLED_E_MESH (-2)     /* connectivity index out of range, or det J0 <= 0 */
#define TLED_E_STATE (-3)    /* call out of order (e.g. step before init) */
#define TLED_E_CUDA (-4)     /* a CUDA runtime call failed */
#define TLED_E_UNSTABLE (-5) /* NaN/Inf in the nodal state (time step too large?) */
#define TLED_E_INVERTED (-6) /* an element reached J <= 0 */
#define TLED_E_TIMEOUT (-7)  /* a bounded device wait ran out */
#define TLED_E_NOMEM (-8)    /* workspace smaller than tled_workspace_size() */
#define TLED_E_FORMAT (-9)   /* checkpoint blob malformed (magic, size, checksum) */

/* element types */
#define TLED_T4 4 /* 4-node linear tetrahedron, corners 0..3, positive volume */
#define TLED_H8 8 /* 8-node hexahedron, VTK corner order, one-point centroid rule */

/* where a read-back goes */
#define TLED_HOST 0
#define TLED_DEVICE 1

/* tled_params.flags */
#define TLED_EXPANSION (1u << 0)   /* thermal expansion split, Eqs. (7)-(11) */
#define TLED_TEMP_DEP (1u << 1)    /* c(T), k(T) linear in T (Table 5) */
#define TLED_COMPENSATED (1u << 2) /* float-float accumulation of u and T */
#define TLED_CEM43 (1u << 3)       /* accumulate the CEM43 thermal dose per node (single problems only) */
#define TLED_GENERAL_H8 (1u << 4)  /* keep the general H8 kernel for brick meshes (every element an
                                      axis-aligned box: reference hourglass projections and off-diagonal
                                      reference Jacobian entries zero in float, e.g. voxels), which otherwise
                                      take a kernel without those zero terms that stores only the diagonal
                                      of J0^-1; the two agree within 1e-6 relative */
#define TLED_STREAMED (1u << 5)    /* keep the streamed step (tile kernel + shared-node kernel per step) when
                                      the problem would fit the resident mode (every scenario in one CTA's
                                      shared memory) or the grid-resident one (a single problem's tiles in
                                      co-resident CTAs); K steps per launch there, same arithmetic and results */

/* boundary mask bits (per node) */
#define TLED_FIX_X 1u
#define TLED_FIX_Y 2u
#define TLED_FIX_Z 4u
#define TLED_FIX_T 8u

/* Uniform material of the tissue.  Mechanics: Table 5's transversely
 * isotropic neo-Hookean law Psi = mu/2 (I1b - 3) + kappa/2 (J - 1)^2 +
 * k1/(2 k2) [exp(k2 (I4b - 1)^2) - 1] (k2 = 0: the quadratic term
 * k1/2 (I4b - 1)^2 of Table 5, eta_a = k1); Prony series of the generalised
 * Maxwell model (Section 2.2).  Heat: Pennes, Eq. (1). */
typedef struct tled_material {
    double rho;           /* density, kg/m^3 */
    double mu, kappa;     /* shear and bulk modulus, Pa */
    double k1, k2;        /* fibre stiffness Pa, fibre exponent (dimensionless) */
    double a0[3];         /* unit fibre direction in the reference configuration */
    int32_t n_prony;      /* number of Prony terms, 0..4 */
    int32_t pad;
    double prony_g[4];    /* phi_i, relative moduli */
    double prony_tau[4];  /* tau_i, s */
    double alpha;         /* isotropic thermal expansion, 1/K (Eq. 11) */
    double k;             /* thermal conductivity at T_ref, W/(m K) */
    double c;             /* specific heat at T_ref, J/(kg K) */
    double beta_k;        /* relative slope of k(T), 1/K (used with TLED_TEMP_DEP) */
    double beta_c;        /* relative slope of c(T), 1/K (used with TLED_TEMP_DEP) */
    double T_ref;         /* temperature at which k and c are given, C */
    double wb_cb;         /* perfusion w_b c_b, W/(m^3 K) */
    double Qm;            /* metabolic heat, W/m^3 */
    double T0;            /* initial and stress-free temperature, C */
    double Ta;            /* arterial blood temperature, C */
    double lnA;           /* natural log of the Arrhenius frequency factor, ln(1/s) */
    double Ea;            /* Arrhenius activation energy, J/mol */
    /* Anisotropic thermal physics (0 or 1 = isotropic): thermal expansion along the
     * fibre a0 relative to the transverse alpha, F_th = lambda_i I + (lambda_m - lambda_i)
     * a0 (x) a0 (Eq. 11, transversely isotropic), lambda_m = 1 + alpha_fibre_ratio alpha
     * theta; conductivity along the current fibre F a0 / |F a0| relative to the
     * transverse k.  The H8 thermal hourglass uses the transverse k. */
    double alpha_fibre_ratio;
    double k_fibre_ratio;
} tled_material;

/* A volumetric heat source with centre c(t) = c0 + vel t, active for
 * t_on <= t < t_off.  Heat source shapes: a Gaussian P exp(-|x - c(t)|^2 / (2 sigma^2)), or (the
 * paper's liver case, Section 6.3) a uniform density P inside the sphere
 * |x - c(t)| <= sigma.  x is the current nodal position X + u(t). */
#define TLED_SRC_GAUSSIAN 0
#define TLED_SRC_SPHERE 1

typedef struct tled_source {
    double c0[3], vel[3];
    double sigma;  /* m: standard deviation (Gaussian) or radius (sphere) */
    double power;  /* peak density, W/m^3 */
    double t_on, t_off;
    int32_t shape; /* TLED_SRC_GAUSSIAN or TLED_SRC_SPHERE */
    int32_t pad;
} tled_source;

typedef struct tled_params {
    double dt;          /* time step, s; 0 = dt_safety * stable step */
    double dt_safety;   /* fraction of the stable step used when dt = 0 (default 0.8) */
    double gamma;       /* mass-proportional damping D = gamma M, 1/s (Eq. 21) */
    double mass_scale;  /* mechanical mass multiplier >= 1 (1 = none); < 0 = automatic (needs dt > 0):
                           s_m = max(1, (dt / (dt_safety dt_mech))^2) with dt_mech the CFL bound of the
                           unscaled mesh, which makes dt the safe mechanical step (mass scaling for
                           long heating runs, where inertia barely affects temperature); init and
                           tled_stable_dt then fail with E_ARG if dt exceeds dt_safety x the thermal
                           bound */
    double kappa_hg;    /* H8 hourglass coefficient (default 0.1) */
    double kappa_hgT;   /* H8 thermal hourglass coefficient (default 0.1) */
    uint32_t flags;     /* TLED_EXPANSION | TLED_TEMP_DEP | TLED_COMPENSATED */
    int32_t tile_elems; /* elements per tile, 0 = default (H8 512, T4 1024) */
    int32_t n_sub;      /* mechanical subcycling: n_sub >= 1 mechanical substeps per thermal step (0 = 1).
                           A step (tled_step, n_steps of a batch scenario) is then a mechanical substep
                           of length dt_thermal / n_sub; every substep advances u (Eq. 27) and the Prony
                           state; the last of each n_sub also advances T (Eq. 20), Omega and the CEM43
                           dose by the thermal step, explicit in T at the thermal step's start, with the
                           sources at that start time and the thermal loads of the current displacement.
                           dt (if > 0) is the THERMAL step; dt = 0 takes dt_safety x min(n_sub dt_mech,
                           dt_thermal); an automatic mass scale makes dt / n_sub the safe mechanical step.
                           tled_get_dt and tled_scenario_dt report the substep. */
    int32_t pad;
} tled_params;

typedef struct tled_stats {
    int64_t step;           /* steps taken since t = 0 or the last set_state */
    double t, dt;           /* current time and time step, s */
    double T_max, T_min;    /* nodal temperature extrema, C */
    double u_max;           /* max nodal |u|, m */
    double damage_volume;   /* sum of lumped volumes with Omega >= 1, m^3 */
    double heat_content;    /* sum_i C_i (T_i - T0), J (thermal mass at T_ref) */
    double kinetic_energy;  /* sum_i 1/2 m_i |v_i|^2, J (mechanical, mass-scaled; v at the last half step) */
    double strain_energy;   /* sum_e V0 lambda^3 Psi(F/lambda), J: stored energy of Eq. 9's potential
                               (Table 5 terms, fibre term as in the step) with the thermal split of
                               Eqs. 7-11, at the current u and theta */
    double hourglass_energy;/* sum_e 1/2 k_hg sum_al |q_al|^2, J (H8 hourglass control; 0 for T4) */
    uint32_t status;        /* device status bits (0 = healthy) */
    int32_t pad;
} tled_stats;

typedef struct tled_ctx tled_ctx;

/* Library version (TLED_VERSION). */
int tled_version(void);
/* Static text for a status code. */
const char *tled_status_string(int code);

/* Create a context on CUDA device `device`; all work goes to `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream).  *out receives the context.
 * device = -1 makes a host-only context: set-up, validation, planning and
 * tled_workspace_size() work without a GPU; tled_init() then fails with
 * E_STATE.  Errors: E_ARG (out NULL), E_CUDA (device not usable). */
int tled_create(tled_ctx **out, int device, void *cuda_stream);
/* Destroy a context (and its CUDA graphs).  Does not free the workspace. */
int tled_destroy(tled_ctx *ctx);
/* Last error detail of the context (never NULL; "" if none). */
const char *tled_last_error(const tled_ctx *ctx);

/* Mesh (total Lagrangian reference configuration, Section 4.1).
 * elem_type: TLED_T4 or TLED_H8.  X0: [n_nodes][3] host float64.  conn:
 * [n_elems][elem_type] host int32, 0-based.  Errors: E_ARG, E_MESH (index out
 * of range or det J0 <= 0 -- the detail names the element). */
int tled_set_mesh(tled_ctx *ctx, int elem_type, int64_t n_nodes, const double *X0, int64_t n_elems,
                  const int32_t *conn);

/* Material.  m: uniform values.  per_elem: optional host float64
 * [n_elems][6] = (mu, kappa, k1, k2, k, alpha) per element, overriding the
 * uniform ones.  fibre: optional host float64 [n_elems][3] unit fibre
 * directions.  Errors: E_ARG (NaN/negative moduli, n_prony > 4), E_STATE
 * (no mesh). */
int tled_set_material(tled_ctx *ctx, const tled_material *m, const double *per_elem, const double *fibre);

/* Boundary conditions.  mask: host uint8 [n_nodes] of TLED_FIX_* bits (a
 * fixed displacement component follows ubar; TLED_FIX_T holds the node's
 * temperature).  ubar: optional host float64 [n_nodes][3], the prescribed
 * displacement reached after ramp_time (linear ramp; 0 = at once); NULL
 * means zero.  The exterior is otherwise adiabatic and traction-free. */
int tled_set_bcs(tled_ctx *ctx, const uint8_t *mask, const double *ubar, double ramp_time);

/* Heat sources (n <= 16).  May be called again after init to change the
 * sources (enqueued on the stream; takes effect at the next step). */
int tled_set_heat_sources(tled_ctx *ctx, int32_t n, const tled_source *s);

/* Solver parameters.  p NULL = defaults (auto dt at 0.8, no damping, no mass
 * scaling, hourglass 0.1/0.1, expansion + compensation on). */
int tled_set_params(tled_ctx *ctx, const tled_params *p);

/* Bytes of device workspace tled_init() needs for the current set-up. */
int tled_workspace_size(tled_ctx *ctx, int64_t *bytes);

/* Precompute (shape-function derivatives, volumes, lumped masses, stable
 * step, tiling) and upload into the caller's device buffer; zero state at
 * T = T0.  Synchronises the stream.  Errors: E_NOMEM, E_STATE, E_CUDA. */
int tled_init(tled_ctx *ctx, void *dev_workspace, int64_t bytes);

/* The time step in use (after init) and the two stable-step bounds
 * (mechanical CFL and thermal Gershgorin, before the safety factor). */
int tled_get_dt(tled_ctx *ctx, double *dt, double *dt_mech, double *dt_thermal);

/* The two stable-step bounds of the current set-up (no GPU needed): the
 * mechanical CFL bound (with the set mass scale) and the thermal Gershgorin
 * bound, before the safety factor. */
int tled_stable_dt(tled_ctx *ctx, double *dt_mech, double *dt_thermal);

/* Mechanical mass multiplier in use for scenario `index` (0 for a single
 * problem): tled_params.mass_scale, or the automatic choice described there.
 * No GPU needed.  Errors: E_ARG (index, or dt above the thermal bound with the
 * automatic choice), E_STATE (no mesh or material). */
int tled_get_mass_scale(tled_ctx *ctx, int32_t index, double *mass_scale);

/* Enqueue n explicit coupled steps (element pass, deterministic node gather,
 * nodal updates of u, T and damage).  Asynchronous: device faults such as
 * NaN or inversion are reported by the next tled_sync(). */
int tled_step(tled_ctx *ctx, int64_t n);

/* Wait for the stream; return TLED_OK, or E_UNSTABLE / E_INVERTED if the
 * device flagged the state (the detail names the first node / element). */
int tled_sync(tled_ctx *ctx);

/* Read-back in the caller's node order.  where = TLED_HOST: out is host
 * memory and the call synchronises; TLED_DEVICE: out is device memory and
 * the copy is only enqueued.
 *   displacement: [n_nodes][3] float64, m
 *   temperature:  [n_nodes]    float64, C
 *   damage:       [n_nodes]    float64, fraction 1 - exp(-Omega) */
int tled_get_displacement(tled_ctx *ctx, double *out, int where);
int tled_get_temperature(tled_ctx *ctx, double *out, int where);
int tled_get_damage(tled_ctx *ctx, double *out, int where);
/* CEM43 thermal dose per node, equivalent minutes at 43 C (Sapareto-Dewey:
 * sum of dt/60 R^(43 - T(t)), R = 0.5 at or above 43 C, 0.25 below, explicit
 * in T(t) like the Arrhenius integral), accumulated in FP64 by a small kernel
 * before each step when the flags hold TLED_CEM43; [n_nodes] float64, caller
 * order.  E_STATE without TLED_CEM43. */
int tled_get_cem43(tled_ctx *ctx, double *out, int where);
/* Volume of tissue at or above T_iso (C), sum of the lumped nodal volumes of
 * the nodes with T >= T_iso (the paper reads the ablation zone off the 60 C
 * isotherm, Section 6.3); deterministic FP64 reduction.  Synchronises. */
int tled_get_isotherm_volume(tled_ctx *ctx, double T_iso, double *volume);

/* Overwrite the full state from host float64 arrays (caller order):
 * u [n][3], v [n][3] (velocity at t - dt/2), T [n], Omega [n], and visc
 * [n_elems][n_prony][6] (xx,yy,zz,xy,yz,xz; NULL = zero), at time t after
 * `step` steps.  Synchronises. */
int tled_set_state(tled_ctx *ctx, const double *u, const double *v, const double *T, const double *Omega,
                   const double *visc, double t, int64_t step);
/* Read the full state into host float64 arrays (any pointer may be NULL). */
int tled_get_state(tled_ctx *ctx, double *u, double *v, double *T, double *Omega, double *visc, double *t,
                   int64_t *step);

/* Diagnostic timing: enqueue n steps with the kernels launched one by one (no
 * graph) and CUDA events around each launch on the context stream; ms[0]
 * receives the summed device time of the tile kernel (element pass,
 * in-tile gather, interior-node update), ms[1] that of the shared-node
 * kernel.  The steps are real (the state advances).  Synchronises. */
int tled_step_timed(tled_ctx *ctx, int64_t n, double *ms);

/* Plan summary after tled_workspace_size(): info[0] tiles, [1] interior
 * nodes, [2] shared nodes, [3] partial slots, [4] workspace bytes, [5]
 * element type, [6] scenarios, [7] persistent CTAs of the tile kernel (after
 * init).  info has 8 entries. */
int tled_plan_info(tled_ctx *ctx, int64_t *info);

/* L2 residency of the streamed step (after init): the streamed step kernels are
 * launched with an access-policy window over the shared nodes' (u, theta) and
 * the partial sums, which the tile kernel writes and the shared-node kernel reads
 * back within the step, marked persisting; init raises the CUDA context's
 * persisting set-aside (cudaLimitPersistingL2CacheSize, a limit of the calling
 * process's context) to the window's size, capped by the device's maximum and by
 * 40 % of L2 (the hit ratio then covers the capped share of the window), and
 * tled_destroy puts the previous value back.  out[0] window bytes (0: none, e.g.
 * no shared nodes), out[1] set-aside bytes, out[2] the window's hit ratio times
 * 1e6.  An implementation choice of this library, not part of the paper. */
int tled_l2_window(tled_ctx *ctx, int64_t *out);

/* ---- probes (temperature and damage at points, e.g. a 16^3 lattice) ----
 * Set-up call of a single-scenario context: n points xyz [n][3] (host
 * float64, reference coordinates).  Each point is located in the mesh when
 * the context is planned (E_ARG if a point lies outside every element) and
 * is interpolated with the element's shape functions. */
int tled_set_probes(tled_ctx *ctx, int64_t n, const double *xyz);
/* out [2][n_probes] float64: temperature (C) then damage fraction, in probe
 * order (for a batch: scenario 0's probes, then scenario 1's, ...).  where as
 * for the field read-backs. */
int tled_get_probes(tled_ctx *ctx, double *out, int where);

/* ---- batches: many independent scenarios advanced by the same launches ----
 * Treatment planning runs many scenarios (meshes, sources, tissue parameters,
 * durations) at once.  A batch context holds copies of fully set-up single
 * scenario contexts; their meshes are concatenated (caller numbering:
 * scenario 0 first), tiled without crossing scenarios, and one launch of the
 * step kernels per step advances all unfinished scenarios, each with its own
 * time step.  A scenario stops after n_steps steps (its state then stays
 * fixed).  Scenarios must share the element type, number of Prony terms,
 * T0, Ta, Arrhenius constants, c/k slopes, flags, hourglass coefficients and
 * ramp time (E_ARG otherwise).  After tled_batch_add the usual
 * tled_workspace_size / tled_init / tled_step / tled_get_* / tled_get_probes /
 * checkpoint calls apply to the whole batch. */
int tled_batch_create(tled_ctx **out, int device, void *cuda_stream);
/* Append a copy of `scenario`'s set-up (mesh, material, BCs, sources,
 * params, probes); *index receives its scenario index. */
int tled_batch_add(tled_ctx *batch, const tled_ctx *scenario, int64_t n_steps, int32_t *index);
/* Run until every scenario has taken its n_steps (enqueued; *steps receives
 * the number of launches-steps run). */
int tled_batch_run(tled_ctx *batch, int64_t *steps);
/* info[0] node offset, [1] nodes, [2] element offset, [3] elements, [4]
 * n_steps (-1 = unbounded), [5] steps taken, [6] probe offset, [7] probes. */
int tled_scenario_info(tled_ctx *ctx, int32_t index, int64_t *info);
/* time step of one scenario (after init) */
int tled_scenario_dt(tled_ctx *ctx, int32_t index, double *dt);

/* ---- autotuner ----
 * Time the candidate tilings (elements per tile 256 / 192 / 128, persistent
 * grid of one or two CTAs per SM; and the resident and grid-resident modes
 * where the problem fits them) for `trial_steps` steps each in the
 * caller's workspace (bytes of it), keep the fastest, and leave the context
 * initialised with it at t = 0 (state reset).  The choice is cached in the
 * process per element type, size (log2 of the element count), material
 * layout and scenario count; a cached choice is applied without timing.
 * choice[0] elements per tile, [1] CTAs, [2] 1 if it came from the cache. */
int tled_autotune(tled_ctx *ctx, void *dev_workspace, int64_t bytes, int32_t trial_steps, int32_t *choice);
/* Kernel choice after init, as bits of *mode: bit 0 (TLED_MODE_RESIDENT) when the steps
 * run in the resident mode (each scenario held by one CTA in shared memory for K steps
 * per launch), bit 2 (TLED_MODE_GRID) in the grid-resident mode (a single problem's tiles
 * held by the CTAs of one cooperative launch for K steps, grid barriers between the
 * phases), neither when streamed (tile and shared-node kernels per step); bit 1
 * (TLED_MODE_BRICK) when the H8 brick instance runs. */
#define TLED_MODE_RESIDENT 1
#define TLED_MODE_BRICK 2
#define TLED_MODE_GRID 4
int tled_get_mode(tled_ctx *ctx, int32_t *mode);

/* Self-test of the bounded device waits (after init): runs a kernel whose wait can
 * never complete and returns what a step would report: TLED_E_TIMEOUT after about a
 * second or two.  which = 0: a one-CTA kernel's mbarrier wait (as the tile kernel's
 * copies use); 1: a one-CTA kernel's grid-barrier wait (as the grid-resident mode
 * uses); 2: the step's own tile kernel with the node staging of tile 0 left out, so
 * that the CTA holding it waits in vain, skips its element pass, waits (bounded) for
 * its other copies and leaves while the other CTAs finish their tiles (streamed mode
 * only, else E_STATE; the nodal state is then that of a partial step -- set it again,
 * e.g. with tled_set_state or tled_load_state, before stepping on).  The status is
 * cleared again afterwards, so the context stays usable.  Nothing faults or hangs. */
int tled_selftest_wait(tled_ctx *ctx, int32_t which);

/* Scalar diagnostics, reduced on the device in FP64 in a fixed order
 * (deterministic).  With no damping, no viscous terms, fixed or free
 * boundaries and no thermal load, kinetic_energy + strain_energy +
 * hourglass_energy is the mechanical energy the central-difference scheme
 * conserves up to O(dt^2) oscillation (energy balance).  Synchronises. */
int tled_get_stats(tled_ctx *ctx, tled_stats *s);

/* Allocation-free diagnostics (the paper has no counterpart: this is a
 * service for callers that cannot allocate device memory when they want the
 * numbers -- real-time loops in which an allocation would synchronise the
 * device or take an unbounded time, and processes whose device memory is fully
 * held by another framework's caching allocator).  Enqueues on the context
 * stream the same FP64 reduction as tled_get_stats and writes six doubles to
 * the DEVICE buffer `out` (device or managed memory of the context's device;
 * anything else is refused with E_ARG):
 *   out[0] kinetic energy sum_i 1/2 m_i |v_i|^2          (J)
 *   out[1] heat content sum_i C_i (T_i - T0)              (J)
 *   out[2] max_i (T_i - T0), out[3] min_i (T_i - T0)       (K)
 *   out[4] max_i |u_i|^2                                   (m^2)
 *   out[5] sum of lumped volumes with Omega >= 1           (m^3)
 * n_blocks: reduction blocks, 0 = 296; values above 296 are rejected with
 * E_ARG (the block partial sums live in a static device array of 296 x 8
 * doubles, 18,944 bytes, that every GPU loading the library keeps until the
 * process exits).  Allocates nothing (no cudaMalloc, no allocating library
 * call) and does not synchronise.  The first call on a device looks up that
 * array's device address (with the device current) and keeps it for the
 * process; make that first call before any stream capture.  After a
 * cudaDeviceReset of the device the kept address belongs to the ended context:
 * do not call this entry point in that process again.  All calls in the
 * process share the array: each call overwrites the partial sums it reads, so
 * nothing needs clearing, but calls whose kernels overlap on the GPU
 * (different streams, or different contexts on one device) race on it and
 * must be ordered by the caller. */
int tled_get_stats_noalloc(tled_ctx *ctx, int32_t n_blocks, double *out);

/* Checkpoint: serialise the exact device state (bitwise) with a header and
 * checksum.  Call with buf NULL to get *bytes; then with a buffer of that
 * size.  load verifies magic, sizes, a hash of the set-up and the checksum
 * (E_FORMAT otherwise). */
int tled_save_state(tled_ctx *ctx, void *buf, int64_t *bytes);
int tled_load_state(tled_ctx *ctx, const void *buf, int64_t bytes);

#ifdef __cplusplus
}
#endif
#endif
