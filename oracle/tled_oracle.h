/*
 * Oracle for the coupled thermo-visco-hyperelastic TLED step of
 * Zhang et al., "Towards real-time finite-strain anisotropic
 * thermo-visco-elastodynamic analysis of soft tissues for thermal ablative
 * therapy" (arXiv 2009.10400).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 CPU restatement of
 * the paper's Sections 3-4 (Eqs. 1-28, Tables 1 and 5), written to be checked
 * by eye against the paper.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product (the CUDA library)
 * never includes, links or calls it, and it shares no code with that library.
 *
 * Every function below names the equation it follows.  Where the paper is
 * silent or garbled, the reading taken is stated at the point of use.
 *
 * Parity unpinned (no value of the paper or closed form fixes them; they are
 * held only by the invariants the tests check and by oracle-vs-GPU): the H8
 * hourglass coefficient (reading of the cited stabilisation, no formula in the
 * paper), the perfusion-unit, source-shape and mass-scaling readings, and whole
 * multi-thousand-step trajectories.
 */
#ifndef TLED_ORACLE_H
#define TLED_ORACLE_H
#include <stdint.h>

#define ORA_MAX_PRONY 4

typedef struct {
    /* ---- mesh (caller owned) ---- */
    int32_t npe;               /* 4 = linear tetrahedron (T4), 8 = hexahedron (H8) */
    int32_t pad0;
    int64_t nn, ne;
    const double *X;           /* [nn][3] reference coordinates, m */
    const int32_t *conn;       /* [ne][npe], VTK corner order */
    /* ---- per-element material (caller owned) ---- */
    const double *rho;         /* [ne] kg/m^3 */
    const double *mu;          /* [ne] shear modulus, Pa (Table 1/5) */
    const double *kappa;       /* [ne] bulk modulus, Pa */
    const double *k1;          /* [ne] fibre stiffness, Pa */
    const double *k2;          /* [ne] fibre exponent (0 = quadratic Table 5 term) */
    const double *kc;          /* [ne] thermal conductivity at T_ref, W/(m K) */
    const double *alpha;       /* [ne] thermal expansion coefficient, 1/K */
    const double *a0;          /* [ne][3] unit fibre direction in the reference configuration */
    /* ---- uniform parameters ---- */
    int32_t n_prony, pad1;
    double prony_g[ORA_MAX_PRONY], prony_tau[ORA_MAX_PRONY];
    double c_heat;             /* specific heat at T_ref, J/(kg K) */
    double beta_c, beta_k;     /* relative slopes of c(T), k(T) per K (Table 5 linear interpolation) */
    double T_ref;              /* temperature at which c, k are given, C */
    double wbcb;               /* perfusion w_b c_b, W/(m^3 K) (Eq. 1) */
    double Qm;                 /* metabolic heat, W/m^3 */
    double T0, Ta;             /* initial (stress-free) temperature and arterial temperature, C */
    double lnA, Ea;            /* Arrhenius frequency factor (log) and activation energy J/mol */
    int32_t expansion;         /* 1: thermal expansion split of Eqs. 7-11 on */
    int32_t temp_dep;          /* 1: c(T), k(T) on */
    double gamma;              /* mass-proportional damping coefficient, 1/s (Eq. 21) */
    double mass_scale;         /* mechanical mass multiplier (1 = none) */
    double kappa_hg, kappa_hgT;/* H8 hourglass coefficients (mechanical, thermal) */
    double dt;                 /* time step, s */
    int32_t n_src, pad2;
    const double *src;         /* [n_src][11]: c0 xyz, velocity xyz, sigma (Gaussian) or radius
                                  (sphere), peak W/m^3, t_on, t_off, shape (0 Gaussian, 1 uniform sphere) */
    const uint8_t *mask;       /* [nn] bit0..2: u_x,u_y,u_z prescribed; bit3: T held */
    const double *ubar;        /* [nn][3] prescribed displacement at the end of the ramp (NULL = 0) */
    double ramp_time;          /* prescribed displacement ramps linearly over this time (0 = at once) */
    double aniso_alpha;        /* expansion along the fibre / transverse expansion (Eq. 11, transversely
                                  isotropic form with m = a0); 1 = isotropic */
    double aniso_k;            /* conductivity along the current fibre / transverse conductivity; 1 = isotropic */
    /* ---- precomputed by ora_setup (caller allocated) ---- */
    double *dhdX;              /* [ne][npe][3] shape-function derivatives at the integration point */
    double *V0;                /* [ne] reference element volume (8 det J0 for H8, V0 for T4) */
    double *hg_gamma;          /* [ne][8][4] hourglass shape vectors (H8 only; may be NULL for T4) */
    double *khg;               /* [ne] mechanical hourglass stiffness (H8) */
    double *khgT;              /* [ne] thermal hourglass conductance per unit conductivity (H8) */
    double *M;                 /* [nn] lumped (possibly mass-scaled) mechanical mass */
    double *Cth;               /* [nn] lumped thermal mass rho c V at T_ref */
    double *Vn;                /* [nn] lumped reference volume */
} ora_model;

typedef struct {
    double *u;                 /* [nn][3] displacement at t */
    double *u_prev;            /* [nn][3] displacement at t - dt (Eq. 27) */
    double *T;                 /* [nn] absolute temperature, C */
    double *Omega;             /* [nn] Arrhenius damage integral */
    double *visc;              /* [ne][n_prony][6] Prony state (xx,yy,zz,xy,yz,xz) */
    double t;
    int64_t step;
    double *cem;               /* [nn] CEM43 thermal dose, equivalent minutes at 43 C (NULL: not tracked) */
} ora_state;

#ifdef __cplusplus
extern "C" {
#endif
/* Precompute shape-function derivatives, volumes, hourglass vectors and lumped
 * masses (Section 5, total Lagrangian precomputation).  Returns 0, or -(1+e)
 * for the first element e with non-positive reference Jacobian. */
int ora_setup(ora_model *m);

/* One explicit coupled step t -> t + dt (Eqs. 20, 27, Arrhenius).  Work
 * arrays f [nn][3] and fT [nn] are caller allocated.  Returns 0. */
int ora_step(const ora_model *m, ora_state *s, double *f, double *fT);

/* Element e: internal forces f_e [npe][3] (Eq. 24-28 + hourglass) and thermal
 * loads fT_e [npe] (Eq. 16-19 + thermal hourglass), given the state.  visc_in
 * is the element's Prony state at t - dt, visc_out receives the state at t
 * (both may alias).  Returns det F. */
double ora_element(const ora_model *m, int64_t e, const double *u, const double *T,
                   const double *visc_in, double *visc_out, double *f_e, double *fT_e);

/* Stored energy of element e for elastic checks: V0 det(F_th) Psi(F F_th^-1)
 * + mechanical hourglass energy (Table 1/5, Eq. 10). */
double ora_element_energy(const ora_model *m, int64_t e, const double *u, const double *T);

/* Thermal "energy" 1/2 V0 J k grad0(T) . C^-1 grad0(T) + thermal hourglass
 * energy, at the conductivity of the element temperature Tk_fixed (Eq. 16). */
double ora_element_thermal_energy(const ora_model *m, int64_t e, const double *u,
                                  const double *T, double Tk_fixed);

/* Next state (u, u_prev, T, Omega at t + dt) of the listed nodes only, from
 * the full state s, without modifying s. out_u [k][3], out_T [k], out_O [k]. */
int ora_step_nodes(const ora_model *m, const ora_state *s, const int64_t *nodes, int64_t k,
                   double *out_u, double *out_T, double *out_O);

/* Critical time step reading: safety * min(mechanical CFL, thermal Gershgorin). */
double ora_stable_dt(const ora_model *m, double safety, double *dt_mech, double *dt_th);

/* Temperature and damage fraction at k points xyz [k][3] (reference
 * coordinates) from the state s: the point is located in the first element (in
 * id order) that contains it -- T4 by its affine map, H8 by a Newton solve of
 * the trilinear isoparametric map -- and the nodal temperatures and nodal
 * damage fractions 1 - exp(-Omega) are interpolated with that element's shape
 * functions (the interpolation behind Eqs. 18-19).  Returns 0, or -(1+q) for
 * the first point q that lies in no element. */
int ora_probe(const ora_model *m, const ora_state *s, const double *xyz, int64_t k, double *T_out,
              double *d_out);

/* Node-to-element incidence for ora_step_parallel: offsets [nn + 1] and
 * slots [ne * npe] (entries e * npe + corner, ascending element id within a
 * node).  Returns 0, or -1 if a work allocation failed. */
int ora_incidence(const ora_model *m, int64_t *offsets, int64_t *slots);

/* ora_step on all host cores (OpenMP): elements in parallel into elem_out
 * [ne][npe][4], then every node sums its incident elements' entries in
 * ascending element id from zero -- the additions ora_step makes, in the same
 * order -- so the result is bitwise that of ora_step.  Returns 0. */
int ora_step_parallel(const ora_model *m, ora_state *s, const int64_t *offsets, const int64_t *slots,
                      double *elem_out, double *f, double *fT);

/* Threads ora_step_parallel uses (1 without OpenMP). */
int ora_threads(void);

/* One thermal step of m->dt with mechanical subcycling: n_sub substeps of
 * m->dt / n_sub, each an element pass (Prony recurrence with the substep) and
 * the central-difference update of Eq. (27) over the substep; the temperature
 * is held at T(t) during the substeps, and the last one also advances T, Omega
 * and the CEM43 dose over m->dt (Eq. 20, explicit in T(t)) with its own
 * thermal loads (the current displacement) and the sources at the thermal
 * step's start t.  s->t advances by the substep each substep; n_sub = 1 is
 * ora_step.  Work arrays as for ora_step.  Returns 0. */
int ora_step_subcycled(const ora_model *m, ora_state *s, int n_sub, double *f, double *fT);
#ifdef __cplusplus
}
#endif
#endif
