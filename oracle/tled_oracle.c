/*
 * Oracle: plain FP64 CPU restatement of the coupled thermo-visco-hyperelastic
 * total Lagrangian explicit dynamics step (arXiv 2009.10400, Sections 3-4).
 *
 * TEST INFRASTRUCTURE ONLY -- see tled_oracle.h.  No blocking, no fusion, no
 * reformulation: F is formed as I + H, the stress is the textbook
 * S = 2 dPsi/dC, the thermal load is the literal matrix product of Eq. (16),
 * the displacement update is Eq. (27) with u(t - dt), and nodal sums run in
 * element-id order.
 *
 * Readings where the paper is silent or garbled (all listed in the design
 * notes of the repository):
 *   R1  conduction enters Eq. (20) with the physical sign: dT/dt gets -K T.
 *   R2  F_ij = delta_ij + sum_a u_ai dh_a/dX_j (Eq. 17);
 *       K_e = V J (B F^-1) D (B F^-1)^T with B = [npe x 3] (Eqs. 16, 18, 19).
 *   R3  the element temperature (for lambda and k(T)) is the mean of its nodes.
 *   R4  lambda = 1 + alpha (T_e - T0), exactly linear (Eq. 11, isotropic).
 *   R6  the Prony recurrence acts on the total pulled-back stress S0.
 *   R7  fibre term Psi_f = k1/(2 k2) [exp(k2 (I4b - 1)^2) - 1]; k2 = 0 gives the
 *       quadratic Table 5 term with eta_a = k1.
 *   R8  H8 one-point integration with a stiffness-type hourglass control
 *       (Flanagan-Belytschko shape vectors, total Lagrangian form).
 *   R9  H8 derivatives at the centroid, volume 8 det J0 (Eqs. 18, 25).
 *   R10 lumped masses / volumes from reference volumes split evenly per node.
 *   R11 c(T), k(T) linear in T, evaluated at the time-t temperature.
 *   R14 Gaussian heat sources evaluated at the current nodal position.
 *   R16 stable dt = safety * min(element CFL, thermal Gershgorin bound).
 *   R18 Arrhenius rate A exp(-Ea / (R T_abs)) evaluated at T(t).
 *   R24 CEM43 dose accumulated explicitly at T(t): dt R^(43 - T) / 60 minutes,
 *       R = 0.5 (T >= 43 C) or 0.25.
 *   R26 anisotropic thermal physics: transversely isotropic F_th about m = a0
 *       (Eq. 11) with fibre expansion aniso_alpha * alpha; conductivity
 *       D = k (I + (aniso_k - 1) a a), a = F a0 / |F a0|; the H8 thermal
 *       hourglass keeps the transverse k.
 */
#include "tled_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define R_GAS 8.314
#define KELVIN 273.15

/* ------------------------------------------------------------------ */
/* small 3x3 helpers (row-major a[i][j])                               */
/* ------------------------------------------------------------------ */
static void m_zero(double a[3][3]) { memset(a, 0, 9 * sizeof(double)); }
static void m_eye(double a[3][3], double s) {
    m_zero(a);
    a[0][0] = a[1][1] = a[2][2] = s;
}
static void m_mul(const double a[3][3], const double b[3][3], double c[3][3]) {
    double r[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += a[i][k] * b[k][j];
            r[i][j] = s;
        }
    memcpy(c, r, sizeof(r));
}
static void m_transpose(const double a[3][3], double b[3][3]) {
    double r[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) r[i][j] = a[j][i];
    memcpy(b, r, sizeof(r));
}
static double m_det(const double a[3][3]) {
    return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
           a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
           a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}
static void m_inv(const double a[3][3], double b[3][3]) {
    double d = m_det(a);
    double r[3][3];
    r[0][0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) / d;
    r[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / d;
    r[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / d;
    r[1][0] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) / d;
    r[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / d;
    r[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / d;
    r[2][0] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) / d;
    r[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / d;
    r[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / d;
    memcpy(b, r, sizeof(r));
}
static double m_trace(const double a[3][3]) { return a[0][0] + a[1][1] + a[2][2]; }

/* symmetric storage order used for the Prony state */
static const int SYM_I[6] = {0, 1, 2, 0, 1, 0};
static const int SYM_J[6] = {0, 1, 2, 1, 2, 2};

/* ------------------------------------------------------------------ */
/* element shape functions                                             */
/* ------------------------------------------------------------------ */
/* H8 corner natural coordinates, VTK order. */
static const double H8_NAT[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                    {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
/* T4: N0 = 1 - xi - eta - zeta, N1 = xi, N2 = eta, N3 = zeta. */
static const double T4_DN[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

/* natural-coordinate derivatives dN_a/dxi at the single integration point */
static void natural_derivs(int npe, double dN[8][3]) {
    for (int a = 0; a < npe; a++)
        for (int k = 0; k < 3; k++)
            dN[a][k] = (npe == 8) ? H8_NAT[a][k] / 8.0 /* centroid of the trilinear brick */
                                  : T4_DN[a][k];
}

/* H8 hourglass base vectors h_alpha evaluated at the corners:
 * xi*eta, eta*zeta, xi*zeta, xi*eta*zeta. */
static double hg_base(int a, int alpha) {
    const double *c = H8_NAT[a];
    switch (alpha) {
        case 0: return c[0] * c[1];
        case 1: return c[1] * c[2];
        case 2: return c[0] * c[2];
        default: return c[0] * c[1] * c[2];
    }
}

int ora_setup(ora_model *m) {
    const int npe = m->npe;
    double dN[8][3];
    natural_derivs(npe, dN);
    memset(m->M, 0, m->nn * sizeof(double));
    memset(m->Cth, 0, m->nn * sizeof(double));
    memset(m->Vn, 0, m->nn * sizeof(double));
    for (int64_t e = 0; e < m->ne; e++) {
        const int32_t *cn = m->conn + e * npe;
        /* Jacobian J0_ij = sum_a X_ai dN_a/dxi_j */
        double J[3][3];
        m_zero(J);
        for (int a = 0; a < npe; a++)
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) J[i][j] += m->X[3 * (int64_t)cn[a] + i] * dN[a][j];
        double detJ = m_det(J);
        if (!(detJ > 0)) return -(int)(1 + e);
        double Ji[3][3];
        m_inv(J, Ji);
        /* dh_a/dX_j = sum_k dN_a/dxi_k (J0^-1)_kj */
        double *B = m->dhdX + e * npe * 3;
        for (int a = 0; a < npe; a++)
            for (int j = 0; j < 3; j++) {
                double s = 0;
                for (int k = 0; k < 3; k++) s += dN[a][k] * Ji[k][j];
                B[3 * a + j] = s;
            }
        /* element volume: 8 det J0 for one-point H8 (Eq. 18), det J0 / 6 for T4 */
        double V = (npe == 8) ? 8.0 * detJ : detJ / 6.0;
        m->V0[e] = V;
        /* R8: hourglass shape vectors gamma_a,alpha = h_a,alpha - (sum_b h_b,alpha X_b) . dh_a/dX */
        if (npe == 8) {
            double BB = 0;
            for (int a = 0; a < 8; a++)
                for (int j = 0; j < 3; j++) BB += B[3 * a + j] * B[3 * a + j];
            double *G = m->hg_gamma + e * 32;
            for (int al = 0; al < 4; al++) {
                double cx[3] = {0, 0, 0};
                for (int b = 0; b < 8; b++)
                    for (int j = 0; j < 3; j++) cx[j] += hg_base(b, al) * m->X[3 * (int64_t)cn[b] + j];
                for (int a = 0; a < 8; a++) {
                    double proj = 0;
                    for (int j = 0; j < 3; j++) proj += cx[j] * B[3 * a + j];
                    G[4 * a + al] = hg_base(a, al) - proj;
                }
            }
            double Pmod = m->kappa[e] + 4.0 * m->mu[e] / 3.0; /* P-wave modulus */
            m->khg[e] = m->kappa_hg * Pmod * V * BB / 8.0;
            m->khgT[e] = m->kappa_hgT * V * BB / 8.0;
        }
        /* R10: lumped masses, reference volumes split evenly over the corners */
        for (int a = 0; a < npe; a++) {
            int64_t i = cn[a];
            m->M[i] += m->mass_scale * m->rho[e] * V / npe;
            m->Cth[i] += m->rho[e] * m->c_heat * V / npe;
            m->Vn[i] += V / npe;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* constitutive law                                                    */
/* ------------------------------------------------------------------ */
/* Second Piola-Kirchhoff stress S_i = 2 dPsi/dC of the transversely isotropic
 * neo-Hookean law (Table 5) with the R7 fibre term, at the elastic
 * deformation gradient Fel (Eq. 9). */
static void pk2_stress(const double Fel[3][3], double mu, double kappa, double k1, double k2,
                       const double a[3], double S[3][3]) {
    double Ft[3][3], C[3][3], Ci[3][3];
    m_transpose(Fel, Ft);
    m_mul(Ft, Fel, C);
    m_inv(C, Ci);
    double J = m_det(Fel);
    double I1 = m_trace(C);
    double I4 = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) I4 += a[i] * C[i][j] * a[j];
    double J23 = pow(J, -2.0 / 3.0);
    double I4b = J23 * I4;
    double psi4p = k1 * (I4b - 1.0) * exp(k2 * (I4b - 1.0) * (I4b - 1.0)); /* dPsi_f/dI4b */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double d = (i == j) ? 1.0 : 0.0;
            S[i][j] = mu * J23 * (d - I1 / 3.0 * Ci[i][j])                 /* isochoric */
                      + kappa * J * (J - 1.0) * Ci[i][j]                    /* volumetric */
                      + 2.0 * psi4p * J23 * (a[i] * a[j] - I4 / 3.0 * Ci[i][j]); /* fibre */
        }
}

/* strain energy density Psi(Fel) of Table 5 with the R7 fibre term */
static double strain_energy(const double Fel[3][3], double mu, double kappa, double k1, double k2,
                            const double a[3]) {
    double Ft[3][3], C[3][3];
    m_transpose(Fel, Ft);
    m_mul(Ft, Fel, C);
    double J = m_det(Fel);
    double J23 = pow(J, -2.0 / 3.0);
    double I1b = J23 * m_trace(C);
    double I4 = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) I4 += a[i] * C[i][j] * a[j];
    double x = J23 * I4 - 1.0;
    double psif = (k2 > 0) ? k1 / (2.0 * k2) * (exp(k2 * x * x) - 1.0) : 0.5 * k1 * x * x;
    return 0.5 * mu * (I1b - 3.0) + 0.5 * kappa * (J - 1.0) * (J - 1.0) + psif;
}

/* ------------------------------------------------------------------ */
/* element kinematics shared by forces and energies                    */
/* ------------------------------------------------------------------ */
static void deformation_gradient(const ora_model *m, int64_t e, const double *u, double F[3][3]) {
    const int npe = m->npe;
    const int32_t *cn = m->conn + e * npe;
    const double *B = m->dhdX + e * npe * 3;
    /* Eq. (17): F = u_e^T dh/dX + I */
    m_eye(F, 1.0);
    for (int a = 0; a < npe; a++)
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) F[i][j] += u[3 * (int64_t)cn[a] + i] * B[3 * a + j];
}

static double element_temperature(const ora_model *m, int64_t e, const double *T) {
    const int32_t *cn = m->conn + e * m->npe;
    double s = 0;
    for (int a = 0; a < m->npe; a++) s += T[cn[a]];
    return s / m->npe; /* R3 */
}

/* isotropic thermal deformation gradient F_th = lambda I (Eq. 11, R4) */
/* Eq. (11): F_th = lambda_i I + (lambda_m - lambda_i) m (x) m, transversely
 * isotropic about m = a0 (R26), lambda = 1 + alpha (T_e - T0); isotropic when
 * the fibre expansion ratio is 1 */
static void thermal_gradient(const ora_model *m, int64_t e, double Te, double Fth[3][3]) {
    const double th = m->expansion ? Te - m->T0 : 0.0;
    const double li = 1.0 + m->alpha[e] * th, lm = 1.0 + m->aniso_alpha * m->alpha[e] * th;
    const double *a = m->a0 + 3 * e;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) Fth[i][j] = (i == j ? li : 0.0) + (lm - li) * a[i] * a[j];
}

/* spatial conductivity D = k (I + (r_k - 1) a (x) a), a = F a0 / |F a0| the
 * current fibre direction (R26); k = conductivity at T_e */
static void conductivity_tensor(const ora_model *m, int64_t e, const double F[3][3], double k, double D[3][3]) {
    const double *a0 = m->a0 + 3 * e;
    double a[3] = {0, 0, 0}, n = 0;
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) a[i] += F[i][j] * a0[j];
        n += a[i] * a[i];
    }
    n = sqrt(n);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) D[i][j] = k * ((i == j ? 1.0 : 0.0) + (m->aniso_k - 1.0) * a[i] * a[j] / (n * n));
}

static double conductivity(const ora_model *m, int64_t e, double Te) {
    return m->kc[e] * (m->temp_dep ? 1.0 + m->beta_k * (Te - m->T_ref) : 1.0); /* R11 */
}

double ora_element(const ora_model *m, int64_t e, const double *u, const double *T,
                   const double *visc_in, double *visc_out, double *f_e, double *fT_e) {
    const int npe = m->npe;
    const int32_t *cn = m->conn + e * npe;
    const double *B = m->dhdX + e * npe * 3;
    const double V = m->V0[e];
    double F[3][3];
    deformation_gradient(m, e, u, F);
    double Te = element_temperature(m, e, T);

    /* Eqs. (7)-(8): F_el = F F_th^-1 */
    double Fth[3][3], Fthi[3][3], Fthit[3][3], Fel[3][3];
    thermal_gradient(m, e, Te, Fth);
    m_inv(Fth, Fthi);
    m_transpose(Fthi, Fthit);
    m_mul(F, Fthi, Fel);

    /* Eq. (9): stress in the stress-free intermediate configuration */
    double Si[3][3];
    pk2_stress(Fel, m->mu[e], m->kappa[e], m->k1[e], m->k2[e], m->a0 + 3 * e, Si);

    /* Eq. (10): S0 = det(F_th) F_th^-1 S_i F_th^-T */
    double S0[3][3], tmp[3][3];
    m_mul(Fthi, Si, tmp);
    m_mul(tmp, Fthit, S0);
    double dFth = m_det(Fth);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) S0[i][j] *= dFth;

    /* Section 4.3 Prony recurrence (R6):
     * theta_i = dt phi_i/(dt+tau_i) S0 + tau_i/(dt+tau_i) theta_i(t-dt),
     * S~ = S0 - sum_i theta_i */
    double St[3][3];
    memcpy(St, S0, sizeof(St));
    for (int p = 0; p < m->n_prony; p++) {
        double dt = m->dt, tau = m->prony_tau[p];
        double ca = dt * m->prony_g[p] / (dt + tau), cb = tau / (dt + tau);
        for (int s = 0; s < 6; s++) {
            int i = SYM_I[s], j = SYM_J[s];
            double th = ca * S0[i][j] + cb * visc_in[6 * p + s];
            visc_out[6 * p + s] = th;
            St[i][j] -= th;
            if (i != j) St[j][i] -= th;
        }
    }

    /* Eqs. (24)-(28): f_a = V F S~ dh_a/dX */
    double P[3][3];
    m_mul(F, St, P);
    for (int a = 0; a < npe; a++)
        for (int i = 0; i < 3; i++) {
            double s = 0;
            for (int j = 0; j < 3; j++) s += P[i][j] * B[3 * a + j];
            f_e[3 * a + i] = V * s;
        }

    /* Eqs. (16), (18), (19): fT = V (B F^-1) D (B F^-1)^T det F T_e */
    double Fi[3][3];
    m_inv(F, Fi);
    double detF = m_det(F);
    double kT = conductivity(m, e, Te);
    double D[3][3];
    conductivity_tensor(m, e, F, kT, D);
    double G[8][3]; /* rows: spatial gradients of the shape functions, B F^-1 */
    for (int a = 0; a < npe; a++)
        for (int j = 0; j < 3; j++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += B[3 * a + k] * Fi[k][j];
            G[a][j] = s;
        }
    for (int a = 0; a < npe; a++) {
        double s = 0;
        for (int b = 0; b < npe; b++) {
            double Kab = 0;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) Kab += G[a][i] * D[i][j] * G[b][j];
            s += V * detF * Kab * T[cn[b]];
        }
        fT_e[a] = s;
    }

    /* R8: hourglass forces f_a += k_hg sum_alpha gamma_a,alpha (sum_b gamma_b,alpha u_b),
     * and the thermal analogue with conductance k(Te) khgT. */
    if (npe == 8) {
        const double *Gm = m->hg_gamma + e * 32;
        for (int al = 0; al < 4; al++) {
            double qu[3] = {0, 0, 0}, qT = 0;
            for (int b = 0; b < 8; b++) {
                for (int i = 0; i < 3; i++) qu[i] += Gm[4 * b + al] * u[3 * (int64_t)cn[b] + i];
                qT += Gm[4 * b + al] * T[cn[b]];
            }
            for (int a = 0; a < 8; a++) {
                for (int i = 0; i < 3; i++) f_e[3 * a + i] += m->khg[e] * Gm[4 * a + al] * qu[i];
                fT_e[a] += kT * m->khgT[e] * Gm[4 * a + al] * qT;
            }
        }
    }
    return detF;
}

double ora_element_energy(const ora_model *m, int64_t e, const double *u, const double *T) {
    double F[3][3], Fth[3][3], Fthi[3][3], Fel[3][3];
    deformation_gradient(m, e, u, F);
    double Te = element_temperature(m, e, T);
    thermal_gradient(m, e, Te, Fth);
    m_inv(Fth, Fthi);
    m_mul(F, Fthi, Fel);
    /* energy per reference volume of the thermally expanded element: det(F_th) Psi(F_el) */
    double W = m->V0[e] * m_det(Fth) *
               strain_energy(Fel, m->mu[e], m->kappa[e], m->k1[e], m->k2[e], m->a0 + 3 * e);
    if (m->npe == 8) {
        const int32_t *cn = m->conn + e * 8;
        const double *Gm = m->hg_gamma + e * 32;
        for (int al = 0; al < 4; al++)
            for (int i = 0; i < 3; i++) {
                double q = 0;
                for (int b = 0; b < 8; b++) q += Gm[4 * b + al] * u[3 * (int64_t)cn[b] + i];
                W += 0.5 * m->khg[e] * q * q;
            }
    }
    return W;
}

double ora_element_thermal_energy(const ora_model *m, int64_t e, const double *u, const double *T,
                                  double Tk_fixed) {
    const int npe = m->npe;
    const int32_t *cn = m->conn + e * npe;
    const double *B = m->dhdX + e * npe * 3;
    double F[3][3], Fi[3][3], D[3][3];
    deformation_gradient(m, e, u, F);
    m_inv(F, Fi);
    double J = m_det(F);
    double kT = conductivity(m, e, Tk_fixed);
    conductivity_tensor(m, e, F, kT, D);
    double g[3] = {0, 0, 0}, h[3] = {0, 0, 0};
    for (int a = 0; a < npe; a++)
        for (int j = 0; j < 3; j++) g[j] += T[cn[a]] * B[3 * a + j];
    for (int i = 0; i < 3; i++) /* spatial gradient F^-T grad0 T */
        for (int j = 0; j < 3; j++) h[i] += Fi[j][i] * g[j];
    double q = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) q += h[i] * D[i][j] * h[j];
    double W = 0.5 * m->V0[e] * J * q;
    if (npe == 8) {
        const double *Gm = m->hg_gamma + e * 32;
        for (int al = 0; al < 4; al++) {
            double qT = 0;
            for (int b = 0; b < 8; b++) qT += Gm[4 * b + al] * T[cn[b]];
            W += 0.5 * kT * m->khgT[e] * qT * qT;
        }
    }
    return W;
}

/* ------------------------------------------------------------------ */
/* nodal updates                                                       */
/* ------------------------------------------------------------------ */
static double ramp(const ora_model *m, double t) {
    if (m->ramp_time <= 0) return 1.0;
    return t >= m->ramp_time ? 1.0 : t / m->ramp_time;
}

/* regional heat source Q_r at node i (R14), W/m^3: a Gaussian of standard
 * deviation sigma, or (the paper's liver case) a uniform sphere of that radius */
static double heat_source(const ora_model *m, int64_t i, const double *u, double t) {
    double q = 0;
    for (int s = 0; s < m->n_src; s++) {
        const double *p = m->src + 11 * s;
        if (t < p[8] || t >= p[9]) continue;
        double r2 = 0;
        for (int j = 0; j < 3; j++) {
            double x = m->X[3 * i + j] + u[3 * i + j];
            double c = p[j] + p[3 + j] * t;
            r2 += (x - c) * (x - c);
        }
        if (p[10] == 1.0)
            q += r2 <= p[6] * p[6] ? p[7] : 0.0;
        else
            q += p[7] * exp(-r2 / (2.0 * p[6] * p[6]));
    }
    return q;
}

/* CEM43 rate, equivalent minutes per second at temperature T (C):
 * R^(43 - T) / 60 with R = 0.5 at or above 43 C and 0.25 below */
static double cem43_rate(double T) {
    const double R = T >= 43.0 ? 0.5 : 0.25;
    return pow(R, 43.0 - T) / 60.0;
}

/* Eqs. (27), (20) and the Arrhenius integral for one node. */
static void node_update(const ora_model *m, const ora_state *s, int64_t i, const double *f,
                        double fT, double *u_new, double *T_new, double *O_new) {
    const double dt = m->dt, t = s->t;
    /* Eq. (27): central difference with D = gamma M, R = 0 (no applied loads) */
    for (int d = 0; d < 3; d++) {
        if (m->mask[i] & (1u << d)) {
            u_new[d] = (m->ubar ? m->ubar[3 * i + d] : 0.0) * ramp(m, t + dt);
            continue;
        }
        double M = m->M[i], D = m->gamma * m->M[i], R = 0.0;
        double num = R - f[d] + 2.0 * M / (dt * dt) * s->u[3 * i + d] +
                     (D / (2.0 * dt) - M / (dt * dt)) * s->u_prev[3 * i + d];
        u_new[d] = num / (D / (2.0 * dt) + M / (dt * dt));
    }
    /* Eq. (20) with the physical conduction sign (R1) */
    double T = s->T[i];
    if (m->mask[i] & 8u) {
        *T_new = T;
    } else {
        double C = m->Cth[i] * (m->temp_dep ? 1.0 + m->beta_c * (T - m->T_ref) : 1.0);
        double Kb = m->wbcb * m->Vn[i];
        double Qb = Kb * m->Ta;
        double Qm = m->Qm * m->Vn[i];
        double Qr = m->Vn[i] * heat_source(m, i, s->u, t);
        *T_new = T + dt / C * (-fT - Kb * T + Qb + Qm + Qr);
    }
    /* Arrhenius damage integral, explicit in T(t) (R18) */
    *O_new = s->Omega[i] + dt * exp(m->lnA) * exp(-m->Ea / (R_GAS * (T + KELVIN)));
}

int ora_step(const ora_model *m, ora_state *s, double *f, double *fT) {
    const int npe = m->npe;
    memset(f, 0, 3 * m->nn * sizeof(double));
    memset(fT, 0, m->nn * sizeof(double));
    double fe[24], fTe[8];
    /* element loop, assembled by plain summation in element-id order (Eqs. 14, 23) */
    for (int64_t e = 0; e < m->ne; e++) {
        double *vs = m->n_prony ? s->visc + e * m->n_prony * 6 : NULL;
        ora_element(m, e, s->u, s->T, vs, vs, fe, fTe);
        const int32_t *cn = m->conn + e * npe;
        for (int a = 0; a < npe; a++) {
            for (int i = 0; i < 3; i++) f[3 * (int64_t)cn[a] + i] += fe[3 * a + i];
            fT[cn[a]] += fTe[a];
        }
    }
    /* node loop: every node independent (Section 4.1) */
    for (int64_t i = 0; i < m->nn; i++) {
        double un[3], Tn, On;
        node_update(m, s, i, f + 3 * i, fT[i], un, &Tn, &On);
        if (s->cem) s->cem[i] += m->dt * cem43_rate(s->T[i]);  /* explicit in T(t), like the damage */
        for (int d = 0; d < 3; d++) {
            s->u_prev[3 * i + d] = s->u[3 * i + d];
            s->u[3 * i + d] = un[d];
        }
        s->T[i] = Tn;
        s->Omega[i] = On;
    }
    s->t += m->dt;
    s->step += 1;
    return 0;
}

int ora_step_nodes(const ora_model *m, const ora_state *s, const int64_t *nodes, int64_t k,
                   double *out_u, double *out_T, double *out_O) {
    const int npe = m->npe;
    int64_t *slot = (int64_t *)malloc(m->nn * sizeof(int64_t));
    double *acc = (double *)calloc(4 * k, sizeof(double));
    if (!slot || !acc) {
        free(slot);
        free(acc);
        return -1;
    }
    for (int64_t i = 0; i < m->nn; i++) slot[i] = -1;
    for (int64_t q = 0; q < k; q++) slot[nodes[q]] = q;
    double fe[24], fTe[8], vtmp[6 * ORA_MAX_PRONY];
    for (int64_t e = 0; e < m->ne; e++) {
        const int32_t *cn = m->conn + e * npe;
        int touches = 0;
        for (int a = 0; a < npe; a++) touches |= slot[cn[a]] >= 0;
        if (!touches) continue;
        const double *vs = m->n_prony ? s->visc + e * m->n_prony * 6 : vtmp;
        ora_element(m, e, s->u, s->T, vs, vtmp, fe, fTe);
        for (int a = 0; a < npe; a++) {
            int64_t q = slot[cn[a]];
            if (q < 0) continue;
            for (int i = 0; i < 3; i++) acc[4 * q + i] += fe[3 * a + i];
            acc[4 * q + 3] += fTe[a];
        }
    }
    for (int64_t q = 0; q < k; q++)
        node_update(m, s, nodes[q], acc + 4 * q, acc[4 * q + 3], out_u + 3 * q, out_T + q, out_O + q);
    free(slot);
    free(acc);
    return 0;
}

/* ------------------------------------------------------------------ */
/* critical time step (R16)                                            */
/* ------------------------------------------------------------------ */
static double quad_area(const double *p0, const double *p1, const double *p2, const double *p3) {
    double d1[3], d2[3], c[3];
    for (int j = 0; j < 3; j++) {
        d1[j] = p2[j] - p0[j];
        d2[j] = p3[j] - p1[j];
    }
    c[0] = d1[1] * d2[2] - d1[2] * d2[1];
    c[1] = d1[2] * d2[0] - d1[0] * d2[2];
    c[2] = d1[0] * d2[1] - d1[1] * d2[0];
    return 0.5 * sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
}
static double tri_area(const double *p0, const double *p1, const double *p2) {
    double d1[3], d2[3], c[3];
    for (int j = 0; j < 3; j++) {
        d1[j] = p1[j] - p0[j];
        d2[j] = p2[j] - p0[j];
    }
    c[0] = d1[1] * d2[2] - d1[2] * d2[1];
    c[1] = d1[2] * d2[0] - d1[0] * d2[2];
    c[2] = d1[0] * d2[1] - d1[1] * d2[0];
    return 0.5 * sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
}

double ora_stable_dt(const ora_model *m, double safety, double *dt_mech, double *dt_th) {
    static const int HF[6][4] = {{0, 1, 2, 3}, {4, 5, 6, 7}, {0, 1, 5, 4},
                                 {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}};
    static const int TF[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
    const int npe = m->npe;
    double kfac = m->temp_dep ? fmax(1.0, 1.0 + m->beta_k * (90.0 - m->T_ref)) : 1.0;
    double cfac = m->temp_dep ? fmin(1.0, 1.0 + m->beta_c * (90.0 - m->T_ref)) : 1.0;
    double dtm = INFINITY;
    double *row = (double *)calloc(m->nn, sizeof(double));
    for (int64_t e = 0; e < m->ne; e++) {
        const int32_t *cn = m->conn + e * npe;
        const double *p[8];
        for (int a = 0; a < npe; a++) p[a] = m->X + 3 * (int64_t)cn[a];
        double Amax = 0;
        if (npe == 8)
            for (int f = 0; f < 6; f++)
                Amax = fmax(Amax, quad_area(p[HF[f][0]], p[HF[f][1]], p[HF[f][2]], p[HF[f][3]]));
        else
            for (int f = 0; f < 4; f++) Amax = fmax(Amax, tri_area(p[TF[f][0]], p[TF[f][1]], p[TF[f][2]]));
        double L = (npe == 8 ? 1.0 : 3.0) * m->V0[e] / Amax; /* hex V/A_max, tet min altitude */
        double cd = sqrt((m->kappa[e] + 4.0 * m->mu[e] / 3.0 + 4.0 * m->k1[e]) / (m->rho[e] * m->mass_scale));
        dtm = fmin(dtm, L / cd);
        /* element conduction matrix at F = I and k_max; absolute row sums */
        const double *B = m->dhdX + e * npe * 3;
        double kmax = m->kc[e] * kfac;
        for (int a = 0; a < npe; a++) {
            double rs = 0;
            for (int b = 0; b < npe; b++) {
                /* grad h_a . D grad h_b with D = k_max (I + (r_k - 1) a0 a0) at F = I */
                double K = 0, ma = 0, mb = 0;
                for (int j = 0; j < 3; j++) {
                    K += B[3 * a + j] * B[3 * b + j];
                    ma += B[3 * a + j] * m->a0[3 * e + j];
                    mb += B[3 * b + j] * m->a0[3 * e + j];
                }
                K = (K + (m->aniso_k - 1.0) * ma * mb) * m->V0[e] * kmax;
                if (npe == 8) {
                    const double *Gm = m->hg_gamma + e * 32;
                    double Kh = 0;
                    for (int al = 0; al < 4; al++) Kh += Gm[4 * a + al] * Gm[4 * b + al];
                    K += kmax * m->khgT[e] * Kh;
                }
                rs += fabs(K);
            }
            row[cn[a]] += rs;
        }
    }
    double dtt = INFINITY;
    for (int64_t i = 0; i < m->nn; i++) {
        double r = row[i] + m->wbcb * m->Vn[i];
        if (r > 0) dtt = fmin(dtt, 2.0 * m->Cth[i] * cfac / r);
    }
    free(row);
    if (dt_mech) *dt_mech = dtm;
    if (dt_th) *dt_th = dtt;
    return safety * fmin(dtm, dtt);
}

/* ------------------------------------------------------------------ */
/* point probes: temperature and damage fraction at arbitrary points   */
/* ------------------------------------------------------------------ */
/* Shape functions N_a at natural coordinates xi: T4 barycentric (N0 = 1 - xi - eta
 * - zeta, N1 = xi, N2 = eta, N3 = zeta), H8 trilinear (1/8) prod_j (1 + s_aj xi_j)
 * -- the interpolation behind Eqs. (18)-(19). */
static void shape_values(int npe, const double xi[3], double N[8]) {
    if (npe == 4) {
        N[0] = 1.0 - xi[0] - xi[1] - xi[2];
        N[1] = xi[0];
        N[2] = xi[1];
        N[3] = xi[2];
        return;
    }
    for (int a = 0; a < 8; a++)
        N[a] = (1.0 + H8_NAT[a][0] * xi[0]) * (1.0 + H8_NAT[a][1] * xi[1]) * (1.0 + H8_NAT[a][2] * xi[2]) / 8.0;
}

/* Natural coordinates of point x in element e, if it lies in the element.
 * T4: the map is affine, solved once.  H8: Newton iteration on the trilinear
 * isoparametric map x(xi) = sum_a N_a(xi) X_a from the centroid.  Returns 1 if
 * the point is inside (tolerance 1e-9 in natural coordinates). */
static int point_in_element(const ora_model *m, int64_t e, const double x[3], double xi[3]) {
    const int npe = m->npe;
    const int32_t *cn = m->conn + e * npe;
    const double *P[8];
    for (int a = 0; a < npe; a++) P[a] = m->X + 3 * (int64_t)cn[a];
    /* quick reject: outside the element's bounding box (with a margin) */
    for (int j = 0; j < 3; j++) {
        double lo = P[0][j], hi = P[0][j];
        for (int a = 1; a < npe; a++) {
            lo = fmin(lo, P[a][j]);
            hi = fmax(hi, P[a][j]);
        }
        double pad = 1e-9 * (hi - lo);
        if (x[j] < lo - pad || x[j] > hi + pad) return 0;
    }
    if (npe == 4) {
        double J[3][3], Ji[3][3];
        for (int i = 0; i < 3; i++)
            for (int k = 0; k < 3; k++) J[i][k] = P[k + 1][i] - P[0][i];
        if (m_det(J) == 0.0) return 0;
        m_inv(J, Ji);
        for (int k = 0; k < 3; k++) {
            xi[k] = 0;
            for (int i = 0; i < 3; i++) xi[k] += Ji[k][i] * (x[i] - P[0][i]);
        }
        const double tol = 1e-9;
        return xi[0] >= -tol && xi[1] >= -tol && xi[2] >= -tol && xi[0] + xi[1] + xi[2] <= 1.0 + tol;
    }
    xi[0] = xi[1] = xi[2] = 0.0;
    for (int it = 0; it < 60; it++) {
        double N[8], r[3], J[3][3], Ji[3][3];
        shape_values(8, xi, N);
        m_zero(J);
        for (int i = 0; i < 3; i++) r[i] = -x[i];
        for (int a = 0; a < 8; a++) {
            double dN[3];
            for (int k = 0; k < 3; k++) {
                dN[k] = H8_NAT[a][k] / 8.0;
                for (int l = 0; l < 3; l++)
                    if (l != k) dN[k] *= 1.0 + H8_NAT[a][l] * xi[l];
            }
            for (int i = 0; i < 3; i++) {
                r[i] += N[a] * P[a][i];
                for (int k = 0; k < 3; k++) J[i][k] += P[a][i] * dN[k];
            }
        }
        if (!(m_det(J) > 0)) return 0;
        m_inv(J, Ji);
        double step = 0;
        for (int k = 0; k < 3; k++) {
            double d = 0;
            for (int i = 0; i < 3; i++) d += Ji[k][i] * r[i];
            xi[k] -= d;
            step += fabs(d);
        }
        if (fabs(xi[0]) > 4 || fabs(xi[1]) > 4 || fabs(xi[2]) > 4) return 0;
        if (step < 1e-15) break;
    }
    const double tol = 1e-9;
    return fabs(xi[0]) <= 1 + tol && fabs(xi[1]) <= 1 + tol && fabs(xi[2]) <= 1 + tol;
}

int ora_probe(const ora_model *m, const ora_state *s, const double *xyz, int64_t k, double *T_out,
              double *d_out) {
    const int npe = m->npe;
    for (int64_t q = 0; q < k; q++) {
        int64_t found = -1;
        double xi[3];
        for (int64_t e = 0; e < m->ne && found < 0; e++)
            if (point_in_element(m, e, xyz + 3 * q, xi)) found = e;
        if (found < 0) return -(int)(1 + q);
        double N[8];
        shape_values(npe, xi, N);
        const int32_t *cn = m->conn + found * npe;
        double T = 0, d = 0;
        for (int a = 0; a < npe; a++) {
            T += N[a] * s->T[cn[a]];
            d += N[a] * (1.0 - exp(-s->Omega[cn[a]])); /* nodal damage fraction, interpolated */
        }
        T_out[q] = T;
        d_out[q] = d;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* the same step on all host cores                                     */
/* ------------------------------------------------------------------ */
int ora_incidence(const ora_model *m, int64_t *offsets, int64_t *slots) {
    const int npe = m->npe;
    memset(offsets, 0, (m->nn + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < m->ne; e++)
        for (int a = 0; a < npe; a++) offsets[m->conn[e * npe + a] + 1]++;
    for (int64_t i = 0; i < m->nn; i++) offsets[i + 1] += offsets[i];
    int64_t *fill = (int64_t *)malloc(m->nn * sizeof(int64_t));
    if (!fill) return -1;
    memcpy(fill, offsets, m->nn * sizeof(int64_t));
    for (int64_t e = 0; e < m->ne; e++) /* ascending element id within every node's list */
        for (int a = 0; a < npe; a++) slots[fill[m->conn[e * npe + a]]++] = e * npe + a;
    free(fill);
    return 0;
}

int ora_step_parallel(const ora_model *m, ora_state *s, const int64_t *offsets, const int64_t *slots,
                      double *elem_out, double *f, double *fT) {
    const int npe = m->npe;
    const int64_t ne = m->ne, nn = m->nn;
    /* element loop: every element independent; results kept per (element, corner) */
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; e++) {
        double fe[24], fTe[8];
        double *vs = m->n_prony ? s->visc + e * m->n_prony * 6 : NULL;
        ora_element(m, e, s->u, s->T, vs, vs, fe, fTe);
        for (int a = 0; a < npe; a++) {
            double *o = elem_out + 4 * (e * npe + a);
            o[0] = fe[3 * a];
            o[1] = fe[3 * a + 1];
            o[2] = fe[3 * a + 2];
            o[3] = fTe[a];
        }
    }
    /* node gather in ascending element order from zero: the additions of
     * ora_step's element-order assembly, in the same order */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nn; i++) {
        double acc[4] = {0, 0, 0, 0};
        for (int64_t r = offsets[i]; r < offsets[i + 1]; r++) {
            const double *o = elem_out + 4 * slots[r];
            for (int d = 0; d < 4; d++) acc[d] += o[d];
        }
        f[3 * i] = acc[0];
        f[3 * i + 1] = acc[1];
        f[3 * i + 2] = acc[2];
        fT[i] = acc[3];
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nn; i++) {
        double un[3], Tn, On;
        node_update(m, s, i, f + 3 * i, fT[i], un, &Tn, &On);
        if (s->cem) s->cem[i] += m->dt * cem43_rate(s->T[i]);
        for (int d = 0; d < 3; d++) {
            s->u_prev[3 * i + d] = s->u[3 * i + d];
            s->u[3 * i + d] = un[d];
        }
        s->T[i] = Tn;
        s->Omega[i] = On;
    }
    s->t += m->dt;
    s->step += 1;
    return 0;
}

int ora_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* mechanical subcycling: n_sub mechanical substeps per thermal step   */
/* ------------------------------------------------------------------ */
int ora_step_subcycled(const ora_model *m, ora_state *s, int n_sub, double *f, double *fT) {
    const int npe = m->npe;
    /* the mechanical substep: the Prony recurrence and Eq. (27) with dt / n_sub */
    ora_model mm = *m;
    mm.dt = m->dt / n_sub;
    /* the thermal step starts here: the temperature is held at T(t_th) during the
     * substeps and advances once, explicit in T(t_th), with the sources at t_th */
    const double t_th = s->t;
    double fe[24], fTe[8];
    for (int j = 0; j < n_sub; j++) {
        memset(f, 0, 3 * m->nn * sizeof(double));
        memset(fT, 0, m->nn * sizeof(double));
        for (int64_t e = 0; e < m->ne; e++) {
            double *vs = m->n_prony ? s->visc + e * m->n_prony * 6 : NULL;
            ora_element(&mm, e, s->u, s->T, vs, vs, fe, fTe);
            const int32_t *cn = m->conn + e * npe;
            for (int a = 0; a < npe; a++) {
                for (int i = 0; i < 3; i++) f[3 * (int64_t)cn[a] + i] += fe[3 * a + i];
                fT[cn[a]] += fTe[a];
            }
        }
        const int thermal = j == n_sub - 1; /* the last substep also advances T and the damage */
        ora_state st = *s;
        st.t = t_th;
        for (int64_t i = 0; i < m->nn; i++) {
            double un[3], Tn, On, u_th[3], T_th, O_th;
            node_update(&mm, s, i, f + 3 * i, fT[i], un, &Tn, &On); /* u over the substep */
            if (thermal) {
                /* T and Omega over the whole thermal step, with this substep's thermal loads
                 * (current displacement, T(t_th)) and the sources at t_th */
                node_update(m, &st, i, f + 3 * i, fT[i], u_th, &T_th, &O_th);
                if (s->cem) s->cem[i] += m->dt * cem43_rate(s->T[i]);
                s->T[i] = T_th;
                s->Omega[i] = O_th;
            }
            for (int d = 0; d < 3; d++) {
                s->u_prev[3 * i + d] = s->u[3 * i + d];
                s->u[3 * i + d] = un[d];
            }
        }
        s->t += mm.dt;
        s->step += 1;
    }
    return 0;
}
