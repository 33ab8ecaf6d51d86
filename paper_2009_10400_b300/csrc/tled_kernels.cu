// Device kernels of libtled (sm_103a): one explicit coupled TLED step.
//
// Step = tile kernel + shared-node kernel.
//  * tile kernel, one CTA per tile of Morton-ordered elements:
//      1. gather (u, theta, X0) of the tile's nodes into shared memory,
//      2. per element (one thread each): deformation gradient (Eq. 17),
//         thermal split (Eqs. 7-11), transversely isotropic neo-Hookean stress
//         (Table 5, Eq. 9), pull-back (Eq. 10), Prony recurrence (Section 4.3),
//         nodal forces (Eqs. 24-28) + hourglass control, deformed-configuration
//         thermal loads (Eqs. 16-19); contributions go to per-corner slots in
//         shared memory,
//      3. node-centric gather of the slots in a fixed order (no float atomics),
//         then, for the tile's interior nodes, the central-difference
//         displacement update (Eq. 27), the explicit bioheat update (Eq. 20)
//         and the Arrhenius damage update; boundary nodes of the tile store
//         their partial sums instead.
//  * shared-node kernel: each node touched by several tiles sums its partials
//    in tile order and applies the same nodal update.
//
// Floating point: FP32 throughout; kinematics are written in H = du/dX so
// that J - 1, E and I4b - 1 never cancel; nodal u and theta accumulate in
// float-float (TwoSum) pairs; theta is stored relative to T0.
#include <cstdint>

#include "tled_internal.h"

namespace tled {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
// VTK hexahedron corner signs (xi, eta, zeta) and hourglass base vectors.
__device__ __forceinline__ constexpr float sgn_xi(int a) { return (a == 1 || a == 2 || a == 5 || a == 6) ? 1.f : -1.f; }
__device__ __forceinline__ constexpr float sgn_eta(int a) { return (a == 2 || a == 3 || a == 6 || a == 7) ? 1.f : -1.f; }
__device__ __forceinline__ constexpr float sgn_zeta(int a) { return a >= 4 ? 1.f : -1.f; }
__device__ __forceinline__ constexpr float sgn(int a, int j) {
    return j == 0 ? sgn_xi(a) : j == 1 ? sgn_eta(a) : sgn_zeta(a);
}
__device__ __forceinline__ constexpr float hgv(int a, int al) {
    return al == 0 ? sgn_xi(a) * sgn_eta(a)
         : al == 1 ? sgn_eta(a) * sgn_zeta(a)
         : al == 2 ? sgn_xi(a) * sgn_zeta(a)
                   : sgn_xi(a) * sgn_eta(a) * sgn_zeta(a);
}

// hi + lo += d, keeping hi the nearest float of the pair (TwoSum, then
// FastTwoSum renormalisation); explicit _rn intrinsics forbid FMA contraction.
__device__ __forceinline__ void add_ff(float &hi, float &lo, float d) {
    float s = __fadd_rn(hi, d);
    float bb = __fsub_rn(s, hi);
    float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(d, bb));
    float l = __fadd_rn(lo, err);
    float h2 = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(h2, s));
    hi = h2;
}

struct SrcSmem {
    float cx[kMaxSources], cy[kMaxSources], cz[kMaxSources], inv2s2[kMaxSources], P[kMaxSources];
    double t;
    int n;
};

// Source centres c(t) = c0 + vel t at this step's time, once per CTA.
__device__ __forceinline__ void prepare_sources(const StepArgs &A, int k, SrcSmem &S) {
    if (threadIdx.x == 0) {
        S.t = *A.time_base + (double)k * A.dt;
        S.n = *A.n_src;
    }
    __syncthreads();
    const int s = threadIdx.x;
    if (s < S.n) {
        const double *p = A.src + 10 * s;
        const double t = S.t;
        S.cx[s] = (float)(p[0] + p[3] * t);
        S.cy[s] = (float)(p[1] + p[4] * t);
        S.cz[s] = (float)(p[2] + p[5] * t);
        S.inv2s2[s] = (float)(0.5 / (p[6] * p[6]));
        S.P[s] = (t >= p[8] && t < p[9]) ? (float)p[7] : 0.f;
    }
}

// ---------------------------------------------------------------------------
// nodal update: Eq. (27) in velocity form, Eq. (20), Arrhenius
// ---------------------------------------------------------------------------
__device__ __forceinline__ void node_update(const StepArgs &A, int64_t g, float4 f, float4 xu, float4 X,
                                            const SrcSmem &S) {
    const float4 lo = A.lo[g];
    const float4 vo = A.vel[g];
    const float4 nc = __ldg(&A.nodec[g]);
    const unsigned mask = __float_as_uint(nc.z);
    const bool comp = (A.flags & TLED_COMPENSATED) != 0;
    const float dt = A.dtf;
    // current position for the heat source (state at t)
    const float px = X.x + (xu.x + lo.x), py = X.y + (xu.y + lo.y), pz = X.z + (xu.z + lo.z);

    float u[3] = {xu.x, xu.y, xu.z}, ul[3] = {lo.x, lo.y, lo.z}, v[3] = {vo.x, vo.y, vo.z};
    const float fv[3] = {f.x, f.y, f.z};
    const float im = 1.f / nc.x;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (mask & (1u << d)) {
            // prescribed: u(t+dt) = ubar * ramp(t+dt), v consistent with it
            float target = 0.f;
            if (A.ubar) {
                const double tn = S.t + A.dt;
                const double r = (A.ramp_time > 0.0 && tn < A.ramp_time) ? tn / A.ramp_time : 1.0;
                const float4 ub = __ldg(&A.ubar[g]);
                target = (float)((d == 0 ? ub.x : d == 1 ? ub.y : ub.z) * r);
            }
            v[d] = (target - u[d] - ul[d]) / dt;
            u[d] = target;
            ul[d] = 0.f;
        } else {
            // v+ = [(1 - g dt/2) v + dt (R - f)/m] / (1 + g dt/2), R = 0; u+ = u + dt v+
            v[d] = A.damp_a * v[d] - A.damp_b * fv[d] * im;
            if (comp)
                add_ff(u[d], ul[d], dt * v[d]);
            else
                u[d] += dt * v[d];
        }
    }
    // Eq. (20), physical conduction sign: C dtheta/dt = -fT - wbcb V (theta - theta_a) + V (Qm + Qr)
    float th = xu.w, tl = lo.w;
    const float theta = th + tl;
    float C = nc.y;
    if (A.flags & TLED_TEMP_DEP) C *= 1.f + A.beta_c * (theta - A.Tref_m_T0);
    float Q = A.Qm;
    for (int s = 0; s < S.n; s++) {
        const float dx = px - S.cx[s], dy = py - S.cy[s], dz = pz - S.cz[s];
        Q += S.P[s] * __expf(-(dx * dx + dy * dy + dz * dz) * S.inv2s2[s]);
    }
    if (!(mask & TLED_FIX_T)) {
        const float dth = dt / C * (-f.w + X.w * (Q - A.wbcb * (theta - A.theta_a)));
        if (comp)
            add_ff(th, tl, dth);
        else
            th += dth;
    }
    // Arrhenius damage integral, explicit in T(t); exp(ln A - Ea/(R T)) avoids A > FLT_MAX
    const float Om = vo.w + dt * expf(A.lnA - A.Ea_R / (theta + A.T0_K));
    if (!(isfinite(th) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]))) {
        atomicOr(A.status, kStatusNaN);
        atomicMin(A.status + 2, (unsigned)g);
    }
    A.xu[g] = make_float4(u[0], u[1], u[2], th);
    A.lo[g] = make_float4(ul[0], ul[1], ul[2], tl);
    A.vel[g] = make_float4(v[0], v[1], v[2], Om);
}

// ---------------------------------------------------------------------------
// element pass
// ---------------------------------------------------------------------------
template <int NPE>
__device__ __forceinline__ void element_step(const StepArgs &A, int64_t e, int el, const float4 *__restrict__ s_xu,
                                             const float4 *__restrict__ s_X, float4 *__restrict__ s_slot) {
    const int64_t ne = A.ne;
    // ---- loads: connectivity, reference geometry, material, Prony state
    int cl[NPE];
    if constexpr (NPE == 8) {
        const uint4 c = __ldg(reinterpret_cast<const uint4 *>(A.conn_local) + e);
        cl[0] = c.x & 0xffff; cl[1] = c.x >> 16; cl[2] = c.y & 0xffff; cl[3] = c.y >> 16;
        cl[4] = c.z & 0xffff; cl[5] = c.z >> 16; cl[6] = c.w & 0xffff; cl[7] = c.w >> 16;
    } else {
        const uint2 c = __ldg(reinterpret_cast<const uint2 *>(A.conn_local) + e);
        cl[0] = c.x & 0xffff; cl[1] = c.x >> 16; cl[2] = c.y & 0xffff; cl[3] = c.y >> 16;
    }
    float Ji[9];
#pragma unroll
    for (int q = 0; q < 9; q++) Ji[q] = __ldg(A.jinv + q * ne + e);
    const float V = __ldg(A.V0 + e);
    float mu = A.mu, kap = A.kappa, k1 = A.k1, k2 = A.k2, kc = A.kc, al = A.alpha;
    if (A.mat) {
        mu = __ldg(A.mat + e);
        kap = __ldg(A.mat + ne + e);
        k1 = __ldg(A.mat + 2 * ne + e);
        k2 = __ldg(A.mat + 3 * ne + e);
        kc = __ldg(A.mat + 4 * ne + e);
        al = __ldg(A.mat + 5 * ne + e);
    }
    float ax = A.a0x, ay = A.a0y, az = A.a0z;
    if (A.fib) {
        ax = __ldg(A.fib + e);
        ay = __ldg(A.fib + ne + e);
        az = __ldg(A.fib + 2 * ne + e);
    }
    float vs[4][6];
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
        for (int s = 0; s < 6; s++) vs[p][s] = (p < A.n_prony) ? A.visc[(int64_t)(p * 6 + s) * ne + e] : 0.f;

    // ---- gather nodal displacement and temperature rise from shared memory
    float ux[NPE], uy[NPE], uz[NPE], th[NPE];
#pragma unroll
    for (int a = 0; a < NPE; a++) {
        const float4 q = s_xu[cl[a]];
        ux[a] = q.x; uy[a] = q.y; uz[a] = q.z; th[a] = q.w;
    }
    // ---- Eq. (17) without forming I + H: H = sum_a u_a (x) dh_a/dX with
    //      dh/dX = s * Xi * J0^-1 (Xi: corner signs for H8 with s = 1/8; T4 derivative table)
    float G[3][3], gt[3];
    if constexpr (NPE == 8) {
#pragma unroll
        for (int j = 0; j < 3; j++) {
            float gx = 0.f, gy = 0.f, gz = 0.f, gT = 0.f;
#pragma unroll
            for (int a = 0; a < 8; a++) {
                gx += sgn(a, j) * ux[a]; gy += sgn(a, j) * uy[a]; gz += sgn(a, j) * uz[a]; gT += sgn(a, j) * th[a];
            }
            G[0][j] = gx; G[1][j] = gy; G[2][j] = gz; gt[j] = gT;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 3; j++) {
            G[0][j] = ux[j + 1] - ux[0]; G[1][j] = uy[j + 1] - uy[0]; G[2][j] = uz[j + 1] - uz[0];
            gt[j] = th[j + 1] - th[0];
        }
    }
    constexpr float sc = NPE == 8 ? 0.125f : 1.f;
    float H[3][3], gth[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
#pragma unroll
        for (int i = 0; i < 3; i++) H[i][j] = sc * (G[i][0] * Ji[j] + G[i][1] * Ji[3 + j] + G[i][2] * Ji[6 + j]);
        gth[j] = sc * (gt[0] * Ji[j] + gt[1] * Ji[3 + j] + gt[2] * Ji[6 + j]);
    }
    float the = 0.f;
#pragma unroll
    for (int a = 0; a < NPE; a++) the += th[a];
    the *= 1.f / NPE;

    // ---- thermal split (Eqs. 7-11, isotropic): lambda = 1 + delta, delta = alpha theta_e
    const float dl = (A.flags & TLED_EXPANSION) ? al * the : 0.f;
    const float lam = 1.f + dl;
    // J - 1 = tr H + [(tr H)^2 - tr(H^2)]/2 + det H
    const float trH = H[0][0] + H[1][1] + H[2][2];
    const float trH2 = H[0][0] * H[0][0] + H[1][1] * H[1][1] + H[2][2] * H[2][2] +
                       2.f * (H[0][1] * H[1][0] + H[0][2] * H[2][0] + H[1][2] * H[2][1]);
    const float detH = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) -
                       H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
                       H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
    const float Jm1 = trH + 0.5f * (trH * trH - trH2) + detH;
    // Green-Lagrange E = (H + H^T + H^T H)/2, then E_el = (E - (delta + delta^2/2) I) / lambda^2
    float E[6];  // xx yy zz xy yz xz
    E[0] = H[0][0] + 0.5f * (H[0][0] * H[0][0] + H[1][0] * H[1][0] + H[2][0] * H[2][0]);
    E[1] = H[1][1] + 0.5f * (H[0][1] * H[0][1] + H[1][1] * H[1][1] + H[2][1] * H[2][1]);
    E[2] = H[2][2] + 0.5f * (H[0][2] * H[0][2] + H[1][2] * H[1][2] + H[2][2] * H[2][2]);
    E[3] = 0.5f * (H[0][1] + H[1][0] + H[0][0] * H[0][1] + H[1][0] * H[1][1] + H[2][0] * H[2][1]);
    E[4] = 0.5f * (H[1][2] + H[2][1] + H[0][1] * H[0][2] + H[1][1] * H[1][2] + H[2][1] * H[2][2]);
    E[5] = 0.5f * (H[0][2] + H[2][0] + H[0][0] * H[0][2] + H[1][0] * H[1][2] + H[2][0] * H[2][2]);
    const float il2 = 1.f / (lam * lam);
    const float d1 = dl + 0.5f * dl * dl;
    E[0] = (E[0] - d1) * il2; E[1] = (E[1] - d1) * il2; E[2] = (E[2] - d1) * il2;
    E[3] *= il2; E[4] *= il2; E[5] *= il2;
    // J_el - 1 = ((J - 1) - (lambda^3 - 1)) / lambda^3
    const float l3m1 = dl * (3.f + dl * (3.f + dl));
    const float jel = (Jm1 - l3m1) / (lam * lam * lam);
    const float Jel = 1.f + jel;
    if (!(Jel > 0.f)) {
        atomicOr(A.status, kStatusInverted);
        atomicMin(A.status + 1, (unsigned)e);
    }
    // C_el = I + 2 E_el and its inverse adj(C_el) / J_el^2
    const float c00 = 1.f + 2.f * E[0], c11 = 1.f + 2.f * E[1], c22 = 1.f + 2.f * E[2];
    const float c01 = 2.f * E[3], c12 = 2.f * E[4], c02 = 2.f * E[5];
    const float iJ2 = 1.f / (Jel * Jel);
    float Ci[6];
    Ci[0] = (c11 * c22 - c12 * c12) * iJ2;
    Ci[1] = (c00 * c22 - c02 * c02) * iJ2;
    Ci[2] = (c00 * c11 - c01 * c01) * iJ2;
    Ci[3] = (c02 * c12 - c01 * c22) * iJ2;
    Ci[4] = (c01 * c02 - c00 * c12) * iJ2;
    Ci[5] = (c01 * c12 - c02 * c11) * iJ2;
    // J_el^(-2/3) and J_el^(-2/3) - 1 without cancellation
    const float lg = log1pf(jel);
    const float Jm23 = expf(-(2.f / 3.f) * lg);
    const float Jm23m1 = expm1f(-(2.f / 3.f) * lg);
    // isochoric part: mu J^-2/3 (I - I1/3 C^-1) = 2 mu J^-2/3 C^-1 dev(E_el)
    const float tr3 = (E[0] + E[1] + E[2]) * (1.f / 3.f);
    const float D[6] = {E[0] - tr3, E[1] - tr3, E[2] - tr3, E[3], E[4], E[5]};
    // symmetric product M = Ci * D (both symmetric and commuting)
    float M[6];
    M[0] = Ci[0] * D[0] + Ci[3] * D[3] + Ci[5] * D[5];
    M[1] = Ci[3] * D[3] + Ci[1] * D[1] + Ci[4] * D[4];
    M[2] = Ci[5] * D[5] + Ci[4] * D[4] + Ci[2] * D[2];
    M[3] = Ci[0] * D[3] + Ci[3] * D[1] + Ci[5] * D[4];
    M[4] = Ci[3] * D[5] + Ci[1] * D[4] + Ci[4] * D[2];
    M[5] = Ci[0] * D[5] + Ci[3] * D[4] + Ci[5] * D[2];
    // fibre term: I4b - 1 = (J^-2/3 - 1) + 2 J^-2/3 a.E_el.a
    const float aEa = ax * ax * E[0] + ay * ay * E[1] + az * az * E[2] + 2.f * (ax * ay * E[3] + ay * az * E[4] + ax * az * E[5]);
    const float I4 = 1.f + 2.f * aEa;
    const float x4 = Jm23m1 + 2.f * Jm23 * aEa;
    const float psi4 = k1 * x4 * expf(k2 * x4 * x4);
    const float cf = 2.f * psi4 * Jm23;
    const float cI4 = I4 * (1.f / 3.f);
    const float ciso = 2.f * mu * Jm23;
    const float cvol = kap * Jel * jel;
    const float aa[6] = {ax * ax, ay * ay, az * az, ax * ay, ay * az, ax * az};
    // S_0 = lambda S_i (Eq. 10 for F_th = lambda I), then Prony: S~ = S_0 - sum theta_p
    float St[6];
#pragma unroll
    for (int s = 0; s < 6; s++) St[s] = lam * (ciso * M[s] + cvol * Ci[s] + cf * (aa[s] - cI4 * Ci[s]));
    {
        float S0[6];
#pragma unroll
        for (int s = 0; s < 6; s++) S0[s] = St[s];
#pragma unroll
        for (int p = 0; p < 4; p++) {
            if (p < A.n_prony) {
#pragma unroll
                for (int s = 0; s < 6; s++) {
                    const float tp = A.pr_a[p] * S0[s] + A.pr_b[p] * vs[p][s];
                    A.visc[(int64_t)(p * 6 + s) * ne + e] = tp;
                    St[s] -= tp;
                }
            }
        }
    }
    const float Sm[3][3] = {{St[0], St[3], St[5]}, {St[3], St[1], St[4]}, {St[5], St[4], St[2]}};
    // first Piola-Kirchhoff P = F S~ = S~ + H S~
    float P[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) P[i][j] = Sm[i][j] + H[i][0] * Sm[0][j] + H[i][1] * Sm[1][j] + H[i][2] * Sm[2][j];
    // f_a = V P dh_a/dX = Q Xi_a with Q = s V P J0^-T (Eqs. 24-26, 28)
    float Qm[3][3];
    const float sV = sc * V;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++)
            Qm[i][k] = sV * (P[i][0] * Ji[3 * k] + P[i][1] * Ji[3 * k + 1] + P[i][2] * Ji[3 * k + 2]);
    // thermal: q = k J C^-1 grad0 theta = k lambda J_el C_el^-1 grad0 theta (Eq. 16);
    // fT_a = V dh_a/dX . q = r . Xi_a with r = s V J0^-1 q
    float kT = kc;
    if (A.flags & TLED_TEMP_DEP) kT *= 1.f + A.beta_k * (the - A.Tref_m_T0);
    const float kq = kT * lam * Jel;
    const float q0 = kq * (Ci[0] * gth[0] + Ci[3] * gth[1] + Ci[5] * gth[2]);
    const float q1 = kq * (Ci[3] * gth[0] + Ci[1] * gth[1] + Ci[4] * gth[2]);
    const float q2 = kq * (Ci[5] * gth[0] + Ci[4] * gth[1] + Ci[2] * gth[2]);
    float r[3];
#pragma unroll
    for (int k = 0; k < 3; k++) r[k] = sV * (Ji[3 * k] * q0 + Ji[3 * k + 1] * q1 + Ji[3 * k + 2] * q2);

    if constexpr (NPE == 8) {
        // hourglass control: gamma_a,al = h_a,al - c_al . dh_a/dX with c_al = sum_b h_b,al X_b;
        // f_a += k_hg sum_al gamma_a,al q_al with q_al = sum_b h_b,al u_b - H c_al
        float Xr[8][3];
        {
            const float4 x0 = s_X[cl[0]];
#pragma unroll
            for (int a = 0; a < 8; a++) {
                const float4 xa = s_X[cl[a]];
                Xr[a][0] = xa.x - x0.x; Xr[a][1] = xa.y - x0.y; Xr[a][2] = xa.z - x0.z;
            }
        }
        float jn2 = 0.f;
#pragma unroll
        for (int q = 0; q < 9; q++) jn2 += Ji[q] * Ji[q];
        const float khg = A.khg * (kap + (4.f / 3.f) * mu) * V * jn2 * (1.f / 64.f);
        const float khgT = A.khgT * kT * V * jn2 * (1.f / 64.f);
        float qa[4][3], qT[4];
        float Wm[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        float wT[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int l = 0; l < 4; l++) {
            float c[3] = {0.f, 0.f, 0.f}, hu[3] = {0.f, 0.f, 0.f}, ht = 0.f;
#pragma unroll
            for (int b = 0; b < 8; b++) {
                c[0] += hgv(b, l) * Xr[b][0]; c[1] += hgv(b, l) * Xr[b][1]; c[2] += hgv(b, l) * Xr[b][2];
                hu[0] += hgv(b, l) * ux[b]; hu[1] += hgv(b, l) * uy[b]; hu[2] += hgv(b, l) * uz[b];
                ht += hgv(b, l) * th[b];
            }
#pragma unroll
            for (int i = 0; i < 3; i++) {
                qa[l][i] = hu[i] - (H[i][0] * c[0] + H[i][1] * c[1] + H[i][2] * c[2]);
#pragma unroll
                for (int j = 0; j < 3; j++) Wm[i][j] += qa[l][i] * c[j];
            }
            qT[l] = ht - (c[0] * gth[0] + c[1] * gth[1] + c[2] * gth[2]);
            wT[0] += qT[l] * c[0]; wT[1] += qT[l] * c[1]; wT[2] += qT[l] * c[2];
        }
        // fold the -k_hg W dh_a/dX part into Q and r
        const float hs = 0.125f;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int k = 0; k < 3; k++)
                Qm[i][k] -= khg * hs * (Wm[i][0] * Ji[3 * k] + Wm[i][1] * Ji[3 * k + 1] + Wm[i][2] * Ji[3 * k + 2]);
#pragma unroll
        for (int k = 0; k < 3; k++) r[k] -= khgT * hs * (Ji[3 * k] * wT[0] + Ji[3 * k + 1] * wT[1] + Ji[3 * k + 2] * wT[2]);
#pragma unroll
        for (int a = 0; a < 8; a++) {
            float f[3], fT;
#pragma unroll
            for (int i = 0; i < 3; i++)
                f[i] = sgn(a, 0) * Qm[i][0] + sgn(a, 1) * Qm[i][1] + sgn(a, 2) * Qm[i][2] +
                       khg * (hgv(a, 0) * qa[0][i] + hgv(a, 1) * qa[1][i] + hgv(a, 2) * qa[2][i] + hgv(a, 3) * qa[3][i]);
            fT = sgn(a, 0) * r[0] + sgn(a, 1) * r[1] + sgn(a, 2) * r[2] +
                 khgT * (hgv(a, 0) * qT[0] + hgv(a, 1) * qT[1] + hgv(a, 2) * qT[2] + hgv(a, 3) * qT[3]);
            s_slot[el * 8 + a] = make_float4(f[0], f[1], f[2], fT);
        }
    } else {
        // T4: dh_0 = -(dh_1 + dh_2 + dh_3), dh_{j+1} = row j of J0^-1
        s_slot[el * 4 + 0] = make_float4(-(Qm[0][0] + Qm[0][1] + Qm[0][2]), -(Qm[1][0] + Qm[1][1] + Qm[1][2]),
                                         -(Qm[2][0] + Qm[2][1] + Qm[2][2]), -(r[0] + r[1] + r[2]));
#pragma unroll
        for (int j = 0; j < 3; j++) s_slot[el * 4 + 1 + j] = make_float4(Qm[0][j], Qm[1][j], Qm[2][j], r[j]);
    }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <int NPE>
__global__ void __launch_bounds__(kBlock, 2) tile_step_kernel(const StepArgs A, const int k) {
    extern __shared__ float4 smem[];
    float4 *s_xu = smem;
    float4 *s_X = smem + kMaxLocal;
    float4 *s_slot = smem + 2 * kMaxLocal;
    __shared__ SrcSmem S;
    const int *ti = A.tile_info + (size_t)blockIdx.x * kTileInfo;
    const int e0 = ti[0], ne_t = ti[1], ib = ti[2], n_int = ti[3], nl = ti[4], sh_off = ti[5], row_off = ti[6],
              part_off = ti[7];
    // 1. gather the tile's nodes
    for (int l = threadIdx.x; l < nl; l += kBlock) {
        const int64_t g = l < n_int ? (int64_t)ib + l : (int64_t)__ldg(A.tile_shared + sh_off + l - n_int);
        s_xu[l] = A.xu[g];
        s_X[l] = __ldg(&A.X0[g]);
    }
    prepare_sources(A, k, S);  // contains __syncthreads
    __syncthreads();
    // 2. element pass
    for (int el = threadIdx.x; el < ne_t; el += kBlock) element_step<NPE>(A, (int64_t)e0 + el, el, s_xu, s_X, s_slot);
    __syncthreads();
    // 3. node-centric gather in a fixed order, then nodal update or partial store
    const uint16_t *rp = A.rowptr + row_off;
    const uint16_t *sl = A.slots + (size_t)e0 * NPE;
    for (int l = threadIdx.x; l < nl; l += kBlock) {
        const int r0 = __ldg(rp + l), r1 = __ldg(rp + l + 1);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int r = r0; r < r1; r++) {
            const float4 c = s_slot[__ldg(sl + r)];
            acc.x += c.x; acc.y += c.y; acc.z += c.z; acc.w += c.w;
        }
        if (l < n_int)
            node_update(A, (int64_t)ib + l, acc, s_xu[l], s_X[l], S);
        else
            A.partials[part_off + l - n_int] = acc;
    }
}

__global__ void __launch_bounds__(256) shared_step_kernel(const StepArgs A, const int k) {
    __shared__ SrcSmem S;
    prepare_sources(A, k, S);
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.n_shared) return;
    const int64_t g = A.n_interior + s;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const int r0 = __ldg(A.sh_rowptr + s), r1 = __ldg(A.sh_rowptr + s + 1);
    for (int r = r0; r < r1; r++) {
        const float4 c = A.partials[__ldg(A.sh_list + r)];
        acc.x += c.x; acc.y += c.y; acc.z += c.z; acc.w += c.w;
    }
    node_update(A, g, acc, A.xu[g], __ldg(&A.X0[g]), S);
}

__global__ void bump_kernel(double *time_base, int64_t *step_base, int K, double dt) {
    *time_base += (double)K * dt;
    *step_base += K;
}

__global__ void readback_kernel(const float4 *__restrict__ hi, const float4 *__restrict__ lo,
                                const float4 *__restrict__ vel, const int32_t *__restrict__ node_new, int64_t nn,
                                double T0, int mode, double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const int64_t g = node_new[i];
    if (mode == 0) {
        const float4 h = hi[g], l = lo[g];
        out[3 * i + 0] = (double)h.x + (double)l.x;
        out[3 * i + 1] = (double)h.y + (double)l.y;
        out[3 * i + 2] = (double)h.z + (double)l.z;
    } else if (mode == 1) {
        out[i] = T0 + ((double)hi[g].w + (double)lo[g].w);
    } else {
        out[i] = -expm1(-(double)vel[g].w);
    }
}

// Deterministic FP64 diagnostics: fixed grid, fixed per-thread stride, fixed tree.
__global__ void __launch_bounds__(256) stats_partial_kernel(const StepArgs A, int64_t nn, double *partials) {
    double ke = 0, heat = 0, tmax = -1e300, tmin = 1e300, umax = 0, dvol = 0;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        const float4 h = A.xu[g], l = A.lo[g], v = A.vel[g], nc = A.nodec[g], X = A.X0[g];
        const double ux = (double)h.x + l.x, uy = (double)h.y + l.y, uz = (double)h.z + l.z;
        const double th = (double)h.w + l.w;
        ke += 0.5 * (double)nc.x * ((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z);
        heat += (double)nc.y * th;
        tmax = fmax(tmax, th);
        tmin = fmin(tmin, th);
        umax = fmax(umax, ux * ux + uy * uy + uz * uz);
        if (v.w >= 1.f) dvol += (double)X.w;
    }
    __shared__ double sh[6][256];
    sh[0][threadIdx.x] = ke; sh[1][threadIdx.x] = heat; sh[2][threadIdx.x] = tmax;
    sh[3][threadIdx.x] = tmin; sh[4][threadIdx.x] = umax; sh[5][threadIdx.x] = dvol;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const int o = threadIdx.x + w;
            sh[0][threadIdx.x] += sh[0][o];
            sh[1][threadIdx.x] += sh[1][o];
            sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][o]);
            sh[3][threadIdx.x] = fmin(sh[3][threadIdx.x], sh[3][o]);
            sh[4][threadIdx.x] = fmax(sh[4][threadIdx.x], sh[4][o]);
            sh[5][threadIdx.x] += sh[5][o];
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) partials[(size_t)blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void stats_final_kernel(const double *partials, int nb, double *out) {
    if (threadIdx.x != 0) return;
    double ke = 0, heat = 0, tmax = -1e300, tmin = 1e300, umax = 0, dvol = 0;
    for (int b = 0; b < nb; b++) {
        const double *p = partials + (size_t)b * 8;
        ke += p[0]; heat += p[1]; tmax = fmax(tmax, p[2]); tmin = fmin(tmin, p[3]); umax = fmax(umax, p[4]);
        dvol += p[5];
    }
    out[0] = ke; out[1] = heat; out[2] = tmax; out[3] = tmin; out[4] = umax; out[5] = dvol;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t tile_smem_bytes(int npe) { return (size_t)(2 * kMaxLocal + kMaxSlots) * sizeof(float4); }

cudaError_t tile_kernel_setup(int npe) {
    const int bytes = (int)tile_smem_bytes(npe);
    if (npe == 8) return cudaFuncSetAttribute(tile_step_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return cudaFuncSetAttribute(tile_step_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_tile_step(const StepArgs &a, int n_tiles, int npe, int k, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    const size_t sm = tile_smem_bytes(npe);
    if (npe == 8)
        tile_step_kernel<8><<<n_tiles, kBlock, sm, s>>>(a, k);
    else
        tile_step_kernel<4><<<n_tiles, kBlock, sm, s>>>(a, k);
    return cudaGetLastError();
}

cudaError_t launch_shared_step(const StepArgs &a, int npe, int k, cudaStream_t s) {
    (void)npe;
    if (a.n_shared <= 0) return cudaSuccess;
    const int nb = (int)((a.n_shared + 255) / 256);
    shared_step_kernel<<<nb, 256, 0, s>>>(a, k);
    return cudaGetLastError();
}

cudaError_t launch_bump(double *time_base, int64_t *step_base, int K, double dt, cudaStream_t s) {
    bump_kernel<<<1, 1, 0, s>>>(time_base, step_base, K, dt);
    return cudaGetLastError();
}

cudaError_t launch_readback(const StepArgs &a, const int32_t *node_new, int64_t nn, double T0, int mode, double *out,
                            cudaStream_t s) {
    const int nb = (int)((nn + 255) / 256);
    readback_kernel<<<nb, 256, 0, s>>>(a.xu, a.lo, a.vel, node_new, nn, T0, mode, out);
    return cudaGetLastError();
}

cudaError_t launch_stats(const StepArgs &a, int64_t nn, double *partials, double *out, cudaStream_t s) {
    stats_partial_kernel<<<kStatBlocks, 256, 0, s>>>(a, nn, partials);
    stats_final_kernel<<<1, 32, 0, s>>>(partials, kStatBlocks, out);
    return cudaGetLastError();
}

}  // namespace tled
