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
//  * resident kernel (problems, or batch scenarios, that fit one CTA's shared
//    memory): one CTA per scenario runs the same phases for K steps with block
//    barriers in place of kernel boundaries.
// Instances: element type (H8, T4 or a mixed batch), Prony term count,
// transversely isotropic thermal physics, and for H8 meshes of axis-aligned
// bricks an instance without the (exactly zero) reference hourglass projections.
//
// Floating point: FP32 throughout; kinematics are written in H = du/dX so
// that J - 1, E and I4b - 1 never cancel; nodal u and theta accumulate in
// float-float (TwoSum) pairs; theta is stored relative to T0.
#include <algorithm>
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

// Per-scenario values of one step: time, step size, damping and Prony
// coefficients, and the heat sources' centres c(t) = c0 + v t and powers.
// With mechanical subcycling (n_sub > 1) a step is a mechanical substep: every
// substep advances u by dt; the last of each group of n_sub (thermal = 1)
// also advances T, Omega and the dose by the thermal step dt_th = n_sub dt,
// with the sources at the group's start time t_th (explicit in T(t_th)).
struct ScenStep {
    double t, dt, dt_th;
    float dtf, inv_dt, damp_a, damp_b, Qm, dtf_th;
    int thermal;
    float pr_a[4], pr_b[4];
    int n;
    int sph;  // 1 if a source is a uniform sphere
    // source s adds P exp(-d^2 inv2s2) where d^2 <= r2: a Gaussian (r2 infinite) or a
    // uniform sphere (inv2s2 = 0, r2 = radius^2)
    float cx[kMaxSources], cy[kMaxSources], cz[kMaxSources], inv2s2[kMaxSources], r2[kMaxSources], P[kMaxSources];
};

// Fill P for scenario s at step k of the current chunk.  Called by all threads of
// a group; thread `lane` handles source `lane`, lane 0 the scalars (no barrier inside).
__device__ __forceinline__ void prepare_scen(const StepArgs &A, int s, int k, ScenStep &P, int lane, int nlanes) {
    const ScenDev &D = A.scn[s];
    const int64_t n = A.scn_step[s] + k;
    const double t = A.scn_time[s] + (double)n * D.dt;  // t0 + n dt, no accumulation
    // the thermal step this (sub)step belongs to starts at t_th; sources are evaluated there
    const double t_th = D.n_sub > 1 ? A.scn_time[s] + (double)(n - n % D.n_sub) * D.dt : t;
    if (lane == 0) {
        P.t = t;
        P.dt = D.dt;
        P.dtf = D.dtf;
        P.dt_th = D.dt_th;
        P.dtf_th = D.dtf_th;
        P.thermal = D.n_sub <= 1 || n % D.n_sub == D.n_sub - 1;
        P.inv_dt = D.inv_dt;
        P.damp_a = D.damp_a;
        P.damp_b = D.damp_b;
        P.Qm = D.Qm;
        for (int i = 0; i < 4; i++) {
            P.pr_a[i] = D.pr_a[i];
            P.pr_b[i] = D.pr_b[i];
        }
        P.n = D.n_src;
        P.sph = 0;
        for (int q = 0; q < D.n_src; q++) P.sph |= A.src[kSrcRow * (int64_t)(D.src_off + q) + 10] == 1.0;
    }
    for (int q = lane; q < D.n_src; q += nlanes) {
        const double *p = A.src + kSrcRow * (int64_t)(D.src_off + q);
        P.cx[q] = (float)(p[0] + p[3] * t_th);
        P.cy[q] = (float)(p[1] + p[4] * t_th);
        P.cz[q] = (float)(p[2] + p[5] * t_th);
        const bool sphere = p[10] == 1.0;
        P.inv2s2[q] = sphere ? 0.f : (float)(0.5 / (p[6] * p[6]));
        P.r2[q] = sphere ? (float)(p[6] * p[6]) : INFINITY;
        P.P[q] = (t_th >= p[8] && t_th < p[9]) ? (float)p[7] : 0.f;
    }
}

// ---------------------------------------------------------------------------
// TMA bulk copies and mbarriers (inline PTX, sm_90+ / sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// 16-byte asynchronous global -> shared copy (L2 only); completion by cp_async_wait_all
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait (about 2^31 SM cycles, i.e. around a second): on time-out the
// caller flags the device status instead of hanging.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// nodal update: Eq. (27) in velocity form, Eq. (20), Arrhenius
// ---------------------------------------------------------------------------
// xu: (u_hi, theta_hi); X: (X0, V_i); lo: (u_lo, theta_lo); vo: (v, Omega);
// nc: (1/m_i, 1/C_i, mask bits, K_b,i); f: (internal force, thermal load).
// nc.w: perfusion conductance w_b c_b V_i of the node.
// The new state goes to xo (u_hi, theta_hi), lo_o (u_lo, theta_lo), vo_o (v, Omega).
// dose: accumulate the CEM43 dose (off for the redundant copies of a shared node's update)
__device__ __forceinline__ void node_advance(const StepArgs &A, const ScenStep &S, int64_t g, float4 f, float4 xu,
                                             float4 X, float4 lo, float4 vo, float4 nc, float4 &xo, float4 &lo_o,
                                             float4 &vo_o, bool dose = true) {
    const unsigned mask = __float_as_uint(nc.z);
    const bool comp = (A.flags & TLED_COMPENSATED) != 0;
    const float dt = S.dtf;
    if (A.cem && dose && S.thermal) {  // CEM43 dose (Sapareto-Dewey) at T(t): dt R^(43 - T) / 60 minutes,
                  // R = 0.5 at or above 43 C, 0.25 below; FP64 (single problems)
        const double T = A.T0 + ((double)xu.w + (double)lo.w);
        const double x = T - 43.0;  // R^(43 - T) = 2^(x) or 4^(x)
        A.cem[g] += S.dt_th * exp2(T >= 43.0 ? x : 2.0 * x) / 60.0;
    }
    // current position for the heat source (state at t)
    const float px = X.x + (xu.x + lo.x), py = X.y + (xu.y + lo.y), pz = X.z + (xu.z + lo.z);

    float u[3] = {xu.x, xu.y, xu.z}, ul[3] = {lo.x, lo.y, lo.z}, v[3] = {vo.x, vo.y, vo.z};
    const float fv[3] = {f.x, f.y, f.z};
    const float im = nc.x;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (mask & (1u << d)) {
            // prescribed: u(t+dt) = ubar * ramp(t+dt), v consistent with it
            float target = 0.f;
            if (A.ubar) {
                const double tn = S.t + S.dt;
                const double r = (A.ramp_time > 0.0 && tn < A.ramp_time) ? tn / A.ramp_time : 1.0;
                const float4 ub = __ldg(&A.ubar[g]);
                target = (float)((d == 0 ? ub.x : d == 1 ? ub.y : ub.z) * r);
            }
            v[d] = (target - u[d] - ul[d]) * S.inv_dt;
            u[d] = target;
            ul[d] = 0.f;
        } else {
            // v+ = [(1 - g dt/2) v + dt (R - f)/m] / (1 + g dt/2), R = 0; u+ = u + dt v+
            v[d] = S.damp_a * v[d] - S.damp_b * fv[d] * im;
            if (comp)
                add_ff(u[d], ul[d], dt * v[d]);
            else
                u[d] += dt * v[d];
        }
    }
    // Eq. (20), physical conduction sign: C dtheta/dt = -fT - wbcb V (theta - theta_a) + V (Qm + Qr)
    float th = xu.w, tl = lo.w;
    const float theta = th + tl;
    float iC = nc.y;
    if (A.flags & TLED_TEMP_DEP) iC = __fdividef(iC, 1.f + A.beta_c * (theta - A.Tref_m_T0));
    float Q = S.Qm;
    if (S.sph) {  // some source is a uniform sphere: P inside radius^2, or a Gaussian
        for (int s = 0; s < S.n; s++) {
            const float dx = px - S.cx[s], dy = py - S.cy[s], dz = pz - S.cz[s];
            const float d2 = dx * dx + dy * dy + dz * dz;
            Q += d2 <= S.r2[s] ? S.P[s] * __expf(-d2 * S.inv2s2[s]) : 0.f;
        }
    } else {
        for (int s = 0; s < S.n; s++) {
            const float dx = px - S.cx[s], dy = py - S.cy[s], dz = pz - S.cz[s];
            Q += S.P[s] * __expf(-(dx * dx + dy * dy + dz * dz) * S.inv2s2[s]);
        }
    }
    const float dtt = S.dtf_th;
    if (!(mask & TLED_FIX_T) && S.thermal) {
        const float dth = dtt * iC * (-f.w + X.w * Q - nc.w * (theta - A.theta_a));
        if (comp)
            add_ff(th, tl, dth);
        else
            th += dth;
    }
    // Arrhenius damage integral, explicit in T(t); exp(ln A - Ea/(R T)) avoids A > FLT_MAX
    const float Om = S.thermal ? vo.w + dtt * __expf(A.lnA - __fdividef(A.Ea_R, theta + A.T0_K)) : vo.w;
    if (!(isfinite(th) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]))) {
        atomicOr(A.status, kStatusNaN);
        atomicMin(A.status + 2, (unsigned)g);
    }
    xo = make_float4(u[0], u[1], u[2], th);
    lo_o = make_float4(ul[0], ul[1], ul[2], tl);
    vo_o = make_float4(v[0], v[1], v[2], Om);
}
// ... stored to node g's state in global memory
__device__ __forceinline__ void node_update(const StepArgs &A, const ScenStep &S, int64_t g, float4 f, float4 xu,
                                            float4 X, float4 lo, float4 vo, float4 nc) {
    float4 a, b, c;
    node_advance(A, S, g, f, xu, X, lo, vo, nc, a, b, c);
    A.xu[g] = a;
    A.lo[g] = b;
    A.vel[g] = c;
}

// ---------------------------------------------------------------------------
// element pass
// ---------------------------------------------------------------------------
// In-place unnormalised Walsh-Hadamard transform of 8 values:
// X_k = sum_i x_i (-1)^popcount(i & k).  With hexahedron corners ordered by
// i = [xi > 0] + 2 [eta > 0] + 4 [zeta > 0], the coefficients are the corner
// sums against the sign vectors: xi -> -X1, eta -> -X2, zeta -> -X4,
// xi eta -> X3, eta zeta -> X6, xi zeta -> X5, xi eta zeta -> -X7; the
// transform is its own inverse up to a factor 8.
__device__ __forceinline__ void wht8(float *x) {
#pragma unroll
    for (int h = 1; h < 8; h <<= 1)
#pragma unroll
        for (int i = 0; i < 8; i++)
            if ((i & h) == 0) {
                const float a = x[i], b = x[i + h];
                x[i] = a + b;
                x[i + h] = a - b;
            }
}
// Paired form: two independent transforms (the two lanes of a float2) with
// one packed f32x2 add or subtract per butterfly (sm_100+); same roundings.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ void wht8x2(float2 *x) {
#pragma unroll
    for (int h = 1; h < 8; h <<= 1)
#pragma unroll
        for (int i = 0; i < 8; i++)
            if ((i & h) == 0) {
                const float2 a = x[i], b = x[i + h];
                x[i] = add2(a, b);
                x[i + h] = sub2(a, b);
            }
}
// WHT index -> VTK corner (an involution)
__device__ __forceinline__ constexpr int wht_corner(int i) { return i == 2 ? 3 : i == 3 ? 2 : i == 6 ? 7 : i == 7 ? 6 : i; }

// Corner values of an H8 element (local corner ids cl) transformed against the
// shape-function sign vectors by Walsh-Hadamard butterflies: (u_x, u_y) and (u_z,
// theta) in pairs and, with WITH_X, (X, Y) in a pair and Z alone.  Mode i of the
// transform: 0 the corner sum, 1/2/4 minus the xi/eta/zeta sums, 3/6/5 the xi eta /
// eta zeta / xi zeta hourglass sums, 7 minus the xi eta zeta sum.
template <bool WITH_X>
__device__ __forceinline__ void h8_modes(const int *cl, const float4 *__restrict__ s_xu,
                                         const float4 *__restrict__ s_X, float *wx, float *wy, float *wz, float *wt,
                                         float *px, float *py, float *pz) {
    float2 uxy[8], uzt[8], pxy[8];
    float qz[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int a = cl[wht_corner(i)];
        const float4 q = s_xu[a];
        uxy[i] = make_float2(q.x, q.y);
        uzt[i] = make_float2(q.z, q.w);
        if constexpr (WITH_X) {
            const float4 x = s_X[a];
            pxy[i] = make_float2(x.x, x.y);
            qz[i] = x.z;
        }
    }
    wht8x2(uxy); wht8x2(uzt);
    if constexpr (WITH_X) {
        wht8x2(pxy); wht8(qz);
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
        wx[i] = uxy[i].x; wy[i] = uxy[i].y; wz[i] = uzt[i].x; wt[i] = uzt[i].y;
        if constexpr (WITH_X) {
            px[i] = pxy[i].x; py[i] = pxy[i].y; pz[i] = qz[i];
        }
    }
}

// NPR: Prony terms (a compile-time count, so that only the terms in use take registers)
template <int NPR>
struct ElemIn {
    float Ji[9];
    float V;
    float mu, kap, k1, k2, kc, al;
    float ax, ay, az;
    float vs[NPR > 0 ? NPR : 1][6];
};

// Element inputs staged in shared memory for one tile: the local connectivity
// [kTile][NPE] (uint16, head of the structure record) and the float components
// [q][kTile]: J0^-1 (9; bricks: its diagonal, 3), V0, [mu kappa k1 k2 k alpha], [fibre xyz],
// Prony state (6 per term).
template <int NPE, int NPR, bool BRICK = false>
__device__ __forceinline__ void load_elem(const StepArgs &A, const char *base, const uint16_t *conn, int ec, int *cl,
                                          ElemIn<NPR> &E) {
    if constexpr (NPE == 8) {
        const uint4 c = reinterpret_cast<const uint4 *>(conn)[ec];
        cl[0] = c.x & 0xffff; cl[1] = c.x >> 16; cl[2] = c.y & 0xffff; cl[3] = c.y >> 16;
        cl[4] = c.z & 0xffff; cl[5] = c.z >> 16; cl[6] = c.w & 0xffff; cl[7] = c.w >> 16;
    } else {
        const uint2 c = reinterpret_cast<const uint2 *>(conn)[ec];
        cl[0] = c.x & 0xffff; cl[1] = c.x >> 16; cl[2] = c.y & 0xffff; cl[3] = c.y >> 16;
    }
    const float *cp = reinterpret_cast<const float *>(base) + ec;
    int q = 0;
    if constexpr (BRICK) {
#pragma unroll
        for (int k = 0; k < 9; k++) E.Ji[k] = 0.f;
        E.Ji[0] = cp[(q++) * kTile]; E.Ji[4] = cp[(q++) * kTile]; E.Ji[8] = cp[(q++) * kTile];
    } else {
#pragma unroll
        for (int k = 0; k < 9; k++) E.Ji[k] = cp[(q++) * kTile];
    }
    E.V = cp[(q++) * kTile];
    if (A.has_mat) {
        E.mu = cp[(q++) * kTile]; E.kap = cp[(q++) * kTile]; E.k1 = cp[(q++) * kTile];
        E.k2 = cp[(q++) * kTile]; E.kc = cp[(q++) * kTile]; E.al = cp[(q++) * kTile];
    } else {
        E.mu = A.mu; E.kap = A.kappa; E.k1 = A.k1; E.k2 = A.k2; E.kc = A.kc; E.al = A.alpha;
    }
    if (A.has_fib) {
        E.ax = cp[(q++) * kTile]; E.ay = cp[(q++) * kTile]; E.az = cp[(q++) * kTile];
    } else {
        E.ax = A.a0x; E.ay = A.a0y; E.az = A.a0z;
    }
#pragma unroll
    for (int p = 0; p < NPR; p++)
#pragma unroll
        for (int s = 0; s < 6; s++) E.vs[p][s] = cp[(q + p * 6 + s) * kTile];
}

// One element: deformation gradient, thermal split, stress, Prony, nodal
// forces + hourglass, thermal loads.  Corner contributions are written to the
// chunk's slot buffer at [corner][ec] (conflict-free).
// ANI: transversely isotropic thermal expansion about the fibre (Eq. 11) and
// conductivity along the current fibre; otherwise isotropic (F_th = lambda I).
// BRICK (H8): every element an axis-aligned box: J0^-1 is diagonal (its off-diagonal
// products are dropped) and the reference hourglass projections c_al vanish exactly,
// so the terms they multiply (and the corner coordinates) are dropped too.
template <int NPE, int NPR, bool ANI, bool BRICK>
__device__ __forceinline__ void element_step(const StepArgs &A, const ScenStep &SP, int64_t e, int ec, const int *cl,
                                             ElemIn<NPR> &E, const float4 *__restrict__ s_xu,
                                             const float4 *__restrict__ s_X, float4 *__restrict__ slot,
                                             float *__restrict__ gvisc) {
    const float *Ji = E.Ji;
    const float V = E.V, mu = E.mu, kap = E.kap, k1 = E.k1, k2 = E.k2, kc = E.kc, al = E.al;
    const float ax = E.ax, ay = E.ay, az = E.az;

    // ---- corner values and the sums against the shape-function sign vectors: here the
    //      constant and linear modes; the H8 hourglass modes are transformed again where
    //      they are used (from the same shared-memory values, so bitwise the same), which
    //      keeps them out of the registers the stress evaluation needs
    float G[3][3], gt[3], the;
    float hu[4][3], ht[4];  // H8 hourglass modes of u and theta (bricks: kept from this transform)
    if constexpr (NPE == 8) {
        float wx[8], wy[8], wz[8], wt[8];
        h8_modes<false>(cl, s_xu, s_X, wx, wy, wz, wt, nullptr, nullptr, nullptr);
        G[0][0] = -wx[1]; G[0][1] = -wx[2]; G[0][2] = -wx[4];
        G[1][0] = -wy[1]; G[1][1] = -wy[2]; G[1][2] = -wy[4];
        G[2][0] = -wz[1]; G[2][1] = -wz[2]; G[2][2] = -wz[4];
        gt[0] = -wt[1]; gt[1] = -wt[2]; gt[2] = -wt[4];
        the = 0.125f * wt[0];
        if constexpr (BRICK) {
            hu[0][0] = wx[3]; hu[1][0] = wx[6]; hu[2][0] = wx[5]; hu[3][0] = -wx[7];
            hu[0][1] = wy[3]; hu[1][1] = wy[6]; hu[2][1] = wy[5]; hu[3][1] = -wy[7];
            hu[0][2] = wz[3]; hu[1][2] = wz[6]; hu[2][2] = wz[5]; hu[3][2] = -wz[7];
            ht[0] = wt[3]; ht[1] = wt[6]; ht[2] = wt[5]; ht[3] = -wt[7];
        }
    } else {
        float ux[4], uy[4], uz[4], th[4];
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const float4 q = s_xu[cl[a]];
            ux[a] = q.x; uy[a] = q.y; uz[a] = q.z; th[a] = q.w;
        }
#pragma unroll
        for (int j = 0; j < 3; j++) {
            G[0][j] = ux[j + 1] - ux[0]; G[1][j] = uy[j + 1] - uy[0]; G[2][j] = uz[j + 1] - uz[0];
            gt[j] = th[j + 1] - th[0];
        }
        the = 0.25f * ((th[0] + th[1]) + (th[2] + th[3]));
    }
    // ---- Eq. (17) without forming I + H: H = s G J0^-1 (s = 1/8 for H8)
    constexpr float sc = NPE == 8 ? 0.125f : 1.f;
    float H[3][3], gth[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        if constexpr (BRICK) {
#pragma unroll
            for (int i = 0; i < 3; i++) H[i][j] = sc * (G[i][j] * Ji[4 * j]);
            gth[j] = sc * (gt[j] * Ji[4 * j]);
        } else {
#pragma unroll
            for (int i = 0; i < 3; i++) H[i][j] = sc * (G[i][0] * Ji[j] + G[i][1] * Ji[3 + j] + G[i][2] * Ji[6 + j]);
            gth[j] = sc * (gt[0] * Ji[j] + gt[1] * Ji[3 + j] + gt[2] * Ji[6 + j]);
        }
    }

    // ---- thermal split (Eqs. 7-11, isotropic): lambda = 1 + delta, delta = alpha theta_e
    const float dl = (A.flags & TLED_EXPANSION) ? al * the : 0.f;
    const float lam = 1.f + dl;
    const float il = __fdividef(1.f, lam);
    const float il2 = il * il;
    // J - 1 = tr H + [(tr H)^2 - tr(H^2)]/2 + det H
    const float trH = H[0][0] + H[1][1] + H[2][2];
    const float trH2 = H[0][0] * H[0][0] + H[1][1] * H[1][1] + H[2][2] * H[2][2] +
                       2.f * (H[0][1] * H[1][0] + H[0][2] * H[2][0] + H[1][2] * H[2][1]);
    const float detH = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) -
                       H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
                       H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
    const float Jm1 = trH + 0.5f * (trH * trH - trH2) + detH;
    // Green-Lagrange E = (H + H^T + H^T H)/2, then E_el = (E - (delta + delta^2/2) I) / lambda^2
    float Ee[6];  // xx yy zz xy yz xz
    Ee[0] = H[0][0] + 0.5f * (H[0][0] * H[0][0] + H[1][0] * H[1][0] + H[2][0] * H[2][0]);
    Ee[1] = H[1][1] + 0.5f * (H[0][1] * H[0][1] + H[1][1] * H[1][1] + H[2][1] * H[2][1]);
    Ee[2] = H[2][2] + 0.5f * (H[0][2] * H[0][2] + H[1][2] * H[1][2] + H[2][2] * H[2][2]);
    Ee[3] = 0.5f * (H[0][1] + H[1][0] + H[0][0] * H[0][1] + H[1][0] * H[1][1] + H[2][0] * H[2][1]);
    Ee[4] = 0.5f * (H[1][2] + H[2][1] + H[0][1] * H[0][2] + H[1][1] * H[1][2] + H[2][1] * H[2][2]);
    Ee[5] = 0.5f * (H[0][2] + H[2][0] + H[0][0] * H[0][2] + H[1][0] * H[1][2] + H[2][0] * H[2][2]);
    const float d1 = dl + 0.5f * dl * dl;
    // anisotropic: F_th^-1 = (I - g m m) / lambda_i, g = (lambda_m - lambda_i) / lambda_m, m = fibre,
    // E_el = [E - d1 I - g (m Em + Em m) + (g^2 m.E.m - g + g^2/2) m m] / lambda_i^2 (Em = E m)
    float dm = dl, lm = lam, gam = 0.f, mEm = 0.f, det_th = 1.f;  // delta_m kept: 1 + tiny - 1 would lose it
    if constexpr (ANI) {
        dm = (A.flags & TLED_EXPANSION) ? A.ani_alpha * al * the : 0.f;
        lm = 1.f + dm;
        gam = __fdividef(dm - dl, lm);
        const float Emx = Ee[0] * ax + Ee[3] * ay + Ee[5] * az;
        const float Emy = Ee[3] * ax + Ee[1] * ay + Ee[4] * az;
        const float Emz = Ee[5] * ax + Ee[4] * ay + Ee[2] * az;
        mEm = ax * Emx + ay * Emy + az * Emz;
        const float cmm = gam * gam * mEm - gam + 0.5f * gam * gam;
        Ee[0] += -2.f * gam * ax * Emx + cmm * ax * ax;
        Ee[1] += -2.f * gam * ay * Emy + cmm * ay * ay;
        Ee[2] += -2.f * gam * az * Emz + cmm * az * az;
        Ee[3] += -gam * (ax * Emy + Emx * ay) + cmm * ax * ay;
        Ee[4] += -gam * (ay * Emz + Emy * az) + cmm * ay * az;
        Ee[5] += -gam * (ax * Emz + Emx * az) + cmm * ax * az;
    }
    Ee[0] = (Ee[0] - d1) * il2; Ee[1] = (Ee[1] - d1) * il2; Ee[2] = (Ee[2] - d1) * il2;
    Ee[3] *= il2; Ee[4] *= il2; Ee[5] *= il2;
    // J_el - 1 = ((J - 1) - (det F_th - 1)) / det F_th; det F_th = lambda_i^2 lambda_m
    float jel;
    if constexpr (ANI) {
        const float t3m1 = dl * (2.f + dl) + dm * (1.f + dl) * (1.f + dl);
        det_th = 1.f + t3m1;
        jel = __fdividef(Jm1 - t3m1, det_th);
    } else {
        const float l3m1 = dl * (3.f + dl * (3.f + dl));
        jel = (Jm1 - l3m1) * (il2 * il);
    }
    const float Jel = 1.f + jel;
    if (!(Jel > 0.f)) {
        atomicOr(A.status, kStatusInverted);
        atomicMin(A.status + 1, (unsigned)e);
    }
    // C_el = I + 2 E_el and its inverse adj(C_el) / J_el^2
    const float c00 = 1.f + 2.f * Ee[0], c11 = 1.f + 2.f * Ee[1], c22 = 1.f + 2.f * Ee[2];
    const float c01 = 2.f * Ee[3], c12 = 2.f * Ee[4], c02 = 2.f * Ee[5];
    const float iJ2 = __fdividef(1.f, Jel * Jel);
    float Ci[6];
    Ci[0] = (c11 * c22 - c12 * c12) * iJ2;
    Ci[1] = (c00 * c22 - c02 * c02) * iJ2;
    Ci[2] = (c00 * c11 - c01 * c01) * iJ2;
    Ci[3] = (c02 * c12 - c01 * c22) * iJ2;
    Ci[4] = (c01 * c02 - c00 * c12) * iJ2;
    Ci[5] = (c01 * c12 - c02 * c11) * iJ2;
    // J_el^(-2/3) - 1 without cancellation: binomial series of (1 + j)^(-2/3) for
    // |j| < 0.1 (terms to j^8, truncation below 4e-9 relative), else expm1(-2/3 log1p(j))
    float Jm23m1;
    if (fabsf(jel) < 0.1f) {
        Jm23m1 = jel * (-0.66666667f + jel * (0.55555556f + jel * (-0.49382716f + jel * (0.45267490f +
                 jel * (-0.42249657f + jel * (0.39902454f + jel * (-0.38002337f + jel * 0.36418906f)))))));
    } else {
        Jm23m1 = expm1f(-(2.f / 3.f) * log1pf(jel));
    }
    const float Jm23 = 1.f + Jm23m1;
    // isochoric part: mu J^-2/3 (I - I1/3 C^-1) = 2 mu J^-2/3 C^-1 dev(E_el)
    const float tr3 = (Ee[0] + Ee[1] + Ee[2]) * (1.f / 3.f);
    const float D[6] = {Ee[0] - tr3, Ee[1] - tr3, Ee[2] - tr3, Ee[3], Ee[4], Ee[5]};
    float M[6];  // C^-1 dev(E), symmetric (the two commute)
    M[0] = Ci[0] * D[0] + Ci[3] * D[3] + Ci[5] * D[5];
    M[1] = Ci[3] * D[3] + Ci[1] * D[1] + Ci[4] * D[4];
    M[2] = Ci[5] * D[5] + Ci[4] * D[4] + Ci[2] * D[2];
    M[3] = Ci[0] * D[3] + Ci[3] * D[1] + Ci[5] * D[4];
    M[4] = Ci[3] * D[5] + Ci[1] * D[4] + Ci[4] * D[2];
    M[5] = Ci[0] * D[5] + Ci[3] * D[4] + Ci[5] * D[2];
    // fibre term: I4b - 1 = (J^-2/3 - 1) + 2 J^-2/3 a.E_el.a
    const float aEa = ax * ax * Ee[0] + ay * ay * Ee[1] + az * az * Ee[2] +
                      2.f * (ax * ay * Ee[3] + ay * az * Ee[4] + ax * az * Ee[5]);
    const float I4 = 1.f + 2.f * aEa;
    const float x4 = Jm23m1 + 2.f * Jm23 * aEa;
    const float psi4 = k1 * x4 * __expf(k2 * x4 * x4);
    const float cf = 2.f * psi4 * Jm23;
    const float cI4 = I4 * (1.f / 3.f);
    const float ciso = 2.f * mu * Jm23;
    const float cvol = kap * Jel * jel;
    const float aa[6] = {ax * ax, ay * ay, az * az, ax * ay, ay * az, ax * az};
    // S_0 = lambda S_i (Eq. 10 for F_th = lambda I), then Prony: S~ = S_0 - sum theta_p
    float St[6];
#pragma unroll
    for (int s = 0; s < 6; s++) St[s] = lam * (ciso * M[s] + cvol * Ci[s] + cf * (aa[s] - cI4 * Ci[s]));
    if constexpr (ANI) {
        // Eq. (10): S_0 = det F_th F_th^-1 S_i F_th^-T = lambda_m [S_i - g (m Sm + Sm m) + g^2 (m.S.m) m m]
#pragma unroll
        for (int s = 0; s < 6; s++) St[s] = ciso * M[s] + cvol * Ci[s] + cf * (aa[s] - cI4 * Ci[s]);  // S_i
        const float Smx = St[0] * ax + St[3] * ay + St[5] * az;
        const float Smy = St[3] * ax + St[1] * ay + St[4] * az;
        const float Smz = St[5] * ax + St[4] * ay + St[2] * az;
        const float g2 = gam * gam * (ax * Smx + ay * Smy + az * Smz);
        St[0] = lm * (St[0] - 2.f * gam * ax * Smx + g2 * ax * ax);
        St[1] = lm * (St[1] - 2.f * gam * ay * Smy + g2 * ay * ay);
        St[2] = lm * (St[2] - 2.f * gam * az * Smz + g2 * az * az);
        St[3] = lm * (St[3] - gam * (ax * Smy + Smx * ay) + g2 * ax * ay);
        St[4] = lm * (St[4] - gam * (ay * Smz + Smy * az) + g2 * ay * az);
        St[5] = lm * (St[5] - gam * (ax * Smz + Smx * az) + g2 * ax * az);
    }
    {
        float S0[6];
#pragma unroll
        for (int s = 0; s < 6; s++) S0[s] = St[s];
#pragma unroll
        for (int p = 0; p < NPR; p++) {
#pragma unroll
            for (int s = 0; s < 6; s++) {
                const float tp = SP.pr_a[p] * S0[s] + SP.pr_b[p] * E.vs[p][s];
                gvisc[(p * 6 + s) * kTile] = tp;
                St[s] -= tp;
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
            Qm[i][k] = BRICK ? sV * (P[i][k] * Ji[4 * k])
                             : sV * (P[i][0] * Ji[3 * k] + P[i][1] * Ji[3 * k + 1] + P[i][2] * Ji[3 * k + 2]);
    // thermal: q = k J C^-1 grad0 theta = k lambda J_el C_el^-1 grad0 theta (Eq. 16);
    // fT_a = V dh_a/dX . q = r . Xi_a with r = s V J0^-1 q
    float kT = kc;
    if (A.flags & TLED_TEMP_DEP) kT *= 1.f + A.beta_k * (the - A.Tref_m_T0);
    float q0, q1, q2;
    if constexpr (ANI) {
        // J C^-1 = det F_th J_el F_th^-1 C_el^-1 F_th^-T, plus the conduction along the current
        // fibre a = F m / |F m|: F^-1 (k_f - k) a a F^-T = (k_f - k) m m / (m.C.m), m.C.m = 1 + 2 m.E.m
        const float mg = ax * gth[0] + ay * gth[1] + az * gth[2];
        const float p0 = il * (gth[0] - gam * mg * ax), p1 = il * (gth[1] - gam * mg * ay), p2 = il * (gth[2] - gam * mg * az);
        const float c0 = Ci[0] * p0 + Ci[3] * p1 + Ci[5] * p2;
        const float c1 = Ci[3] * p0 + Ci[1] * p1 + Ci[4] * p2;
        const float c2 = Ci[5] * p0 + Ci[4] * p1 + Ci[2] * p2;
        const float mc = ax * c0 + ay * c1 + az * c2;
        const float kq = kT * det_th * Jel * il;
        const float kf = __fdividef(kT * (A.ani_k - 1.f) * (1.f + Jm1) * mg, 1.f + 2.f * mEm);
        q0 = kq * (c0 - gam * mc * ax) + kf * ax;
        q1 = kq * (c1 - gam * mc * ay) + kf * ay;
        q2 = kq * (c2 - gam * mc * az) + kf * az;
    } else {
        const float kq = kT * lam * Jel;
        q0 = kq * (Ci[0] * gth[0] + Ci[3] * gth[1] + Ci[5] * gth[2]);
        q1 = kq * (Ci[3] * gth[0] + Ci[1] * gth[1] + Ci[4] * gth[2]);
        q2 = kq * (Ci[5] * gth[0] + Ci[4] * gth[1] + Ci[2] * gth[2]);
    }
    float r[3];
    if constexpr (BRICK) {
        r[0] = sV * (Ji[0] * q0); r[1] = sV * (Ji[4] * q1); r[2] = sV * (Ji[8] * q2);
    } else {
#pragma unroll
        for (int k = 0; k < 3; k++) r[k] = sV * (Ji[3 * k] * q0 + Ji[3 * k + 1] * q1 + Ji[3 * k + 2] * q2);
    }

    if constexpr (NPE == 8) {
        // hourglass control: gamma_a,al = h_a,al - c_al . dh_a/dX with c_al = sum_b h_b,al X_b;
        // f_a += k_hg sum_al gamma_a,al q_al with q_al = sum_b h_b,al u_b - H c_al (thermal alike)
        float jn2 = 0.f;
#pragma unroll
        for (int q = 0; q < 9; q++)
            if (!BRICK || q % 4 == 0) jn2 += Ji[q] * Ji[q];
        const float khg = A.khg * (kap + (4.f / 3.f) * mu) * V * jn2 * (1.f / 64.f);
        const float khgT = A.khgT * kT * V * jn2 * (1.f / 64.f);
        float qa[4][3], qT[4];
        // general hexahedra: the hourglass modes of u, theta and X, transformed again from
        // shared memory (the empty asm keeps the compiler from carrying the first transform's
        // values across the stress evaluation, where the registers are scarcest)
        float cX[4][3];
        if constexpr (!BRICK) {
            asm volatile("" ::: "memory");
            float wx[8], wy[8], wz[8], wt[8], px[8], py[8], pz[8];
            h8_modes<true>(cl, s_xu, s_X, wx, wy, wz, wt, px, py, pz);
            hu[0][0] = wx[3]; hu[1][0] = wx[6]; hu[2][0] = wx[5]; hu[3][0] = -wx[7];
            hu[0][1] = wy[3]; hu[1][1] = wy[6]; hu[2][1] = wy[5]; hu[3][1] = -wy[7];
            hu[0][2] = wz[3]; hu[1][2] = wz[6]; hu[2][2] = wz[5]; hu[3][2] = -wz[7];
            ht[0] = wt[3]; ht[1] = wt[6]; ht[2] = wt[5]; ht[3] = -wt[7];
            cX[0][0] = px[3]; cX[1][0] = px[6]; cX[2][0] = px[5]; cX[3][0] = -px[7];
            cX[0][1] = py[3]; cX[1][1] = py[6]; cX[2][1] = py[5]; cX[3][1] = -py[7];
            cX[0][2] = pz[3]; cX[1][2] = pz[6]; cX[2][2] = pz[5]; cX[3][2] = -pz[7];
        }
        if constexpr (BRICK) {  // c_al = 0: gamma_a,al = h_a,al and q_al = sum_b h_b,al u_b
#pragma unroll
            for (int l = 0; l < 4; l++) {
                qa[l][0] = hu[l][0]; qa[l][1] = hu[l][1]; qa[l][2] = hu[l][2];
                qT[l] = ht[l];
            }
        } else {
            float Wm[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
            float wT[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int l = 0; l < 4; l++) {
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    qa[l][i] = hu[l][i] - (H[i][0] * cX[l][0] + H[i][1] * cX[l][1] + H[i][2] * cX[l][2]);
#pragma unroll
                    for (int j = 0; j < 3; j++) Wm[i][j] += qa[l][i] * cX[l][j];
                }
                qT[l] = ht[l] - (cX[l][0] * gth[0] + cX[l][1] * gth[1] + cX[l][2] * gth[2]);
                wT[0] += qT[l] * cX[l][0]; wT[1] += qT[l] * cX[l][1]; wT[2] += qT[l] * cX[l][2];
            }
            // fold the -k_hg W dh_a/dX part into Q and r
            const float kh8 = 0.125f * khg, kT8 = 0.125f * khgT;
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int k = 0; k < 3; k++)
                    Qm[i][k] -= kh8 * (Wm[i][0] * Ji[3 * k] + Wm[i][1] * Ji[3 * k + 1] + Wm[i][2] * Ji[3 * k + 2]);
#pragma unroll
            for (int k = 0; k < 3; k++) r[k] -= kT8 * (Ji[3 * k] * wT[0] + Ji[3 * k + 1] * wT[1] + Ji[3 * k + 2] * wT[2]);
        }
        // corner values by the inverse transform of the sign-vector coefficients
        float fx[8], fy[8], fz[8], ft[8];
        fx[0] = 0.f; fx[1] = -Qm[0][0]; fx[2] = -Qm[0][1]; fx[4] = -Qm[0][2];
        fx[3] = khg * qa[0][0]; fx[6] = khg * qa[1][0]; fx[5] = khg * qa[2][0]; fx[7] = -khg * qa[3][0];
        fy[0] = 0.f; fy[1] = -Qm[1][0]; fy[2] = -Qm[1][1]; fy[4] = -Qm[1][2];
        fy[3] = khg * qa[0][1]; fy[6] = khg * qa[1][1]; fy[5] = khg * qa[2][1]; fy[7] = -khg * qa[3][1];
        fz[0] = 0.f; fz[1] = -Qm[2][0]; fz[2] = -Qm[2][1]; fz[4] = -Qm[2][2];
        fz[3] = khg * qa[0][2]; fz[6] = khg * qa[1][2]; fz[5] = khg * qa[2][2]; fz[7] = -khg * qa[3][2];
        ft[0] = 0.f; ft[1] = -r[0]; ft[2] = -r[1]; ft[4] = -r[2];
        ft[3] = khgT * qT[0]; ft[6] = khgT * qT[1]; ft[5] = khgT * qT[2]; ft[7] = -khgT * qT[3];
        float2 fxy[8], fzt[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            fxy[i] = make_float2(fx[i], fy[i]);
            fzt[i] = make_float2(fz[i], ft[i]);
        }
        wht8x2(fxy); wht8x2(fzt);
#pragma unroll
        for (int i = 0; i < 8; i++)
            slot[slot_pos(ec, wht_corner(i))] = make_float4(fxy[i].x, fxy[i].y, fzt[i].x, fzt[i].y);
    } else {
        // T4: dh_0 = -(dh_1 + dh_2 + dh_3), dh_{j+1} = row j of J0^-1
        slot[slot_pos(ec, 0)] = make_float4(-(Qm[0][0] + Qm[0][1] + Qm[0][2]), -(Qm[1][0] + Qm[1][1] + Qm[1][2]),
                               -(Qm[2][0] + Qm[2][1] + Qm[2][2]), -(r[0] + r[1] + r[2]));
#pragma unroll
        for (int j = 0; j < 3; j++) slot[slot_pos(ec, 1 + j)] = make_float4(Qm[0][j], Qm[1][j], Qm[2][j], r[j]);
    }
}

// ---------------------------------------------------------------------------
// tile kernel (persistent: CTA b handles tiles b, b + gridDim.x, ...)
// ---------------------------------------------------------------------------

struct TileInfo {
    int e0, ne_t, ib, n_int, nl, sh_off, pat, npe;  // pat: structure record id
};
__device__ __forceinline__ TileInfo tile_info(const StepArgs &A, int t) {
    const int4 a = __ldg(reinterpret_cast<const int4 *>(A.tile_info) + 2 * t);
    const int4 b = __ldg(reinterpret_cast<const int4 *>(A.tile_info) + 2 * t + 1);
    return TileInfo{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
}
// bytes of a tile's element record (float components; the stride is rec_bytes)
__device__ __forceinline__ uint32_t rec_len(const StepArgs &A) { return (uint32_t)((A.n_comp - 6 * A.n_prony) * kTile * 4); }

__device__ __forceinline__ uint32_t visc_tile_bytes(const StepArgs &A) { return (uint32_t)(A.n_prony * 6 * kTile * 4); }

// element record + Prony state of tile t -> buf
__device__ __forceinline__ void stage_elem(const StepArgs &A, int t, char *buf, uint64_t *bar) {
    const uint32_t rb = rec_len(A), vb = visc_tile_bytes(A);
    mbar_expect_tx(bar, rb + vb);
    bulk_g2s(buf, A.elem_rec + (int64_t)t * A.rec_bytes, rb, bar);
    if (vb) bulk_g2s(buf + rb, A.visc + (int64_t)t * (vb / 4), vb, bar);
}
// structure record and interior (u, theta, X0) of tile T; the record is left out when the
// buffer already holds it (have_pat: the previous tile named the same record, the norm in
// block and voxel meshes, whose tiles share a few records)
template <int NPE>
__device__ __forceinline__ void stage_nodes(const StepArgs &A, const TileInfo &T, char *smem, uint64_t *bar,
                                            bool have_pat = false) {
    const uint32_t cb = have_pat ? 0u : (uint32_t)pattern_u16(NPE ? NPE : T.npe) * 2;
    mbar_expect_tx(bar, cb + 32u * T.n_int);
    if (cb) bulk_g2s(smem + A.sm_pat, A.pattern + (int64_t)T.pat * A.pat_stride, cb, bar);
    if (T.n_int > 0) {
        bulk_g2s(smem + A.sm_xu, A.xu + T.ib, 16u * T.n_int, bar);
        bulk_g2s(smem + A.sm_X, A.X0 + T.ib, 16u * T.n_int, bar);
    }
}
// shared-node lists of tile T (global index, partial position; they start on 16-byte
// boundaries, the copy is rounded up to 4 entries) into list buffer b: two buffers, so that
// the next tile's lists arrive while this tile still reads its own
template <int NPE>
__device__ __forceinline__ int *list_buf(const StepArgs &A, char *smem, int b) {
    return reinterpret_cast<int *>(smem + A.sm_sh) + b * 2 * max_local(NPE);
}
template <int NPE>
__device__ __forceinline__ void stage_lists(const StepArgs &A, const TileInfo &T, char *smem, int b, uint64_t *bar) {
    const uint32_t sb = 4u * (uint32_t)((T.nl - T.n_int + 3) & ~3);
    mbar_expect_tx(bar, 2u * sb);  // 0 bytes: the arrival alone completes the phase
    if (sb) {
        int *lb = list_buf<NPE>(A, smem, b);
        bulk_g2s(lb, A.tile_shared + T.sh_off, sb, bar);
        bulk_g2s(lb + max_local(NPE), A.part_pos + T.sh_off, sb, bar);
    }
}
// the shared nodes' (u, theta) (and, for general elements, X0) of tile T by 16-byte
// asynchronous copies (mostly L2 hits), from list buffer lb; completion by cp_async_wait_all
template <int NPE, bool BRICK>
__device__ __forceinline__ void gather_shared(const StepArgs &A, const TileInfo &T, const int *lb, float4 *s_xu,
                                              float4 *s_X) {
    for (int l = T.n_int + threadIdx.x; l < T.nl; l += kBlock) {
        const int64_t g = lb[l - T.n_int];
        cp_async16(&s_xu[l], &A.xu[g]);
        if constexpr (!BRICK) cp_async16(&s_X[l], &A.X0[g]);  // bricks: only interior X0 is read
    }
}

// fixed-order sum of local node l's corner slots (ascending corner, element): two
// running sums (even and odd entries), each as (x, y) and (z, w) pairs
__device__ __forceinline__ float4 gather_node(const float4 *slot, const uint16_t *s_code, const uint16_t *s_row, int l) {
    int r = s_row[l];
    const int r1 = s_row[l + 1];
    float2 a0 = make_float2(0.f, 0.f), b0 = a0, a1 = a0, b1 = a0;
    for (; r + 1 < r1; r += 2) {
        const float4 v0 = slot[s_code[r]];
        const float4 v1 = slot[s_code[r + 1]];
        a0 = add2(a0, make_float2(v0.x, v0.y)); b0 = add2(b0, make_float2(v0.z, v0.w));
        a1 = add2(a1, make_float2(v1.x, v1.y)); b1 = add2(b1, make_float2(v1.z, v1.w));
    }
    if (r < r1) {
        const float4 v0 = slot[s_code[r]];
        a0 = add2(a0, make_float2(v0.x, v0.y)); b0 = add2(b0, make_float2(v0.z, v0.w));
    }
    const float2 sxy = add2(a0, a1), szw = add2(b0, b1);
    return make_float4(sxy.x, sxy.y, szw.x, szw.y);
}

// CPS: resident CTAs per SM the instance is built for (its register budget)
template <int NPE, int NPR, bool ANI, bool BRICK, int CPS>
__global__ void __launch_bounds__(kBlock, CPS) tile_step_kernel(const StepArgs A, const int k) {
    extern __shared__ __align__(128) char smem[];
    __shared__ ScenStep S;
    __shared__ int s_abort;
    const uint16_t *s_pat = reinterpret_cast<const uint16_t *>(smem + A.sm_pat);  // structure record
    float4 *s_xu = reinterpret_cast<float4 *>(smem + A.sm_xu);
    float4 *s_X = reinterpret_cast<float4 *>(smem + A.sm_X);
    float4 *ns = reinterpret_cast<float4 *>(smem + A.sm_ns);
    // [0] element buffer, [1] shared-node lists, [2] structure record and interior nodes, [3] node state
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + A.sm_bar);
    const int G = gridDim.x;

    const int n_tiles = min(*A.n_active, A.n_tiles);  // tiles of unfinished scenarios form a prefix
    TileInfo T{};
    int scn = 0;
    if ((int)blockIdx.x < n_tiles) {
        T = tile_info(A, blockIdx.x);
        scn = __ldg(A.tile_scn + blockIdx.x);
    }
    if (threadIdx.x == 0) {
        for (int b = 0; b < 4; b++) mbar_init(&bar[b], 1);
        fence_barrier_init();
        s_abort = 0;
        if ((int)blockIdx.x < n_tiles) {
            stage_elem(A, blockIdx.x, smem, &bar[0]);
            if (A.stage_skip != 1 + (int)blockIdx.x) stage_nodes<NPE>(A, T, smem, &bar[2]);
            stage_lists<NPE>(A, T, smem, 0, &bar[1]);
        }
    }
    __syncthreads();  // barrier init visible to all
    // the first tile's shared nodes; a thread reads a list only once it has seen its copy complete
    bool ok1 = true;
    if ((int)blockIdx.x < n_tiles) {
        ok1 = mbar_wait(&bar[1], 0);
        if (ok1) gather_shared<NPE, BRICK>(A, T, list_buf<NPE>(A, smem, 0), s_xu, s_X);
    }
    uint32_t ph_s = 0;
    int i = 0, cur_scn = -1;
    for (int t = blockIdx.x; t < n_tiles; t += G, i++) {
        // the records of the next tile, loaded here so that their latency hides behind this
        // tile (an L2 prefetch of the tile after next was measured slower: 151.4 against 147.2
        // us per 128^3 step, the general H8 instance 195.5 against 185.3)
        const bool has_next = t + G < n_tiles;
        TileInfo Tn = T;
        int scn_n = scn;
        if (has_next) {
            Tn = tile_info(A, t + G);
            scn_n = __ldg(A.tile_scn + t + G);
        }
        const int npe = NPE ? NPE : T.npe;
        const uint16_t *s_code = s_pat + kTile * npe;  // gather slot offsets
        const uint16_t *s_row = s_code + kTile * npe;   // and their row offsets
        char *buf = smem;  // element inputs, then this tile's corner slots
        float4 *slot = reinterpret_cast<float4 *>(buf);
        const bool ns_smem = T.n_int > 0 && T.n_int <= kNsMax;
        if (scn != cur_scn) {  // published by the barrier after the element inputs are read
            prepare_scen(A, scn, k, S, threadIdx.x, kBlock);
            cur_scn = scn;
        }
        const int *s_shg = list_buf<NPE>(A, smem, i & 1);  // shared node -> global index
        const int *s_ppos = s_shg + max_local(NPE);        // shared node -> partial position
        // ---- 1. structure record and interior nodes, element record (bulk copies); the shared
        //         nodes' gathers were issued with those copies (or before the loop)
        const bool ok2 = mbar_wait(&bar[2], i & 1);
        const bool ok0 = mbar_wait(&bar[0], i & 1);
        if (!(ok0 && ok2 && ok1)) {
            atomicOr(A.status, kStatusTimeout);
            s_abort = 1;
        }
        // ---- 2. element inputs -> registers; the buffer then becomes the slot buffer
        const int ec = threadIdx.x;
        const bool active = ec < T.ne_t;
        int cl[NPE ? NPE : 8];
        ElemIn<NPR> E;
        if (active) {
            if constexpr (NPE != 0) load_elem<NPE, NPR, BRICK>(A, buf, s_pat, ec, cl, E);
            else if (npe == 8) load_elem<8, NPR>(A, buf, s_pat, ec, cl, E);
            else load_elem<4, NPR>(A, buf, s_pat, ec, cl, E);
        }
        cp_async_wait_all();
        __syncthreads();
        if (s_abort) {  // the status says why; no copy of this CTA may still be in flight when it leaves
            if (threadIdx.x == 0) {
                mbar_wait(&bar[0], i & 1);
                mbar_wait(&bar[2], i & 1);
                mbar_wait(&bar[1], i & 1);
            }
            return;
        }
        if (threadIdx.x == 0) {
            fence_proxy_async();
            if (has_next) stage_lists<NPE>(A, Tn, smem, (i + 1) & 1, &bar[1]);  // the other buffer is free
            if (ns_smem) {
                mbar_expect_tx(&bar[3], 48u * T.n_int);
                bulk_g2s(ns, A.lo + T.ib, 16u * T.n_int, &bar[3]);
                bulk_g2s(ns + T.n_int, A.vel + T.ib, 16u * T.n_int, &bar[3]);
                bulk_g2s(ns + 2 * T.n_int, A.nodec + T.ib, 16u * T.n_int, &bar[3]);
            }
        }
        // ---- 3. element pass
        if (active) {
            float *gv = A.visc + (int64_t)t * A.n_prony * 6 * kTile + ec;
            if constexpr (NPE != 0) element_step<NPE, NPR, ANI, BRICK>(A, S, (int64_t)t * kTile + ec, ec, cl, E, s_xu, s_X, slot, gv);
            else if (npe == 8) element_step<8, NPR, ANI, false>(A, S, (int64_t)t * kTile + ec, ec, cl, E, s_xu, s_X, slot, gv);
            else element_step<4, NPR, ANI, false>(A, S, (int64_t)t * kTile + ec, ec, cl, E, s_xu, s_X, slot, gv);
        }
        __syncthreads();
        // ---- 4. fixed-order gather into nodes, nodal update; shared nodes: partial sum
        bool ok3 = true;
        if (ns_smem) {
            ok3 = mbar_wait(&bar[3], ph_s);
            if (!ok3) {
                atomicOr(A.status, kStatusTimeout);
                s_abort = 1;
            }
        }
        for (int l = threadIdx.x; l < T.nl && ok3; l += kBlock) {
            const float4 acc = gather_node(slot, s_code, s_row, l);
            if (l < T.n_int) {
                const int64_t g = (int64_t)T.ib + l;
                float4 lo, vo, nc;
                if (ns_smem) {
                    lo = ns[l]; vo = ns[T.n_int + l]; nc = ns[2 * T.n_int + l];
                } else {
                    lo = A.lo[g]; vo = A.vel[g]; nc = __ldg(&A.nodec[g]);
                }
                node_update(A, S, g, acc, s_xu[l], s_X[l], lo, vo, nc);
            } else {
                A.partials[s_ppos[l - T.n_int]] = acc;
            }
        }
        __syncthreads();
        if (s_abort) {  // a node-state copy timed out: wait (bounded) for it and the next lists, then leave
            if (threadIdx.x == 0) {
                mbar_wait(&bar[3], ph_s);
                if (has_next) mbar_wait(&bar[1], (i + 1) & 1);
            }
            return;
        }
        ph_s ^= (uint32_t)ns_smem;
        // ---- 5. stage the next tile's element record (into the consumed slot buffer), structure
        //         record and interior nodes, and gather its shared nodes at the same time
        if (has_next) {
            if (threadIdx.x == 0) {
                fence_proxy_async();
                stage_elem(A, t + G, smem, &bar[0]);
                stage_nodes<NPE>(A, Tn, smem, &bar[2], Tn.pat == T.pat);
            }
            ok1 = mbar_wait(&bar[1], (i + 1) & 1);
            if (ok1) gather_shared<NPE, BRICK>(A, Tn, list_buf<NPE>(A, smem, (i + 1) & 1), s_xu, s_X);
        }
        T = Tn;
        scn = scn_n;
    }
}

// Nodes touched by several tiles: sum the node's partial sums in tile order,
// then the same nodal update as the tile kernel.  Persistent: block b takes the
// 256-node chunks b, b + gridDim.x, ...; the scenario's step values are
// prepared only when a chunk's first node belongs to another scenario than the
// previous chunk's (once per launch for a single problem).
__global__ void __launch_bounds__(256) shared_step_kernel(const StepArgs A, const int k) {
    __shared__ ScenStep S;
    const int64_t n_sh = min((int64_t)A.n_active[1], A.n_shared);  // shared nodes of unfinished scenarios: a prefix
    const bool multi = A.n_scn > 1;      // a batch: nodes carry their scenario
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int cur = -1;
    // the node's partial-sum range, loaded one chunk ahead so that the partial sums
    // themselves can be requested as soon as a chunk starts
    int64_t c0 = (int64_t)blockIdx.x * blockDim.x;
    int rn0 = 0, rn1 = 0;
    if (c0 + threadIdx.x < n_sh) {
        rn0 = __ldg(A.sh_rowptr + c0 + threadIdx.x);
        rn1 = __ldg(A.sh_rowptr + c0 + threadIdx.x + 1);
    }
    for (; c0 < n_sh; c0 += stride) {
        const int64_t s = c0 + threadIdx.x;
        const bool live = s < n_sh;
        const int r0 = rn0, r1 = rn1;
        rn0 = 0;
        rn1 = 0;
        if (s + stride < n_sh) {
            rn0 = __ldg(A.sh_rowptr + s + stride);
            rn1 = __ldg(A.sh_rowptr + s + stride + 1);
        }
        // every load of the node issued up front: its state, then its first four partial
        // sums (a node of a tile-boundary face has 2, of an edge 4); more follow in order
        const int64_t g = A.n_interior + (live ? s : c0);
        const float4 xu = A.xu[g], X = __ldg(&A.X0[g]), lo = A.lo[g], vo = A.vel[g], nc = __ldg(&A.nodec[g]);
        const int scn = !multi ? 0 : live ? __ldg(A.shared_scn + s) : -1;
        float4 c[4];
#pragma unroll
        for (int j = 0; j < 4; j++) c[j] = r0 + j < r1 ? A.partials[r0 + j] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int scn0 = multi ? __ldg(A.shared_scn + c0) : 0;  // the chunk's first node's scenario (block-uniform)
        if (scn0 != cur) {
            __syncthreads();  // nobody still reads the previous step values
            prepare_scen(A, scn0, k, S, threadIdx.x, blockDim.x);
            __syncthreads();
            cur = scn0;
        }
        if (!live) continue;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 4; j++) {  // the node's partial sums, in tile order (adding 0 changes nothing)
            acc.x += c[j].x; acc.y += c[j].y; acc.z += c[j].z; acc.w += c[j].w;
        }
        for (int r = r0 + 4; r < r1; r++) {
            const float4 d = A.partials[r];
            acc.x += d.x; acc.y += d.y; acc.z += d.z; acc.w += d.w;
        }
        if (scn == scn0) {
            node_update(A, S, g, acc, xu, X, lo, vo, nc);
        } else {  // chunk spans a scenario boundary: this thread's own step values
            ScenStep L;
            prepare_scen(A, scn, k, L, 0, 1);
            node_update(A, L, g, acc, xu, X, lo, vo, nc);
        }
    }
}

// ---------------------------------------------------------------------------
// resident mode: one CTA per scenario holds the whole scenario in shared memory
// and runs K steps.  Per step, the scenario's tiles two at a time (two lanes of
// 256 threads: element pass, fixed-order gather, interior node updates, partial
// sums of shared nodes -- two tiles share no interior node), then its shared
// nodes (partials in tile order): the arithmetic and its order are those of the
// tile and shared-node kernels.
// ---------------------------------------------------------------------------
template <int NPE, int NPR, bool ANI, bool BRICK>
__global__ void __launch_bounds__(kResBlock, 1) resident_step_kernel(const StepArgs A, const int K) {
    extern __shared__ __align__(128) char smem[];
    __shared__ ScenStep S;
    const ResDesc D = A.res[blockIdx.x];
    if (D.t0 >= *A.n_active) return;  // a finished scenario (active tiles form a prefix)
    float4 *r_xu = reinterpret_cast<float4 *>(smem + A.rs_xu);
    float4 *r_lo = reinterpret_cast<float4 *>(smem + A.rs_lo);
    float4 *r_vel = reinterpret_cast<float4 *>(smem + A.rs_vel);
    float4 *r_X = reinterpret_cast<float4 *>(smem + A.rs_X);
    float4 *r_nc = reinterpret_cast<float4 *>(smem + A.rs_nc);
    int *r_rowptr = reinterpret_cast<int *>(smem + A.rs_rowptr);
    float4 *r_part = reinterpret_cast<float4 *>(smem + A.rs_part);
    const int tid = threadIdx.x;
    const int lane = tid / kBlock, lt = tid % kBlock;  // tile lane, thread within it
    float4 *slot = reinterpret_cast<float4 *>(smem + A.rs_slot) + lane * kTile * NPE;
    const int nn_s = D.n_int + D.n_sh;
    const int nfix = A.n_comp - 6 * A.n_prony;  // record floats before the Prony state
    // scenario-local node q: interior nodes first, then shared nodes
    auto gnode = [&](int q) -> int64_t { return q < D.n_int ? (int64_t)D.i0 + q : A.n_interior + D.s0 + (q - D.n_int); };

    // ---- the scenario into shared memory: node state, and per tile its element record and
    //      Prony state, its connectivity in scenario-local node numbers, gather lists and
    //      shared-node partial positions
    for (int q = tid; q < nn_s; q += kResBlock) {
        const int64_t g = gnode(q);
        r_xu[q] = A.xu[g];
        r_lo[q] = A.lo[g];
        r_vel[q] = A.vel[g];
        r_X[q] = __ldg(&A.X0[g]);
        r_nc[q] = __ldg(&A.nodec[g]);
    }
    for (int q = tid; q <= D.n_sh; q += kResBlock) r_rowptr[q] = __ldg(A.sh_rowptr + D.s0 + q) - D.p0;
    for (int j = 0; j < D.n_t; j++) {
        const int t = D.t0 + j;
        const TileInfo T = tile_info(A, t);
        char *blk = smem + A.rs_tiles + j * A.rs_tile;
        float *rec = reinterpret_cast<float *>(blk);
        const float *grec = reinterpret_cast<const float *>(A.elem_rec + (int64_t)t * A.rec_bytes);
        for (int i = tid; i < nfix * kTile; i += kResBlock) rec[i] = __ldg(grec + i);
        const float *gvs = A.visc + (int64_t)t * A.n_prony * 6 * kTile;
        for (int i = tid; i < 6 * A.n_prony * kTile; i += kResBlock) rec[nfix * kTile + i] = gvs[i];
        const uint16_t *pat = A.pattern + (int64_t)T.pat * A.pat_stride;
        uint16_t *conn = reinterpret_cast<uint16_t *>(blk + A.rt_conn);
        for (int i = tid; i < kTile * NPE; i += kResBlock) {
            int q = 0;
            if (i < T.ne_t * NPE) {
                const int l = pat[i];
                q = l < T.n_int ? (T.ib - D.i0) + l
                                : D.n_int + (__ldg(A.tile_shared + T.sh_off + l - T.n_int) - (int)A.n_interior - D.s0);
            }
            conn[i] = (uint16_t)q;
        }
        uint16_t *codes = reinterpret_cast<uint16_t *>(blk + A.rt_codes);
        for (int i = tid; i < kTile * NPE + kMaxLocal + 8; i += kResBlock) codes[i] = pat[kTile * NPE + i];
        int *ppos = reinterpret_cast<int *>(blk + A.rt_ppos);
        for (int m = tid; m < T.nl - T.n_int; m += kResBlock) ppos[m] = __ldg(A.part_pos + T.sh_off + m) - D.p0;
        if (tid == 0) {
            int *ti = reinterpret_cast<int *>(blk + A.rt_info);
            ti[0] = T.ne_t; ti[1] = T.ib - D.i0; ti[2] = T.n_int; ti[3] = T.nl;
        }
    }
    __syncthreads();

    // ---- K steps
    for (int k = 0; k < K; k++) {
        prepare_scen(A, D.scn, k, S, tid, kResBlock);
        __syncthreads();
        for (int j0 = 0; j0 < D.n_t; j0 += kResLanes) {
            const int j = j0 + lane;
            const bool on = j < D.n_t;  // this lane has a tile in this pass
            char *blk = smem + A.rs_tiles + (on ? j : j0) * A.rs_tile;
            const int *ti = reinterpret_cast<const int *>(blk + A.rt_info);
            const int ne_t = on ? ti[0] : 0, q0 = on ? ti[1] : 0, n_int = on ? ti[2] : 0, nl = on ? ti[3] : 0;
            const uint16_t *codes = reinterpret_cast<const uint16_t *>(blk + A.rt_codes);
            const uint16_t *rows = codes + kTile * NPE;
            const int *ppos = reinterpret_cast<const int *>(blk + A.rt_ppos);
            if (lt < ne_t) {
                int cl[NPE];
                ElemIn<NPR> E;
                load_elem<NPE, NPR, BRICK>(A, blk, reinterpret_cast<const uint16_t *>(blk + A.rt_conn), lt, cl, E);
                element_step<NPE, NPR, ANI, BRICK>(A, S, (int64_t)(D.t0 + j) * kTile + lt, lt, cl, E, r_xu, r_X, slot,
                                                   reinterpret_cast<float *>(blk) + nfix * kTile + lt);
            }
            __syncthreads();
            for (int l = lt; l < nl; l += kBlock) {
                const float4 acc = gather_node(slot, codes, rows, l);
                if (l < n_int) {
                    const int q = q0 + l;
                    node_advance(A, S, (int64_t)D.i0 + q, acc, r_xu[q], r_X[q], r_lo[q], r_vel[q], r_nc[q], r_xu[q], r_lo[q],
                                 r_vel[q]);
                } else {
                    r_part[ppos[l - n_int]] = acc;
                }
            }
            __syncthreads();
        }
        for (int q = tid; q < D.n_sh; q += kResBlock) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int r = r_rowptr[q]; r < r_rowptr[q + 1]; r++) {
                const float4 d = r_part[r];
                acc.x += d.x; acc.y += d.y; acc.z += d.z; acc.w += d.w;
            }
            const int qq = D.n_int + q;
            node_advance(A, S, A.n_interior + D.s0 + q, acc, r_xu[qq], r_X[qq], r_lo[qq], r_vel[qq], r_nc[qq], r_xu[qq],
                         r_lo[qq], r_vel[qq]);
        }
        __syncthreads();
    }

    // ---- state back to global memory
    for (int q = tid; q < nn_s; q += kResBlock) {
        const int64_t g = gnode(q);
        A.xu[g] = r_xu[q];
        A.lo[g] = r_lo[q];
        A.vel[g] = r_vel[q];
    }
    for (int j = 0; j < D.n_t; j++) {
        const float *rec = reinterpret_cast<const float *>(smem + A.rs_tiles + j * A.rs_tile);
        float *gvs = A.visc + (int64_t)(D.t0 + j) * A.n_prony * 6 * kTile;
        for (int i = tid; i < 6 * A.n_prony * kTile; i += kResBlock) gvs[i] = rec[nfix * kTile + i];
    }
}

// ---------------------------------------------------------------------------
// grid-resident mode (single problems whose tiles all fit co-resident CTAs): a
// cooperative launch of one CTA per tile runs K steps.  The tile's element record,
// Prony state, structure record, shared-node lists, reference coordinates and the
// state of all its nodes stay in the CTA's shared memory.  Per step the CTA runs
// the element pass and the node phase (interior nodes updated in shared memory,
// shared nodes' partial sums to global memory, double-buffered by step parity);
// after one grid barrier every CTA updates its own copy of each of its shared
// nodes from all the node's partial sums in tile order -- the copies of a node
// in different CTAs are computed from the same values in the same order and stay
// identical, and only the node's first tile writes it back and adds its dose.
// Same functions and order as the tile and shared-node kernels.
// ---------------------------------------------------------------------------
// Grid barrier over all CTAs of a cooperative launch: a monotonic arrival count in
// global memory (zeroed before the launch); barrier j opens when it reaches
// j * gridDim.x.  Arrival with release semantics (the CTA's writes, ordered by the
// block barrier, before it), acquire on the wait; the wait is bounded (about a
// second), after which the CTA flags the device status and reports failure.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ bool grid_barrier(const StepArgs &A, unsigned &target) {
    __shared__ int s_ok;
    target += gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        red_release_add(&A.gbar[0], 1u);
        const long long t0 = clock64();
        while (ld_acquire_u32(&A.gbar[0]) < target) {
            if (clock64() - t0 > (1ll << 31)) {
                atomicOr(A.status, kStatusTimeout);
                s_ok = 0;
                break;
            }
        }
    }
    __syncthreads();
    return s_ok != 0;
}

// Self-test of the bounded device waits: which = 0 waits on an mbarrier nothing
// arrives at, which = 1 on a grid barrier whose arrival count is never reached.
// Either wait gives up after about a second and sets the timeout status bit.
__global__ void wait_selftest_kernel(const StepArgs A, int which) {
    __shared__ __align__(8) uint64_t bar;
    if (which == 0) {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            fence_barrier_init();
        }
        __syncthreads();
        if (threadIdx.x == 0 && !mbar_wait(&bar, 0)) atomicOr(A.status, kStatusTimeout);
    } else {
        unsigned target = 1u << 30;  // far beyond the arrivals of this one-CTA launch
        grid_barrier(A, target);
    }
}

template <int NPE, int NPR, bool ANI, bool BRICK>
__global__ void __launch_bounds__(kBlock, 2) coop_step_kernel(const StepArgs A, const int K) {
    extern __shared__ __align__(128) char smem[];
    __shared__ ScenStep S;
    const int t = blockIdx.x, tid = threadIdx.x;
    const TileInfo T = tile_info(A, t);
    constexpr int ML = max_local(NPE);
    char *rec = smem + A.cs_rec;
    const uint16_t *s_pat = reinterpret_cast<const uint16_t *>(smem + A.cs_pat);
    const uint16_t *s_code = s_pat + kTile * NPE, *s_row = s_code + kTile * NPE;
    int *s_shg = reinterpret_cast<int *>(smem + A.cs_sh);  // per shared node: global index,
    int *s_ppos = s_shg + ML;                               // this tile's partial position,
    int *s_r0 = s_shg + 2 * ML;                             // the node's first partial,
    int *s_cnt = s_shg + 3 * ML;                            // and its tile count
    float4 *s_xu = reinterpret_cast<float4 *>(smem + A.cs_xu);
    float4 *s_X = reinterpret_cast<float4 *>(smem + A.cs_X);
    float4 *s_lo = reinterpret_cast<float4 *>(smem + A.cs_lo);
    float4 *s_vo = reinterpret_cast<float4 *>(smem + A.cs_vo);
    float4 *s_nc = reinterpret_cast<float4 *>(smem + A.cs_nc);
    float4 *slot = reinterpret_cast<float4 *>(smem + A.cs_slot);
    const int nfix = A.n_comp - 6 * A.n_prony;
    const int n_sh = T.nl - T.n_int;
    unsigned target = 0;  // arrivals that open the next grid barrier

    // ---- the tile into shared memory
    {
        const float *grec = reinterpret_cast<const float *>(A.elem_rec + (int64_t)t * A.rec_bytes);
        float *r = reinterpret_cast<float *>(rec);
        for (int i = tid; i < nfix * kTile; i += kBlock) r[i] = __ldg(grec + i);
        const float *gvs = A.visc + (int64_t)t * A.n_prony * 6 * kTile;
        for (int i = tid; i < 6 * A.n_prony * kTile; i += kBlock) r[nfix * kTile + i] = gvs[i];
        const uint16_t *pat = A.pattern + (int64_t)T.pat * A.pat_stride;
        uint16_t *sp = reinterpret_cast<uint16_t *>(smem + A.cs_pat);
        for (int i = tid; i < pattern_u16(NPE); i += kBlock) sp[i] = pat[i];
        for (int m = tid; m < n_sh; m += kBlock) {
            const int g = __ldg(A.tile_shared + T.sh_off + m);
            const int64_t s = g - A.n_interior;
            s_shg[m] = g;
            s_ppos[m] = __ldg(A.part_pos + T.sh_off + m);
            s_r0[m] = __ldg(A.sh_rowptr + s);
            s_cnt[m] = __ldg(A.sh_rowptr + s + 1) - s_r0[m];
        }
        for (int l = tid; l < T.nl; l += kBlock) {
            const int64_t g = l < T.n_int ? (int64_t)T.ib + l : (int64_t)__ldg(A.tile_shared + T.sh_off + l - T.n_int);
            s_X[l] = __ldg(&A.X0[g]);
            s_xu[l] = A.xu[g];
            s_lo[l] = A.lo[g];
            s_vo[l] = A.vel[g];
            s_nc[l] = __ldg(&A.nodec[g]);
        }
    }
    __syncthreads();

    for (int k = 0; k < K; k++) {
        float4 *part = A.partials + (k & 1) * A.n_partials;  // this step's partial sums
        prepare_scen(A, 0, k, S, tid, kBlock);
        __syncthreads();
        if (tid < T.ne_t) {
            int cl[NPE];
            ElemIn<NPR> E;
            load_elem<NPE, NPR, BRICK>(A, rec, s_pat, tid, cl, E);
            element_step<NPE, NPR, ANI, BRICK>(A, S, (int64_t)t * kTile + tid, tid, cl, E, s_xu, s_X, slot,
                                               reinterpret_cast<float *>(rec) + nfix * kTile + tid);
        }
        __syncthreads();
        for (int l = tid; l < T.nl; l += kBlock) {
            const float4 acc = gather_node(slot, s_code, s_row, l);
            if (l < T.n_int)
                node_advance(A, S, (int64_t)T.ib + l, acc, s_xu[l], s_X[l], s_lo[l], s_vo[l], s_nc[l], s_xu[l], s_lo[l],
                             s_vo[l]);
            else
                part[s_ppos[l - T.n_int]] = acc;
        }
        if (!grid_barrier(A, target)) return;  // every tile's partial sums of this step are in memory
        // this CTA's copy of each of its shared nodes: all the node's partial sums in tile order
        for (int m = tid; m < n_sh; m += kBlock) {
            const int r0 = s_r0[m], cnt = s_cnt[m];
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int r = 0; r < cnt; r++) {
                const float4 d = __ldcg(&part[r0 + r]);
                acc.x += d.x; acc.y += d.y; acc.z += d.z; acc.w += d.w;
            }
            const int l = T.n_int + m;
            node_advance(A, S, (int64_t)s_shg[m], acc, s_xu[l], s_X[l], s_lo[l], s_vo[l], s_nc[l], s_xu[l], s_lo[l],
                         s_vo[l], s_ppos[m] == r0);
        }
        __syncthreads();
    }

    // ---- node state (interior nodes, and the shared nodes this tile is the first of) and
    //      Prony state back to global memory
    for (int l = tid; l < T.nl; l += kBlock) {
        const bool own = l < T.n_int || s_ppos[l - T.n_int] == s_r0[l - T.n_int];
        if (!own) continue;
        const int64_t g = l < T.n_int ? (int64_t)T.ib + l : (int64_t)s_shg[l - T.n_int];
        A.xu[g] = s_xu[l];
        A.lo[g] = s_lo[l];
        A.vel[g] = s_vo[l];
    }
    float *gvs = A.visc + (int64_t)t * A.n_prony * 6 * kTile;
    const float *r = reinterpret_cast<const float *>(rec);
    for (int i = tid; i < 6 * A.n_prony * kTile; i += kBlock) gvs[i] = r[nfix * kTile + i];
}

// volume at or above an isotherm: sum of V_i over theta_i >= theta_iso (fixed grid, fixed tree)
__global__ void __launch_bounds__(256) isotherm_partial_kernel(const StepArgs A, int64_t nn, double th_iso,
                                                               double *partials) {
    double v = 0.0;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x)
        if ((double)A.xu[g].w + (double)A.lo[g].w >= th_iso) v += (double)A.X0[g].w;
    __shared__ double sh[256];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}
__global__ void sum_final_kernel(const double *partials, int n, double *out) {
    if (threadIdx.x) return;
    double s = 0.0;
    for (int i = 0; i < n; i++) s += partials[i];
    out[0] = s;
}

// advance every scenario's step counter by K (its time is t0 + n dt)
__global__ void bump_kernel(const StepArgs A, int K) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < A.n_scn; s += gridDim.x * blockDim.x) A.scn_step[s] += K;
}

// Temperature and damage fraction at probe points: shape-function weights of
// the containing element applied to the nodal fields; out [2][n].
__global__ void probe_kernel(const float4 *__restrict__ hi, const float4 *__restrict__ lo,
                             const float4 *__restrict__ vel, const int32_t *__restrict__ node,
                             const float *__restrict__ w, int64_t n, double T0, double *__restrict__ out) {
    // eight lanes per probe, one per weight; the eight terms are summed by a fixed
    // butterfly (pairs, then quads, then the two halves)
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = i >> 3;
    const int a = (int)(i & 7);
    double th = 0.0, dmg = 0.0;
    if (p < n) {
        const double wa = w[8 * p + a];
        if (wa != 0.0) {
            const int64_t g = node[8 * p + a];
            th = wa * ((double)hi[g].w + (double)lo[g].w);
            dmg = wa * -expm1(-(double)vel[g].w);
        }
    }
#pragma unroll
    for (int m = 1; m < 8; m <<= 1) {
        th += __shfl_xor_sync(0xffffffffu, th, m);
        dmg += __shfl_xor_sync(0xffffffffu, dmg, m);
    }
    if (p < n && a == 0) {
        out[p] = T0 + th;
        out[n + p] = dmg;
    }
}

__global__ void readback_kernel(const float4 *__restrict__ hi, const float4 *__restrict__ lo,
                                const float4 *__restrict__ vel, const double *__restrict__ cem,
                                const int32_t *__restrict__ node_new, int64_t nn, double T0, int mode,
                                double *__restrict__ out) {
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
    } else if (mode == 2) {
        out[i] = -expm1(-(double)vel[g].w);
    } else {
        out[i] = cem[g];
    }
}

// Deterministic FP64 diagnostics: fixed grid, fixed per-thread stride, fixed tree.
__global__ void __launch_bounds__(256) stats_partial_kernel(const StepArgs A, int64_t nn, double *partials) {
    double ke = 0, heat = 0, tmax = -1e300, tmin = 1e300, umax = 0, dvol = 0;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        const float4 h = A.xu[g], l = A.lo[g], v = A.vel[g], nc = A.nodec[g], X = A.X0[g];
        const double ux = (double)h.x + l.x, uy = (double)h.y + l.y, uz = (double)h.z + l.z;
        const double th = (double)h.w + l.w;
        ke += 0.5 / (double)nc.x * ((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z);
        heat += th / (double)nc.y;
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

// n_out = 6 (nodal diagnostics) or 8 (with the two energy sums of energy_partial_kernel)
__global__ void stats_final_kernel(const double *partials, int nb, int n_out, double *out) {
    if (threadIdx.x != 0) return;
    double ke = 0, heat = 0, tmax = -1e300, tmin = 1e300, umax = 0, dvol = 0, wel = 0, whg = 0;
    for (int b = 0; b < nb; b++) {
        const double *p = partials + (size_t)b * 8;
        ke += p[0]; heat += p[1]; tmax = fmax(tmax, p[2]); tmin = fmin(tmin, p[3]); umax = fmax(umax, p[4]);
        dvol += p[5];
        if (n_out > 6) {
            wel += p[6];
            whg += p[7];
        }
    }
    out[0] = ke; out[1] = heat; out[2] = tmax; out[3] = tmin; out[4] = umax; out[5] = dvol;
    if (n_out > 6) {
        out[6] = wel;
        out[7] = whg;
    }
}

// Mechanical energy in FP64 (diagnostics): per element the stored energy of
// the thermally split potential in the reference configuration, V0 lambda^3
// Psi(F_el) (Eqs. 7-11, Table 5, fibre term as in the step), and the H8
// hourglass energy 1/2 k_hg sum_al |q_al|^2 whose gradient is the hourglass
// force of the step.  Block b sums tiles b, b + gridDim.x, ... in a fixed tree
// and writes partials[8 b + 6] (stored energy) and [8 b + 7] (hourglass).
template <int NPE>
__global__ void __launch_bounds__(256) energy_partial_kernel(const StepArgs A, double *partials) {
    double w_el = 0.0, w_hg = 0.0;
    for (int t = blockIdx.x; t < A.n_tiles; t += gridDim.x) {
        const TileInfo T = tile_info(A, t);
        const int npe = NPE ? NPE : T.npe;
        const int ec = threadIdx.x;
        if (ec >= T.ne_t) continue;
        const char *base = A.elem_rec + (int64_t)t * A.rec_bytes;
        const uint16_t *cl = A.pattern + (int64_t)T.pat * A.pat_stride + ec * npe;
        const float *cp = reinterpret_cast<const float *>(base) + ec;
        double Ji[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int q = 0;
        if (A.brick) {  // diagonal of J0^-1
            for (int k = 0; k < 9; k += 4) Ji[k] = cp[(q++) * kTile];
        } else {
            for (int k = 0; k < 9; k++) Ji[k] = cp[(q++) * kTile];
        }
        const double V = cp[(q++) * kTile];
        double mu = A.mu, kap = A.kappa, k1 = A.k1, k2 = A.k2, al = A.alpha;
        if (A.has_mat) {
            mu = cp[q * kTile]; kap = cp[(q + 1) * kTile]; k1 = cp[(q + 2) * kTile]; k2 = cp[(q + 3) * kTile];
            al = cp[(q + 5) * kTile];
            q += 6;
        }
        double a0[3] = {A.a0x, A.a0y, A.a0z};
        if (A.has_fib)
            for (int j = 0; j < 3; j++) a0[j] = cp[(q + j) * kTile];
        double u[8][3], X[8][3], the = 0.0;
        for (int a = 0; a < npe; a++) {
            const int l = cl[a];
            const int64_t g = l < T.n_int ? (int64_t)T.ib + l : (int64_t)__ldg(A.tile_shared + T.sh_off + l - T.n_int);
            const float4 h = A.xu[g], lo = A.lo[g], x = A.X0[g];
            u[a][0] = (double)h.x + lo.x; u[a][1] = (double)h.y + lo.y; u[a][2] = (double)h.z + lo.z;
            the += (double)h.w + lo.w;
            X[a][0] = x.x; X[a][1] = x.y; X[a][2] = x.z;
        }
        the /= npe;
        // shape-function derivatives dh_a/dX_j (H8: centroid, corner signs; T4: rows of J0^-1)
        double dh[8][3];
        for (int a = 0; a < npe; a++)
            for (int j = 0; j < 3; j++) {
                if (npe == 8) {
                    dh[a][j] = 0.125 * (sgn(a, 0) * Ji[j] + sgn(a, 1) * Ji[3 + j] + sgn(a, 2) * Ji[6 + j]);
                } else {
                    dh[a][j] = a == 0 ? -(Ji[j] + Ji[3 + j] + Ji[6 + j]) : Ji[3 * (a - 1) + j];
                }
            }
        double H[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int a = 0; a < npe; a++)
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) H[i][j] += u[a][i] * dh[a][j];
        const double dl = (A.flags & TLED_EXPANSION) ? al * the : 0.0;
        const double lam = 1.0 + dl;
        const double trH = H[0][0] + H[1][1] + H[2][2];
        double trH2 = 0.0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) trH2 += H[i][j] * H[j][i];
        const double detH = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) -
                            H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
                            H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
        const double Jm1 = trH + 0.5 * (trH * trH - trH2) + detH;
        // E_el = F_th^-T E F_th^-1 + (F_th^-T F_th^-1 - I) / 2, E = (H + H^T + H^T H) / 2, with
        // F_th^-1 = (I - g m m) / lambda_i, g = (lambda_m - lambda_i) / lambda_m (m the fibre;
        // isotropic: g = 0, lambda_m = lambda_i)
        const double dm = A.ani && (A.flags & TLED_EXPANSION) ? (double)A.ani_alpha * al * the : dl;
        const double lm = 1.0 + dm, g = (dm - dl) / lm;
        double E[3][3], Em[3] = {0, 0, 0}, mEm = 0.0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double e = 0.5 * (H[i][j] + H[j][i]);
                for (int k = 0; k < 3; k++) e += 0.5 * H[k][i] * H[k][j];
                E[i][j] = e;
            }
        for (int i = 0; i < 3; i++) {
            for (int j = 0; j < 3; j++) Em[i] += E[i][j] * a0[j];
            mEm += a0[i] * Em[i];
        }
        double Ee[3][3];
        const double d1 = dl + 0.5 * dl * dl, il2 = 1.0 / (lam * lam), cmm = g * g * mEm - g + 0.5 * g * g;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                Ee[i][j] = (E[i][j] - (i == j ? d1 : 0.0) - g * (a0[i] * Em[j] + Em[i] * a0[j]) + cmm * a0[i] * a0[j]) * il2;
        const double th3m1 = dl * (2.0 + dl) + dm * (1.0 + dl) * (1.0 + dl);  // det F_th - 1
        const double jel = (Jm1 - th3m1) / (1.0 + th3m1);                      // J_el - 1
        const double Jm23m1 = expm1(-(2.0 / 3.0) * log1p(jel));
        const double Jm23 = 1.0 + Jm23m1;
        const double trE = Ee[0][0] + Ee[1][1] + Ee[2][2];
        double aEa = 0.0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) aEa += a0[i] * Ee[i][j] * a0[j];
        const double I1m3 = 3.0 * Jm23m1 + 2.0 * Jm23 * trE;  // I1bar - 3
        const double x4 = Jm23m1 + 2.0 * Jm23 * aEa;          // I4bar - 1
        const double psif = k2 > 0.0 ? k1 / (2.0 * k2) * expm1(k2 * x4 * x4) : 0.5 * k1 * x4 * x4;
        w_el += V * (1.0 + th3m1) * (0.5 * mu * I1m3 + 0.5 * kap * jel * jel + psif);
        if (npe == 8) {
            double jn2 = 0.0;
            for (int k = 0; k < 9; k++) jn2 += Ji[k] * Ji[k];
            const double khg = (double)A.khg * (kap + (4.0 / 3.0) * mu) * V * jn2 / 64.0;
            for (int l = 0; l < 4; l++) {
                double hu[3] = {0, 0, 0}, cX[3] = {0, 0, 0};
                for (int b = 0; b < 8; b++) {
                    const double h = hgv(b, l);
                    for (int i = 0; i < 3; i++) {
                        hu[i] += h * u[b][i];
                        cX[i] += h * X[b][i];
                    }
                }
                for (int i = 0; i < 3; i++) {
                    const double qi = hu[i] - (H[i][0] * cX[0] + H[i][1] * cX[1] + H[i][2] * cX[2]);
                    w_hg += 0.5 * khg * qi * qi;
                }
            }
        }
    }
    __shared__ double sh[2][256];
    sh[0][threadIdx.x] = w_el;
    sh[1][threadIdx.x] = w_hg;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x < 2) partials[(size_t)blockIdx.x * 8 + 6 + threadIdx.x] = sh[threadIdx.x][0];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int align128(int x) { return (x + 127) & ~127; }

void tile_smem_layout(StepArgs &a, int npe) {
    if (npe == 0) npe = 8;  // a mixed batch sizes everything for the larger element
    a.n_comp = (a.brick ? 4 : 10) + (a.has_mat ? 6 : 0) + (a.has_fib ? 3 : 0) + 6 * a.n_prony;
    a.sm_in = align128(a.n_comp * kTile * 4);
    a.sm_buf = std::max(a.sm_in, kTile * npe * 16);
    int off = a.sm_buf;  // element inputs; once read into registers, the corner slot buffer
    a.sm_ns = off;
    off = align128(off + kNsMax * 48);
    a.sm_pat = off;
    off = align128(off + pattern_u16(npe) * 2);
    a.sm_sh = off;  // two list buffers of (global index, partial position)
    off = align128(off + 4 * max_local(npe) * 4);
    a.sm_xu = off;
    off = align128(off + max_local(npe) * 16);
    a.sm_X = off;
    off = align128(off + max_local(npe) * 16);
    a.sm_bar = off;
    off = align128(off + 32);
    a.sm_total = off;
}

template <class K>
static cudaError_t set_smem(K kern, int bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// the tile kernel instance for (element type, Prony terms, anisotropic thermal physics,
// brick H8, CTAs per SM): npe 8, 4 or 0 (mixed), n_prony 0..4; T4 problems with more
// tiles than three CTAs per SM cover take the 4-CTA (64-register) instance
using TileKernel = void (*)(const StepArgs, const int);
template <int NPE, bool ANI, bool BRICK = false, int CPS = kTileCtasPerSm>
static TileKernel tile_kernel_npr(int n_prony) {
    switch (n_prony) {
        case 0: return tile_step_kernel<NPE, 0, ANI, BRICK, CPS>;
        case 1: return tile_step_kernel<NPE, 1, ANI, BRICK, CPS>;
        case 2: return tile_step_kernel<NPE, 2, ANI, BRICK, CPS>;
        case 3: return tile_step_kernel<NPE, 3, ANI, BRICK, CPS>;
        default: return tile_step_kernel<NPE, 4, ANI, BRICK, CPS>;
    }
}
template <bool ANI>
static TileKernel tile_kernel_ani(int npe, bool brick, bool wide, int n_prony) {
    return npe == 8 ? (brick ? tile_kernel_npr<8, ANI, true>(n_prony) : tile_kernel_npr<8, ANI>(n_prony))
         : npe == 4 ? (wide ? tile_kernel_npr<4, ANI, false, kTileCtasPerSmT4>(n_prony) : tile_kernel_npr<4, ANI>(n_prony))
                    : tile_kernel_npr<0, ANI>(n_prony);
}
static TileKernel tile_kernel(const StepArgs &a, int npe) {
    const bool brick = a.brick != 0, wide = a.wide != 0;
    return a.ani ? tile_kernel_ani<true>(npe, brick, wide, a.n_prony) : tile_kernel_ani<false>(npe, brick, wide, a.n_prony);
}

cudaError_t tile_kernel_setup(const StepArgs &a, int npe) { return set_smem(tile_kernel(a, npe), a.sm_total); }

// resident kernel instance (element type 4 or 8, Prony terms, anisotropic, brick)
template <int NPE, bool ANI, bool BRICK = false>
static TileKernel resident_kernel_npr(int n_prony) {
    switch (n_prony) {
        case 0: return resident_step_kernel<NPE, 0, ANI, BRICK>;
        case 1: return resident_step_kernel<NPE, 1, ANI, BRICK>;
        case 2: return resident_step_kernel<NPE, 2, ANI, BRICK>;
        case 3: return resident_step_kernel<NPE, 3, ANI, BRICK>;
        default: return resident_step_kernel<NPE, 4, ANI, BRICK>;
    }
}
template <bool ANI>
static TileKernel resident_kernel_ani(int npe, bool brick, int n_prony) {
    return npe == 8 ? (brick ? resident_kernel_npr<8, ANI, true>(n_prony) : resident_kernel_npr<8, ANI>(n_prony))
                    : resident_kernel_npr<4, ANI>(n_prony);
}
static TileKernel resident_kernel(const StepArgs &a, int npe) {
    const bool brick = a.brick != 0;
    return a.ani ? resident_kernel_ani<true>(npe, brick, a.n_prony) : resident_kernel_ani<false>(npe, brick, a.n_prony);
}

static int align16(int x) { return (x + 15) & ~15; }

int resident_smem_layout(StepArgs &a, int npe, int nn_max, int nt_max, int npart_max, int nsh_max) {
    int off = 0;
    auto take = [&](int bytes) {
        const int o = off;
        off = align128(off + bytes);
        return o;
    };
    a.rs_xu = take(16 * nn_max);
    a.rs_lo = take(16 * nn_max);
    a.rs_vel = take(16 * nn_max);
    a.rs_X = take(16 * nn_max);
    a.rs_nc = take(16 * nn_max);
    a.rs_rowptr = take(4 * (nsh_max + 1));
    a.rs_part = take(16 * npart_max);
    a.rs_slot = take(kResLanes * kTile * npe * 16);  // one corner slot buffer per tile lane
    int to = align128(a.n_comp * kTile * 4);  // element record and Prony state
    a.rt_conn = to;
    to = align16(to + kTile * npe * 2);
    a.rt_codes = to;
    to = align16(to + (kTile * npe + kMaxLocal + 8) * 2);
    a.rt_ppos = to;
    to = align16(to + kMaxLocal * 4);
    a.rt_info = to;
    a.rs_tile = align128(to + 16);
    a.rs_tiles = take(nt_max * a.rs_tile);
    a.rs_total = off;
    return off;
}

// dynamic shared memory a resident CTA may use (the opt-in limit less the static part)
int resident_smem_limit() {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return optin - 1024;
}

cudaError_t resident_kernel_setup(const StepArgs &a, int npe) { return set_smem(resident_kernel(a, npe), a.rs_total); }

// grid-resident kernel instance (element type 4 or 8, Prony terms, anisotropic, brick)
template <int NPE, bool ANI, bool BRICK = false>
static TileKernel coop_kernel_npr(int n_prony) {
    switch (n_prony) {
        case 0: return coop_step_kernel<NPE, 0, ANI, BRICK>;
        case 1: return coop_step_kernel<NPE, 1, ANI, BRICK>;
        case 2: return coop_step_kernel<NPE, 2, ANI, BRICK>;
        case 3: return coop_step_kernel<NPE, 3, ANI, BRICK>;
        default: return coop_step_kernel<NPE, 4, ANI, BRICK>;
    }
}
template <bool ANI>
static TileKernel coop_kernel_ani(int npe, bool brick, int n_prony) {
    return npe == 8 ? (brick ? coop_kernel_npr<8, ANI, true>(n_prony) : coop_kernel_npr<8, ANI>(n_prony))
                    : coop_kernel_npr<4, ANI>(n_prony);
}
static TileKernel coop_kernel(const StepArgs &a, int npe) {
    const bool brick = a.brick != 0;
    return a.ani ? coop_kernel_ani<true>(npe, brick, a.n_prony) : coop_kernel_ani<false>(npe, brick, a.n_prony);
}

int coop_smem_layout(StepArgs &a, int npe) {
    const int ml = max_local(npe);
    int off = 0;
    auto take = [&](int bytes) {
        const int o = off;
        off = align128(off + bytes);
        return o;
    };
    a.cs_rec = take(a.n_comp * kTile * 4);
    a.cs_pat = take(pattern_u16(npe) * 2);
    a.cs_sh = take(4 * ml * 4);
    a.cs_xu = take(ml * 16);
    a.cs_X = take(ml * 16);
    a.cs_lo = take(ml * 16);  // interior node state: up to every local node
    a.cs_vo = take(ml * 16);
    a.cs_nc = take(ml * 16);
    a.cs_slot = take(kTile * npe * 16);
    a.cs_total = off;
    return off;
}

int coop_ctas_per_sm(const StepArgs &a, int npe) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coop_kernel(a, npe), kBlock, a.cs_total) != cudaSuccess)
        return 0;
    return per_sm;
}

cudaError_t coop_kernel_setup(const StepArgs &a, int npe) { return set_smem(coop_kernel(a, npe), a.cs_total); }

// single problem: its scenario table and source rows from the kernel's parameters
__global__ void single_upload_kernel(const SingleScenUpload u, ScenDev *scn, double *src) {
    if (threadIdx.x == 0) *scn = u.d;
    for (int i = threadIdx.x; i < kMaxSources * kSrcRow; i += blockDim.x) src[i] = u.src[i];
}

cudaError_t launch_single_upload(const SingleScenUpload &u, ScenDev *scn, double *src, cudaStream_t s) {
    single_upload_kernel<<<1, 64, 0, s>>>(u, scn, src);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(const StepArgs &a, int which, cudaStream_t s) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(a, which);
    return cudaGetLastError();
}

cudaError_t launch_coop_step(const StepArgs &a, int npe, int K, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.gbar, 0, sizeof(unsigned), s);  // arrivals start at zero
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.n_tiles);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = (size_t)a.cs_total;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, coop_kernel(a, npe), a, K);
}

cudaError_t launch_resident_step(const StepArgs &a, int n_ctas, int npe, int K, cudaStream_t s) {
    if (n_ctas <= 0) return cudaSuccess;
    resident_kernel(a, npe)<<<n_ctas, kResBlock, (size_t)a.rs_total, s>>>(a, K);
    return cudaGetLastError();
}

int tile_grid(const StepArgs &a, int npe, int n_sm) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tile_kernel(a, npe), kBlock, a.sm_total);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return std::max(1, std::min(a.n_tiles, per_sm * n_sm));
}

// a streamed step kernel's launch, with the persisting-L2 window when the context set one
static cudaError_t launch_step_kernel(void (*kern)(const StepArgs, const int), int grid, int block, size_t smem,
                                     cudaStream_t s, const StepArgs &a, int k) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    if (a.l2_bytes > 0) {
        at[0].id = cudaLaunchAttributeAccessPolicyWindow;
        at[0].val.accessPolicyWindow.base_ptr = a.l2_base;
        at[0].val.accessPolicyWindow.num_bytes = a.l2_bytes;
        at[0].val.accessPolicyWindow.hitRatio = a.l2_hit;
        at[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        at[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        cfg.attrs = at;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kern, a, k);
}

cudaError_t launch_tile_step(const StepArgs &a, int n_ctas, int npe, int k, cudaStream_t s) {
    if (a.n_tiles <= 0) return cudaSuccess;
    return launch_step_kernel(tile_kernel(a, npe), n_ctas, kBlock, (size_t)a.sm_total, s, a, k);
}

int shared_grid(const StepArgs &a, int n_sm) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, shared_step_kernel, 256, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return (int)std::max<int64_t>(1, std::min<int64_t>((a.n_shared + 255) / 256, (int64_t)per_sm * n_sm));
}

cudaError_t launch_shared_step(const StepArgs &a, int n_blocks, int k, cudaStream_t s) {
    if (a.n_shared <= 0) return cudaSuccess;
    return launch_step_kernel(shared_step_kernel, n_blocks, 256, 0, s, a, k);
}

cudaError_t launch_isotherm(const StepArgs &a, int64_t nn, double theta_iso, double *partials, double *out,
                            cudaStream_t s) {
    isotherm_partial_kernel<<<kStatBlocks, 256, 0, s>>>(a, nn, theta_iso, partials);
    sum_final_kernel<<<1, 32, 0, s>>>(partials, kStatBlocks, out);
    return cudaGetLastError();
}

cudaError_t launch_bump(const StepArgs &a, int K, cudaStream_t s) {
    bump_kernel<<<(a.n_scn + 255) / 256, 256, 0, s>>>(a, K);
    return cudaGetLastError();
}

cudaError_t launch_readback(const StepArgs &a, const int32_t *node_new, int64_t nn, double T0, int mode, double *out,
                            cudaStream_t s) {
    const int nb = (int)((nn + 255) / 256);
    readback_kernel<<<nb, 256, 0, s>>>(a.xu, a.lo, a.vel, a.cem, node_new, nn, T0, mode, out);
    return cudaGetLastError();
}

cudaError_t launch_probes(const StepArgs &a, const int32_t *node, const float *w, int64_t n, double T0, double *out,
                          cudaStream_t s) {
    probe_kernel<<<(int)((8 * n + 255) / 256), 256, 0, s>>>(a.xu, a.lo, a.vel, node, w, n, T0, out);
    return cudaGetLastError();
}

cudaError_t launch_stats(const StepArgs &a, int npe, int64_t nn, double *partials, double *out, cudaStream_t s) {
    stats_partial_kernel<<<kStatBlocks, 256, 0, s>>>(a, nn, partials);
    if (npe == 8)
        energy_partial_kernel<8><<<kStatBlocks, 256, 0, s>>>(a, partials);
    else if (npe == 4)
        energy_partial_kernel<4><<<kStatBlocks, 256, 0, s>>>(a, partials);
    else
        energy_partial_kernel<0><<<kStatBlocks, 256, 0, s>>>(a, partials);
    stats_final_kernel<<<1, 32, 0, s>>>(partials, kStatBlocks, 8, out);
    return cudaGetLastError();
}

cudaError_t launch_stats_blocks(const StepArgs &a, int64_t nn, int n_blocks, double *partials, double *out,
                                cudaStream_t s) {
    stats_partial_kernel<<<n_blocks, 256, 0, s>>>(a, nn, partials);
    stats_final_kernel<<<1, 32, 0, s>>>(partials, n_blocks, 6, out);
    return cudaGetLastError();
}

}  // namespace tled
