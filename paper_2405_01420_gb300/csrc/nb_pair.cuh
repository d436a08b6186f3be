// One atom pair of the LJ + Ewald real-space interaction, FP32.
//
//   E_LJ  = C12/r^12 - C6/r^6 - (C12/rc^12 - C6/rc^6)
//   E_C   = f q_i q_j erfc(beta r)/r
//   s     = -(1/r) dE/dr
//         = f q_i q_j [erfc(beta r)/r + (2 beta/sqrt(pi)) exp(-beta^2 r^2)] / r^2
//           + (12 C12/r^12 - 6 C6/r^6) / r^2
//   F_i  += s d,  F_j -= s d
//
// erfc(x) = exp(-x^2) R(x) with R(x) = P(x)/Q(x) a degree-4/4 rational fit
// of erfcx on [0, 3.2] (relative error 1.6e-8 in FP64, 2.9e-7 evaluated in
// FP32; coefficients from fit_coeffs.py). 1/sqrt(r2) is the hardware
// estimate refined by a Newton step; exp and the division are chosen by
// NB_EXP_MODE / NB_RCP_NR below. The energies are summed over ~10^7 terms
// that cancel to ~1/400 of their absolute sum in water, so any error that
// varies systematically with r is amplified; the refined forms keep every
// factor free of approximation bias beyond FP32 rounding.
#pragma once

#include <cmath>

#include "nb_internal.cuh"

#define NB_ERFCX_P1 8.430113792e-01f
#define NB_ERFCX_P2 3.496225476e-01f
#define NB_ERFCX_P3 5.748734251e-02f
#define NB_ERFCX_P4 1.737346247e-05f
#define NB_ERFCX_Q1 1.971389651e+00f
#define NB_ERFCX_Q2 1.574109197e+00f
#define NB_ERFCX_Q3 6.144732237e-01f
#define NB_ERFCX_Q4 1.024811342e-01f

__device__ __forceinline__ float nb_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float nb_rsqrt(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float nb_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Variants of the two function approximations (compile-time):
//   NB_EXP_MODE 0: 2^t by ex2.approx; 1: Cody-Waite reduction t = n + f and a
//                  degree-6 polynomial for 2^f (fit_coeffs.py), no hardware
//                  approximation in the result.
//   NB_RCP_NR   0: 1/q by rcp.approx; 1: plus one Newton step.
#ifndef NB_EXP_MODE
#define NB_EXP_MODE 1
#endif
#ifndef NB_RCP_NR
#define NB_RCP_NR 1
#endif

#define NB_EXP2_C1 6.931471825e-01f
#define NB_EXP2_C2 2.402264923e-01f
#define NB_EXP2_C3 5.550362542e-02f
#define NB_EXP2_C4 9.618407115e-03f
#define NB_EXP2_C5 1.338712522e-03f
#define NB_EXP2_C6 1.533757168e-04f

// 2^t for -125 <= t <= 0. Pairs inside the cutoff have t >= -(beta rc)^2
// log2(e) > -15; for t below -125 the result is meaningless, which is
// harmless because the callers select such pairs away (never multiply).
__device__ __forceinline__ float nb_exp2(float t) {
#if NB_EXP_MODE == 0
    return nb_ex2(t);
#else
    const float magic = 12582912.0f;          // 1.5 * 2^23: adding it rounds to an integer
    const float tn = t + magic;
    const float n = tn - magic;               // rint(t)
    const float f = t - n;                    // in [-0.5, 0.5]
    float p = fmaf(NB_EXP2_C6, f, NB_EXP2_C5);
    p = fmaf(p, f, NB_EXP2_C4);
    p = fmaf(p, f, NB_EXP2_C3);
    p = fmaf(p, f, NB_EXP2_C2);
    p = fmaf(p, f, NB_EXP2_C1);
    p = fmaf(p, f, 1.0f);                     // 2^f in [0.70, 1.42]
    // bits(tn) = bits(magic) + n and bits(magic) * 2^23 = 0 (mod 2^32), so
    // adding bits(tn) * 2^23 to the bits of p multiplies p by 2^n.
    return __int_as_float(__float_as_int(p) + __float_as_int(tn) * (1 << 23));
#endif
}

__device__ __forceinline__ float nb_recip(float q) {
    float y = nb_rcp(q);
#if NB_RCP_NR
    const float e = fmaf(-q, y, 1.0f);
    y = fmaf(y, e, y);
#endif
    return y;
}

// R(x) = erfc(x) exp(x^2) for x in [0, 3.2].
__device__ __forceinline__ float nb_erfcx(float x) {
    float p = fmaf(fmaf(fmaf(fmaf(NB_ERFCX_P4, x, NB_ERFCX_P3), x, NB_ERFCX_P2), x, NB_ERFCX_P1), x, 1.0f);
    float q = fmaf(fmaf(fmaf(fmaf(NB_ERFCX_Q4, x, NB_ERFCX_Q3), x, NB_ERFCX_Q2), x, NB_ERFCX_Q1), x, 1.0f);
    return p * nb_recip(q);
}

// Coulomb flavour of the pair kernels (their COUL template parameter):
//   NB_COULK_EWALD        f qi qj erfc(beta r)/r
//   NB_COULK_EWALD_SHIFT  the same minus f qi qj erfc(beta rc)/rc (energies only)
//   NB_COULK_RF           reaction field f qi qj (1/r + k_rf r^2 - c_rf)
#define NB_COULK_EWALD 0
#define NB_COULK_EWALD_SHIFT 1
#define NB_COULK_RF 2

// Constants of one force call, shared by all pairs.
struct nb_coul {
    float rc2;   // fl(rc * rc): a pair counts iff r2 < rc2
    float beta;  // Ewald splitting parameter
    float kexp;  // -beta^2 log2(e): exp(-beta^2 r^2) = 2^(kexp r^2)
    float c2b;   // 2 beta / sqrt(pi)
    float sh;    // erfc(beta rc)/rc (Ewald shift)
    float krf;   // k_rf (reaction field)
    float crf;   // c_rf = 1/rc + k_rf rc^2
    // k_rf - krf and c_rf - crf: the energy adds these residuals, since
    // f sum q q c_rf cancels to ~1/60 of itself in water and the FP32
    // rounding of the constants alone biases E_coul by ~1e-6
    float krf_lo, crf_lo;
};

// Fills the constants for cutoff rc, Ewald beta and the pair list's
// Coulomb setting (kind NB_COUL_*, eps_rf with 0 meaning infinity, flags
// NB_COUL_SHIFT / NB_COUL_EXCL_CORR); returns the NB_COULK_* mode.
inline int nb_fill_coul(nb_coul &cc, float rc, float beta, int kind, float eps_rf, unsigned flags) {
    cc.rc2 = rc * rc;
    cc.beta = beta;
    cc.kexp = (float)(-(double)beta * beta * 1.4426950408889634);
    cc.c2b = (float)(2.0 * beta / 1.7724538509055159);
    cc.sh = (float)(std::erfc((double)beta * rc) / rc);
    const double rc3 = (double)rc * rc * rc;
    const double krf = eps_rf == 0.0f ? 1.0 / (2.0 * rc3) : ((double)eps_rf - 1.0) / ((2.0 * eps_rf + 1.0) * rc3);
    const double crf = 1.0 / rc + krf * (double)rc * rc;
    cc.krf = (float)krf;
    cc.crf = (float)crf;
    cc.krf_lo = (float)(krf - (double)cc.krf);
    cc.crf_lo = (float)(crf - (double)cc.crf);
    if (kind == NB_COUL_RF) return NB_COULK_RF;
    return (flags & NB_COUL_SHIFT) ? NB_COULK_EWALD_SHIFT : NB_COULK_EWALD;
}

// Accumulates one pair into fi (+) and fj (-). in_mask: the list mask bit.
// SHIFT: add the periodic shift S to (y_a - y_b). ENERGY: also accumulate
// the pair energies. Returns 1 if the pair was within rc and counted.
template <bool SHIFT, bool ENERGY, int COUL = NB_COULK_EWALD>
__device__ __forceinline__ int nb_pair(const float4 xi, const float qi_f, const float4 xj,
                                       const float4 lj, const float Sx, const float Sy,
                                       const float Sz, const bool in_mask, const nb_coul &cc,
                                       float3 &fi, float3 &fj, float &ec, float &elj) {
    float dx = __fsub_rn(xi.x, xj.x);
    float dy = __fsub_rn(xi.y, xj.y);
    float dz = __fsub_rn(xi.z, xj.z);
    if (SHIFT) {
        dx = __fadd_rn(dx, Sx);
        dy = __fadd_rn(dy, Sy);
        dz = __fadd_rn(dz, Sz);
    }
    const float r2 = nb_r2(dx, dy, dz);
    const bool in = in_mask && (r2 < cc.rc2);
    // 1/sqrt(r2): hardware estimate plus one Newton step on the residual
    // e = 1 - r2 y^2, so that the LJ terms (which carry 1/r to the 12th
    // power) see no systematic bias from the estimate.
    const float y0 = nb_rsqrt(r2);
    const float res = fmaf(-(r2 * y0), y0, 1.0f);
    const float rinv = fmaf(0.5f * y0, res, y0);
    const float rinv2 = rinv * rinv;
    const float rinv6 = rinv2 * rinv2 * rinv2;
    const float v6 = lj.x * rinv6;           // C6 / r^6
    const float v12 = lj.y * rinv6 * rinv6;  // C12 / r^12
    const float slj = fmaf(12.0f, v12, -6.0f * v6) * rinv2;
    float s, a = 0.0f, qq;  // qq = f q_i q_j
    if (COUL == NB_COULK_RF) {
        // f q q (1/r + k_rf r^2 - c_rf); s = f q q (1/r^3 - 2 k_rf)
        qq = qi_f * xj.w;
        s = fmaf(qq, fmaf(rinv, rinv2, -2.0f * cc.krf), slj);
    } else {
        const float r = r2 * rinv;
        const float ex = nb_exp2(cc.kexp * r2);  // exp(-beta^2 r^2)
        a = ex * nb_erfcx(cc.beta * r) * rinv;   // erfc(beta r) / r
        qq = qi_f * xj.w;
        s = fmaf(qq * fmaf(cc.c2b, ex, a), rinv2, slj);
    }
    s = in ? s : 0.0f;
    fi.x = fmaf(s, dx, fi.x);
    fi.y = fmaf(s, dy, fi.y);
    fi.z = fmaf(s, dz, fi.z);
    fj.x = fmaf(-s, dx, fj.x);
    fj.y = fmaf(-s, dy, fj.y);
    fj.z = fmaf(-s, dz, fj.z);
    if (ENERGY) {
        // RF: the residual term enters through the FMA's addend, against the
        // unrounded product (added to a rounded sum it would be absorbed)
        const float e_c = COUL == NB_COULK_RF
                              ? fmaf(qq, rinv + fmaf(cc.krf, r2, -cc.crf), qq * fmaf(cc.krf_lo, r2, -cc.crf_lo))
                          : COUL == NB_COULK_EWALD_SHIFT ? qq * (a - cc.sh) : qq * a;
        const float e_lj = v12 - v6 - lj.z;
        ec += in ? e_c : 0.0f;
        elj += in ? e_lj : 0.0f;
    }
    return in ? 1 : 0;
}

// One pair of the adjoint of nb_pair (same distance contract, same pair
// terms), for g = dL/dF with u = g_a - g_b:
//   dL/dx_a += s u + (s'/r)(u.d) d,  dL/dx_b -= the same
//   dL/dq_a += f q_b B (u.d),        dL/dq_b += f q_a B (u.d)
//   dL/dC6 = -6 r^-8 (u.d),          dL/dC12 = 12 r^-14 (u.d)
// bi/bj accumulate (dL/dx, dL/dq); d6/d12 return the pair's dL/dC6 and
// dL/dC12 (0 when the pair does not count). k2 = 2 (2 beta/sqrt(pi)) beta^2.
template <bool SHIFT, int COUL = NB_COULK_EWALD>
__device__ __forceinline__ void nb_pair_adj(const float4 xi, const float qi_f, const float4 gi, const float4 xj,
                                            const float qj_f, const float4 gj, const float4 lj, const float Sx,
                                            const float Sy, const float Sz, const bool in_mask, const nb_coul &cc,
                                            const float k2, float4 &bi, float4 &bj, float &d6, float &d12) {
    float dx = __fsub_rn(xi.x, xj.x), dy = __fsub_rn(xi.y, xj.y), dz = __fsub_rn(xi.z, xj.z);
    if (SHIFT) {
        dx = __fadd_rn(dx, Sx);
        dy = __fadd_rn(dy, Sy);
        dz = __fadd_rn(dz, Sz);
    }
    const float r2 = nb_r2(dx, dy, dz);
    const bool in = in_mask && (r2 < cc.rc2);
    const float y0 = nb_rsqrt(r2);
    const float rinv = fmaf(0.5f * y0, fmaf(-(r2 * y0), y0, 1.0f), y0);
    const float rinv2 = rinv * rinv;
    const float rinv6 = rinv2 * rinv2 * rinv2;
    const float v6 = lj.x * rinv6, v12 = lj.y * rinv6 * rinv6;
    const float slj = fmaf(12.0f, v12, -6.0f * v6) * rinv2;
    const float qq = qi_f * xj.w;                          // f q_a q_b
    float Bc, cpr;  // B, and r^2 (1/r) dB/dr times f q_a q_b
    if (COUL == NB_COULK_RF) {
        const float rinv3 = rinv * rinv2;
        Bc = rinv3 - 2.0f * cc.krf;  // 1/r^3 - 2 k_rf
        cpr = -3.0f * qq * rinv3;    // (1/r) dB/dr = -3/r^5
    } else {
        const float r = r2 * rinv;
        const float ex = nb_exp2(cc.kexp * r2);
        const float a = ex * nb_erfcx(cc.beta * r) * rinv;  // erfc(beta r)/r
        Bc = fmaf(cc.c2b, ex, a) * rinv2;
        cpr = fmaf(-3.0f, qq * Bc, -k2 * qq * ex);
    }
    const float sC = qq * Bc;
    const float s = sC + slj;
    const float spr = rinv2 * fmaf(rinv2, fmaf(48.0f, v6, -168.0f * v12), cpr);
    const float ux = gi.x - gj.x, uy = gi.y - gj.y, uz = gi.z - gj.z;
    const float ud = fmaf(ux, dx, fmaf(uy, dy, uz * dz));
    // Pairs that do not count can carry inf/NaN in their pair terms (r2 = 0
    // on a masked diagonal): select, never multiply by a zero factor.
    const float sm = in ? s : 0.0f;
    const float t = in ? spr * ud : 0.0f;
    const float vx = fmaf(sm, ux, t * dx), vy = fmaf(sm, uy, t * dy), vz = fmaf(sm, uz, t * dz);
    bi.x += vx;
    bi.y += vy;
    bi.z += vz;
    bj.x -= vx;
    bj.y -= vy;
    bj.z -= vz;
    const float bud = in ? Bc * ud : 0.0f;
    bi.w = fmaf(qj_f, bud, bi.w);
    bj.w = fmaf(qi_f, bud, bj.w);
    const float r8ud = rinv6 * rinv2 * ud;
    d6 = in ? -6.0f * r8ud : 0.0f;
    d12 = in ? 12.0f * rinv6 * r8ud : 0.0f;
}
