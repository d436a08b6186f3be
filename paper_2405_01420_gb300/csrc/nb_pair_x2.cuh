// The pair arithmetic of nb_pair for two i rows at once, on the packed
// two-wide FP32 instructions of sm_100 and later (__fadd2_rn, __fmul2_rn,
// __ffma2_rn): row a in .x, row b in .y, against one j atom. Each lane of a
// packed operation is the IEEE operation of its scalar counterpart, so the
// displacement and r^2 (and with them the in-range decision) are bit-equal
// to nb_pair's; the other terms follow nb_pair's formulas step by step with
// explicit rounding (no contraction), negated where a packed operation has
// no subtract form:
//   a - b        as  a + (-b)            (exact negation)
//   1 - t y      as  -(t y - 1)          (round-to-nearest is odd-symmetric)
//   -Q(x)        from the negated coefficients, each Horner step negated
// The j forces are summed per row pair and negated once per j atom.
#pragma once

#include "nb_pair.cuh"

__device__ __forceinline__ float2 nb_f2(float v) { return make_float2(v, v); }

// Constants of one force call in packed form (both lanes equal).
struct nb_coul2 {
    float2 kexp, beta, c2b;
    float2 nsh;              // -erfc(beta rc)/rc
    float2 m2krf, krf, ncrf;  // -2 k_rf, k_rf, -c_rf
    float2 krf_lo, ncrf_lo;   // k_rf and -c_rf residuals
};

inline nb_coul2 nb_pack_coul(const nb_coul &c) {
    nb_coul2 r;
    r.kexp = make_float2(c.kexp, c.kexp);
    r.beta = make_float2(c.beta, c.beta);
    r.c2b = make_float2(c.c2b, c.c2b);
    r.nsh = make_float2(-c.sh, -c.sh);
    r.m2krf = make_float2(-2.0f * c.krf, -2.0f * c.krf);
    r.krf = make_float2(c.krf, c.krf);
    r.ncrf = make_float2(-c.crf, -c.crf);
    r.krf_lo = make_float2(c.krf_lo, c.krf_lo);
    r.ncrf_lo = make_float2(-c.crf_lo, -c.crf_lo);
    return r;
}

// 2^t, nb_exp2's reduction and polynomial per lane.
__device__ __forceinline__ float2 nb_exp2_x2(float2 t) {
    const float2 magic = nb_f2(12582912.0f);
    const float2 tn = __fadd2_rn(t, magic);
    const float2 nn = __ffma2_rn(tn, nb_f2(-1.0f), magic);  // -rint(t)
    const float2 f = __fadd2_rn(t, nn);
    float2 p = __ffma2_rn(nb_f2(NB_EXP2_C6), f, nb_f2(NB_EXP2_C5));
    p = __ffma2_rn(p, f, nb_f2(NB_EXP2_C4));
    p = __ffma2_rn(p, f, nb_f2(NB_EXP2_C3));
    p = __ffma2_rn(p, f, nb_f2(NB_EXP2_C2));
    p = __ffma2_rn(p, f, nb_f2(NB_EXP2_C1));
    p = __ffma2_rn(p, f, nb_f2(1.0f));
    return make_float2(__int_as_float(__float_as_int(p.x) + __float_as_int(tn.x) * (1 << 23)),
                       __int_as_float(__float_as_int(p.y) + __float_as_int(tn.y) * (1 << 23)));
}

// erfcx on [0, 3.2], nb_erfcx per lane.
__device__ __forceinline__ float2 nb_erfcx_x2(float2 x) {
    float2 p = __ffma2_rn(nb_f2(NB_ERFCX_P4), x, nb_f2(NB_ERFCX_P3));
    p = __ffma2_rn(p, x, nb_f2(NB_ERFCX_P2));
    p = __ffma2_rn(p, x, nb_f2(NB_ERFCX_P1));
    p = __ffma2_rn(p, x, nb_f2(1.0f));
    float2 nq = __ffma2_rn(nb_f2(-NB_ERFCX_Q4), x, nb_f2(-NB_ERFCX_Q3));
    nq = __ffma2_rn(nq, x, nb_f2(-NB_ERFCX_Q2));
    nq = __ffma2_rn(nq, x, nb_f2(-NB_ERFCX_Q1));
    nq = __ffma2_rn(nq, x, nb_f2(-1.0f));  // -Q(x)
    float2 y = make_float2(nb_rcp(-nq.x), nb_rcp(-nq.y));
#if NB_RCP_NR
    const float2 e = __ffma2_rn(nq, y, nb_f2(1.0f));  // 1 - Q y
    y = __ffma2_rn(y, e, y);
#endif
    return __fmul2_rn(p, y);
}

// Rows a, b (positions xi*, f q_i in qi) against j (negated position
// nxj*, charge qj, all lanes equal) with shift S*. lj = (C6_a, C6_b,
// C12_a, C12_b), nshlj = minus the LJ shifts of a and b. in_a, in_b: the
// list mask bits. Adds the rows' forces to fi*, the j force (positive sign,
// summed over rows) to gj*, and with ENERGY the pair energies to ec, elj.
// Returns the number of the two pairs within rc.
template <bool ENERGY, int COUL>
__device__ __forceinline__ int nb_pair_x2(const float2 xix, const float2 xiy, const float2 xiz, const float2 qi,
                                          const float2 nxjx, const float2 nxjy, const float2 nxjz, const float2 qj,
                                          const float2 Sx, const float2 Sy, const float2 Sz, const float4 lj,
                                          const float2 nshlj, const bool in_a, const bool in_b, const float rc2,
                                          const nb_coul2 &cc, float2 &fix, float2 &fiy, float2 &fiz, float2 &gjx,
                                          float2 &gjy, float2 &gjz, float2 &ec, float2 &elj) {
    const float2 dx = __fadd2_rn(__fadd2_rn(xix, nxjx), Sx);
    const float2 dy = __fadd2_rn(__fadd2_rn(xiy, nxjy), Sy);
    const float2 dz = __fadd2_rn(__fadd2_rn(xiz, nxjz), Sz);
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
    const bool ia = in_a && (r2.x < rc2);
    const bool ib = in_b && (r2.y < rc2);
    const float2 y0 = make_float2(nb_rsqrt(r2.x), nb_rsqrt(r2.y));
    const float2 nres = __ffma2_rn(__fmul2_rn(r2, y0), y0, nb_f2(-1.0f));  // -(1 - r2 y0^2)
    const float2 rinv = __ffma2_rn(__fmul2_rn(nb_f2(-0.5f), y0), nres, y0);
    const float2 rinv2 = __fmul2_rn(rinv, rinv);
    const float2 rinv6 = __fmul2_rn(__fmul2_rn(rinv2, rinv2), rinv2);
    const float2 v6 = __fmul2_rn(make_float2(lj.x, lj.y), rinv6);
    const float2 v12 = __fmul2_rn(__fmul2_rn(make_float2(lj.z, lj.w), rinv6), rinv6);
    const float2 slj = __fmul2_rn(__ffma2_rn(nb_f2(12.0f), v12, __fmul2_rn(nb_f2(-6.0f), v6)), rinv2);
    const float2 qq = __fmul2_rn(qi, qj);
    float2 s, a;
    if (COUL == NB_COULK_RF) {
        s = __ffma2_rn(qq, __ffma2_rn(rinv, rinv2, cc.m2krf), slj);
    } else {
        const float2 r = __fmul2_rn(r2, rinv);
        const float2 ex = nb_exp2_x2(__fmul2_rn(cc.kexp, r2));
        a = __fmul2_rn(__fmul2_rn(ex, nb_erfcx_x2(__fmul2_rn(cc.beta, r))), rinv);
        s = __ffma2_rn(__fmul2_rn(qq, __ffma2_rn(cc.c2b, ex, a)), rinv2, slj);
    }
    s.x = ia ? s.x : 0.0f;
    s.y = ib ? s.y : 0.0f;
    fix = __ffma2_rn(s, dx, fix);
    fiy = __ffma2_rn(s, dy, fiy);
    fiz = __ffma2_rn(s, dz, fiz);
    gjx = __ffma2_rn(s, dx, gjx);
    gjy = __ffma2_rn(s, dy, gjy);
    gjz = __ffma2_rn(s, dz, gjz);
    if (ENERGY) {
        float2 e_c;
        if (COUL == NB_COULK_RF) {
            const float2 lo = __fmul2_rn(qq, __ffma2_rn(cc.krf_lo, r2, cc.ncrf_lo));
            e_c = __ffma2_rn(qq, __fadd2_rn(rinv, __ffma2_rn(cc.krf, r2, cc.ncrf)), lo);
        } else if (COUL == NB_COULK_EWALD_SHIFT) {
            e_c = __fmul2_rn(qq, __fadd2_rn(a, cc.nsh));
        } else {
            e_c = __fmul2_rn(qq, a);
        }
        float2 e_lj = __fadd2_rn(__ffma2_rn(v6, nb_f2(-1.0f), v12), nshlj);  // v12 - v6 - shift
        e_c.x = ia ? e_c.x : 0.0f;
        e_c.y = ib ? e_c.y : 0.0f;
        e_lj.x = ia ? e_lj.x : 0.0f;
        e_lj.y = ib ? e_lj.y : 0.0f;
        ec = __fadd2_rn(ec, e_c);
        elj = __fadd2_rn(elj, e_lj);
    }
    return (ia ? 1 : 0) + (ib ? 1 : 0);
}

// Rows a, b (.x, .y) of the adjoint pair nb_pair_adj<true, COUL> against
// one j atom, on the packed instructions: each lane performs the scalar
// form's operations in its order (negations exact), so a row's values are
// bit-equal to nb_pair_adj's. Inputs: the rows' positions xi*, f q_i in
// qi_f and g in gi*; the j atom's negated position nxj*, charge qj, f q_j
// in qj_f and negated g in ngj*; the shift S*; the rows' C6, C12 against
// the j atom's type; the list mask bits in_a, in_b. Adds to the rows'
// (dL/dx, dL/dq) in bi*; adds to vj* the vector v that the j atom's dL/dx
// loses (subtract it once per j atom), and to bjq the j atom's dL/dq; d6,
// d12 receive the two pairs' dL/dC6, dL/dC12 (0 when a pair does not count).
template <int COUL>
__device__ __forceinline__ void nb_pair_adj_x2(const float2 xix, const float2 xiy, const float2 xiz, const float2 qi_f,
                                               const float2 gix, const float2 giy, const float2 giz,
                                               const float2 nxjx, const float2 nxjy, const float2 nxjz,
                                               const float2 qj, const float2 qj_f, const float2 ngjx,
                                               const float2 ngjy, const float2 ngjz, const float2 Sx, const float2 Sy,
                                               const float2 Sz, const float2 c6, const float2 c12, const bool in_a,
                                               const bool in_b, const float rc2, const nb_coul2 &cc, const float2 nk2,
                                               float2 &bix, float2 &biy, float2 &biz, float2 &biq, float2 &vjx,
                                               float2 &vjy, float2 &vjz, float2 &bjq, float2 &d6, float2 &d12) {
    const float2 dx = __fadd2_rn(__fadd2_rn(xix, nxjx), Sx);
    const float2 dy = __fadd2_rn(__fadd2_rn(xiy, nxjy), Sy);
    const float2 dz = __fadd2_rn(__fadd2_rn(xiz, nxjz), Sz);
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
    const bool ia = in_a && (r2.x < rc2);
    const bool ib = in_b && (r2.y < rc2);
    const float2 y0 = make_float2(nb_rsqrt(r2.x), nb_rsqrt(r2.y));
    const float2 nres = __ffma2_rn(__fmul2_rn(r2, y0), y0, nb_f2(-1.0f));  // -(1 - r2 y0^2)
    const float2 rinv = __ffma2_rn(__fmul2_rn(nb_f2(-0.5f), y0), nres, y0);
    const float2 rinv2 = __fmul2_rn(rinv, rinv);
    const float2 rinv6 = __fmul2_rn(__fmul2_rn(rinv2, rinv2), rinv2);
    const float2 v6 = __fmul2_rn(c6, rinv6);
    const float2 v12 = __fmul2_rn(__fmul2_rn(c12, rinv6), rinv6);
    const float2 slj = __fmul2_rn(__ffma2_rn(nb_f2(12.0f), v12, __fmul2_rn(nb_f2(-6.0f), v6)), rinv2);
    const float2 qq = __fmul2_rn(qi_f, qj);
    float2 Bc, cpr;  // B, and r^2 (1/r) dB/dr times f q_a q_b
    if (COUL == NB_COULK_RF) {
        const float2 rinv3 = __fmul2_rn(rinv, rinv2);
        Bc = __fadd2_rn(rinv3, cc.m2krf);  // 1/r^3 - 2 k_rf
        cpr = __fmul2_rn(__fmul2_rn(nb_f2(-3.0f), qq), rinv3);
    } else {
        const float2 r = __fmul2_rn(r2, rinv);
        const float2 ex = nb_exp2_x2(__fmul2_rn(cc.kexp, r2));
        const float2 a = __fmul2_rn(__fmul2_rn(ex, nb_erfcx_x2(__fmul2_rn(cc.beta, r))), rinv);
        Bc = __fmul2_rn(__ffma2_rn(cc.c2b, ex, a), rinv2);
        cpr = __ffma2_rn(nb_f2(-3.0f), __fmul2_rn(qq, Bc), __fmul2_rn(__fmul2_rn(nk2, qq), ex));
    }
    const float2 s = __fadd2_rn(__fmul2_rn(qq, Bc), slj);
    const float2 spr =
        __fmul2_rn(rinv2, __ffma2_rn(rinv2, __ffma2_rn(nb_f2(48.0f), v6, __fmul2_rn(nb_f2(-168.0f), v12)), cpr));
    const float2 ux = __fadd2_rn(gix, ngjx), uy = __fadd2_rn(giy, ngjy), uz = __fadd2_rn(giz, ngjz);
    const float2 ud = __ffma2_rn(ux, dx, __ffma2_rn(uy, dy, __fmul2_rn(uz, dz)));
    // pairs that do not count can carry inf/NaN (r2 = 0 on a masked diagonal): select, never multiply
    float2 sm = s, t = __fmul2_rn(spr, ud), bud = __fmul2_rn(Bc, ud);
    const float2 r8ud = __fmul2_rn(__fmul2_rn(rinv6, rinv2), ud);
    float2 e6 = __fmul2_rn(nb_f2(-6.0f), r8ud), e12 = __fmul2_rn(__fmul2_rn(nb_f2(12.0f), rinv6), r8ud);
    sm.x = ia ? sm.x : 0.0f;
    sm.y = ib ? sm.y : 0.0f;
    t.x = ia ? t.x : 0.0f;
    t.y = ib ? t.y : 0.0f;
    bud.x = ia ? bud.x : 0.0f;
    bud.y = ib ? bud.y : 0.0f;
    e6.x = ia ? e6.x : 0.0f;
    e6.y = ib ? e6.y : 0.0f;
    e12.x = ia ? e12.x : 0.0f;
    e12.y = ib ? e12.y : 0.0f;
    const float2 vx = __ffma2_rn(sm, ux, __fmul2_rn(t, dx));
    const float2 vy = __ffma2_rn(sm, uy, __fmul2_rn(t, dy));
    const float2 vz = __ffma2_rn(sm, uz, __fmul2_rn(t, dz));
    bix = __fadd2_rn(bix, vx);
    biy = __fadd2_rn(biy, vy);
    biz = __fadd2_rn(biz, vz);
    vjx = __fadd2_rn(vjx, vx);
    vjy = __fadd2_rn(vjy, vy);
    vjz = __fadd2_rn(vjz, vz);
    biq = __ffma2_rn(qj_f, bud, biq);
    bjq = __ffma2_rn(qi_f, bud, bjq);
    d6 = e6;
    d12 = e12;
}
