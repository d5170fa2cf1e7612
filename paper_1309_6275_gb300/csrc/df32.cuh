// df32.cuh -- double-float arithmetic (an unevaluated sum hi + lo of two
// float32 values, ~44 significant bits) and the second-tier evaluation of a
// (hit, rho row, phi0 column) built on it.
//
// Methods: Knuth's TwoSum and the FMA form of Dekker's TwoProduct give the
// exact rounding error of a float32 sum or product; double-float add,
// multiply, divide (one correction step) and square root (one Newton step)
// follow the classical double-length algorithms (Dekker 1971; Hida, Li and
// Bailey 2001).  Each operation here has relative error well below 2^-42 of
// its operands' magnitudes, which is the unit the bounds below use.
#pragma once

#include "ht_internal.cuh"

namespace ht {

struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 two_sum(float a, float b)
{
    const float s = a + b;
    const float v = s - a;
    return F2{s, (a - (s - v)) + (b - v)};
}

__device__ __forceinline__ F2 fast_two_sum(float a, float b)   // |a| >= |b| or a == 0
{
    const float s = a + b;
    return F2{s, b - (s - a)};
}

__device__ __forceinline__ F2 two_prod(float a, float b)
{
    const float p = a * b;
    return F2{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ F2 df_add(F2 a, F2 b)
{
    F2 s = two_sum(a.hi, b.hi);
    const float e = s.lo + (a.lo + b.lo);
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ F2 df_neg(F2 a) { return F2{-a.hi, -a.lo}; }

__device__ __forceinline__ F2 df_mul(F2 a, F2 b)
{
    F2 p = two_prod(a.hi, b.hi);
    float e = fmaf(a.hi, b.lo, p.lo);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ F2 df_mulf(F2 a, float b)
{
    F2 p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}

__device__ __forceinline__ F2 df_div(F2 a, F2 b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const F2 r = df_add(a, df_neg(df_mulf(b, q1)));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ F2 df_sqrt(F2 a)   // a.hi > 0
{
    const float s = __fsqrt_rn(a.hi);
    const F2 r = df_add(a, df_neg(two_prod(s, s)));
    return fast_two_sum(s, __fdiv_rn(r.hi, 2.0f * s));
}

// Bin decision of a double-float bin coordinate u with bound e (bins):
// j >= 0, -1 (outside the axis) or -2 (undecided).
__device__ __forceinline__ int decide_df(F2 u, float e, float nd)
{
    const float uh = u.hi + u.lo;
    if (uh + 2.0f * e < -0.5f || uh - 2.0f * e >= nd + 0.5f) return -1;
    const float f = floorf(uh);
    // distances to the integers below and above, each in double-float so
    // that its leading part is accurate relative to its own (small) size
    const F2 d0 = df_add(u, F2{-f, 0.0f});
    const F2 d1 = df_add(F2{f + 1.0f, 0.0f}, df_neg(u));
    if (!(fminf(d0.hi, d1.hi) > e)) return -2;
    return (f >= 0.0f && f < nd) ? (int)f : -1;
}

// Second tier: both roots in double-float with first-order bounds of the
// same form as eval32's, unit 2^-42 instead of 2^-24.  Returns kDecided
// (jA, jB = bin or -1) or kRedo (redo in float64).
static __device__ __noinline__ int eval_df(const DevGeom &G, float xf, float yf, int i, int k,
                                    int &jA, int &jB)
{
    jA = -1;
    jB = -1;
    const float ud = 2.2737368e-13f;   // 2^-42
    const F2 sn{G.sn32[k], G.snlo[k]}, cs{G.cs32[k], G.cslo[k]};
    const F2 rho{G.rho32[i], G.rholo[i]};
    const F2 s = df_add(df_mulf(sn, xf), df_neg(df_mulf(cs, yf)));
    const F2 c = df_add(df_mulf(cs, xf), df_mulf(sn, yf));
    const float R1 = fabsf(xf) + fabsf(yf);
    const float P = fabsf(rho.hi) * R1 * 1.0001f;
    const float Ec = kSafe * 3.0f * ud * R1;
    if (c.hi <= Ec) return (c.hi < -Ec) ? kDecided : kRedo;
    const F2 r2 = df_add(two_prod(xf, xf), two_prod(yf, yf));
    const F2 b = df_add(F2{1.0f, 0.0f}, df_mul(rho, s));
    const F2 pc = df_mul(rho, c);
    const F2 D = df_add(F2{1.0f, 0.0f}, df_neg(df_mul(pc, pc)));
    const float eD = kSafe * ud * fmaf(10.0f * P, P, 2.0f);
    if (D.hi <= eD) return (D.hi < -eD) ? kDecided : kRedo;
    const F2 sq = df_sqrt(D);
    const F2 q = df_neg(b.hi >= 0.0f ? df_add(b, sq) : df_add(b, df_neg(sq)));
    const F2 C = df_add(df_mul(rho, r2), df_add(s, s));
    const float nd = (float)G.n_d0;
    const float es = kSafe * ud / G.delta_f * 1.0001f;
    const float rs = 1.0f / sq.hi;
    const float Qa = fmaf(6.0f, P, 9.0f), Qb = fmaf(5.0f * P, P, 0.5f);
    const float Q = fmaf(Qb, rs, Qa);
    const float e3 = es * 6.0f * G.dext_f + kSafe * ud * (nd + 1.0f);
    const F2 inv_delta{G.inv_delta_f, G.inv_delta_lo};
    // root A = C / q
    const F2 dA = df_div(C, q);
    const F2 uA = df_add(df_mul(dA, inv_delta), F2{G.off_f, 0.0f});
    const float iq = fabsf(1.0f / q.hi);
    const float Ea = fmaf(3.0f * fabsf(rho.hi), r2.hi, 6.0f * R1);
    const float eA = fmaf(iq * es, fmaf(G.dext_f, Q, Ea), e3);
    jA = decide_df(uA, eA, nd);
    if (jA == -2) return kRedo;
    if (rho.hi != 0.0f) {   // rho == 0 exactly iff its float32 rounding is 0
        const F2 dB = df_div(q, rho);
        const F2 uB = df_add(df_mul(dB, inv_delta), F2{G.off_f, 0.0f});
        const float eB = fmaf(fabsf(1.0f / rho.hi) * es, Q, e3);
        jB = decide_df(uB, eB, nd);
        if (jB == -2) return kRedo;
    }
    return kDecided;
}

// Both tiers behind the float32 one: double-float, then float64 in the
// definition's order.  Returns the number of bins written to jj.
__device__ __forceinline__ int redo_bins(const DevGeom &G, float xf, float yf, int i, int k,
                                         int jj[2])
{
    int jA, jB;
    if (eval_df(G, xf, yf, i, k, jA, jB) == kDecided) {
        int nv = 0;
        if (jA >= 0) jj[nv++] = jA;
        if (jB >= 0) jj[nv++] = jB;
        return nv;
    }
    int edge = 0;
    return cell_bins64(G, xf, yf, i, k, jj, &edge);
}

}  // namespace ht
