// dwmath.cuh -- double-word ("double-float") FP32 arithmetic shared by the
// omega sweep and the derivative's pair sums: error-free transformations
// (TwoSum after Knuth, FastTwoSum after Dekker, TwoProd by FMA), a
// renormalised double-word addition (Joldes, Muller, Popescu 2017) and exp
// of a double-word argument by table-driven reduction (Tang 1989).
#pragma once
#include "common.cuh"

namespace iso {

struct ExpTable {
    float2 t[64];   // 2^(-j/64) as (hi, lo)
};
ExpTable make_exp_table();   // computed on the host in FP64 (weights.cu)

// ln2/64 = C1 + C2 + C3 (C1 has 11 significant bits: k*C1 is exact for |k| < 2^13)
#define ISO_C1 0x1.63p-7f
#define ISO_C2 (-0x1.bd0106p-19f)
#define ISO_C3 0x1.cf79acp-46f
#define ISO_INV_C 92.33248261689366f

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
// (h, l) += (bh, bl), renormalised
__device__ __forceinline__ void dw_add(float &h, float &l, float bh, float bl) {
    float s, e;
    two_sum(h, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(l, bl));
    fast_two_sum(s, e, h, l);
}


// exp(-z) * 1 for z given as a double-word, result as a double-word.
__device__ __forceinline__ void dw_exp_neg(float zh, float zl, const float2 *__restrict__ tab, float &oh, float &ol) {
    const float kf = rintf(__fmul_rn(zh, ISO_INV_C));
    const int k = (int)kf;
    const float t1 = __fmaf_rn(-kf, ISO_C1, zh);        // exact
    float p2, p2e;
    two_prod(kf, ISO_C2, p2, p2e);
    float rh, re;
    two_sum(t1, -p2, rh, re);
    re = __fadd_rn(__fsub_rn(re, p2e), __fmaf_rn(-kf, ISO_C3, zl));
    float rl;
    fast_two_sum(rh, re, rh, rl);
    // exp(-r) = 1 - r + r^2/2 - r^3/6 + r^4/24 - r^5/120
    float s2, s2e;
    two_prod(rh, rh, s2, s2e);
    s2e = __fmaf_rn(__fadd_rn(rh, rh), rl, s2e);
    const float h2 = __fmul_rn(0.5f, s2), h2e = __fmul_rn(0.5f, s2e);
    const float poly = __fmaf_rn(__fmaf_rn(-1.0f / 120.0f, rh, 1.0f / 24.0f), rh, -1.0f / 6.0f);
    const float tail = __fmul_rn(__fmul_rn(s2, rh), poly);
    float eh, el;
    two_sum(1.0f, -rh, eh, el);
    el = __fadd_rn(__fsub_rn(el, rl), __fadd_rn(h2e, tail));
    float eh2, el2;
    two_sum(eh, h2, eh2, el2);
    el2 = __fadd_rn(el2, el);
    float mh, ml;
    fast_two_sum(eh2, el2, mh, ml);
    const float2 T = tab[k & 63];
    float ph, pl;
    two_prod(mh, T.x, ph, pl);
    pl = __fmaf_rn(mh, T.y, pl);
    pl = __fmaf_rn(ml, T.x, pl);
    const float scale = __int_as_float((127 - (k >> 6)) << 23);
    oh = __fmul_rn(ph, scale);
    ol = __fmul_rn(pl, scale);
}

}  // namespace iso
