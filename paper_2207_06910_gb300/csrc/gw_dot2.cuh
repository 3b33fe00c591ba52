// gw_dot2.cuh -- compensated dot products in double-float on packed FP32x2
// operations, and the layout of the per-item copy of the PN polynomial
// coefficients they read.  Used by the mixed point kernel (phase and tau*
// derivatives rounded to FP32) and by the double-float Fisher pass (kept as
// double-float numbers).
#pragma once

#include "gw_dfloat.cuh"
#include "gw_internal.cuh"

namespace gw {

// packed FP32x2 subtraction (sm_100+)
__device__ __forceinline__ float2 f2sub(float2 a, float2 b)
{
    unsigned long long ra = *reinterpret_cast<unsigned long long *>(&a);
    unsigned long long rb = *reinterpret_cast<unsigned long long *>(&b);
    unsigned long long rd;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<float2 *>(&rd);
}

// Compensated dot products sum_q c_q b_q with double-float coefficients and
// basis values (Dot2 of Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26 (2005)): the high products are summed with
// error-free transforms (exact product error by an FMA, Knuth's two-sum) and
// all errors, together with the cross products of high and low parts, are
// summed into one compensation term.  The result is as accurate as if it were
// computed in twice the FP32 precision.  dot2_pk evaluates two such sums at
// once in the two lanes of packed FP32x2 operations: c[q] = (high part of the
// lane-x coefficient, high part of lane y, low part x, low part y).
struct DF2 {
    float2 hi, lo;
};

template <int N>
__device__ __forceinline__ DF2 dot2_pk(const float4 *c, const dfl (&b)[N], const float (&nb)[N])
{
    float4 cq = c[0];
    float2 ch = make_float2(cq.x, cq.y), cl = make_float2(cq.z, cq.w);
    float2 bh = make_float2(b[0].hi, b[0].hi);
    float2 s = __fmul2_rn(ch, bh);
    float2 comp = __ffma2_rn(ch, make_float2(b[0].lo, b[0].lo),
                             __ffma2_rn(ch, bh, __fmul2_rn(ch, make_float2(nb[0], nb[0]))));
    comp = __ffma2_rn(cl, bh, comp);
#pragma unroll
    for (int q = 1; q < N; q++) {
        cq = c[q];
        ch = make_float2(cq.x, cq.y);
        cl = make_float2(cq.z, cq.w);
        bh = make_float2(b[q].hi, b[q].hi);
        // two-sum t = s + p with nbb = s - t = -bb; the correction (s's roundoff
        // t2, p's roundoff p - bb and the product error c b - p) is
        // t2 + (c b - bb), the last term one FMA: the addend's roundoff less
        // the product's rounding error is -(c b + nbb), of roundoff size
        const float2 p = __fmul2_rn(ch, bh);
        const float2 t = __fadd2_rn(s, p);
        const float2 nbb = f2sub(s, t);
        const float2 t2 = f2sub(s, __fadd2_rn(t, nbb));
        const float2 y = __ffma2_rn(ch, bh, nbb);
        s = t;
        comp = __fadd2_rn(comp, __fadd2_rn(t2, y));
        comp = __ffma2_rn(ch, make_float2(b[q].lo, b[q].lo), comp);
        comp = __ffma2_rn(cl, bh, comp);
    }
    return DF2{s, comp};
}

// scalar form: c[q] = (high part, low part)
template <int N>
__device__ __forceinline__ dfl dot2_s(const float2 *c, const dfl (&b)[N])
{
    float2 cq = c[0];
    float s = cq.x * b[0].hi;
    float comp = fmaf(cq.x, b[0].lo, fmaf(cq.x, b[0].hi, -s));
    comp = fmaf(cq.y, b[0].hi, comp);
#pragma unroll
    for (int q = 1; q < N; q++) {
        cq = c[q];
        const float p = cq.x * b[q].hi;
        const float t = s + p;
        const float nbb = s - t;
        const float t2 = s - (t + nbb);
        const float y = fmaf(cq.x, b[q].hi, nbb);   // c b - bb, one rounding
        s = t;
        comp += t2 + y;
        comp = fmaf(cq.x, b[q].lo, comp);
        comp = fmaf(cq.y, b[q].hi, comp);
    }
    return df_fast_two_sum(s, comp);
}

// Layout of a work group's copy of the polynomial coefficients (floats):
// d Psi/d Mc and d Psi/d eta interleaved for dot2_pk (11 x 4), slots 9 and 10
// (4 x 4), d tau*/d Mc and d tau*/d eta (8 x 4), tau* as (hi, lo) pairs (8 x 2).
constexpr int CO_PMPE = 0, CO_P910 = 44, CO_TMTE = 60, CO_T0 = 92;
static_assert(CO_T0 + 16 == 2 * NCOEF, "coefficient copy layout");

// float offset of component part (0 = high, 1 = low) of slot EV_PM + q
__device__ __forceinline__ int coef_pos(int q, int part)
{
    const int s = EV_PM + q;
    if (s < EV_PE) return CO_PMPE + 4 * (s - EV_PM) + 2 * part;
    if (s < EV_P9) return CO_PMPE + 4 * (s - EV_PE) + 2 * part + 1;
    if (s < EV_P10) return CO_P910 + 4 * (s - EV_P9) + 2 * part;
    if (s < EV_T0) return CO_P910 + 4 * (s - EV_P10) + 2 * part + 1;
    if (s < EV_TM) return CO_T0 + 2 * (s - EV_T0) + part;
    if (s < EV_TE) return CO_TMTE + 4 * (s - EV_TM) + 2 * part;
    return CO_TMTE + 4 * (s - EV_TE) + 2 * part + 1;
}


}  // namespace gw
