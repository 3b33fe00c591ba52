// gw_dfloat.cuh -- double-float numbers (an unevaluated sum hi + lo of two
// FP32 numbers, |lo| <= ulp(hi) / 2, ~2^-48 relative) as a scalar type for the
// templated point formulas of gw_points_fp64.cuh, so that the same source
// evaluates the tangents in FP64 (on the FP64 pipe) or in double-float (on the
// FP32 pipe, ~90 times the FP64 rate on this GPU).
//
// Error-free transforms: Knuth's two-sum, Dekker's product with an FMA (the
// product error fma(a, b, -a b) is exact).  Addition is the "sloppy" form (one
// two-sum of the high parts, low parts added, renormalised): its error is
// ~2^-48 of |a| + |b|, i.e. of the operands, which is what the Gram of the
// tangents needs (an error relative to the tangents' own scale perturbs the
// vectors, and a vector perturbation reaches the covariance only through the
// square root of the condition number).  Division, square root and sine and
// cosine take one FP32 estimate and one Newton or Taylor correction in
// double-float.  Range: that of FP32 (the callers keep the noise curve and the
// amplitude in scaled units).
#pragma once

#include <cuda_runtime.h>

namespace gw {

// the FP64 functions keep their names inside the namespace next to the
// double-float overloads below
using ::fma;
using ::sincos;
using ::sqrt;

struct dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    // from a double (folded at compile time for constants; a runtime double
    // costs two conversions on the FP64 pipe)
    __host__ __device__ constexpr explicit dfl(double x)
        : hi((float)x), lo((float)(x - (double)(float)x))
    {
    }
};

__device__ __forceinline__ dfl df_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return dfl(s, (a - (s - bb)) + (b - bb));
}

__device__ __forceinline__ dfl df_fast_two_sum(float a, float b)   // |a| >= |b|
{
    const float s = a + b;
    return dfl(s, b - (s - a));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b)
{
    dfl s = df_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }

__device__ __forceinline__ dfl operator*(dfl a, dfl b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

// by an FP32 number (exact for powers of two)
__device__ __forceinline__ dfl df_mul_f(dfl a, float b)
{
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return df_fast_two_sum(p, e);
}

// mixed forms with double constants (split at compile time)
__device__ __forceinline__ dfl operator*(double c, dfl a) { return dfl(c) * a; }
__device__ __forceinline__ dfl operator*(dfl a, double c) { return a * dfl(c); }
__device__ __forceinline__ dfl operator+(dfl a, double c) { return a + dfl(c); }
__device__ __forceinline__ dfl operator+(double c, dfl a) { return dfl(c) + a; }
__device__ __forceinline__ dfl operator-(dfl a, double c) { return a + dfl(-c); }
__device__ __forceinline__ dfl operator-(double c, dfl a) { return dfl(c) - a; }

__device__ __forceinline__ dfl fma(dfl a, dfl b, dfl c) { return a * b + c; }
__device__ __forceinline__ dfl fma(dfl a, dfl b, double c) { return a * b + dfl(c); }
__device__ __forceinline__ dfl fma(double a, dfl b, dfl c) { return dfl(a) * b + c; }

__device__ __forceinline__ float df_round(dfl a) { return a.hi + a.lo; }

// 1/b: FP32 estimate, one Newton step r = r + r (1 - b r) in double-float
__device__ __forceinline__ dfl df_rcp(dfl b)
{
    const float r = __frcp_rn(b.hi);
    const dfl e = dfl(1.0f, 0.0f) - df_mul_f(b, r);   // 1 - b r, small
    return df_fast_two_sum(r, r * e.hi);
}

__device__ __forceinline__ dfl df_div(dfl a, dfl b)
{
    const float q0 = __fdiv_rn(a.hi, b.hi);
    const dfl r = a - df_mul_f(b, q0);                 // a - b q0
    return df_fast_two_sum(q0, __fdiv_rn(r.hi, b.hi));
}

// sqrt(a), a > 0: y0 = sqrt(a_hi) rounded, y = y0 + (a - y0^2) / (2 y0)
__device__ __forceinline__ dfl df_sqrt(dfl a)
{
    if (!(a.hi > 0.0f)) return dfl(a.hi == 0.0f ? 0.0f : __fsqrt_rn(a.hi), 0.0f);
    const float y0 = __fsqrt_rn(a.hi);
    const float sq = y0 * y0;
    const dfl d = a - dfl(sq, fmaf(y0, y0, -sq));       // a - y0^2 (y0^2 exact as a pair)
    return df_fast_two_sum(y0, d.hi * (0.5f / y0));
}

// integer power, |p| <= 31 (binary powering)
__device__ __forceinline__ dfl df_ipow(dfl x, int p)
{
    dfl r(1.0f, 0.0f);
    if (p < 0) {
        x = df_rcp(x);
        p = -p;
    }
    while (p) {
        if (p & 1) r = r * x;
        x = x * x;
        p >>= 1;
    }
    return r;
}

// Two double-float numbers computed together with the packed FP32x2
// instructions (FADD2, FMUL2, FFMA2): lane x holds one number, lane y the
// other.  Each operation is the double-float operation above applied to both
// lanes (the packed instructions round each lane as the scalar ones do), in
// half the instructions.  Used for quantities that come in pairs: the real and
// imaginary parts of a tangent, the pattern functions F+ and Fx, sine and
// cosine.
struct dfl2 {
    float2 hi, lo;
};

__device__ __forceinline__ dfl2 d2_make(dfl x, dfl y)
{
    return dfl2{make_float2(x.hi, y.hi), make_float2(x.lo, y.lo)};
}
__device__ __forceinline__ dfl2 d2_bcast(dfl s)
{
    return dfl2{make_float2(s.hi, s.hi), make_float2(s.lo, s.lo)};
}
__device__ __forceinline__ dfl d2_x(const dfl2 &a) { return dfl(a.hi.x, a.lo.x); }
__device__ __forceinline__ dfl d2_y(const dfl2 &a) { return dfl(a.hi.y, a.lo.y); }

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

// (x, y) -> (-y, x): the pair times i, read as (Re, Im)
__device__ __forceinline__ dfl2 d2_mul_i(const dfl2 &a)
{
    return dfl2{make_float2(-a.hi.y, a.hi.x), make_float2(-a.lo.y, a.lo.x)};
}

__device__ __forceinline__ dfl2 d2_fast_two_sum(float2 a, float2 b)   // |a| >= |b| per lane
{
    const float2 s = __fadd2_rn(a, b);
    return dfl2{s, __fadd2_rn(b, f2neg(__fadd2_rn(s, f2neg(a))))};
}

__device__ __forceinline__ dfl2 operator+(const dfl2 &a, const dfl2 &b)
{
    // two-sum of the high parts, low parts added, renormalised
    const float2 s = __fadd2_rn(a.hi, b.hi);
    const float2 bb = __fadd2_rn(s, f2neg(a.hi));
    const float2 e = __fadd2_rn(__fadd2_rn(a.hi, f2neg(__fadd2_rn(s, f2neg(bb)))),
                                __fadd2_rn(b.hi, f2neg(bb)));
    return d2_fast_two_sum(s, __fadd2_rn(e, __fadd2_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dfl2 operator-(const dfl2 &a)
{
    return dfl2{f2neg(a.hi), f2neg(a.lo)};
}
__device__ __forceinline__ dfl2 operator-(const dfl2 &a, const dfl2 &b) { return a + (-b); }

__device__ __forceinline__ dfl2 operator*(const dfl2 &a, const dfl2 &b)
{
    const float2 p = __fmul2_rn(a.hi, b.hi);
    float2 e = __ffma2_rn(a.hi, b.hi, f2neg(p));
    e = __ffma2_rn(a.hi, b.lo, e);
    e = __ffma2_rn(a.lo, b.hi, e);
    return d2_fast_two_sum(p, e);
}

// a * s + c with a double-float scalar s in both lanes
__device__ __forceinline__ dfl2 d2_fma(const dfl2 &a, dfl s, const dfl2 &c)
{
    return a * d2_bcast(s) + c;
}


// Overloads with the names the templated formulas call.
__device__ __forceinline__ dfl sqrt(dfl a) { return df_sqrt(a); }

// sine and cosine of x (|x| up to a few hundred): x reduced by multiples of
// pi/2 in double-float (pi/2 to three FP32 parts), then Taylor series of sin
// and cos on |r| <= pi/4 (terms to r^15 and r^16: the first omitted term is
// below 2^-52 of the result), evaluated in double-float by Horner's rule in
// r^2; the quadrant selects and signs the pair.
namespace dfs {
// (-1)^n / m! (m = 2n + 1 for the sine, 2n for the cosine)
__host__ __device__ constexpr double taylor(int m)
{
    double f = 1.0;
    for (int i = 2; i <= m; i++) f *= (double)i;
    return ((m / 2) % 2 ? -1.0 : 1.0) / f;
}
// pi/2 = P1 + P2 + P3 (Cody and Waite): P1 and P2 carry 15 significant bits
// each, so k P1 and k P2 are exact in FP32 for |k| < 2^9; P3 is the rest
constexpr double PIO2 = 1.5707963267948966192;
constexpr double P1D = (double)(long long)(PIO2 * 16384.0) / 16384.0;
constexpr double P2D = (double)(long long)((PIO2 - P1D) * 536870912.0) / 536870912.0;
constexpr float P1 = (float)P1D;
constexpr float P2 = (float)P2D;
constexpr float P3 = (float)(PIO2 - P1D - P2D);
}  // namespace dfs

// the coefficients as double-float pairs, fixed at compile time:
// kTaylor[m] = (-1)^(m/2) / m!, m = 0..16
#define GW_DFL_TAYLOR(m) {(float)dfs::taylor(m), (float)(dfs::taylor(m) - (double)(float)dfs::taylor(m))}
__constant__ const float2 kTaylor[17] = {
    GW_DFL_TAYLOR(0),  GW_DFL_TAYLOR(1),  GW_DFL_TAYLOR(2),  GW_DFL_TAYLOR(3),  GW_DFL_TAYLOR(4),
    GW_DFL_TAYLOR(5),  GW_DFL_TAYLOR(6),  GW_DFL_TAYLOR(7),  GW_DFL_TAYLOR(8),  GW_DFL_TAYLOR(9),
    GW_DFL_TAYLOR(10), GW_DFL_TAYLOR(11), GW_DFL_TAYLOR(12), GW_DFL_TAYLOR(13), GW_DFL_TAYLOR(14),
    GW_DFL_TAYLOR(15), GW_DFL_TAYLOR(16)};
#undef GW_DFL_TAYLOR

__device__ __forceinline__ dfl taylor_coef(int m) { return dfl(kTaylor[m].x, kTaylor[m].y); }

__device__ __forceinline__ void sincos(dfl x, dfl *sx, dfl *cx)
{
    const float k = rintf(x.hi * 0.636619772f);          // nearest multiple of pi/2
    // r = x - k pi/2: k P1 and k P2 exact, k P3 rounded (|k P3| < 1e-6)
    dfl r = x + dfl(-k * dfs::P1, 0.0f);
    r = r + dfl(-k * dfs::P2, 0.0f);
    r = r + dfl(-k * dfs::P3, 0.0f);
    const dfl r2 = r * r;
    // both series in one rolled loop, as one packed pair (sine in lane x,
    // cosine in lane y; rolled to keep the callers' code small)
    const dfl2 R2 = d2_bcast(r2);
    dfl2 sc = d2_make(taylor_coef(15), taylor_coef(16) * r2 + taylor_coef(14));
#pragma unroll 1
    for (int n = 6; n >= 0; n--) sc = sc * R2 + d2_make(taylor_coef(2 * n + 1), taylor_coef(2 * n));
    const dfl s = d2_x(sc) * r, c = d2_y(sc);
    const int q = ((int)k) & 3;
    const dfl sn = (q == 0) ? s : (q == 1) ? c : (q == 2) ? -s : -c;
    const dfl cs = (q == 0) ? c : (q == 1) ? -s : (q == 2) ? -c : s;
    *sx = sn;
    *cx = cs;
}

}  // namespace gw
