// gw_points_fp64_tc.cu -- the Fisher pass with its Gram accumulation on the
// tensor cores (tcgen05), exactly, fed by tangents in FP64 or in double-float.
//
// The Fisher matrix of a work item is the Gram matrix of its tangent rows,
//     Gamma_ij = sum_k y_ik y_jk,   y_.k = (Re g, Im g) of one interferometer at
//     one grid point, tangents pre-scaled by sigma = A sqrt(4 w / S_n)
// (Sec. 3.2, Eqs. 3.1-3.3).  Every tangent value is written, per item and
// column, relative to the column's largest exponent E_i (y' = y 2^(1022 - E_i),
// |y'| < 1) as eight digits: digit a is a multiple of q_a = 2^(-7(a+1)) of
// magnitude at most 128 q_a, exact in bf16, the sum of the digits y' to 2^-57
// (FP64 values; double-float values use seven digits, y' to 2^-50).
// The tensor core forms all digit products with FP32 accumulation; a product
// of digits a and b is a multiple of q_a q_b below 2^14 q_a q_b and an item has
// at most 1024 rows (256 points x 2 interferometers x real/imaginary), so
// every partial sum is such a multiple below 2^24 q_a q_b: the accumulation is
// exact.  The digit Gram D[(i,a),(j,b)] is then summed exactly (integers) and
// rounded once to FP64,
//     Gamma_ij = 2^(E_i + E_j - 2044) sum_ab D[(i,a),(j,b)],
// so the item's Fisher matrix is the exact Gram of the tangents rounded to 56
// bits (relative to the column maximum), rounded once to FP64.
//
// The tangents come from the templated formulas of gw_points_fp64.cuh with
// scalar type T:
//  * T = double (GW_FP64 with the tensor-core Gram): the FP64 pass, every
//    operation on the FP64 pipe except the Gram;
//  * T = dfl (GW_DFLOAT): the same formulas in double-float arithmetic
//    (gw_dfloat.cuh, ~2^-48) on the FP32 pipe.  An error of the tangents
//    relative to their own scale is a perturbation of the Gram's vectors, which
//    reaches the covariance only through the square root of the condition
//    number, so double-float tangents with an exact Gram give FP64-class
//    covariances at FP32-pipe speed.  The noise curve and the amplitude are
//    carried relative to the network's reference PSD scale (FP32 range); a
//    tabulated PSD's weight is taken in FP64 and converted.
//
// Shape.  Work items of at most TC_CHUNK = 128 points (the event set-up splits
// events accordingly), one grid point per thread of a 128-thread CTA, three
// CTAs per SM, persistent: each CTA takes a contiguous range of items, finds
// the event of its first item by bisection and then walks forward, and loads
// an event's constants (and builds its power tables) once for the event's
// consecutive items.  An event's items take the even share of its points
// rounded up to whole warps (the last item the rest), and warp 3, whose TMEM
// lanes hold no Gram rows, prepares the next item while warps 0-2 read the
// current one's Gram.  Each thread writes its point's values (rows r =
// interferometer x {Re, Im}, then columns) to shared memory as it forms them
// (FP64 or double-float pairs, 8 bytes each), so that no value stays in
// registers and the kernel fits three CTAs per SM (~168 registers); the column
// maxima are reduced once the item's points are done.  The digits go to shared
// memory in the MN-major, no-swizzle operand layout (8 digits of one value =
// one 16-byte row of a core matrix; K groups of 8 rows at stride KG, MN groups
// at 128 bytes), one K block of 128 rows per row r, alternating between two
// operand buffers: a dedicated one and the staged rows 0 and 1, which are free
// once they have been turned into digits.  One thread issues a block's eight
// M=128 x N x K=16 MMAs (A = B = the block) into the item's TMEM accumulator and
// commits them to the buffer's mbarrier; the digits of the next block are
// formed meanwhile, and a buffer is rewritten only after its previous MMAs are
// done.  After the item's last block the four warps read their 32 TMEM lanes
// (rows (i, a)) and reduce over the digit pairs in 128-bit integer arithmetic,
// one rounding to FP64 per Fisher entry.  Networks of at most two
// interferometers per point (one triangle or up to two L-shaped detectors) take
// this kernel; wider networks, and the SNR, SNR-gradient and log-det passes,
// run the FP64-pipe kernel.
//
// Every wait is bounded (about a second of wall time); a wait that runs out
// sets *kerr, writes NaN into the item's sums and ends the CTA after freeing
// its TMEM.
#include <type_traits>

#include <cuda_bf16.h>

#include "gw_points_fp64.cuh"

namespace gw {

namespace {

constexpr int TC_T = 128;                 // threads = points per round
constexpr int TC_KROWS = 128;             // K rows per block (one value per thread)
constexpr int TC_MG = 128;                // bytes between MN groups (8 digits x 8 rows)
constexpr int TC_PW = 104;                // power tables (96) and per-item bases (8)

constexpr int TC_CTAS = 3;                // CTAs per SM (registers, shared memory, TMEM)
constexpr int TC_SITES = 2;               // sites of a supported network (<= 2 interferometers)

template <int NP>
struct TcShape {
    static constexpr int KG = NP * 128;                    // bytes between K groups
    static constexpr int BLK = (TC_KROWS / 8) * KG;        // one K block (the operand buffer)
    static constexpr int N = ((NP * 8 + 15) / 16) * 16;    // MMA N (digit rows used, padded)
    // The staged values follow operand buffer 0, and their rows 0 and 1 (one
    // block: 2 x NP x TC_T values of 8 bytes) are operand buffer 1: an M = 128
    // read of the last MMA step of a block reaches 2047 - KG bytes past the
    // block, into the staged values (finite data, only for accumulator rows
    // and columns never read).
    static constexpr int STAGE_BYTES = NP * 4 * TC_T * 8;
    // double-float copies: event constants, site constants, interferometer
    // (s2g, c2g, amp) and PSD constants (inverse f0, f0, coefficients)
    static constexpr int DF_WORDS = EVC + TC_SITES * SC_N + 3 * MAX_IFO +
                                    MAX_PSD * (2 + MAX_TERM) + TC_PW;
    static constexpr size_t smem(bool df)
    {
        return (size_t)BLK + STAGE_BYTES + (size_t)EVC * 8 + TC_PW * 8 + 32 * 4 + 8 + 8 + 16 + 32 +
               (df ? (size_t)DF_WORDS * 8 : 0);
    }
    static_assert(2 * BLK == STAGE_BYTES, "staged rows 0 and 1 hold one operand block");
    static_assert(2047 - KG <= STAGE_BYTES - BLK, "operand over-read stays in shared memory");
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the completion of the mbarrier phase of the given parity, for at
// most about a second
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done = 0;
    const uint64_t t0 = globaltimer();
    for (;;) {
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
        if (globaltimer() - t0 > 1000000000ull) return false;
    }
}

// shared-memory matrix descriptor, no swizzle: start, K-group stride (LBO),
// MN-group stride (SBO), descriptor version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t kstride, uint32_t mnstride)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((kstride >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((mnstride >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Digit a of a value y' in (-1, 1) (the value over 2^(ec - 1022), ec the
// column's largest biased FP64 exponent) is a multiple of q_a = 2^(-7(a+1))
// of magnitude <= 128 q_a; the row holds the eight digits as bf16 numbers in
// these absolute units (digit a in element a), so the accumulator's sums are
// exact multiples of q_a q_b below 2^24 q_a q_b and the item's Gram entry is
// the plain sum over the digit pairs.

// the eight 7-bit digits of a 56-bit magnitude N = |y'| 2^56 with the given
// sign, digit a = bits 49 - 7a .. 55 - 7a of N, valued d q_a
__device__ __forceinline__ uint4 pack_digits(unsigned long long N, bool negative)
{
    const unsigned nh = (unsigned)(N >> 28), nl = (unsigned)N & 0x0FFFFFFFu;
    // d q_a as an FP32 number: the integer d (< 2^23) in the mantissa of
    // 2^(23 - 7(a+1)) (exponent field 150 - 7(a+1)), less that power of two
    auto fd = [](unsigned d, int a) {
        const unsigned e = (unsigned)(150 - 7 * (a + 1));
        return __float_as_uint(__uint_as_float((e << 23) | d) - __uint_as_float(e << 23));
    };
    uint4 r;
    r.x = __byte_perm(fd((nh >> 21) & 127u, 0), fd((nh >> 14) & 127u, 1), 0x7632);
    r.y = __byte_perm(fd((nh >> 7) & 127u, 2), fd(nh & 127u, 3), 0x7632);
    r.z = __byte_perm(fd((nl >> 21) & 127u, 4), fd((nl >> 14) & 127u, 5), 0x7632);
    r.w = __byte_perm(fd((nl >> 7) & 127u, 6), fd(nl & 127u, 7), 0x7632);
    if (negative) {
        r.x ^= 0x80008000u;
        r.y ^= 0x80008000u;
        r.z ^= 0x80008000u;
        r.w ^= 0x80008000u;
    }
    return r;
}

// mant x 2^(-sh) rounded to nearest (sh >= -32 here, mant < 2^53), 0 when
// shifted out
__device__ __forceinline__ unsigned long long shift_round(unsigned long long mant, int sh)
{
    if (sh <= 0) return mant << (-sh);
    if (sh >= 62) return 0ull;
    return (mant + (1ull << (sh - 1))) >> sh;
}

// biased FP64 exponent of a value (FP32 exponents rebased; 0 for zero and
// subnormals, 2047 for Inf and NaN)
__device__ __forceinline__ unsigned expo(double y)
{
    return ((unsigned)__double2hiint(y) >> 20) & 0x7FFu;
}
__device__ __forceinline__ unsigned expo(dfl y)
{
    const unsigned e = (__float_as_uint(y.hi) >> 23) & 0xFFu;
    return e == 0u ? 0u : (e == 255u ? 2047u : e + 896u);
}

// digits of |y| as a 56-bit fixed-point number relative to the column's
// largest biased exponent ec: |y| ~ N 2^(ec - 1078), N < 2^56, rounded
__device__ __forceinline__ uint4 digits8(double y, int ec)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(y);
    const int e = (int)((b >> 52) & 0x7FFu);
    unsigned long long N = 0;
    if (e != 0) {
        const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
        N = shift_round(mant, ec - e - 3);    // e <= ec: shift >= -3, N < 2^56
    }
    return pack_digits(N, (b >> 63) != 0);
}

// double-float y = hi + lo: both parts scaled exactly to y' (a power of two),
// then digit by digit, in both lanes of packed FP32x2 operations, rounded to
// the multiple of q_a (adding and subtracting 1.5 2^(23 - 7(a+1)): round to
// nearest) and the remainders kept exactly; digit a is the sum of the two
// lanes' parts (for a >= 1 each is at most 64 q_a; lo has no part in digit 0).
// Seven digits (49 bits; digit 7 is zero): the value is rounded to 2^-49 of
// the column's scale, below the double-float tangents' own error (~2^-48 of
// their size), so the eighth digit would only carry rounding noise.
__device__ __forceinline__ uint4 digits8(dfl y, int ec)
{
    // a column of zeros, or a zero value (rows of idle points, slots switched off)
    if (ec == 0 || y.hi == 0.0f) return make_uint4(0u, 0u, 0u, 0u);
    const int sf = 1149 - ec;                             // 2^(1022 - ec) as FP32
    const float sc = __uint_as_float((unsigned)(sf > 0 ? sf : 1) << 23);
    float2 r = __fmul2_rn(make_float2(y.hi, y.lo), make_float2(sc, sc));
    float d[8];
    d[7] = 0.0f;
#pragma unroll
    for (int a = 0; a < 7; a++) {
        const float M = __uint_as_float(((unsigned)(143 - 7 * a) << 23) | 0x400000u);
        const float2 t = __fadd2_rn(r, make_float2(M, M));
        const float2 q = __fadd2_rn(t, make_float2(-M, -M));
        r = __fadd2_rn(r, make_float2(-q.x, -q.y));
        d[a] = q.x + q.y;
    }
    uint4 o;
    __nv_bfloat162 p0 = __floats2bfloat162_rn(d[0], d[1]), p1 = __floats2bfloat162_rn(d[2], d[3]);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(d[4], d[5]), p3 = __floats2bfloat162_rn(d[6], d[7]);
    o.x = *reinterpret_cast<unsigned *>(&p0);
    o.y = *reinterpret_cast<unsigned *>(&p1);
    o.z = *reinterpret_cast<unsigned *>(&p2);
    o.w = *reinterpret_cast<unsigned *>(&p3);
    return o;
}

// Two double-float values at once (the digits of digits8(dfl) above, the same
// roundings): the high parts of both run as one packed pair, the low parts as
// another.  A low part is below 2^-24 of the column's scale (|lo| <= ulp(hi)/2
// and |hi| < 2^(ec - 1022)), so its rounded parts in digits 0-2 (multiples of
// 2^-7, 2^-14, 2^-21) are zero and those steps are left out for it.
__device__ __forceinline__ void digits8x2(dfl y1, int ec1, dfl y2, int ec2, uint4 &o1, uint4 &o2)
{
    if (y1.hi == 0.0f && y2.hi == 0.0f) {
        o1 = o2 = make_uint4(0u, 0u, 0u, 0u);
        return;
    }
    auto scale = [](int ec) {                               // 2^(1022 - ec); 0 for a zero column
        const int sf = 1149 - ec;
        return ec == 0 ? 0.0f : __uint_as_float((unsigned)(sf > 0 ? sf : 1) << 23);
    };
    const float2 sc = make_float2(scale(ec1), scale(ec2));
    float2 rh = __fmul2_rn(make_float2(y1.hi, y2.hi), sc);
    float2 rl = __fmul2_rn(make_float2(y1.lo, y2.lo), sc);
    float2 d[7];
#pragma unroll
    for (int a = 0; a < 7; a++) {
        const float M = __uint_as_float(((unsigned)(143 - 7 * a) << 23) | 0x400000u);
        const float2 th = __fadd2_rn(rh, make_float2(M, M));
        const float2 qh = __fadd2_rn(th, make_float2(-M, -M));
        rh = __fadd2_rn(rh, make_float2(-qh.x, -qh.y));
        if (a >= 3) {
            const float2 tl = __fadd2_rn(rl, make_float2(M, M));
            const float2 ql = __fadd2_rn(tl, make_float2(-M, -M));
            rl = __fadd2_rn(rl, make_float2(-ql.x, -ql.y));
            d[a] = __fadd2_rn(qh, ql);
        } else {
            d[a] = qh;
        }
    }
    // a digit has at most 8 significant bits: its bf16 form is the upper half
    // of its FP32 bits
    auto b2 = [](float lo, float hi) { return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632); };
    o1 = make_uint4(b2(d[0].x, d[1].x), b2(d[2].x, d[3].x), b2(d[4].x, d[5].x), b2(d[6].x, 0.0f));
    o2 = make_uint4(b2(d[0].y, d[1].y), b2(d[2].y, d[3].y), b2(d[4].y, d[5].y), b2(d[6].y, 0.0f));
}

// 2^x in FP64 (x an integer), NaN when a column held a non-finite value
__device__ __forceinline__ double pow2_scale(int ei, int ej)
{
    if (ei == 2047 || ej == 2047) return __longlong_as_double(0x7FF8000000000000ll);
    const int x = ei + ej - 2044;
    const int be = x + 1023;
    if (be >= 1 && be <= 2046) return __longlong_as_double((long long)be << 52);
    return ldexp(1.0, x);
}

// double-float noise weights sigma_p = A sqrt(4 w / S_p) (A and S relative to
// the reference scale); a tabulated PSD's factor is formed in FP64
template <bool TAB>
__device__ __forceinline__ void psd_sigma_df(const DevNet &net, const dfl *psd_d, const dfl *E,
                                             const double *Ed, int k, dfl f, dfl vi3, dfl w,
                                             dfl Aamp, int (&tseg)[MAX_PSD], dfl (&Wp)[MAX_PSD])
{
#pragma unroll
    for (int p = 0; p < MAX_PSD; p++) {
        const dfl *P = psd_d + p * (2 + MAX_TERM);   // inverse f0, f0, coefficients
        if (TAB && p < net.n_psd && net.psd_kind[p] == 1) {
            const double lnf_k = fma((double)k, Ed[EV_LNR], Ed[EV_LNF0]);
            const double lns = psd_table_lns(net, p, lnf_k, tseg[p]);
            const double wd = (double)w.hi + (double)w.lo;
            Wp[p] = Aamp * dfl(sqrt(4.0 * wd) * exp(-0.5 * (lns - net.ln_scale_ref)));
        } else if (p < net.n_psd) {
            const dfl x = f * P[0];
            const dfl xi = P[1] * E[EV_PIM] * vi3;
            dfl S(0.0f, 0.0f);
            for (int q = 0; q < net.psd_nterm[p]; q++) {
                const int pw = net.psd_pow[p][q];
                S = fma(P[2 + q], df_ipow(pw >= 0 ? x : xi, pw >= 0 ? pw : -pw), S);
            }
            Wp[p] = Aamp * df_sqrt(df_mul_f(w, 4.0f) * df_rcp(S));
        } else {
            Wp[p] = dfl(0.0f, 0.0f);
        }
    }
}

// a work item as the preparing warp leaves it for the CTA
struct __align__(16) TcItem {
    long long e;       // event
    int n, kb, ke;     // the event's grid length, the item's points [kb, ke)
    int pad[3];
};

// The tangents of one interferometer as (Re, Im) pairs of double-float
// numbers, the operations of tangents() (gw_points_fp64.cuh) on both parts at
// once: with Q = (qr, qi) and iQ = (-qi, qr),
//   g_Mc = aMc Q + dPhi/dMc iQ [+ Omega dtau*/dMc dQ/dx],  g_eta, g_theta,
//   g_phi, g_tc, g_9, g_10 likewise, g_dL = -Q/d_L, g_iota = dQ/diota,
//   g_psi = 2 (Acp Fx, -Acx F+), g_Phic = -iQ.
// F = (F+, Fx), FT, FX their theta- and x-derivatives; A = (Acp, Acx),
// Ad = (Adcp, Adcx) the amplitudes times the noise weight.
template <int NP, bool ROT>
__device__ __forceinline__ void tangents2(const dfl2 &F, const dfl2 &FT, const dfl2 &FX,
                                          const dfl2 &A, const dfl2 &Ad, dfl aMc, dfl invdL,
                                          const PhaseT<dfl> &ph, dfl2 (&g)[NP])
{
    const dfl2 Q = A * F, X = A * FX, Tt = A * FT;
    const dfl2 iQ = d2_mul_i(Q);
    g[0] = Q * d2_bcast(aMc) + iQ * d2_bcast(ph.Mc);
    g[1] = iQ * d2_bcast(ph.eta);
    if (ROT) {
        g[0] = d2_fma(X, ph.tMc, g[0]);
        g[1] = d2_fma(X, ph.teta, g[1]);
    }
    g[2] = Q * d2_bcast(-invdL);
    g[3] = Tt + iQ * d2_bcast(ph.th);
    g[4] = X + iQ * d2_bcast(ph.ph);
    g[5] = Ad * F;
    // psi: dF+/dpsi = 2 Fx, dFx/dpsi = -2 F+
    g[6] = dfl2{make_float2(2.0f * A.hi.x, -2.0f * A.hi.y), make_float2(2.0f * A.lo.x, -2.0f * A.lo.y)} *
           dfl2{make_float2(F.hi.y, F.hi.x), make_float2(F.lo.y, F.lo.x)};
    g[7] = iQ * d2_bcast(ph.tc);
    if (ROT) g[7] = d2_fma(X, dfl(-OMEGA_E), g[7]);
    g[8] = -iQ;
    if (NP == 11) {
        g[NP - 2] = iQ * d2_bcast(ph.p9);
        g[NP - 1] = iQ * d2_bcast(ph.p10);
    }
}

// (F+, Fx) = P1 (a, b) + P2 (b, -a): one pattern pair from the JKS coefficients
__device__ __forceinline__ dfl2 pattern_pair(dfl a, dfl b, const dfl2 &P1, const dfl2 &P2)
{
    return d2_make(a, b) * P1 + d2_make(b, -a) * P2;
}

template <int NP, bool ROT, bool TAB, typename T>
__global__ void __launch_bounds__(TC_T, TC_CTAS) k_fisher_tc(PointArgs A)
{
    using SH = TcShape<NP>;
    constexpr bool DF = std::is_same<T, dfl>::value;
    constexpr int KG = SH::KG, NMMA = SH::N;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    // operand buffer 0, then the staged values [4 rows r][NP columns][TC_T
    // points]; the first two rows' values (2 x NP x TC_T x 8 bytes = one operand
    // block) become operand buffer 1 once they have been turned into digits
    unsigned char *ops0 = tc_smem;
    T *stage = reinterpret_cast<T *>(tc_smem + SH::BLK);
    unsigned char *ops1 = reinterpret_cast<unsigned char *>(stage);
    double *cs = reinterpret_cast<double *>(stage + NP * 4 * TC_T);   // event constants
    double *pw = cs + EVC;                   // [3][2][16] powers, then bases
    unsigned *emax = reinterpret_cast<unsigned *>(pw + TC_PW);   // [2][16]: column maxima
    uint64_t *mbar = reinterpret_cast<uint64_t *>(emax + 32);   // one per operand buffer
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 2);
    TcItem *item = reinterpret_cast<TcItem *>(tmem_slot + 4);   // the next item to run
    // double-float copies (T = dfl only)
    dfl *Ed = reinterpret_cast<dfl *>(item + 1);
    dfl *Sd = Ed + EVC;                       // [TC_SITES][SC_N]
    dfl *Qd = Sd + TC_SITES * SC_N;           // [MAX_IFO][3]: s2g, c2g, amp
    dfl *Pd = Qd + 3 * MAX_IFO;               // [MAX_PSD][2 + MAX_TERM]
    dfl *pwd = Pd + MAX_PSD * (2 + MAX_TERM);  // powers and bases

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const DevNet &net = A.net;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(tmem_slot)), "r"(128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(&mbar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(&mbar[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (DF) {
        // network constants: interferometers, and the PSDs relative to the
        // reference scale (S / scale_ref; the amplitude carries 1/sqrt(scale_ref))
        const double inv_ref = net.inv_sqrt_scale_ref * net.inv_sqrt_scale_ref;
        for (int q = t; q < net.n_ifo; q += TC_T) {
            Qd[3 * q + 0] = dfl(net.ifo_s2g[q]);
            Qd[3 * q + 1] = dfl(net.ifo_c2g[q]);
            Qd[3 * q + 2] = dfl(net.ifo_amp[q]);
        }
        for (int i = t; i < net.n_psd * (2 + MAX_TERM); i += TC_T) {
            const int p = i / (2 + MAX_TERM), j = i % (2 + MAX_TERM);
            const double v = j == 0 ? net.psd_inv_f0[p]
                           : j == 1 ? net.psd_f0[p]
                           : (j - 2 < net.psd_nterm[p] ? net.psd_coef[p][j - 2] * inv_ref : 0.0);
            Pd[i] = dfl(v);
        }
    }
    // the staged values are read past either operand buffer (see TcShape):
    // keep them finite from the start
    for (int i = t; i < (SH::BLK + SH::STAGE_BYTES) / 16; i += TC_T)
        reinterpret_cast<uint4 *>(ops0)[i] = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t ops_addr0 = smem_addr(ops0), ops_addr1 = smem_addr(ops1);
    // instruction descriptor: D FP32, A and B bf16, both MN-major, N, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                           ((uint32_t)(NMMA >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    uint32_t par = 0u;   // bit b: parity of the next mbarrier phase of buffer b
    bool ok = true;

    // this CTA's contiguous range of work items: consecutive items mostly
    // belong to one event, whose constants then stay in shared memory
    const int64_t n_total = A.item_off[A.n_ev];
    const int64_t n_items = n_total < A.n_items ? n_total : A.n_items;
    const int64_t it_begin = n_items * blockIdx.x / gridDim.x;
    const int64_t it_end = n_items * (blockIdx.x + 1) / gridDim.x;
    // Warp 3 prepares each item: the event (a search for the range's first
    // item, then forward), the event's constants and power tables when the
    // event changes, the item's starting values, a cleared column-maximum
    // buffer and the item descriptor.  It does so for the next item while
    // warps 0-2 read the current item's Gram out of TMEM (TMEM rows 96-127,
    // warp 3's lanes, hold no Gram rows), so only the range's first item waits
    // for it.
    int64_t e_w = -1;   // warp 3: the event of the last prepared item
    auto prepare = [&](int64_t itp, unsigned *emx_next) {
        int64_t en;
        if (e_w < 0) {
            en = find_event(A.item_off, A.n_ev, itp);
        } else {
            en = e_w;
            while (__ldg(A.item_off + en + 1) <= itp) en++;
        }
        const bool new_event = en != e_w;
        e_w = en;
        const int64_t off0 = __ldg(A.item_off + en);
        const int64_t jit = itp - off0, nj = __ldg(A.item_off + en + 1) - off0;
        if (new_event) {
            const double *Eg = A.evc + en * (int64_t)EVC;
            for (int q = lane; q < EVC; q += 32) {
                const double v = Eg[q];
                cs[q] = v;
                if (DF) Ed[q] = dfl(v);
            }
            if (DF) {
                for (int i = lane; i < net.n_site * SC_N; i += 32)
                    Sd[i] = dfl(A.sitec[en * net.n_site * (int64_t)SC_N + i]);
            }
        }
        __syncwarp();
        const int N = (int)cs[EV_NPTS];
        // the event's nj = ceil(N / 128) items take isz points each, isz the
        // even share rounded up to whole warps (<= 128), the last item the rest:
        // fewer partly filled warps than an even split ((nj - 1) isz < N holds
        // because N > 128 (nj - 1))
        const int isz = (int)(((N + nj - 1) / nj + 31) & ~31);
        const int kb = (int)jit * isz, ke = min(N, kb + isz);
        const double lnr = cs[EV_LNR];
        // powers of the per-point factors of v, 1/v and the amplitude (steps 1
        // and 16 points; lanes 0-5, once per event) and their values at the
        // item's first point (lanes 8-11, every item)
        if (new_event && lane < 6) {
            const int q = lane % 3, big = lane / 3;
            const double l = q == 0 ? lnr * (1.0 / 3.0) : (q == 1 ? -lnr * (1.0 / 3.0) : -7.0 / 6.0 * lnr);
            const double fct = exp(big ? 16.0 * l : l);
            if (DF) {
                // the chain in double-float on the FP32 pipe (~16 x 2^-48)
                const dfl fc(fct);
                dfl val(1.0f, 0.0f);
                for (int i = 0; i < 16; i++) {
                    pwd[(q * 2 + big) * 16 + i] = val;
                    val = val * fc;
                }
            } else {
                double val = 1.0;
                for (int i = 0; i < 16; i++) {
                    pw[(q * 2 + big) * 16 + i] = val;
                    val *= fct;
                }
            }
        } else if (lane >= 8 && lane < 12) {
            const double lnf0 = fma((double)kb, lnr, cs[EV_LNF0]);
            const double lnv0 = (lnf0 + cs[EV_LNPIM]) * (1.0 / 3.0);
            const int q = lane - 8;
            const double bv = q == 0 ? exp(lnv0)
                            : q == 1 ? exp(-lnv0)
                            : q == 2 ? cs[EV_A0] * exp(-7.0 / 6.0 * lnf0)
                                     : lnv0;
            pw[96 + q] = bv;
            if (DF) {
                // amplitude relative to sqrt(scale_ref); ln v step per point
                pwd[96 + q] = dfl(q == 2 ? bv * net.inv_sqrt_scale_ref : bv);
                if (q == 3) pwd[100] = dfl(lnr * (1.0 / 3.0));
            }
        }
        if (lane < 16) emx_next[lane] = 0u;
        if (lane == 0) {
            item->e = en;
            item->n = N;
            item->kb = kb;
            item->ke = ke;
        }
        __syncwarp();
    };
    int cur = 1;   // column-maximum buffer of the current item
    // (the first pass, it = it_begin - 1, only prepares the range's first item:
    // one call site keeps the kernel's code small)
    for (int64_t it = it_begin - 1; it < it_end; it++) {
      unsigned *emx = emax + 16 * cur;
      double *out = A.partial + (it < 0 ? 0 : it) * (int64_t)A.nacc;   // the item's row
      bool bad = false;
      if (it >= it_begin) {
        const int64_t e = item->e;
        const int N = item->n, kb = item->kb, ke = item->ke;
        const double lnr = cs[EV_LNR];

        // per-thread copies of the event's scalar constants
        const T *E;
        if constexpr (DF) E = Ed;
        else E = cs;
        int tseg[MAX_PSD];
#pragma unroll
        for (int p = 0; p < MAX_PSD; p++) tseg[p] = -1;

        // ---- tangents of this thread's point, staged as they are formed:
        // rows r = 2 L + {Re, Im} of interferometer slot L (0 or 1)
        unsigned lmax[NP];
#pragma unroll
        for (int c = 0; c < NP; c++) lmax[c] = 0u;
        unsigned written = 0u;
        const int k = kb + t;
        if (k < ke) {
            const int lo = t & 15, hi = t >> 4;
            T v, vinv, Aamp, lnv;
            if constexpr (DF) {
                v = pwd[96] * pwd[0 * 16 + lo] * pwd[1 * 16 + hi];
                vinv = pwd[97] * pwd[2 * 16 + lo] * pwd[3 * 16 + hi];
                Aamp = pwd[98] * pwd[4 * 16 + lo] * pwd[5 * 16 + hi];
                lnv = pwd[99] + df_mul_f(pwd[100], (float)t);
            } else {
                const double lnf = fma((double)k, lnr, cs[EV_LNF0]);
                lnv = (lnf + cs[EV_LNPIM]) * (1.0 / 3.0);
                v = pw[96] * pw[0 * 16 + lo] * pw[1 * 16 + hi];
                vinv = pw[97] * pw[2 * 16 + lo] * pw[3 * 16 + hi];
                Aamp = pw[98] * pw[4 * 16 + lo] * pw[5 * 16 + hi];
            }
            const PnTermsT<T> pn = pn_terms<NP, ROT>(E, v, vinv, lnv);
            const T w = pn.f * (k == 0 ? E[EV_WC0] : (k == N - 1 ? E[EV_WCN] : E[EV_WCM]));
            const T twopif = T(TWO_PI) * pn.f;
            T Wp[MAX_PSD];
            if constexpr (DF)
                psd_sigma_df<TAB>(net, Pd, E, cs, k, pn.f, pn.vi3, w, Aamp, tseg, Wp);
            else
                psd_sigma<TAB>(net, E, k, pn.f, pn.vi3, w, Aamp, tseg, Wp);
            int L = 0;
#pragma unroll 1
            for (int s = 0; s < net.n_site; s++) {
                const double *Sg = A.sitec + (e * net.n_site + s) * (int64_t)SC_N;
                if (net.masked && Sg[SC_SLOT0] < 0.0) {   // every arm of the site off
                    L += net.site_nslot[s];
                    continue;
                }
                const T *S;
                if constexpr (DF) S = Sd + s * SC_N;
                else S = Sg;
                T J[12];
                PhaseT<T> ph;
                site_terms<MODE_FISHER, ROT>(S, pn, twopif, J, ph);
#pragma unroll 1
                for (int slot = 0; slot < net.site_nslot[s]; slot++, L++) {
                    int q = net.masked ? (int)Sg[SC_SLOT0 + slot] : net.site_ifo0[s] + slot;
                    bool on = true;
                    if (q < 0) {
                        q = net.site_ifo0[s];
                        on = false;
                    }
                    T s2g, c2g, amp;
                    if constexpr (DF) {
                        s2g = Qd[3 * q];
                        c2g = Qd[3 * q + 1];
                        amp = on ? Qd[3 * q + 2] : T(0.0);
                    } else {
                        s2g = net.ifo_s2g[q];
                        c2g = net.ifo_c2g[q];
                        amp = net.ifo_amp[q] * (on ? 1.0 : 0.0);
                    }
                    // A triangle's two virtual interferometers (at gamma_T and
                    // gamma_T + 45 deg, same amplitude and noise) enter the
                    // patterns through (sin 2g, cos 2g) and (cos 2g, -sin 2g): an
                    // orthogonal pair, so the sum over the two of the outer
                    // products of anything linear in the patterns is unchanged
                    // with (1, 0) and (0, 1) in their place -- the pair's Gram
                    // is that of the unrotated coefficients, 18 operations less
                    // per slot and point
                    const int L1 = q - net.site_ifo0[s];
                    const bool unit = net.site_nslot[s] == 2 && L1 >= 0 && L1 < 2;
                    const T sg = Wp[net.ifo_psd[q]];
                    T *row = stage + (2 * L) * NP * TC_T + t;
                    if constexpr (DF) {
                        // (Re, Im) pairs on the packed FP32x2 instructions
                        const dfl2 P1 = d2_bcast(amp * E[EV_C2PSI]), P2 = d2_bcast(amp * E[EV_S2PSI]);
                        dfl2 F, FT, FX;
                        if (unit) {
                            F = pattern_pair(L1 ? J[1] : J[0], L1 ? J[2] : J[3], P1, P2);
                            FT = pattern_pair(L1 ? J[5] : J[4], L1 ? J[6] : J[7], P1, P2);
                            FX = pattern_pair(L1 ? J[9] : J[8], L1 ? J[10] : J[11], P1, P2);
                        } else {
                            const PatT<T> pt = patterns(s2g, c2g, amp * E[EV_C2PSI], amp * E[EV_S2PSI], J);
                            F = d2_make(pt.fp, pt.fx);
                            FT = d2_make(pt.fpT, pt.fxT);
                            FX = d2_make(pt.fpX, pt.fxX);
                        }
                        const dfl2 sg2 = d2_bcast(sg);
                        dfl2 g[NP];
                        tangents2<NP, ROT>(F, FT, FX, sg2 * d2_make(E[EV_CP], E[EV_CX]),
                                           sg2 * d2_make(E[EV_DCP], E[EV_DCX]), E[EV_AMC],
                                           E[EV_INVDL], ph, g);
#pragma unroll
                        for (int c = 0; c < NP; c++) {
                            const dfl gr = d2_x(g[c]), gi = d2_y(g[c]);
                            row[c * TC_T] = gr;
                            row[(NP + c) * TC_T] = gi;
                            const unsigned er = expo(gr), ei = expo(gi);
                            const unsigned em2 = er > ei ? er : ei;
                            lmax[c] = em2 > lmax[c] ? em2 : lmax[c];
                        }
                    } else {
                        const PatT<T> pt =
                            unit ? patterns_ab(amp * E[EV_C2PSI], amp * E[EV_S2PSI], L1 ? J[1] : J[0],
                                               L1 ? J[2] : J[3], L1 ? J[5] : J[4], L1 ? J[6] : J[7],
                                               L1 ? J[9] : J[8], L1 ? J[10] : J[11])
                                 : patterns(s2g, c2g, amp * E[EV_C2PSI], amp * E[EV_S2PSI], J);
                        T gr[NP], gi[NP], qr, qi;
                        tangents<NP, ROT>(pt, sg * E[EV_CP], sg * E[EV_CX], sg * E[EV_DCP],
                                          sg * E[EV_DCX], E[EV_AMC], E[EV_INVDL], ph, gr, gi, qr, qi);
#pragma unroll
                        for (int c = 0; c < NP; c++) {
                            row[c * TC_T] = gr[c];
                            row[(NP + c) * TC_T] = gi[c];
                            const unsigned er = expo(gr[c]), ei = expo(gi[c]);
                            const unsigned em2 = er > ei ? er : ei;
                            lmax[c] = em2 > lmax[c] ? em2 : lmax[c];
                        }
                    }
                    written |= 1u << L;
                }
            }
        }
        // rows of slots this point did not fill (absent or switched-off
        // interferometers, points past the item) are zero
#pragma unroll
        for (int L = 0; L < 2; L++)
            if (!((written >> L) & 1u)) {
#pragma unroll
                for (int c = 0; c < NP; c++) {
                    stage[(2 * L * NP + c) * TC_T + t] = T(0.0);
                    stage[((2 * L + 1) * NP + c) * TC_T + t] = T(0.0);
                }
            }
        // ---- column maxima of the item's biased exponents
#pragma unroll
        for (int c = 0; c < NP; c++) {
            const unsigned m = __reduce_max_sync(0xffffffffu, lmax[c]);
            if (lane == 0) atomicMax(&emx[c], m);
        }
        __syncthreads();
        int em[NP];
#pragma unroll
        for (int c = 0; c < NP; c++) em[c] = (int)emx[c];

        // ---- digits of row r into operand buffer r % 2; buffer 1 overlays the
        // staged rows 0 and 1, so it is written only after every thread has read
        // them, and each buffer's previous MMAs must be done before it is
        // rewritten.  The digits of the next row are formed while the tensor
        // core works on the previous one.
        const int koff = (t & 7) * 16 + (t >> 3) * KG;   // this thread's K row in a buffer
        // (a rolled loop: the kernel's code size is what limits instruction fetch)
#pragma unroll 1
        for (int r = 0; r < 4; r++) {
            uint4 dg[NP];
            if constexpr (DF) {
#pragma unroll
                for (int c = 0; c + 1 < NP; c += 2)
                    digits8x2(stage[(r * NP + c) * TC_T + t], em[c], stage[(r * NP + c + 1) * TC_T + t],
                              em[c + 1], dg[c], dg[c + 1]);
                if (NP & 1) dg[NP - 1] = digits8(stage[(r * NP + NP - 1) * TC_T + t], em[NP - 1]);
            } else {
#pragma unroll
                for (int c = 0; c < NP; c++) dg[c] = digits8(stage[(r * NP + c) * TC_T + t], em[c]);
            }
            const int b = r & 1;
            if (r == 1) __syncthreads();   // staged rows 0 and 1 read by every thread
            if (r >= 2) {
                ok = mbar_wait(smem_addr(&mbar[b]), (par >> b) & 1u) && ok;
                par ^= 1u << b;
                asm volatile("tcgen05.fence::after_thread_sync;");
            }
            unsigned char *B = (b ? ops1 : ops0) + koff;
#pragma unroll
            for (int c = 0; c < NP; c++) *reinterpret_cast<uint4 *>(B + c * TC_MG) = dg[c];
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            if (t == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                for (int st = 0; st < TC_KROWS / 16; st++) {
                    const uint64_t d = smem_desc((b ? ops_addr1 : ops_addr0) + st * 2 * KG, KG, TC_MG);
                    const uint32_t accum = (r > 0 || st > 0) ? 1u : 0u;
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                 :: "r"(tmem), "l"(d), "l"(d), "r"(idesc), "r"(accum));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(smem_addr(&mbar[b])));
            }
        }
#pragma unroll
        for (int b = 0; b < 2; b++) {
            ok = mbar_wait(smem_addr(&mbar[b]), (par >> b) & 1u) && ok;
            par ^= 1u << b;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        bad = __syncthreads_or(!ok || ke - kb > TC_T);
        if (bad) {
            // a wait that ran out, or an item longer than the kernel's round
            for (int a = t; a < A.nacc; a += TC_T) out[a] = __longlong_as_double(0x7FF8000000000000ll);
            if (t == 0 && A.kerr) atomicExch(A.kerr, 1);
            if (!ok) break;
        }
      }
        if (warp == 3) {
            // the next item's set-up (warp 3 holds no Gram rows)
            if (it + 1 < it_end) prepare(it + 1, emax + 16 * (cur ^ 1));
        } else if (it >= it_begin && !bad) {
        // ---- read the digit Gram: thread t holds TMEM lane t = row (i, a),
        // i = t / 8, a = t % 8; columns (j, b) at 8 j + b.  The rows sit in
        // warps 0-2 (rows 4w .. 4w + 3); warp w reads its own four column
        // groups (entries (i, j), i <= j, of its own rows) and the next warp's
        // (w + 1 mod 3: every (i, j) of its rows with them), so each unordered
        // pair is formed once and a warp reads at most 8 groups, three per
        // batch of TMEM loads.  The products D[(i,a),(j,b)] are exact multiples of q_a q_b
        // below 2^24 q_a q_b: with n_ab = D / (q_a q_b), the entry is
        //     sum_ab D = 2^-112 I,   I = sum_a 2^(7 (7 - a)) sum_b 2^(7 (7 - b)) n_ab,
        // an integer below 2^123 in magnitude, formed exactly in 128-bit
        // integer arithmetic (per lane over b, across the row's eight lanes with
        // shuffles) and rounded once to FP64.
        const int i = t >> 3, a = t & 7;
        static_assert(NP <= 12, "Gram rows in warps 0-2");
        constexpr int NGRP = 8;       // column groups read per warp (at most)
        const int nxt = warp == 2 ? 0 : warp + 1;
        const int own_n = NP - 4 * warp < 4 ? NP - 4 * warp : 4;
        const int nxt_n = NP - 4 * nxt < 4 ? NP - 4 * nxt : 4;
        // (a warp whose rows are all padding, 4w >= P, reads nothing)
        const int ngrp = 4 * warp >= NP ? 0 : own_n + nxt_n;
        auto col_of = [&](int g) { return g < own_n ? 4 * warp + g : 4 * nxt + (g - own_n); };
        constexpr int GB = 3;          // column groups per batch of TMEM loads
#pragma unroll 1
        for (int g0 = 0; g0 < NGRP; g0 += GB) {
            if (g0 >= ngrp) break;
            uint32_t dd[GB][8];
#pragma unroll
            for (int g = 0; g < GB; g++) {
                if (g0 + g < ngrp) {
                    const int j = col_of(g0 + g);
                    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 8);
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(dd[g][0]), "=r"(dd[g][1]), "=r"(dd[g][2]), "=r"(dd[g][3]),
                                   "=r"(dd[g][4]), "=r"(dd[g][5]), "=r"(dd[g][6]), "=r"(dd[g][7])
                                 : "r"(ta));
                }
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int g = 0; g < GB; g++) {
                if (g0 + g >= ngrp) break;
                const int j = col_of(g0 + g);
                // W = sum_b 2^(7 (7 - b)) n_ab (|W| < 2^74), as hs 2^28 + ls
                long long hs = 0, ls = 0;
#pragma unroll
                for (int b = 0; b < 8; b++) {
                    // D / (q_a q_b): an integer below 2^24 (exact FP32 scaling by 2^(7(a+b+2)))
                    const float sb = __uint_as_float((unsigned)(127 + 7 * (a + b + 2)) << 23);
                    const long long n = (long long)__float2int_rn(__uint_as_float(dd[g][b]) * sb);
                    if (b < 4) hs += n << (7 * (3 - b));
                    else ls += n << (7 * (7 - b));
                }
                // X = W 2^(7 (7 - a)) as a 128-bit two's-complement integer, summed
                // over the row's eight lanes
                using u128 = unsigned __int128;
                u128 X = (((u128)(__int128)hs << 28) + (u128)(__int128)ls) << (7 * (7 - a));
#pragma unroll
                for (int m = 1; m < 8; m <<= 1) {
                    const unsigned long long yl = __shfl_xor_sync(0xffffffffu, (unsigned long long)X, m);
                    const unsigned long long yh =
                        __shfl_xor_sync(0xffffffffu, (unsigned long long)(X >> 64), m);
                    X += ((u128)yh << 64) | (u128)yl;
                }
                // own groups: the pairs i <= j; the next warp's: every pair
                if (a == 0 && i < NP && (g0 + g >= own_n || i <= j)) {
                    const int lo = i < j ? i : j, hi = i < j ? j : i;
                    // |I| rounded to FP64 (high word, exact below 2^53, times 2^64
                    // plus the low word), the sign, then the scale 2^-112 (exact)
                    const bool neg = (long long)(unsigned long long)(X >> 64) < 0;
                    const u128 M = neg ? (u128)0 - X : X;
                    const double mag = fma((double)(unsigned long long)(M >> 64), 0x1p64,
                                           (double)(unsigned long long)M);
                    const double P = (neg ? -mag : mag) * 0x1p-112;
                    const double gv = P == 0.0 ? 0.0 : P * pow2_scale((int)emx[i], (int)emx[j]);
                    const int idx = 1 + lo * NP - lo * (lo - 1) / 2 + (hi - lo);
                    if (idx < A.nacc) out[idx] = gv;
                    // SNR^2 = sum |Q|^2 = the (Phic, Phic) entry: g_Phic = -i Q
                    if (i == 8 && j == 8) out[0] = gv;
                }
            }
        }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();   // TMEM, emax and the buffers are free for the next item
        cur ^= 1;
    }

    // ---- teardown.  Normally every commit has been waited on.  After a wait
    // that ran out, give the MMAs in flight one more bounded wait; then free
    // the TMEM columns.
    if (!ok) {
        // (each wait flipped its parity: par ^ 1 is the phase last waited for)
        mbar_wait(smem_addr(&mbar[0]), (par & 1u) ^ 1u);
        mbar_wait(smem_addr(&mbar[1]), ((par >> 1) & 1u) ^ 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(128));
}

template <int NP, bool ROT, bool TAB, typename T>
cudaError_t launch_tc(const PointArgs &a, cudaStream_t s)
{
    const size_t smem = TcShape<NP>::smem(std::is_same<T, dfl>::value);
    static PerDeviceOnce attr;
    cudaError_t err = set_smem_once(attr, k_fisher_tc<NP, ROT, TAB, T>, smem);
    if (err != cudaSuccess) return err;
    if (a.n_items <= 0) return cudaSuccess;
    k_fisher_tc<NP, ROT, TAB, T><<<points_grid_size(TC_CTAS), TC_T, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tc_t(int np, int rot, const PointArgs &a, cudaStream_t s)
{
    const bool tab = has_psd_table(a.net);
    if (np == 9) {
        if (rot) return tab ? launch_tc<9, true, true, T>(a, s) : launch_tc<9, true, false, T>(a, s);
        return tab ? launch_tc<9, false, true, T>(a, s) : launch_tc<9, false, false, T>(a, s);
    }
    if (rot) return tab ? launch_tc<11, true, true, T>(a, s) : launch_tc<11, true, false, T>(a, s);
    return tab ? launch_tc<11, false, true, T>(a, s) : launch_tc<11, false, false, T>(a, s);
}

}  // namespace

bool fisher_fp64_tc_supported(const DevNet &net)
{
    int slots = 0;
    for (int s = 0; s < net.n_site; s++) slots += net.site_nslot[s];
    return slots <= 2;
}

cudaError_t launch_fisher_fp64_tc(int np, int rot, const PointArgs &a, cudaStream_t s)
{
    return launch_tc_t<double>(np, rot, a, s);
}

cudaError_t launch_fisher_dfloat_tc(int np, int rot, const PointArgs &a, cudaStream_t s)
{
    return launch_tc_t<dfl>(np, rot, a, s);
}

}  // namespace gw
