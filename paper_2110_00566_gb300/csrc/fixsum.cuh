// Exact stencil sums of the FP64 nDGP kernels on the integer pipe.
//
// On this GPU the FP64 pipe issues about 2 lane-operations per clock per SM
// and the integer ALU about 64, and the GPU's own int64 <-> FP64 conversion
// instructions issue at the FP64 rate.  About half of the FP64 nDGP cell
// update is signed sums of neighbour values (S_x - S_y, the mixed
// differences C_xy, C_xz, C_yz, S6, S6 - 6u); those are computed here
// exactly in 64-bit integer arithmetic, with conversions written as bit
// manipulations of the IEEE 754 binary64 layout (sign bit, 11-bit biased
// exponent field E, 52-bit fraction; x = M 2^(E - 1075) with M the 53-bit
// significand including its leading one).
//
// Format.  The values of one stencil share a scale set by the largest
// exponent field emax among them: x becomes the integer
//     V = sign(x) floor(M 2^6 / 2^(emax - E)),
// so x = V 2^(emax - 1081) exactly whenever emax - E <= 6, and to within
// 2^(emax - 1081) (1/64 of an ulp of the largest value) otherwise.  |V| <
// 2^59, so any signed sum of up to 12 such values fits in an int64 without
// overflow.  A sum is rounded once on the way back to binary64 (to nearest,
// ties away from zero), where an FP64 evaluation rounds after every add.
//
// The nDGP update also needs the quadratic form of the differences,
// Q = 16 (a (a - b) + b^2) + 3 (C_xy^2 + C_xz^2 + C_yz^2); with the
// differences exact integers (|.| < 2^61) Q is formed exactly in 128-bit
// integer arithmetic (64 x 64 -> 128-bit products, which issue as integer
// multiply-adds on the otherwise idle FMA pipe): Q >= 0 (both parts are
// positive semi-definite) and Q < 57 * 2^122 < 2^128, so it is exact as an
// unsigned 128-bit integer and is rounded once to binary64.
//
// Domain.  The fixed-point path needs 570 <= emax <= 1529 (fx_ok): every
// value finite, the largest between 2^-453 and 2^506 in magnitude.  Zeros and
// values below 2^(emax - 1081) then shift out to 0, and the converted sums and
// Q stay in the normal range.  Callers fall back to FP64 arithmetic outside
// it (a NaN or an infinity, extreme magnitudes); an all-zero stencil takes
// the fixed-point path at the scale of 1.0 (fx_zero_scale).
#pragma once
#include "common.cuh"

namespace mg {

// biased exponent field of x, in place (bits 20..30 of the high word)
__device__ __forceinline__ int fx_ef(double x) { return __double2hiint(x) & 0x7FF00000; }

// the scale's exponent field (in place) admits the fixed-point path: the
// quadratic form below (at the squared scale) and every converted sum stay
// in binary64's normal range for 570 <= emax <= 1529, i.e. the largest value
// of a stencil between 2^-453 and 2^506 in magnitude
__device__ __forceinline__ bool fx_ok(int ef) { return ef >= (570 << 20) && ef <= (1529 << 20); }

// x as a fixed-point integer at the scale of exponent field ef (in place):
// sign(x) floor(M 2^S / 2^(emax - E)), so x = V 2^(emax - 1075 - S); S = 6
// for the stencil sums (|V| < 2^59), S = 3 where up to 64 values are summed
// with integer weights (|V| < 2^56)
template <int S = 6>
__device__ __forceinline__ long long fx_in(double x, int ef)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned sh = (unsigned)(ef - (hi & 0x7FF00000)) >> 20;            // emax - E >= 0
    const unsigned mh = ((unsigned)hi & 0x000FFFFFu) | 0x00100000u;          // top 21 bits of M
    const unsigned long long M6 = ((((unsigned long long)mh) << 32) | lo) << S;  // M 2^S < 2^(53 + S)
    const unsigned long long a = sh < 64 ? (M6 >> sh) : 0ull;
    const unsigned long long neg = (unsigned long long)(long long)(hi >> 31);  // all ones for x < 0
    return (long long)((a ^ neg) - neg);
}

// the same conversion for an exponent gap emax - E below 32 (a stencil whose
// exponents span fewer than 32 binades, the usual case away from exact
// zeros): two 32-bit funnel shifts instead of a general 64-bit shift; the
// result is identical
template <int S = 6>
__device__ __forceinline__ long long fx_in_near(double x, int ef)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned sh = (unsigned)(ef - (hi & 0x7FF00000)) >> 20;            // 0 .. 31
    const unsigned mh = ((unsigned)hi & 0x000FFFFFu) | 0x00100000u;
    const unsigned h6 = __funnelshift_l(lo, mh, S), l6 = lo << S;           // M 2^S
    const unsigned long long a = ((unsigned long long)(h6 >> sh) << 32) | __funnelshift_r(l6, h6, sh);
    const unsigned long long neg = (unsigned long long)(long long)(hi >> 31);
    return (long long)((a ^ neg) - neg);
}

template <bool NEAR, int S = 6>
__device__ __forceinline__ long long fx_cv(double x, int ef)
{
    return NEAR ? fx_in_near<S>(x, ef) : fx_in<S>(x, ef);
}

// a fixed-point integer v, worth v 2^(emax - 1075 - S) with ef the exponent
// field emax in place, back to binary64, rounded once to nearest (ties away
// from zero); |v| < 2^63.  (S larger than the conversion's folds a power of
// two into the result: fx_out<S + 6> returns the value divided by 64.)
template <int S = 6>
__device__ __forceinline__ double fx_out(long long v, int ef)
{
    const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ull;
    unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)a);          // 64 for v = 0
    a <<= (lz & 63);                               // leading one at bit 63
    const unsigned long long m = ((a >> 10) + 1ull) >> 1;  // 53 bits, rounded (2^53 carries into the exponent)
    // leading one at bit 63 - lz of v, so the value's exponent field is
    // (63 - lz) + emax - 1075 - S + 1023; m carries the leading one at bit
    // 52, so the field is added as (field - 1) << 52
    const unsigned long long e = (unsigned long long)(long long)((ef >> 20) + 10 - S - lz) << 52;
    return lz == 64 ? 0.0 : __longlong_as_double((long long)(sgn | (e + m)));
}

// running minimum and maximum of the exponent fields of the 18 stencil
// neighbours (lo, hi in place)
__device__ __forceinline__ void fx_range(const Nb<double> &v, int &lo, int &hi)
{
    const int f[18] = {fx_ef(v.xp),   fx_ef(v.xm),   fx_ef(v.yp),   fx_ef(v.ym),   fx_ef(v.zp),   fx_ef(v.zm),
                       fx_ef(v.xpyp), fx_ef(v.xmym), fx_ef(v.xpym), fx_ef(v.xmyp), fx_ef(v.xpzp), fx_ef(v.xmzm),
                       fx_ef(v.xpzm), fx_ef(v.xmzp), fx_ef(v.ypzp), fx_ef(v.ymzm), fx_ef(v.ypzm), fx_ef(v.ymzp)};
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        lo = min(lo, f[q]);
        hi = max(hi, f[q]);
    }
}

// a stencil whose exponent fields are all zero (+-0; subnormals, which this
// treats as 0) has exact-zero sums at any scale: give it the scale of 1.0, so
// that it takes the fixed-point path (the first sweep of a solve from phi = 0)
__device__ __forceinline__ int fx_zero_scale(int hi) { return hi == 0 ? (1023 << 20) : hi; }

// the exponents of a stencil (lo, hi from fx_range) take the near conversion
__device__ __forceinline__ bool fx_near(int lo, int hi) { return hi - lo < (32 << 20); }

// unsigned 128-bit integers (two's complement modulo 2^128 for intermediate
// negative products; every final value here is non-negative)
struct U128 {
    unsigned long long lo, hi;
};
__device__ __forceinline__ U128 mul_s64(long long a, long long b)
{
    U128 r;
    r.lo = (unsigned long long)a * (unsigned long long)b;
    r.hi = (unsigned long long)__mul64hi(a, b);
    return r;
}
__device__ __forceinline__ U128 add128(U128 x, U128 y)
{
    U128 r;
    asm("add.cc.u64 %0, %2, %4;\n\taddc.u64 %1, %3, %5;"
        : "=l"(r.lo), "=l"(r.hi)
        : "l"(x.lo), "l"(x.hi), "l"(y.lo), "l"(y.hi));
    return r;
}
__device__ __forceinline__ U128 shl128(U128 x, int k)  // 0 < k < 64
{
    U128 r;
    r.hi = (x.hi << k) | (x.lo >> (64 - k));
    r.lo = x.lo << k;
    return r;
}

// x^2 as an unsigned 128-bit integer (|x| < 2^63)
__device__ __forceinline__ U128 sqr_s64(long long x)
{
    const unsigned long long a = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
    U128 r;
    r.lo = a * a;
    r.hi = __umul64hi(a, a);
    return r;
}

// trunc(x / 6) for |x| < 2^63 without a division: floor(a / 6) =
// floor(a (2^65 + 1) / 3 / 2^66) for a < 2^64, because a / (3 2^66) < 1/24 and
// the fractional part of a / 6 is at most 5/6
__device__ __forceinline__ long long fx_div6(long long x)
{
    const unsigned long long a = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
    const long long q = (long long)(__umul64hi(a, 0xAAAAAAAAAAAAAAABull) >> 2);
    return x < 0 ? -q : q;
}

// Q (an unsigned 128-bit integer at the squared scale of exponent field ef,
// in place) to binary64, rounded once to nearest (ties away from zero)
__device__ __forceinline__ double fx_out_q(U128 q, int ef)
{
    const bool big = q.hi != 0;
    const int lzh = __clzll((long long)q.hi), lzl = __clzll((long long)q.lo);
    const int lz = big ? lzh : 64 + lzl;                  // 128 for Q = 0
    // the top 64 bits of Q << lz (leading one at bit 63)
    const unsigned long long top =
        big ? (lzh == 0 ? q.hi : (q.hi << lzh) | (q.lo >> (64 - lzh))) : (q.lo << (lzl & 63));
    const unsigned long long m = ((top >> 10) + 1ull) >> 1;
    // value = Q 2^(2 emax - 2162); leading one at bit 127 - lz of Q, so the
    // exponent field is (127 - lz) + 2 emax - 1139, added as (field - 1) << 52
    const unsigned long long e = (unsigned long long)(long long)(2 * (ef >> 20) - 1013 - lz) << 52;
    return lz == 128 ? 0.0 : __longlong_as_double((long long)(e + m));
}

// the stencil's signed sums, exact: a = Sx - Sy, b = Sx - Sz, a - b = Sz - Sy,
// the mixed differences C_xy, C_xz, C_yz and S6 = Sx + Sy + Sz; returns the
// quadratic form Q of the differences (rounded once) and S6 (as a fixed-point
// integer), for the nDGP update
struct FxQuad {
    double q;
    long long s6;
};
template <bool NEAR>
__device__ __forceinline__ FxQuad fx_quad(const Nb<double> &v, int ef)
{
    const long long X = fx_cv<NEAR>(v.xp, ef) + fx_cv<NEAR>(v.xm, ef);
    const long long Y = fx_cv<NEAR>(v.yp, ef) + fx_cv<NEAR>(v.ym, ef);
    const long long Z = fx_cv<NEAR>(v.zp, ef) + fx_cv<NEAR>(v.zm, ef);
    const long long a = X - Y, b = X - Z, amb = Z - Y;
    const long long cxy = (fx_cv<NEAR>(v.xpyp, ef) + fx_cv<NEAR>(v.xmym, ef)) -
                          (fx_cv<NEAR>(v.xpym, ef) + fx_cv<NEAR>(v.xmyp, ef));
    const long long cxz = (fx_cv<NEAR>(v.xpzp, ef) + fx_cv<NEAR>(v.xmzm, ef)) -
                          (fx_cv<NEAR>(v.xpzm, ef) + fx_cv<NEAR>(v.xmzp, ef));
    const long long cyz = (fx_cv<NEAR>(v.ypzp, ef) + fx_cv<NEAR>(v.ymzm, ef)) -
                          (fx_cv<NEAR>(v.ypzm, ef) + fx_cv<NEAR>(v.ymzp, ef));
    const U128 E = add128(mul_s64(a, amb), sqr_s64(b));                                      // E / 2 >= 0
    const U128 C = add128(add128(sqr_s64(cxy), sqr_s64(cxz)), sqr_s64(cyz));                 // >= 0
    const U128 Q = add128(shl128(E, 4), add128(C, shl128(C, 1)));                             // 16 E/2 + 3 C
    FxQuad r;
    r.q = fx_out_q(Q, ef);
    r.s6 = (X + Y) + Z;
    return r;
}

}  // namespace mg
