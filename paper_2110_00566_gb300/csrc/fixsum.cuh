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
// Domain.  The fixed-point path needs 60 <= emax <= 2040: every value finite
// and the largest at least 2^-963 in magnitude.  Zeros and values below
// 2^(emax - 1081) then shift out to 0, and a converted sum stays in the
// normal range.  Callers fall back to FP64 arithmetic outside it (a zero
// field, a NaN or an infinity).
#pragma once
#include "common.cuh"

namespace mg {

// biased exponent field of x, in place (bits 20..30 of the high word)
__device__ __forceinline__ int fx_ef(double x) { return __double2hiint(x) & 0x7FF00000; }

// the scale's exponent field (in place) admits the fixed-point path
__device__ __forceinline__ bool fx_ok(int ef) { return ef >= (60 << 20) && ef <= (2040 << 20); }

// x as a fixed-point integer at the scale of exponent field ef (in place)
__device__ __forceinline__ long long fx_in(double x, int ef)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned sh = (unsigned)(ef - (hi & 0x7FF00000)) >> 20;            // emax - E >= 0
    const unsigned mh = ((unsigned)hi & 0x000FFFFFu) | 0x00100000u;          // top 21 bits of M
    const unsigned long long M6 = ((((unsigned long long)mh) << 32) | lo) << 6;  // M 2^6 < 2^59
    const unsigned long long a = sh < 64 ? (M6 >> sh) : 0ull;
    const unsigned long long neg = (unsigned long long)(long long)(hi >> 31);  // all ones for x < 0
    return (long long)((a ^ neg) - neg);
}

// the same conversion for an exponent gap emax - E below 32 (a stencil whose
// exponents span fewer than 32 binades, the usual case away from exact
// zeros): two 32-bit funnel shifts instead of a general 64-bit shift; the
// result is identical
__device__ __forceinline__ long long fx_in_near(double x, int ef)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned sh = (unsigned)(ef - (hi & 0x7FF00000)) >> 20;            // 0 .. 31
    const unsigned mh = ((unsigned)hi & 0x000FFFFFu) | 0x00100000u;
    const unsigned h6 = __funnelshift_l(lo, mh, 6), l6 = lo << 6;           // M 2^6
    const unsigned long long a = ((unsigned long long)(h6 >> sh) << 32) | __funnelshift_r(l6, h6, sh);
    const unsigned long long neg = (unsigned long long)(long long)(hi >> 31);
    return (long long)((a ^ neg) - neg);
}

template <bool NEAR>
__device__ __forceinline__ long long fx_cv(double x, int ef)
{
    return NEAR ? fx_in_near(x, ef) : fx_in(x, ef);
}

// a fixed-point integer at the scale of exponent field ef (in place) back to
// binary64, rounded once to nearest (ties away from zero); |v| < 2^63
__device__ __forceinline__ double fx_out(long long v, int ef)
{
    const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ull;
    unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)a);          // 64 for v = 0
    a <<= (lz & 63);                               // leading one at bit 63
    const unsigned long long m = ((a >> 10) + 1ull) >> 1;  // 53 bits, rounded (2^53 carries into the exponent)
    // leading one at bit 63 - lz of V, so the value's exponent field is
    // (63 - lz) + emax - 58; m carries the leading one at bit 52, so the
    // field is added as (field - 1) << 52
    const unsigned long long e = (unsigned long long)(long long)((ef >> 20) + 4 - lz) << 52;
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

// the exponents of a stencil (lo, hi from fx_range) take the near conversion
__device__ __forceinline__ bool fx_near(int lo, int hi) { return hi - lo < (32 << 20); }

// the signed sums of the 19-point stencil, each exact and rounded once:
// a = Sx - Sy, b = Sx - Sz, amb = a - b = Sz - Sy, the three mixed
// differences, and S6 = Sx + Sy + Sz as a fixed-point integer
struct FxSums {
    double a, b, amb, cxy, cxz, cyz;
    long long s6;
};
template <bool NEAR>
__device__ __forceinline__ FxSums fx_sums(const Nb<double> &v, int ef)
{
    FxSums r;
    const long long X = fx_cv<NEAR>(v.xp, ef) + fx_cv<NEAR>(v.xm, ef);
    const long long Y = fx_cv<NEAR>(v.yp, ef) + fx_cv<NEAR>(v.ym, ef);
    const long long Z = fx_cv<NEAR>(v.zp, ef) + fx_cv<NEAR>(v.zm, ef);
    r.a = fx_out(X - Y, ef);
    r.b = fx_out(X - Z, ef);
    r.amb = fx_out(Z - Y, ef);
    r.cxy = fx_out((fx_cv<NEAR>(v.xpyp, ef) + fx_cv<NEAR>(v.xmym, ef)) -
                   (fx_cv<NEAR>(v.xpym, ef) + fx_cv<NEAR>(v.xmyp, ef)), ef);
    r.cxz = fx_out((fx_cv<NEAR>(v.xpzp, ef) + fx_cv<NEAR>(v.xmzm, ef)) -
                   (fx_cv<NEAR>(v.xpzm, ef) + fx_cv<NEAR>(v.xmzp, ef)), ef);
    r.cyz = fx_out((fx_cv<NEAR>(v.ypzp, ef) + fx_cv<NEAR>(v.ymzm, ef)) -
                   (fx_cv<NEAR>(v.ypzm, ef) + fx_cv<NEAR>(v.ymzp, ef)), ef);
    r.s6 = (X + Y) + Z;
    return r;
}

}  // namespace mg
