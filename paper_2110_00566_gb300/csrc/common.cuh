// Shared device code of the GB300 MG-GLAM solvers (arXiv:2110.00566).
//
// Layout.  Every multigrid level of n^3 cells (n even) is stored
// colour-split: cells with (i+j+k) even (colour 0) and odd (colour 1) live in
// two arrays of n*n*(n/2) elements, index (i*n + j)*(n/2) + m with m = k/2.
// In row (i, j) the cells of colour c sit at k = 2m + p, p = (c+i+j) & 1.
// With this layout all 6 face neighbours of a colour-c cell are in the other
// array and all 12 edge neighbours of the 19-point stencil are in the same
// array; the rows (i+-1, j), (i, j+-1), (i+-1, j+-1) are read at the same m,
// except the k+-1 neighbours, which sit at m + p and m + p - 1 (wrapped).
// A half-sweep of one colour therefore reads both arrays and writes a third
// (ping-pong for the updated colour), which makes the colour-simultaneous
// update race-free; the centre value is never read by the smoother.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mg {

// -------------------------------------------------------------------------
// per-level scalars kept in device memory (FP64)
// -------------------------------------------------------------------------
struct LevScal {
    double c;       // compatibility constant <N> used by the smoother
    double fshift;  // constant part of the FAS source (f = f' + fshift)
    double dc;      // c_new - c_old of the last residual pass
    double eps2;    // mean d^2 of the last residual pass (with c_new)
    double sumN;    // sum of N of the last residual pass
    double clamps;  // sqrt clamps counted in the last residual pass
    double mean;    // scratch mean (delta or u)
    double aux;     // scratch
    float cf32;     // (float)(fshift - c), the smoother's constant for FP32 kernels
    float pad_;
};

// (i, j, k) of the natural-layout index q = (i n + j) nz + k on an
// n x n x nz mesh, by 32-bit unsigned divisions where q fits (this GPU has
// no 64-bit integer divider: a 64-bit division or remainder is a long
// instruction sequence)
__device__ __forceinline__ void split3(long long q, int n, int nz, int &i, int &j, int &k)
{
    if (q < 4294967296LL) {
        const unsigned u = (unsigned)q, r = u / (unsigned)nz, a = r / (unsigned)n;
        k = (int)(u - r * (unsigned)nz);
        j = (int)(r - a * (unsigned)n);
        i = (int)a;
    } else {
        const long long r = q / nz;
        k = (int)(q - r * nz);
        j = (int)(r % n);
        i = (int)(r / n);
    }
}

// update c (and the FP32 copy of fshift - c) from a finalising thread
__device__ __forceinline__ void set_c(LevScal *sc, double c)
{
    sc->c = c;
    sc->cf32 = (float)(sc->fshift - c);
}
__device__ __forceinline__ void set_c_fshift(LevScal *sc, double c, double fshift)
{
    sc->c = c;
    sc->fshift = fshift;
    sc->cf32 = (float)(fshift - c);
}

// the smoother's constant fshift - c in the kernel's precision
template <typename T>
__device__ __forceinline__ T smooth_cf(const LevScal *sc);
template <>
__device__ __forceinline__ double smooth_cf<double>(const LevScal *sc) { return sc->fshift - sc->c; }
template <>
__device__ __forceinline__ float smooth_cf<float>(const LevScal *sc) { return sc->cf32; }

// reduction scratch shared by the reduction kernels of one pyramid
struct RedBuf {
    double *partials;       // [MAX_RED_BLOCKS * 4]
    unsigned int *counter;  // one arrival counter, reset by the last block
    int cap;                // blocks the partials buffer holds
};
constexpr int MAX_RED_BLOCKS = 4096;

// -------------------------------------------------------------------------
// operator parameters, with the h-dependent constants folded in on the host
// -------------------------------------------------------------------------
template <typename T>
struct OpK {
    int model;   // 0 nDGP, 1 Kmouflage
    int nkmo;
    T alpha, abs_alpha, sgn_alpha, alpha2, c83;  // nDGP
    T a75, sgn75;                                // nDGP: (3/4) alpha, (3/4) sgn(alpha)
    T k1, k2, k3;                                // Kmouflage: 1+gamma b^(n-1), (2n+1)gamma/3, 2(n-1)gamma
};

template <typename T>
struct LevK {
    int n, half;
    T h2;        // h^2
    T inv_h2;    // 1/h^2
    T qd, qo;    // nDGP: 1/(3h^4), 1/(8h^4)
    T td, to;    // Kmouflage: 1/(12h^4), 1/(8h^4)
    T g2s;       // Kmouflage: 1/(4h^2)
};

template <typename T>
__host__ __device__ inline LevK<T> make_levk(int n, double h)
{
    LevK<T> L{};
    L.n = n;
    L.half = n / 2;
    const double h2 = h * h, h4 = h2 * h2;
    L.h2 = (T)h2;
    L.inv_h2 = (T)(1.0 / h2);
    L.qd = (T)(1.0 / (3.0 * h4));
    L.qo = (T)(1.0 / (8.0 * h4));
    L.td = (T)(1.0 / (12.0 * h4));
    L.to = (T)(1.0 / (8.0 * h4));
    L.g2s = (T)(1.0 / (4.0 * h2));
    return L;
}

// the 18 neighbours of the 19-point stencil
template <typename T>
struct Nb {
    T xp, xm, yp, ym, zp, zm;          // faces
    T xpyp, xmym, xpym, xmyp;          // xy edges
    T xpzp, xmzm, xpzm, xmzp;          // xz edges
    T ypzp, ymzm, ypzm, ymzp;          // yz edges
};

__device__ __forceinline__ int wrap_p(int i, int n) { return i + 1 == n ? 0 : i + 1; }
__device__ __forceinline__ int wrap_m(int i, int n) { return i == 0 ? n - 1 : i - 1; }

__device__ __forceinline__ long long row_of(int i, int j, int n, int half)
{
    return ((long long)i * n + j) * half;
}

// Gather the 18 neighbours of the colour-c cell (i, j, m) whose row parity
// is p = (c+i+j)&1.  S: array of colour c, O: array of the other colour.
template <typename T>
__device__ __forceinline__ void gather(Nb<T> &v, const T *__restrict__ S, const T *__restrict__ O,
                                       int n, int half, int i, int j, int m, int p)
{
    const int ip = wrap_p(i, n), im = wrap_m(i, n), jp = wrap_p(j, n), jm = wrap_m(j, n);
    int mp = m + p;
    if (mp == half) mp = 0;
    int mm = m - 1 + p;
    if (mm < 0) mm = half - 1;
    const long long r00 = row_of(i, j, n, half);
    const long long rp0 = row_of(ip, j, n, half), rm0 = row_of(im, j, n, half);
    const long long r0p = row_of(i, jp, n, half), r0m = row_of(i, jm, n, half);
    v.xp = __ldg(O + rp0 + m);
    v.xm = __ldg(O + rm0 + m);
    v.yp = __ldg(O + r0p + m);
    v.ym = __ldg(O + r0m + m);
    v.zp = __ldg(O + r00 + mp);
    v.zm = __ldg(O + r00 + mm);
    v.xpyp = __ldg(S + row_of(ip, jp, n, half) + m);
    v.xmym = __ldg(S + row_of(im, jm, n, half) + m);
    v.xpym = __ldg(S + row_of(ip, jm, n, half) + m);
    v.xmyp = __ldg(S + row_of(im, jp, n, half) + m);
    v.xpzp = __ldg(S + rp0 + mp);
    v.xmzm = __ldg(S + rm0 + mm);
    v.xpzm = __ldg(S + rp0 + mm);
    v.xmzp = __ldg(S + rm0 + mp);
    v.ypzp = __ldg(S + r0p + mp);
    v.ymzm = __ldg(S + r0m + mm);
    v.ypzm = __ldg(S + r0p + mm);
    v.ymzp = __ldg(S + r0m + mp);
}

// the same 18 neighbours of two fields at once (unknown and base field)
template <typename T>
__device__ __forceinline__ void gather2(Nb<T> &v, Nb<T> &w, const T *__restrict__ S, const T *__restrict__ O,
                                        const T *__restrict__ BS, const T *__restrict__ BO, int n, int half, int i,
                                        int j, int m, int p)
{
    const int ip = wrap_p(i, n), im = wrap_m(i, n), jp = wrap_p(j, n), jm = wrap_m(j, n);
    int mp = m + p;
    if (mp == half) mp = 0;
    int mm = m - 1 + p;
    if (mm < 0) mm = half - 1;
    const long long r00 = row_of(i, j, n, half);
    const long long rp0 = row_of(ip, j, n, half), rm0 = row_of(im, j, n, half);
    const long long r0p = row_of(i, jp, n, half), r0m = row_of(i, jm, n, half);
    const long long rpp = row_of(ip, jp, n, half), rmm = row_of(im, jm, n, half);
    const long long rpm = row_of(ip, jm, n, half), rmp = row_of(im, jp, n, half);
    v.xp = __ldg(O + rp0 + m);   w.xp = __ldg(BO + rp0 + m);
    v.xm = __ldg(O + rm0 + m);   w.xm = __ldg(BO + rm0 + m);
    v.yp = __ldg(O + r0p + m);   w.yp = __ldg(BO + r0p + m);
    v.ym = __ldg(O + r0m + m);   w.ym = __ldg(BO + r0m + m);
    v.zp = __ldg(O + r00 + mp);  w.zp = __ldg(BO + r00 + mp);
    v.zm = __ldg(O + r00 + mm);  w.zm = __ldg(BO + r00 + mm);
    v.xpyp = __ldg(S + rpp + m); w.xpyp = __ldg(BS + rpp + m);
    v.xmym = __ldg(S + rmm + m); w.xmym = __ldg(BS + rmm + m);
    v.xpym = __ldg(S + rpm + m); w.xpym = __ldg(BS + rpm + m);
    v.xmyp = __ldg(S + rmp + m); w.xmyp = __ldg(BS + rmp + m);
    v.xpzp = __ldg(S + rp0 + mp); w.xpzp = __ldg(BS + rp0 + mp);
    v.xmzm = __ldg(S + rm0 + mm); w.xmzm = __ldg(BS + rm0 + mm);
    v.xpzm = __ldg(S + rp0 + mm); w.xpzm = __ldg(BS + rp0 + mm);
    v.xmzp = __ldg(S + rm0 + mp); w.xmzp = __ldg(BS + rm0 + mp);
    v.ypzp = __ldg(S + r0p + mp); w.ypzp = __ldg(BS + r0p + mp);
    v.ymzm = __ldg(S + r0m + mm); w.ymzm = __ldg(BS + r0m + mm);
    v.ypzm = __ldg(S + r0p + mm); w.ypzm = __ldg(BS + r0p + mm);
    v.ymzp = __ldg(S + r0m + mp); w.ymzp = __ldg(BS + r0m + mp);
}

// square root and quotient in the kernel's precision: IEEE in FP64; in FP32
// the PTX approximate forms (sqrt.approx, div.approx: a few ulp), since every
// FP32 result feeds a correction that the FP64 defect of the mixed solve
// re-measures
// FP64 square root by one Newton (Heron) step on a single-precision estimate:
// s0 = x y0 with y0 ~ 1/sqrt(x) (relative error e0 ~ 2^-22 from the FP32
// special-function unit), then s1 = s0 + (y0 / 2)(x - s0^2), which
// approximates s0 + (x - s0^2)/(2 s0); relative error ~ e0^2, about 5e-14,
// far below the residuals any solve resolves.  FP64 runs at 1/63 of the FP32
// rate on this GPU, so the estimate is formed with integer operations on the
// IEEE 754 layouts and the FP64 pipe issues three instructions: with
// x = 1.m 2^(2k + r) (r = 0 or 1), the float 1.m 2^r in [1, 4) (x's mantissa
// truncated to 23 bits, which only perturbs the estimate) gives
// rsqrtf = 1.m' 2^q, and y0 = 1.m' 2^(q - k) is that float's bit pattern
// re-biased to binary64 (exponent + 1023 - 127 - k).  Valid for every
// positive normal x (and +-0, which return +-0); NaN and infinity give NaN.
__device__ __forceinline__ double k_sqrt(double x)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int E = ((hi >> 20) & 0x7FF) - 1023;   // unbiased exponent (sign ignored: x >= 0 or -0)
    const int k = E >> 1, r = E & 1;           // E = 2k + r (floor)
    const float xf = __int_as_float(((127 + r) << 23) | ((hi & 0x000FFFFF) << 3) | (int)(lo >> 29));
    const int yb = __float_as_int(rsqrtf(xf));
    const double y = __hiloint2double((yb >> 3) + ((896 - k) << 20), yb << 29);
    const double hy = __hiloint2double((yb >> 3) + ((895 - k) << 20), yb << 29);   // y / 2
    const double s0 = x * y;
    return fma(hy, fma(-s0, s0, x), s0);
}
// FP64 reciprocal estimate of a positive normal d (below 2^1022) from the
// single-precision special-function unit: with d = 1.m 2^E, the float 1.m
// in [1, 2) (d's mantissa truncated to 23 bits) gives rcp = 1.m' 2^q, and the
// estimate 1.m' 2^(q - E) is that float's bit pattern re-biased to binary64
// (exponent + 1023 - 127 - E); relative error below 2^-22 (the truncation
// and the approximate reciprocal, each under 2^-23), no FP64 instruction
__device__ __forceinline__ double k_rcp_est(double d)
{
    const int hi = __double2hiint(d);
    const unsigned lo = (unsigned)__double2loint(d);
    const int E = ((hi >> 20) & 0x7FF) - 1023;
    const float xf = __int_as_float((127 << 23) | ((hi & 0x000FFFFF) << 3) | (int)(lo >> 29));
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(xf));
    const int yb = __float_as_int(rf);
    return __hiloint2double((yb >> 3) + ((896 - E) << 20), yb << 29);
}

// FP64 quotient a / d for a positive normal d (below 2^1022): q0 = a y with
// y = k_rcp_est(d) = (1 + e)/d, then one correction by the exact residual
// a - d q0 (a fused multiply-add): q = q0 + y (a - d q0) = (a/d)(1 - e^2 + ...),
// relative error about e^2 < 2^-44, three FP64 instructions
__device__ __forceinline__ double k_quot(double a, double d)
{
    const double y = k_rcp_est(d);
    const double q0 = a * y;
    return fma(y, fma(-d, q0, a), q0);
}
__device__ __forceinline__ double k_div(double a, double b) { return a / b; }
__device__ __forceinline__ float k_sqrt(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float k_div(float a, float b)
{
    float r;
    asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

template <typename T>
__device__ __forceinline__ T ipow(T x, int p)
{
    T r = T(1);
    for (int q = 0; q < p; ++q) r *= x;
    return r;
}

// N(u) at a cell, the right-hand side of Lap u = N(u).
//  nDGP (Sec. 3.2.3, Eq. DGP): Sigma = Q + s with
//    Q = [(Sx-Sy)^2 + (Sx-Sz)^2 + (Sy-Sz)^2]/(3h^4) + (Cxy^2+Cxz^2+Cyz^2)/(8h^4)
//  (the printed (2/3h^4)[Dxx^2+... - DxxDyy - ...] rewritten with
//  D_aa - D_bb = S_a - S_b, which shows that Sigma has no centre term), and
//    N = 2 sgn(alpha) Sigma / (|alpha| + sqrt(alpha^2 + 8 Sigma/3)),
//  the rationalised form of (3/4)[-alpha + sgn(alpha) sqrt(...)]; a negative
//  sqrt argument gives -(3/4) alpha and is counted.
//  Kmouflage (Sec. 3.2.4, Eq. kmf_eqn_codeunit_final / c~):
//    N = (s - 2(n-1) gamma (G^2)^(n-2) T) / (1 + gamma b^(n-1) + (2n+1)gamma/3 (G^2)^(n-1))
// MODEL: 0 or 1 compiles only that operator (the caller knows the model);
// -1 dispatches on op.model at run time
template <typename T, int MODEL = -1>
__device__ __forceinline__ T op_N(const OpK<T> &op, const LevK<T> &L, const Nb<T> &v, T s, int &clamp)
{
    const T Sx = v.xp + v.xm, Sy = v.yp + v.ym, Sz = v.zp + v.zm;
    const T Cxy = (v.xpyp + v.xmym) - (v.xpym + v.xmyp);
    const T Cxz = (v.xpzp + v.xmzm) - (v.xpzm + v.xmzp);
    const T Cyz = (v.ypzp + v.ymzm) - (v.ypzm + v.ymzp);
    if (MODEL == 0 || (MODEL < 0 && op.model == 0)) {
        const T a = Sx - Sy, b = Sx - Sz, c = Sy - Sz;
        const T Q = (a * a + b * b + c * c) * L.qd + (Cxy * Cxy + Cxz * Cxz + Cyz * Cyz) * L.qo;
        const T sig = Q + s;
        const T arg = op.alpha2 + op.c83 * sig;
        if (arg < T(0)) {
            clamp = 1;
            return T(-0.75) * op.alpha;
        }
        // the rationalised form in both precisions: its error is relative to
        // N itself for any Sigma (the printed difference r - |alpha| cancels
        // for Sigma << alpha^2, where it would carry the square root's error
        // relative to alpha)
        return k_div(T(2) * op.sgn_alpha * sig, op.abs_alpha + k_sqrt(arg));
    } else {
        const T dx = v.xp - v.xm, dy = v.yp - v.ym, dz = v.zp - v.zm;
        const T dx2 = dx * dx, dy2 = dy * dy, dz2 = dz * dz;
        const T G2 = (dx2 + dy2 + dz2) * L.g2s;
        const T Tt = (dx2 * (T(2) * Sx - Sy - Sz) + dy2 * (T(2) * Sy - Sx - Sz) + dz2 * (T(2) * Sz - Sx - Sy)) * L.td
                   + (Cxy * dx * dy + Cxz * dx * dz + Cyz * dy * dz) * L.to;
        const T pw2 = ipow(G2, op.nkmo - 2);
        const T sigma1 = op.k1 + op.k2 * pw2 * G2;
        return k_div(s - op.k3 * pw2 * Tt, sigma1);
    }
}

// dN = N(b + e) - N(b) at a cell, for the correction form of the mixed
// precision solve: e (neighbours v) is the unknown correction, b (neighbours
// w) the frozen base field.  Every difference is expanded so that no two
// large terms cancel, which keeps the FP32 evaluation accurate relative to
// the correction itself:
//  nDGP: dSigma = sum_t t(e) (2 t(b) + t(e)) over the linear terms t of Q,
//        dN = 2 sgn(alpha) dSigma / (r0 + r1), r = sqrt(alpha^2 + 8 Sigma/3)
//        (from r1^2 - r0^2 = 8 dSigma / 3); a negative sqrt argument falls
//        back to the clamped difference N1 - N0.
//  Kmouflage: N = A/B with A = s - k3 G2^(n-2) T, B = k1 + k2 G2^(n-1):
//        dN = (dA - N0 dB) / B1, where dG2, dT and the powers' differences
//        are formed from products of the differenced linear terms.
template <typename T>
__device__ __forceinline__ T nd_clamped(const OpK<T> &op, T sig)
{
    const T arg = op.alpha2 + op.c83 * sig;
    if (arg < T(0)) return T(-0.75) * op.alpha;
    return k_div(T(2) * op.sgn_alpha * sig, op.abs_alpha + k_sqrt(arg));
}

template <typename T, int MODEL = -1>
__device__ __forceinline__ T op_dN(const OpK<T> &op, const LevK<T> &L, const Nb<T> &v, const Nb<T> &w, T s,
                                   int &clamp)
{
    const T eSx = v.xp + v.xm, eSy = v.yp + v.ym, eSz = v.zp + v.zm;
    const T bSx = w.xp + w.xm, bSy = w.yp + w.ym, bSz = w.zp + w.zm;
    const T eCxy = (v.xpyp + v.xmym) - (v.xpym + v.xmyp);
    const T eCxz = (v.xpzp + v.xmzm) - (v.xpzm + v.xmzp);
    const T eCyz = (v.ypzp + v.ymzm) - (v.ypzm + v.ymzp);
    const T bCxy = (w.xpyp + w.xmym) - (w.xpym + w.xmyp);
    const T bCxz = (w.xpzp + w.xmzm) - (w.xpzm + w.xmzp);
    const T bCyz = (w.ypzp + w.ymzm) - (w.ypzm + w.ymzp);
    if (MODEL == 0 || (MODEL < 0 && op.model == 0)) {
        const T ea = eSx - eSy, eb = eSx - eSz, ec = eSy - eSz;
        const T ba = bSx - bSy, bb = bSx - bSz, bc = bSy - bSz;
        const T dQ = (ea * (T(2) * ba + ea) + eb * (T(2) * bb + eb) + ec * (T(2) * bc + ec)) * L.qd +
                     (eCxy * (T(2) * bCxy + eCxy) + eCxz * (T(2) * bCxz + eCxz) + eCyz * (T(2) * bCyz + eCyz)) * L.qo;
        const T Q0 = (ba * ba + bb * bb + bc * bc) * L.qd + (bCxy * bCxy + bCxz * bCxz + bCyz * bCyz) * L.qo;
        const T sig0 = Q0 + s, sig1 = sig0 + dQ;
        const T arg0 = op.alpha2 + op.c83 * sig0, arg1 = op.alpha2 + op.c83 * sig1;
        if (arg0 < T(0) || arg1 < T(0)) {
            clamp = 1;
            return nd_clamped(op, sig1) - nd_clamped(op, sig0);
        }
        const T den = k_sqrt(arg0) + k_sqrt(arg1);
        return den > T(0) ? k_div(T(2) * op.sgn_alpha * dQ, den) : T(0);
    } else {
        const T edx = v.xp - v.xm, edy = v.yp - v.ym, edz = v.zp - v.zm;
        const T bdx = w.xp - w.xm, bdy = w.yp - w.ym, bdz = w.zp - w.zm;
        const T dx1 = bdx + edx, dy1 = bdy + edy, dz1 = bdz + edz;
        const T bWx = T(2) * bSx - bSy - bSz, bWy = T(2) * bSy - bSx - bSz, bWz = T(2) * bSz - bSx - bSy;
        const T eWx = T(2) * eSx - eSy - eSz, eWy = T(2) * eSy - eSx - eSz, eWz = T(2) * eSz - eSx - eSy;
        const T qx = edx * (T(2) * bdx + edx), qy = edy * (T(2) * bdy + edy), qz = edz * (T(2) * bdz + edz);
        const T G20 = (bdx * bdx + bdy * bdy + bdz * bdz) * L.g2s;
        const T dG2 = (qx + qy + qz) * L.g2s;
        const T G21 = G20 + dG2;
        const T T0 = (bdx * bdx * bWx + bdy * bdy * bWy + bdz * bdz * bWz) * L.td +
                     (bCxy * bdx * bdy + bCxz * bdx * bdz + bCyz * bdy * bdz) * L.to;
        const T dTd = qx * (bWx + eWx) + bdx * bdx * eWx + qy * (bWy + eWy) + bdy * bdy * eWy + qz * (bWz + eWz) +
                      bdz * bdz * eWz;
        const T dTc = eCxy * dx1 * dy1 + bCxy * edx * dy1 + bCxy * bdx * edy + eCxz * dx1 * dz1 + bCxz * edx * dz1 +
                      bCxz * bdx * edz + eCyz * dy1 * dz1 + bCyz * edy * dz1 + bCyz * bdy * edz;
        const T dT = dTd * L.td + dTc * L.to;
        const int nk = op.nkmo;
        // G21^j G20^(m-1-j) summed over j: the factor of dG2 in G21^m - G20^m
        T g_nm2 = T(0), g_nm1 = T(0);
        {
            T pa = T(1);
            for (int jx = 0; jx <= nk - 2; ++jx) {
                T pb = T(1);
                for (int q = 0; q < nk - 2 - jx; ++q) pb *= G20;
                g_nm1 += pa * pb;
                pa *= G21;
            }
            pa = T(1);
            for (int jx = 0; jx <= nk - 3; ++jx) {
                T pb = T(1);
                for (int q = 0; q < nk - 3 - jx; ++q) pb *= G20;
                g_nm2 += pa * pb;
                pa *= G21;
            }
        }
        const T pw0 = ipow(G20, nk - 2), pw1 = ipow(G21, nk - 2);
        const T dP = pw1 * dT + T0 * dG2 * g_nm2;
        const T B0 = op.k1 + op.k2 * pw0 * G20, B1 = op.k1 + op.k2 * pw1 * G21;
        const T N0 = k_div(s - op.k3 * pw0 * T0, B0);
        return k_div(-op.k3 * dP - N0 * op.k2 * dG2 * g_nm1, B1);
    }
}

// -------------------------------------------------------------------------
// deterministic block reduction of NV doubles (warp shuffles, fixed order)
// -------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *sh /* >= 32*NV */)
{
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5, nwarps = (nthreads + 31) >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[warp * NV + q] = v[q];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            v[q] = lane < nwarps ? sh[lane * NV + q] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
        }
    }
}

// Store this block's NV sums as partials; the block that arrives last sums
// all partials in block order (so the result does not depend on scheduling)
// and returns true in every one of its threads with the totals in tot[]
// (valid in thread 0).  Blocks must be launched with >= 32 threads.
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], const RedBuf &rb, double (&tot)[NV])
{
    __shared__ double sh[32 * NV];
    __shared__ bool last;
    block_sum<NV>(v, sh);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) rb.partials[(size_t)bid * NV + q] = v[q];
        __threadfence();
        const unsigned t = atomicAdd(rb.counter, 1u);
        last = (t == nb - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0;
    // each thread sums a contiguous chunk in order, then the block tree
    const unsigned per = (nb + nthreads - 1) / nthreads;
    const unsigned b0 = tid * per, b1 = min(nb, b0 + per);
    for (unsigned b = b0; b < b1; ++b)
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += __ldcg(rb.partials + (size_t)b * NV + q);
    block_sum<NV>(acc, sh);
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = acc[q];
    if (tid == 0) *rb.counter = 0u;
    return true;
}

// grid_sum for NV FP64 sums and one integer count per thread (a flag count:
// reduced on the integer pipe, so that it costs no FP64 add per thread);
// tot[0 .. NV-1] are the sums, tot[NV] the count (exact as a double).  The
// sums come out bit-identical to grid_sum's: each value's reduction tree
// does not depend on the others.  Every thread of the block must call it.
template <int NV>
__device__ __forceinline__ bool grid_sum_cnt(double (&v)[NV], int cnt, const RedBuf &rb, double (&tot)[NV + 1])
{
    __shared__ double sh[32 * (NV + 1)];
    __shared__ bool last;
    __shared__ unsigned int scnt;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    if (tid == 0) scnt = 0u;
    __syncthreads();
    const unsigned wc = __reduce_add_sync(0xffffffffu, (unsigned)cnt);
    if ((tid & 31) == 0) atomicAdd(&scnt, wc);
    block_sum<NV>(v, sh);   // (its barriers also order the count's atomics before thread 0 reads it)
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) rb.partials[(size_t)bid * (NV + 1) + q] = v[q];
        rb.partials[(size_t)bid * (NV + 1) + NV] = (double)scnt;
        __threadfence();
        const unsigned t = atomicAdd(rb.counter, 1u);
        last = (t == nb - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[NV + 1];
#pragma unroll
    for (int q = 0; q <= NV; ++q) acc[q] = 0.0;
    const unsigned per = (nb + nthreads - 1) / nthreads;
    const unsigned b0 = tid * per, b1 = min(nb, b0 + per);
    for (unsigned b = b0; b < b1; ++b)
#pragma unroll
        for (int q = 0; q <= NV; ++q) acc[q] += __ldcg(rb.partials + (size_t)b * (NV + 1) + q);
    block_sum<NV + 1>(acc, sh);
#pragma unroll
    for (int q = 0; q <= NV; ++q) tot[q] = acc[q];
    if (tid == 0) *rb.counter = 0u;
    return true;
}

// The same deterministic reduction over `nb` work tiles of one problem when
// a persistent block processes tiles of several problems: tile `bid`
// stores its block sums, and the block that stores the last one sums all
// partials in tile order and returns true (totals valid in thread 0).
template <int NV>
__device__ __forceinline__ bool tile_sum(double (&v)[NV], double *partials, unsigned int *counter, unsigned bid,
                                         unsigned nb, double (&tot)[NV])
{
    __shared__ double sh[32 * NV];
    __shared__ bool last;
    block_sum<NV>(v, sh);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) partials[(size_t)bid * NV + q] = v[q];
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == nb - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0;
    const unsigned per = (nb + nthreads - 1) / nthreads;
    const unsigned b0 = tid * per, b1 = min(nb, b0 + per);
    for (unsigned b = b0; b < b1; ++b)
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += __ldcg(partials + (size_t)b * NV + q);
    block_sum<NV>(acc, sh);
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = acc[q];
    if (tid == 0) *counter = 0u;
    __syncthreads();
    return true;
}

}  // namespace mg
