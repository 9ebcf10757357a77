// Block fixed-point staging of the FP64 nDGP kernels: a block owns a tile of
// 32 split-index columns by 8 rows of one level and walks consecutive planes;
// a ring of three planes (both colour arrays, the tile plus its one-cell
// halo) holds the level's values in shared memory converted once to the
// fixed-point integers of fixsum.cuh, so that the 19-point stencil's signed
// sums and quadratic form are formed from shared-memory integers with no
// per-use conversion.
//
// Scale.  The three staged planes share one scale, the largest exponent field
// E among their values (each plane's maximum over the tile and its halo, both
// colours, is kept): x = M 2^(e - 1075) becomes sign(x) floor(M 2^6 / 2^(E - e)),
// exact when E - e <= 6 and otherwise within 2^(E - 1081), 1/64 of an ulp of
// the largest value of the three planes.  When the next plane raises E the
// staged planes are shifted down to it (sign and magnitude: exactly the
// values a direct conversion at the new scale gives); when E falls by more
// than two binades they are read again (from L2) and converted at the new
// scale, so that the scale never exceeds the local largest value by more
// than 2^2.  Outside the fixed-point domain (fx_ok: a value above 2^506,
// NaN or infinity) the caller evaluates those planes' cells in FP64.
//
// Use: construct, fill(i0), then per plane i: prefetch(i + 2) before the
// update of plane i, the update (slots sm, s0, sp hold planes i - 1, i, i + 1),
// and advance(step) after it.  Every thread of the block must make the same
// calls (they contain barriers).
#pragma once
#include "fixsum.cuh"

namespace mg {
namespace bfp {

constexpr int TM = 32;                  // split-index columns of the stencil kernels' tiles
constexpr int W = TM + 2;               // with the k+-1 halo columns
constexpr int THREADS = 256;

// a tile of TMc split-index columns and TJ rows with a one-cell halo: values
// per colour and plane, values staged per plane (both colours)
template <int TJ, int TMc = TM>
struct Tile {
    static constexpr int Wc = TMc + 2;
    static constexpr int H = TJ + 2;
    static constexpr int PLANE = Wc * H;
    static constexpr int LOAD = 2 * PLANE;
};

template <int TJ, int TMc = TM>
struct Shared {
    long long v[3][Tile<TJ, TMc>::LOAD];   // slot -> [colour][row][column]
    int pmax[3];                           // each slot's largest exponent field
    int emax[2];                           // block maximum of a plane being reduced (double-buffered)
};

// sign-and-magnitude shift to a coarser scale: the truncation toward zero of
// the conversion itself
__device__ __forceinline__ long long down(long long v, unsigned d)
{
    if (d >= 63) return 0;
    const long long a = v < 0 ? -v : v;
    const long long r = a >> d;
    return v < 0 ? -r : r;
}

__device__ __forceinline__ int ef_of(double x) { return __double2hiint(x) & 0x7FF00000; }

// a constant K at the block's scale ef, for folding into a fixed-point sum
// whose terms stay below 1.5 2^62 (S6, S6 - 6u): exact to the scale for |K|
// up to four times the scale's largest value (|V| < 2^61, so the sum stays
// below 2^63); ok = false beyond that (or for K not finite): the caller adds
// K in FP64 instead
__device__ __forceinline__ long long fold(double K, int ef, bool &ok)
{
    const int d = ef_of(K) - ef;   // in place
    ok = d <= (2 << 20);
    if (!ok) return 0;
    if (d <= 0) return fx_in<6>(K, ef);
    return fx_in<6>(K, ef + d) << (d >> 20);
}

// the value of colour slot c (0: A0, 1: A1) at tile row r, column col
template <int TJ, int TMc = TM>
__device__ __forceinline__ long long at(const long long *slot, int c, int r, int col)
{
    return slot[c * Tile<TJ, TMc>::PLANE + r * Tile<TJ, TMc>::Wc + col];
}

// S: guard bits of the conversion (fixsum.cuh): 6 for the stencil sums
// (|V| < 2^59), 3 where 64 values are summed with integer weights.  Each half
// of the block stages one colour: thread tid holds elements
// e = tid % HT + q HT (q < PC) of colour tid / HT's plane, so that its global
// array and shared-memory row are fixed and only the last element can fall
// outside the plane.  NEAR: stage each value by two 32-bit funnel shifts
// where it lies within 32 binades of the scale (the usual case; identical
// result), the general 64-bit shift otherwise (fewer instructions per
// staged value, more live registers: the smoother takes it).
template <int TJ, int TMc = TM, int S = 6, bool NEAR = false>
struct Stager {
    static constexpr int PLANE = Tile<TJ, TMc>::PLANE, LOAD = Tile<TJ, TMc>::LOAD;
    static constexpr int Wc = Tile<TJ, TMc>::Wc;
    static constexpr int HT = THREADS / 2;               // threads per colour
    static constexpr int PC = (PLANE + HT - 1) / HT;     // elements per thread
    Shared<TJ, TMc> &t;
    const double *A;         // this thread's colour array
    int n, tid, sb;          // sb: shared-memory index of element q = 0
    long long pstride;
    int goff[PC];
    double x[PC];            // a plane in flight
    int E = 0;               // the staged planes' largest exponent field (0: all zero)
    int ef = 1023 << 20;     // the conversion scale
    int sm = 0, s0 = 1, sp = 2;

    // element e of colour c is tile row jj = e / Wc, column mm = e % Wc: row
    // j0 - 1 + jj and split index m0 - 1 + mm (wrapped)
    __device__ Stager(Shared<TJ, TMc> &sh, const double *a0, const double *a1, int n_, int half, int m0, int j0,
                      int tid_)
        : t(sh), A((tid_ / HT) ? a1 : a0), n(n_), tid(tid_), sb((tid_ / HT) * PLANE + tid_ % HT),
          pstride((long long)n_ * half)
    {
#pragma unroll
        for (int q = 0; q < PC; ++q) {
            const int e = tid % HT + q * HT;
            const int ee = e < PLANE ? e : 0;
            const int jj = ee / Wc, mm = ee - jj * Wc;
            int j = j0 - 1 + jj, m = m0 - 1 + mm;
            j = j < 0 ? j + n : (j >= n ? j - n : j);
            m = m < 0 ? m + half : (m >= half ? m - half : m);
            goff[q] = j * half + m;
        }
    }
    // element q lies in the plane (always for q < PC - 1)
    __device__ bool in(int q) const { return q < PC - 1 || tid % HT + q * HT < PLANE; }
    __device__ int wrap(int i) const { return i < 0 ? i + n : (i >= n ? i - n : i); }
    __device__ void prefetch(int ip)
    {
        const double *Ap = A + (long long)wrap(ip) * pstride;
#pragma unroll
        for (int q = 0; q < PC; ++q) x[q] = in(q) ? __ldg(Ap + goff[q]) : 0.0;
    }
    __device__ int xmax() const
    {
        int e = 0;
#pragma unroll
        for (int q = 0; q < PC; ++q) e = max(e, ef_of(x[q]));
        return e;
    }
    __device__ void block_max(int slot, int e)
    {
        e = __reduce_max_sync(0xffffffffu, e);
        if ((tid & 31) == 0) atomicMax(&t.emax[slot], e);
    }
    __device__ static long long cv(double v, int e)
    {
        if (!NEAR) return fx_in<S>(v, e);
        const unsigned sh = (unsigned)(e - (__double2hiint(v) & 0x7FF00000)) >> 20;
        return sh < 32 ? fx_in_near<S>(v, e) : fx_in<S>(v, e);
    }
    __device__ void store(int s)
    {
        long long *d = t.v[s] + sb;
#pragma unroll
        for (int q = 0; q < PC; ++q)
            if (in(q)) d[q * HT] = cv(x[q], ef);
    }
    __device__ void shift_down(int s, unsigned d)
    {
        for (int e = tid; e < LOAD; e += THREADS) t.v[s][e] = down(t.v[s][e], d);
    }
    // plane ip read again into slot s at the current scale (x is in use for
    // the next plane, so this thread's elements are read one at a time)
    __device__ void reconvert(int s, int ip)
    {
        const double *Ap = A + (long long)wrap(ip) * pstride;
        long long *d = t.v[s] + sb;
#pragma unroll
        for (int q = 0; q < PC; ++q)
            if (in(q)) d[q * HT] = fx_in<S>(__ldg(Ap + goff[q]), ef);
    }
    // planes i0 - 1, i0, i0 + 1 into slots 0, 1, 2; each plane's maximum is
    // reduced on its own (reduction slot q & 1; the other slot, read before
    // the previous barrier, is cleared between this plane's two barriers)
    __device__ void fill(int i0)
    {
        if (tid == 0) {
            t.emax[0] = 0;
            t.emax[1] = 0;
        }
        __syncthreads();
        double xs[2][PC];
        for (int q3 = 0; q3 < 3; ++q3) {
            prefetch(i0 + q3 - 1);
            block_max(q3 & 1, xmax());
            __syncthreads();
            const int e3 = t.emax[q3 & 1];
            if (tid == 0) {
                t.pmax[q3] = e3;
                t.emax[(q3 + 1) & 1] = 0;
            }
            __syncthreads();
            E = max(E, e3);
            if (q3 < 2) {
#pragma unroll
                for (int q = 0; q < PC; ++q) xs[q3][q] = x[q];
            }
        }
        ef = fx_zero_scale(E);
        store(2);
#pragma unroll
        for (int q = 0; q < PC; ++q) x[q] = xs[0][q];
        store(0);
#pragma unroll
        for (int q = 0; q < PC; ++q) x[q] = xs[1][q];
        store(1);
        if (tid == 0) t.emax[0] = 0;   // slot 0, last read before the fill's final barrier
        __syncthreads();
        sm = 0;
        s0 = 1;
        sp = 2;
    }
    // after the update of plane i: stage the prefetched plane i + 2 into the
    // slot of plane i - 1, at the scale of planes i, i + 1, i + 2, and rotate
    // the slots (step counts from 0)
    __device__ void advance(int step, int i)
    {
        block_max(step & 1, xmax());
        __syncthreads();
        const int en = t.emax[step & 1];
        const int Et = max(max(t.pmax[s0], t.pmax[sp]), en);
        if (Et > E) {
            if (E != 0) {
                const unsigned d = (unsigned)(Et - E) >> 20;
                shift_down(s0, d);
                shift_down(sp, d);
            }
            E = Et;
            ef = fx_zero_scale(E);
        } else if (Et < E - (2 << 20)) {
            E = Et;
            ef = fx_zero_scale(E);
            reconvert(s0, i);
            reconvert(sp, i + 1);
        }
        store(sm);
        if (tid == 0) {
            t.pmax[sm] = en;
            t.emax[(step + 1) & 1] = 0;
        }
        __syncthreads();
        const int o = s0;
        s0 = sp;
        sp = sm;
        sm = o;
    }
};

// the 19-point stencil of the colour-c cell at tile row jj, column mm of
// plane i (row parity p = (c + i + j) & 1) from the staged integers: the
// face sums X, Y, Z (S6 = X + Y + Z) and the mixed differences C_xy, C_xz,
// C_yz; slot colour c is the cell's own array, 1 - c the other
struct Sums {
    long long X, Y, Z, cxy, cxz, cyz;
};
template <int TJ>
__device__ __forceinline__ Sums stencil(const long long *Sm, const long long *S0, const long long *Sp, int c, int jj,
                                        int mm, int p)
{
    const int o = 1 - c;
    Sums r;
    r.X = at<TJ>(Sp, o, jj, mm) + at<TJ>(Sm, o, jj, mm);
    r.Y = at<TJ>(S0, o, jj + 1, mm) + at<TJ>(S0, o, jj - 1, mm);
    r.Z = at<TJ>(S0, o, jj, mm + p) + at<TJ>(S0, o, jj, mm + p - 1);
    r.cxy = (at<TJ>(Sp, c, jj + 1, mm) + at<TJ>(Sm, c, jj - 1, mm)) -
            (at<TJ>(Sp, c, jj - 1, mm) + at<TJ>(Sm, c, jj + 1, mm));
    r.cxz = (at<TJ>(Sp, c, jj, mm + p) + at<TJ>(Sm, c, jj, mm + p - 1)) -
            (at<TJ>(Sp, c, jj, mm + p - 1) + at<TJ>(Sm, c, jj, mm + p));
    r.cyz = (at<TJ>(S0, c, jj + 1, mm + p) + at<TJ>(S0, c, jj - 1, mm + p - 1)) -
            (at<TJ>(S0, c, jj + 1, mm + p - 1) + at<TJ>(S0, c, jj - 1, mm + p));
    return r;
}

// the central differences of the face neighbours (Kmouflage's gradient):
// Delta_x = u(i+1) - u(i-1) etc., exact in the staged integers
struct Diffs {
    long long dx, dy, dz;
};
template <int TJ>
__device__ __forceinline__ Diffs diffs(const long long *Sm, const long long *S0, const long long *Sp, int c, int jj,
                                       int mm, int p)
{
    const int o = 1 - c;
    Diffs d;
    d.dx = at<TJ>(Sp, o, jj, mm) - at<TJ>(Sm, o, jj, mm);
    d.dy = at<TJ>(S0, o, jj + 1, mm) - at<TJ>(S0, o, jj - 1, mm);
    d.dz = at<TJ>(S0, o, jj, mm + p) - at<TJ>(S0, o, jj, mm + p - 1);
    return d;
}

// N_K of the Kmouflage operator (Sec. 3.2.4, Eq. kmf_eqn_codeunit_final
// over c~) from the staged integers: the linear parts -- Delta_a, the
// combinations 2 S_a - S_b - S_c and 1.5 C_ab -- exact integers rounded once
// to binary64 at the scale ef, the rest in FP64.  With S2 = sum_a Delta_a^2
// (G^2 = S2 / (4 h^2)) and T' = sum_a Delta_a^2 (2 S_a - S_b - S_c) +
// (3/2) sum_{a<b} C_ab Delta_a Delta_b (T = T' / (12 h^4): the cross
// coefficient 1/(8 h^4) is 3/2 of 1/(12 h^4)),
//   N_K = (s - k3 (G^2)^(n-2) T) / (k1 + k2 (G^2)^(n-1))
//       = (s - KA S2^(n-2) T') / (k1 + KB S2^(n-1)),
// KA = k3 g^(n-2) / (12 h^4), KB = k2 g^(n-1), g = 1/(4 h^2) (KmoK, per
// level), so that no power of the level's constants is formed per cell
// (k1 = 1 + gamma (phibar'/H0)^(2(n-1)), k2 = (2n+1) gamma / 3, k3 = 2 (n-1)
// gamma); the quotient by the corrected single-precision reciprocal (k_quot:
// the denominator is at least 1).  19 FP64 instructions for n = 2.
struct KmoK {
    double KA, KB;
    int nm2;   // n - 2
};
__device__ __forceinline__ KmoK make_kmok(const OpK<double> &op, const LevK<double> &L)
{
    double g = 1.0;
    for (int q = 0; q < op.nkmo - 2; ++q) g *= L.g2s;
    return KmoK{op.k3 * L.td * g, op.k2 * g * L.g2s, op.nkmo - 2};
}
__device__ __forceinline__ double kmo64_N(const OpK<double> &op, const KmoK &kk, const Sums &r, const Diffs &d,
                                          double s, int ef)
{
    const double dx = fx_out(d.dx, ef), dy = fx_out(d.dy, ef), dz = fx_out(d.dz, ef);
    const double px = fx_out(2 * r.X - r.Y - r.Z, ef), py = fx_out(2 * r.Y - r.X - r.Z, ef);
    const double pz = fx_out(2 * r.Z - r.X - r.Y, ef);
    // 1.5 C_ab exactly: 3 C_ab (|.| < 2^63) at half the scale
    const double cxy = fx_out<7>(3 * r.cxy, ef), cxz = fx_out<7>(3 * r.cxz, ef), cyz = fx_out<7>(3 * r.cyz, ef);
    const double dx2 = dx * dx, dy2 = dy * dy, dz2 = dz * dz;
    const double S2 = (dx2 + dy2) + dz2;
    double T = fma(dx2, px, fma(dy2, py, dz2 * pz));
    T = fma(cxy, dx * dy, fma(cxz, dx * dz, fma(cyz, dy * dz, T)));
    double B, A;
    if (kk.nm2 == 0) {
        B = fma(kk.KB, S2, op.k1);
        A = fma(-kk.KA, T, s);
    } else {
        double pw = S2;
        for (int q = 1; q < kk.nm2; ++q) pw *= S2;
        B = fma(kk.KB * pw, S2, op.k1);
        A = fma(-kk.KA * pw, T, s);
    }
    // (an IEEE quotient where B is beyond the reciprocal estimate's range)
    return __double2hiint(B) < ((1023 + 1000) << 20) ? k_quot(A, B) : A / B;
}

// Q16 = 16 (a (a - b) + b^2) + 3 (C_xy^2 + C_xz^2 + C_yz^2) with a = X - Y,
// b = X - Z, as 8 G_A + 3 G_C, G_A = a^2 + b^2 + (a - b)^2 and G_C = C_xy^2 +
// C_xz^2 + C_yz^2 (16 (a^2 - a b + b^2) = 8 (2 a^2 + 2 b^2 - 2 a b)), exact in
// 128 bits and rounded once to binary64 at the scale ef.  Each difference
// (|d| < 2^61) is split into 31-bit limbs, d = dh 2^31 + dl with dl in
// [0, 2^31) and |dh| <= 2^30, so d^2 = dh^2 2^62 + dh dl 2^32 + dl^2; over a
// group of three the limb products sum exactly in 64 bits (sum dh^2 <=
// 3 2^60, |sum dh dl| < 3 2^61, sum dl^2 < 3 2^62), one 32 x 32 -> 64-bit
// multiply-add each, and the group is assembled in 128 bits once
struct Limbs {
    long long p2 = 0, p1 = 0;
    unsigned long long p0 = 0;
};
__device__ __forceinline__ void sq_acc(Limbs &g, long long d)
{
    const unsigned lo = (unsigned)d, hi = (unsigned)((unsigned long long)d >> 32);
    const int dh = (int)__funnelshift_r(lo, hi, 31);   // bits 31..62: d >> 31 for |d| < 2^62
    const int dl = (int)(lo & 0x7FFFFFFFu);
    g.p2 += (long long)dh * dh;
    g.p1 += (long long)dh * dl;
    g.p0 += (unsigned long long)(unsigned)dl * (unsigned)dl;
}
// p2 2^62 + p1 2^32 + p0 modulo 2^128 (p1 signed, the total non-negative)
__device__ __forceinline__ U128 limbs128(const Limbs &g)
{
    const U128 t1{(unsigned long long)g.p1 << 32, (unsigned long long)(g.p1 >> 32)};
    const U128 t2{(unsigned long long)g.p2 << 62, (unsigned long long)g.p2 >> 2};
    return add128(add128(U128{g.p0, 0ull}, t1), t2);
}
__device__ __forceinline__ double quad(const Sums &r, int ef)
{
    U128 GA, GC;
    {
        Limbs A;
        sq_acc(A, r.X - r.Y);
        sq_acc(A, r.X - r.Z);
        sq_acc(A, r.Z - r.Y);
        GA = limbs128(A);
    }
    {
        Limbs C;
        sq_acc(C, r.cxy);
        sq_acc(C, r.cxz);
        sq_acc(C, r.cyz);
        GC = limbs128(C);
    }
    return fx_out_q(add128(shl128(GA, 3), add128(GC, shl128(GC, 1))), ef);
}

}  // namespace bfp
}  // namespace mg
