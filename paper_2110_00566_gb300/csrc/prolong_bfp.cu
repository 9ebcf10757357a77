// FP64 prolongation and correction (Sec. 3.2.1 of arXiv:2110.00566:
// u^h += P(u^H - R u^h), the 27/9/3/1 over 64 trilinear weights) with the
// coarse correction staged once per block in shared memory as block fixed
// point (bfp.cuh), for fine levels of 128^3 and more whose rows are a
// multiple of 64 long.
//
// A block owns a fine tile of 32 split-index columns by 16 rows (both
// colours: 64 cells per row; each thread rows ty and ty + 8) and walks pairs
// of fine planes (2I, 2I + 1); every fine cell of the tile draws on the
// coarse cells of split columns m0/2 - 1 .. m0/2 + 16 and rows j0/2 - 1 ..
// j0/2 + 8 of coarse planes I - 1, I, I + 1, which a ring of three coarse
// planes holds, converted once each (0.2 conversions per fine cell, against
// 8 when every thread converts its own eight coarse values).  The weighted
// sum 27 e000 + 9 (faces) + 3 (edges) + e111 is exact in fixed point with 3
// guard bits (the weights sum to 64, |V| < 2^56), divided by 64 in the
// conversion back and rounded once, as in the per-cell kernel; one FP64 add
// per fine cell.  A thread reads its eight fine values of a coarse plane
// before it writes any (the two colour arrays are distinct), so that the
// eight loads are in flight together.
#include <algorithm>

#include "bfp.cuh"
#include "cells.cuh"
#include "kernels.cuh"

namespace mg {

namespace {
constexpr int PF_TJ = 16;                 // fine rows per tile
constexpr int PC_TJ = PF_TJ / 2;          // coarse rows per tile
constexpr int PC_TM = bfp::TM / 2;        // coarse split columns per tile

// the weighted sum in FP64 where the staged planes' scale is outside the
// fixed-point domain (rare)
__device__ __forceinline__ double prolong_fp64(const double *__restrict__ E0, const double *__restrict__ E1, int I,
                                            int I2, int J, int J2, int K, int K2, int nc, int halfc)
{
    const int Iw = I2 < 0 ? I2 + nc : (I2 >= nc ? I2 - nc : I2);
    const int Jw = J2 < 0 ? J2 + nc : (J2 >= nc ? J2 - nc : J2);
    const int Kw = K2 < 0 ? K2 + nc : (K2 >= nc ? K2 - nc : K2);
    const double e000 = coarse_v(E0, E1, I, J, K, nc, halfc), e100 = coarse_v(E0, E1, Iw, J, K, nc, halfc);
    const double e010 = coarse_v(E0, E1, I, Jw, K, nc, halfc), e001 = coarse_v(E0, E1, I, J, Kw, nc, halfc);
    const double e110 = coarse_v(E0, E1, Iw, Jw, K, nc, halfc), e101 = coarse_v(E0, E1, Iw, J, Kw, nc, halfc);
    const double e011 = coarse_v(E0, E1, I, Jw, Kw, nc, halfc), e111 = coarse_v(E0, E1, Iw, Jw, Kw, nc, halfc);
    const double s1 = (e100 + e010) + e001, s2 = (e110 + e101) + e011;
    return fma(27.0 / 64.0, e000, fma(9.0 / 64.0, s1, fma(3.0 / 64.0, s2, (1.0 / 64.0) * e111)));
}

// this thread's fine cells of coarse plane I by prolong_fp64
__device__ __noinline__ void prolong_plane_fp64(double *__restrict__ U0, double *__restrict__ U1,
                                                const double *__restrict__ E0, const double *__restrict__ E1, int n,
                                                int I, int jt, int m)
{
    const int half = n / 2, nc = n / 2, halfc = nc / 2;
    for (int a = 0; a < 2; ++a) {
        const int i = 2 * I + a, I2 = a ? I + 1 : I - 1;
        for (int h = 0; h < PF_TJ / 8; ++h) {
            const int j = jt + 8 * h, J = j >> 1, J2 = (j & 1) ? J + 1 : J - 1;
            const long long row = ((long long)i * n + j) * half + m;
            for (int c = 0; c < 2; ++c) {
                const int p = (c + i + j) & 1, K2 = p ? m + 1 : m - 1;
                double *Ua = c ? U1 : U0;
                Ua[row] += prolong_fp64(E0, E1, I, I2, J, J2, m, K2, nc, halfc);
            }
        }
    }
}
}

__global__ void __launch_bounds__(bfp::THREADS, 3)
k_prolong_bfp(double *__restrict__ U0, double *__restrict__ U1, const double *__restrict__ E0,
              const double *__restrict__ E1, int n, int zc)
{
    constexpr int H = PF_TJ / 8;   // fine rows per thread
    __shared__ bfp::Shared<PC_TJ, PC_TM> t;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * bfp::TM + tx;
    const int half = n / 2, nc = n / 2, halfc = nc / 2;
    const int m0 = blockIdx.x * bfp::TM, j0 = blockIdx.y * PF_TJ;
    const int I0 = blockIdx.z * zc, I1 = min(nc, I0 + zc);   // coarse planes of this block
    const int m0c = m0 / 2, J0 = j0 / 2;
    bfp::Stager<PC_TJ, PC_TM, 3> g(t, E0, E1, nc, halfc, m0c, J0, tid);
    g.fill(I0);
    const int m = m0 + tx;
    const long long pstride = (long long)n * half;
    // planes whose staged scale is outside the fixed-point domain (uniform
    // over the block, rare): their cells get the FP64 sum after the walk, out
    // of line, so that neither its registers nor a call count against the
    // staged path (zc <= 16 planes per block)
    unsigned fp64_planes = 0;
    for (int I = I0, step = 0; I < I1; ++I, ++step) {
        const bool more = I + 1 < I1;
        if (more) g.prefetch(I + 2);
        const bool fx = g.ef >= (64 << 20) && g.ef < (2047 << 20);
        // the thread's fine values of this coarse plane: [fine plane][row][colour]
        double uv[2][H][2];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const long long row = (long long)(2 * I + a) * pstride + (long long)(j0 + ty + 8 * h) * half + m;
                uv[a][h][0] = U0[row];
                uv[a][h][1] = U1[row];
            }
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int i = 2 * I + a;
            const int I2 = a ? I + 1 : I - 1;
            // ring slots of coarse planes I and I2
            const long long *P0 = t.v[g.s0], *P2 = t.v[a ? g.sp : g.sm];
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const int j = j0 + ty + 8 * h;
                const int J = j >> 1, J2 = (j & 1) ? J + 1 : J - 1;   // unwrapped: the tile's halo rows hold the wrap
                const int jjJ = J - J0 + 1, jjJ2 = J2 - J0 + 1;
                const long long row = (long long)i * pstride + (long long)j * half + m;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int p = (c + i + j) & 1;
                    const int K = m, K2 = p ? K + 1 : K - 1;     // k = 2m + p: K = m
                    double corr;
                    // (a branch per cell, not a select: it keeps the compiler from
                    // interleaving all eight cells' shared-memory loads, which
                    // spills at 80 registers)
                    if (fx) {
                        // coarse (Ic, Jc, Kc) lives in colour (Ic + Jc + Kc) & 1 at split
                        // column Kc >> 1 (arithmetic: Kc = -1 is the wrapped column)
                        auto cv = [&](const long long *P, int Ic, int Jc, int jj, int Kc) {
                            return bfp::at<PC_TJ, PC_TM>(P, (Ic + Jc + Kc) & 1, jj, (Kc >> 1) - m0c + 1);
                        };
                        const long long v000 = cv(P0, I, J, jjJ, K), v100 = cv(P2, I2, J, jjJ, K);
                        const long long v010 = cv(P0, I, J2, jjJ2, K), v001 = cv(P0, I, J, jjJ, K2);
                        const long long v110 = cv(P2, I2, J2, jjJ2, K), v101 = cv(P2, I2, J, jjJ, K2);
                        const long long v011 = cv(P0, I, J2, jjJ2, K2), v111 = cv(P2, I2, J2, jjJ2, K2);
                        const long long Wsum =
                            27 * v000 + 9 * ((v100 + v010) + v001) + 3 * ((v110 + v101) + v011) + v111;
                        corr = fx_out<9>(Wsum, g.ef);
                    } else {
                        corr = 0.0;   // added after the walk
                    }
                    (c ? U1 : U0)[row] = uv[a][h][c] + corr;
                }
            }
        }
        if (!fx) fp64_planes |= 1u << step;
        if (!more) break;
        g.advance(step, I);
    }
    for (int q = 0; fp64_planes; ++q, fp64_planes >>= 1)
        if (fp64_planes & 1u) prolong_plane_fp64(U0, U1, E0, E1, n, I0 + q, j0 + ty, m);
}

// false where the fine level is not eligible (FP64 plain form, n >= 128,
// fine rows a multiple of 64 long, n % 16 == 0)
bool launch_prolong_bfp(const LevArrays<double> &Lf, const LevArrays<double> &Lc, cudaStream_t st)
{
    if (Lf.n < 128 || Lf.half % (2 * bfp::TM) != 0 || Lf.n % PF_TJ != 0) return false;
    const int nc = Lf.n / 2;
    const long long tiles = (long long)(Lf.half / bfp::TM) * (Lf.n / PF_TJ);
    int zc = 16;   // at most 16 (the kernel's plane mask)
    while (zc > 1 && tiles * ((nc + zc - 1) / zc) < 600) zc /= 2;
    const dim3 b(bfp::TM, bfp::THREADS / bfp::TM, 1);
    const dim3 g(Lf.half / bfp::TM, Lf.n / PF_TJ, (nc + zc - 1) / zc);
    k_prolong_bfp<<<g, b, 0, st>>>(Lf.U(0), Lf.U(1), Lc.ur[0], Lc.ur[1], Lf.n, zc);
    return true;
}

}  // namespace mg
