// FP64 nDGP red-black half-sweep (Eq. nonlinear_GS_DGP of arXiv:2110.00566,
// Sec. 3.2.3) with the stencil's values staged once per block in shared
// memory as block fixed-point integers (bfp.cuh): the signed sums of the
// 19-point stencil and the quadratic form Q16 exact in 64- and 128-bit
// integers, each result rounded once to binary64, as in fixsum.cuh, but with
// one conversion per staged value (2.7 per updated cell) instead of one per
// use (15.5 per cell when every thread converts its own stencil).  N(Sigma)
// comes from the FP32 estimate with one FP64 Newton step (dgp64_N_nt), and
// from the rationalised FP64 form where that is not safe.
#include <algorithm>

#include "bfp.cuh"
#include "cells.cuh"
#include "kernels.cuh"

namespace mg {

__global__ void __launch_bounds__(bfp::THREADS, 2)
k_smooth_bfp(const double *__restrict__ Uc, const double *__restrict__ Uo, double *__restrict__ Un,
             const double *__restrict__ Sc, const double *__restrict__ Fc, const LevScal *__restrict__ sc,
             LevK<double> L, const OpK<double> *__restrict__ opp, int colour, DgpK64 dk, int zc)
{
    __shared__ bfp::Shared t;
    __shared__ double s_cf;
    __shared__ NtK s_nk;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * bfp::TM + tx;
    const int n = L.n, half = L.half;
    const int m0 = blockIdx.x * bfp::TM, j0 = blockIdx.y * bfp::TJ;
    const int i0 = blockIdx.z * zc, i1 = min(n, i0 + zc);
    if (tid == 0) {
        s_cf = smooth_cf<double>(sc);
        s_nk = make_ntk(*opp, dk);
    }
    // ring colour slot 0: the updated colour's array, 1: the other's
    bfp::Stager g(t, Uc, Uo, n, half, m0, j0, tid);
    g.fill(i0);
    const double cf = s_cf;
    const NtK nk = s_nk;
    const OpK<double> &op = *opp;
    const int j = j0 + ty, m = m0 + tx;
    const int jj = ty + 1, mm = tx + 1;
    const long long rowo = (long long)j * half + m;
    // the cell's s and f are read a plane ahead, like the staged planes
    double s_nx = __ldg(Sc + (long long)i0 * g.pstride + rowo);
    double f_nx = Fc ? __ldg(Fc + (long long)i0 * g.pstride + rowo) : 0.0;
    for (int i = i0, step = 0; i < i1; ++i, ++step) {
        const bool more = i + 1 < i1;
        const long long idx = (long long)i * g.pstride + rowo;
        const double s = s_nx, fcf = Fc ? cf + f_nx : cf;
        if (more) {
            g.prefetch(i + 2);   // the next plane, in flight during the update
            s_nx = __ldg(Sc + idx + g.pstride);
            if (Fc) f_nx = __ldg(Fc + idx + g.pstride);
        }
        const int p = (colour + i + j) & 1;
        double out;
        if (fx_ok(g.ef)) {
            const bfp::Sums r = bfp::stencil(t.v[g.sm], t.v[g.s0], t.v[g.sp], 0, jj, mm, p);
            const double q = bfp::quad(r, g.ef);
            const double s6d = fx_out(fx_div6(r.X + r.Y + r.Z), g.ef);
            int cl = 0;
            out = dgp64_finish(op, dk, nk, q, s, s6d, fcf, cl);
        } else {
            Nb<double> v;
            gather(v, Uc, Uo, n, half, i, j, m, p);
            int cl = 0;
            out = dgp64_update(op, dk, nk, v, s, fcf, cl);
        }
        Un[idx] = out;
        if (!more) break;
        g.advance(step);   // plane i + 2 into the slot of plane i - 1
    }
}

// the block-fixed-point half-sweep for levels with half % 32 == 0 and
// n % 8 == 0 (n >= 64); false otherwise
bool launch_smooth_bfp(const LevArrays<double> &L, const LevK<double> &K, const OpK<double> *op, int colour, int nb,
                       cudaStream_t st)
{
    if (L.base[0] || L.model != 0 || L.half % bfp::TM != 0 || L.n % bfp::TJ != 0) return false;
    const int zc = L.n >= 256 ? 16 : 8;
    const dim3 b(bfp::TM, bfp::TJ, 1);
    const dim3 g(L.half / bfp::TM, L.n / bfp::TJ, (L.n + zc - 1) / zc);
    k_smooth_bfp<<<g, b, 0, st>>>(L.U(colour), L.U(1 - colour), L.u[nb][colour], L.s[colour], L.f[colour], L.sc, K,
                                  op, colour, make_dgpk64(L.h), zc);
    return true;
}

}  // namespace mg
