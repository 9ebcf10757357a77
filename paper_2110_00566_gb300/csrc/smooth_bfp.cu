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

namespace {
constexpr int SM_TJ = 16;   // tile rows: each thread updates rows ty and ty + 8

// the update where the level's constant does not fit the block's scale
// (rare), out of line so that the compiler does not predicate it into every
// cell
__device__ __noinline__ double smooth_unfolded(double mh6, double N, double fcf, long long s6, int ef)
{
    return fma(mh6, N + fcf, fx_out(s6, ef));
}
}

// HASF: the level has a FAS source f (every level but the finest); MODEL:
// 0 nDGP (Eq. nonlinear_GS_DGP), 1 Kmouflage (the same update with N_K)
template <bool HASF, int MODEL>
__global__ void __launch_bounds__(bfp::THREADS, 4)
k_smooth_bfp(const double *__restrict__ Uc, const double *__restrict__ Uo, double *__restrict__ Un,
             const double *__restrict__ Sc, const double *__restrict__ Fc, const LevScal *__restrict__ sc,
             LevK<double> L, const OpK<double> *__restrict__ opp, int colour, DgpK64 dk, int zc)
{
    __shared__ bfp::Shared<SM_TJ> t;
    __shared__ double s_cf;
    __shared__ NtK s_nk;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * bfp::TM + tx;
    const int n = L.n, half = L.half;
    const int m0 = blockIdx.x * bfp::TM, j0 = blockIdx.y * SM_TJ;
    const int i0 = blockIdx.z * zc, i1 = min(n, i0 + zc);
    if (tid == 0) {
        s_cf = smooth_cf<double>(sc);
        s_nk = make_ntk(*opp, dk);
    }
    // ring colour slot 0: the updated colour's array, 1: the other's (the
    // finest level's nDGP half-sweep stages by 32-bit funnel shifts where it
    // can: 1 % faster at 512^3 and 256^3; no gain on the other variants)
    bfp::Stager<SM_TJ, bfp::TM, 6, !HASF && MODEL == 0> g(t, Uc, Uo, n, half, m0, j0, tid);
    g.fill(i0);
    const double cf = s_cf;
    const NtK nk = s_nk;
    const OpK<double> &op = *opp;
    const bfp::KmoK kk = MODEL == 1 ? bfp::make_kmok(op, L) : bfp::KmoK{0.0, 0.0, 0};
    // where the level has no FAS source, the update's constant -h^2 cf / 6 is
    // folded into the fixed-point S6 / 6 (one FP64 add less per cell)
    const double kc = dk.mh6 * cf;
    bool kok;
    long long kv = bfp::fold(kc, g.ef, kok);
    bool fold = !HASF && kok;
    const int m = m0 + tx, mm = tx + 1;
    const long long rowo = (long long)(j0 + ty) * half + m, rows8 = 8LL * half;
    // each cell's s and f are read a plane ahead, like the staged planes
    double s_nx[2], f_nx[2] = {0.0, 0.0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        s_nx[h] = __ldg(Sc + (long long)i0 * g.pstride + rowo + h * rows8);
        if (HASF) f_nx[h] = __ldg(Fc + (long long)i0 * g.pstride + rowo + h * rows8);
    }
    for (int i = i0, step = 0; i < i1; ++i, ++step) {
        const bool more = i + 1 < i1;
        const long long base = (long long)i * g.pstride + rowo;
        const double sv[2] = {s_nx[0], s_nx[1]}, fv[2] = {f_nx[0], f_nx[1]};
        if (more) {
            g.prefetch(i + 2);   // the next plane, in flight during the update
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                s_nx[h] = __ldg(Sc + base + g.pstride + h * rows8);
                if (HASF) f_nx[h] = __ldg(Fc + base + g.pstride + h * rows8);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + ty + 8 * h, jj = ty + 8 * h + 1;
            const int p = (colour + i + j) & 1;
            const double fcf = HASF ? cf + fv[h] : cf;
            double out;
            int cl = 0;
            if (fx_ok(g.ef)) {
                const bfp::Sums r = bfp::stencil<SM_TJ>(t.v[g.sm], t.v[g.s0], t.v[g.sp], 0, jj, mm, p);
                const long long s6 = fx_div6(r.X + r.Y + r.Z);
                double N;
                if (MODEL == 0) {
                    N = dgp64_N_any(op, dk, nk, bfp::quad(r, g.ef), sv[h], cl);
                } else {
                    const bfp::Diffs dd = bfp::diffs<SM_TJ>(t.v[g.sm], t.v[g.s0], t.v[g.sp], 0, jj, mm, p);
                    N = bfp::kmo64_N(op, kk, r, dd, sv[h], g.ef);
                }
                if (HASF)
                    out = fma(dk.mh6, N + fcf, fx_out(s6, g.ef));
                else if (fold)
                    out = fma(dk.mh6, N, fx_out(s6 + kv, g.ef));
                else
                    out = smooth_unfolded(dk.mh6, N, fcf, s6, g.ef);
            } else {
                Nb<double> v;
                gather(v, Uc, Uo, n, half, i, j, m, p);
                if (MODEL == 0) {
                    out = dgp64_update(op, dk, nk, v, sv[h], fcf, cl);
                } else {
                    const double N = op_N<double, 1>(op, L, v, sv[h], cl);
                    const double S6 = (v.xp + v.xm) + (v.yp + v.ym) + (v.zp + v.zm);
                    out = (S6 - L.h2 * (N + fcf)) * (1.0 / 6.0);
                }
            }
            Un[base + h * rows8] = out;
        }
        if (!more) break;
        g.advance(step, i);   // plane i + 2 into the slot of plane i - 1
        kv = bfp::fold(kc, g.ef, kok);
        fold = !HASF && kok;
    }
}

// the block-fixed-point half-sweep for levels of 128^3 and more with
// half % 32 == 0 and n % 16 == 0; false otherwise (coarser levels have too
// few tiles to fill the GPU with marching blocks); planes per block: 16,
// halved (down to 2) while that leaves under about 4 waves of 4 blocks per
// SM (measured at 256^3: 4 planes 0.184 ms, 16 planes 0.193 ms, the last
// wave of 1024 blocks two-thirds full)
bool launch_smooth_bfp(const LevArrays<double> &L, const LevK<double> &K, const OpK<double> *op, int colour, int nb,
                       cudaStream_t st)
{
    if (L.base[0] || (L.model != 0 && L.model != 1) || L.n < 128 || L.half % bfp::TM != 0 || L.n % SM_TJ != 0)
        return false;
    const long long tiles = (long long)(L.half / bfp::TM) * (L.n / SM_TJ);
    int zc = 16;
    while (zc > 2 && tiles * ((L.n + zc - 1) / zc) < 2400) zc /= 2;
    const dim3 b(bfp::TM, bfp::THREADS / bfp::TM, 1);
    const dim3 g(L.half / bfp::TM, L.n / SM_TJ, (L.n + zc - 1) / zc);
#define MG_SBF(HASF, MODEL)                                                                                    \
    k_smooth_bfp<HASF, MODEL><<<g, b, 0, st>>>(L.U(colour), L.U(1 - colour), L.u[nb][colour], L.s[colour],         \
                                               L.f[colour], L.sc, K, op, colour, make_dgpk64(L.h), zc)
    if (L.model == 0) {
        if (L.f[colour]) MG_SBF(true, 0);
        else MG_SBF(false, 0);
    } else {
        if (L.f[colour]) MG_SBF(true, 1);
        else MG_SBF(false, 1);
    }
#undef MG_SBF
    return true;
}

}  // namespace mg
