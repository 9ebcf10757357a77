// FP64 nDGP residual passes (Sec. 3.2.1 of arXiv:2110.00566: d = L(u) - f,
// its rms and <N>) with the stencil staged once per block in shared memory
// as block fixed-point integers (bfp.cuh), for levels whose colour rows are a
// multiple of 32 long:
//   MODE 1 (restriction): the fused residual and FAS restriction (R u, R d of
//               the 8 children of every coarse cell, Eq.
//               general_pde_numerical_coarse), reducing sum N and the clamps,
//   MODE 0 (norm): the residual norm, optionally writing -d as FP32 (the
//               FP64 defect of the mixed-precision solve), reducing sum N,
//               sum d, sum d^2 and the clamps,
//   MODE 2 (coarse source): on the coarse level, the FAS right-hand side
//               f = L(R u) - (R d + dc) written in place over R d, reducing
//               sum N (the coarse level's first compatibility constant).
// Every reduction runs over the grid in a fixed order (deterministic).  Per fine cell: S6 - 6u exact in 64-bit
// integers and Q16 exact in 128 bits, each rounded once (as fixsum.cuh), N
// from the FP32 estimate with one FP64 Newton step (dgp64_N_nt) or the
// rationalised FP64 form where that is not safe; d = (S6 - 6u)/h^2 - N - f
// + cshift.
//
// Threads: a warp covers 16 split-index columns of two rows (2J, 2J + 1) of
// the tile, and each thread the two cells (one of each colour) at its row and
// split index m, which are the children of the coarse cell (J, K = m) in that
// plane; a block walks pairs of planes (2I, 2I + 1), so the 8 children of a
// coarse cell are the two planes of two partner lanes.
#include <algorithm>
#include <type_traits>

#include "bfp.cuh"
#include "cells.cuh"
#include "kernels.cuh"

namespace mg {

namespace {
constexpr int RR_TJ = 8;   // tile rows: a warp covers 16 columns of two rows

}

// MODE: above; HASF: the level has a FAS source f (every level but the
// finest; in MODE 2 f is R d, read and overwritten through FW0, FW1, and the
// shift is -dc of the fine level, scf); MODEL: 0 nDGP, 1 Kmouflage; ZERO
// (MODE 0): u is known to vanish everywhere (a solve from phi = 0), so
// nothing is staged: the stencil's sums are the zeros a staged zero field
// gives at its scale (that of 1.0), and every result is bit-identical to
// the pass over an explicit zero field
template <int MODE, bool HASF, int MODEL, bool ZERO = false>
__global__ void __launch_bounds__(bfp::THREADS, 3)
k_resid_bfp(const double *__restrict__ U0, const double *__restrict__ U1, const double *__restrict__ S0,
            const double *__restrict__ S1, const double *__restrict__ F0, const double *__restrict__ F1, LevScal *sc,
            RedBuf rb, LevK<double> L, const OpK<double> *__restrict__ opp, double *__restrict__ Uc0,
            double *__restrict__ Uc1, double *__restrict__ URc0, double *__restrict__ URc1,
            double *__restrict__ RDc0, double *__restrict__ RDc1, float *__restrict__ D0, float *__restrict__ D1,
            double *FW0, double *FW1, const LevScal *__restrict__ scf, DgpK64 dk, int zc)
{
    constexpr bool RR = MODE == 1, CS = MODE == 2;
    __shared__ bfp::Shared<RR_TJ> t;
    __shared__ double s_c[2];
    __shared__ NtK s_nk;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int jt = 2 * (warp >> 1) + (lane >> 4), mt = 16 * (warp & 1) + (lane & 15);
    const int n = L.n, half = L.half;
    const int m0 = blockIdx.x * bfp::TM, j0 = blockIdx.y * RR_TJ;
    const int i0 = blockIdx.z * zc, i1 = min(n, i0 + zc);
    if (tid == 0) {
        s_c[0] = sc->c;
        s_c[1] = CS ? -scf->dc : sc->c - sc->fshift;
        s_nk = make_ntk(*opp, dk);
    }
    // ring colour slots: 0 = the colour-0 array, 1 = the colour-1 array
    bfp::Stager<RR_TJ, bfp::TM, 6, !HASF> g(t, U0, U1, n, half, m0, j0, tid);
    static_assert(!ZERO || MODE == 0, "the zero-field variant is a norm pass");
    if (!ZERO) g.fill(i0);   // (its barriers also publish thread 0's constants above)
    else __syncthreads();
    const double c_old = s_c[0], cshift = s_c[1];
    const NtK nk = s_nk;
    const OpK<double> &op = *opp;
    const bfp::KmoK kk = MODEL == 1 ? bfp::make_kmok(op, L) : bfp::KmoK{0.0, 0.0, 0};
    const int j = j0 + jt, m = m0 + mt;
    const int jj = jt + 1, mm = mt + 1;
    double acc[3] = {0.0, 0.0, 0.0};        // sum N, sum d, sum d^2
    int nclamp = 0;                         // (counted in an integer: no FP64 add per cell)
    double su = 0.0, sd = 0.0;              // this thread's children of the coarse cell
    // the pass's constant shift h^2 cshift folded into the fixed-point
    // S6 - 6u (one FP64 add less per cell), where it fits the scale
    const double kc = cshift * L.h2;
    bool kok;
    long long kv = bfp::fold(kc, g.ef, kok);
    const long long rowo = (long long)j * half + m;
    // the cells' s and f are read a plane ahead, like the staged planes (f
    // by plain loads where this pass overwrites it: each thread reads its
    // cells' f before it writes them)
    auto ldf = [&](int c, long long r) { return CS ? (c ? FW1 : FW0)[r] : __ldg((c ? F1 : F0) + r); };
    double s_nx[2], f_nx[2] = {0.0, 0.0};
    {
        const long long r0 = (long long)i0 * g.pstride + rowo;
        s_nx[0] = __ldg(S0 + r0);
        s_nx[1] = __ldg(S1 + r0);
        if (HASF) {
            f_nx[0] = ldf(0, r0);
            f_nx[1] = ldf(1, r0);
        }
    }
    for (int i = i0, step = 0; i < i1; ++i, ++step) {
        const bool more = i + 1 < i1;
        const long long rowi = (long long)i * g.pstride + rowo;
        const double sv[2] = {s_nx[0], s_nx[1]}, fv[2] = {f_nx[0], f_nx[1]};
        if (more) {
            if (!ZERO) g.prefetch(i + 2);
            s_nx[0] = __ldg(S0 + rowi + g.pstride);
            s_nx[1] = __ldg(S1 + rowi + g.pstride);
            if (HASF) {
                f_nx[0] = ldf(0, rowi + g.pstride);
                f_nx[1] = ldf(1, rowi + g.pstride);
            }
        }
        const bool fx = fx_ok(g.ef);
        long long Usum = 0;   // the two centre values at this plane's scale (R u)
        // the plane's two cells, with the shift folded (FOLD) or added in FP64:
        // a uniform branch per plane around two straight-line copies
        auto cells = [&](auto fold_tag) {
        constexpr bool FOLD = decltype(fold_tag)::value;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int p = (c + i + j) & 1;
            const double s = sv[c];
            double N, d;
            int cl = 0;
            if (fx) {
                const bfp::Sums r = ZERO ? bfp::Sums{0, 0, 0, 0, 0, 0}
                                         : bfp::stencil<RR_TJ>(t.v[g.sm], t.v[g.s0], t.v[g.sp], c, jj, mm, p);
                const long long U = ZERO ? 0 : bfp::at<RR_TJ>(t.v[g.s0], c, jj, mm);
                Usum += U;
                const long long lap6 = (r.X + r.Y + r.Z) - ((U << 2) + (U << 1));   // |.| < 12 * 2^59
                if (MODEL == 0) {
                    N = dgp64_N_any(op, dk, nk, bfp::quad(r, g.ef), s, cl);
                } else {
                    const bfp::Diffs dd = ZERO ? bfp::Diffs{0, 0, 0}
                                               : bfp::diffs<RR_TJ>(t.v[g.sm], t.v[g.s0], t.v[g.sp], c, jj, mm, p);
                    N = bfp::kmo64_N(op, kk, r, dd, s, g.ef);
                }
                if (FOLD)
                    d = fma(L.inv_h2, fx_out(lap6 + kv, g.ef), -N);
                else
                    d = fma(L.inv_h2, fx_out(lap6, g.ef), cshift - N);
                if (HASF) d -= fv[c];
            } else {
                Nb<double> v;
                gather(v, c ? U1 : U0, c ? U0 : U1, n, half, i, j, m, p);
                const double u = __ldg((c ? U1 : U0) + rowi);
                if (RR) su += u;
                if (MODEL == 0) {
                    d = dgp64_resid(op, dk, nk, v, u, s, (HASF && !CS) ? (c ? F1 : F0) + rowi : nullptr, cshift,
                                    L.inv_h2, N, cl);
                    if (CS) d -= fv[c];
                } else {
                    N = op_N<double, 1>(op, L, v, s, cl);
                    const double S6 = (v.xp + v.xm) + (v.yp + v.ym) + (v.zp + v.zm);
                    d = (S6 - 6.0 * u) * L.inv_h2 - N + cshift;
                    if (HASF) d -= fv[c];
                }
            }
            acc[0] += N;
            nclamp += cl;
            if (RR) {
                sd += d;
            } else if (CS) {
                (c ? FW1 : FW0)[rowi] = d;
            } else {
                acc[1] += d;
                acc[2] = fma(d, d, acc[2]);
                if (D0) (c ? D1 : D0)[rowi] = (float)(-d);
            }
        }
        };
        if (fx && kok)
            cells(std::true_type{});
        else
            cells(std::false_type{});
        if (RR && fx) su += fx_out(Usum, g.ef);
        if (RR && (i & 1)) {
            // the coarse cell (I, J, K) = (i/2, j/2, m): this lane's 4 children
            // plus the partner row's
            sd += __shfl_xor_sync(0xffffffffu, sd, 16);
            su += __shfl_xor_sync(0xffffffffu, su, 16);
            if (!(lane & 16)) {
                const int nc = n / 2, halfc = nc / 2;
                const int I = i >> 1, J = j >> 1, K = m;
                const int C = (I + J + K) & 1;
                const long long cidx = ((long long)I * nc + J) * halfc + (K >> 1);
                const double Ru = su * 0.125;
                (C ? Uc1 : Uc0)[cidx] = Ru;
                (C ? URc1 : URc0)[cidx] = Ru;
                (C ? RDc1 : RDc0)[cidx] = sd * 0.125;
            }
            sd = 0.0;
            su = 0.0;
        }
        if (!more) break;
        if (!ZERO) g.advance(step, i);
        kv = bfp::fold(kc, g.ef, kok);
    }
    // the restriction and coarse-source passes reduce only sum N (and the
    // clamp count, on the integer pipe)
    constexpr int NR = (RR || CS) ? 1 : 3;
    double red[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) red[q] = acc[q];
    double tot[NR + 1];
    if (grid_sum_cnt<NR>(red, nclamp, rb, tot) && tid == 0) {
        const double cnt = (double)n * n * n;
        const double c_new = tot[0] / cnt;
        if constexpr (CS) {
            set_c_fshift(sc, c_new, c_new);
            sc->dc = 0.0;
        } else {
            const double dc = c_new - c_old;
            set_c(sc, c_new);
            sc->dc = dc;
            // (the restriction pass sums neither d nor d^2: its residual norm
            // is not used, and the norm pass gives it where it is)
            if constexpr (RR)
                sc->eps2 = __longlong_as_double(0x7FF8000000000000LL);
            else
                sc->eps2 = (tot[2] + 2.0 * dc * tot[1] + cnt * dc * dc) / cnt;
        }
        sc->sumN = tot[0];
        sc->clamps = tot[NR];
    }
}

// planes per block: an even count (a block walks whole coarse planes) that
// keeps the grid within the reduction buffer's capacity
static int bfp_planes(const LevArrays<double> &L, int cap)
{
    const long long tiles = (long long)(L.half / bfp::TM) * (L.n / RR_TJ);
    int zc = 2;
    while (zc < L.n && tiles * ((L.n + zc - 1) / zc) > cap) zc *= 2;
    return std::min(zc, L.n);
}

static bool bfp_eligible(const LevArrays<double> &L)
{
    return !L.base[0] && (L.model == 0 || L.model == 1) && L.n >= 128 && L.half % bfp::TM == 0 &&
           L.n % RR_TJ == 0;
}

bool launch_resid_restrict_bfp(const LevArrays<double> &Lf, LevArrays<double> &Lc, const OpK<double> *op,
                               const RedBuf &rb, cudaStream_t st)
{
    if (!bfp_eligible(Lf)) return false;
    const int zc = bfp_planes(Lf, rb.cap);
    const dim3 b(bfp::THREADS, 1, 1);
    const dim3 g(Lf.half / bfp::TM, Lf.n / RR_TJ, (Lf.n + zc - 1) / zc);
    if ((long long)g.x * g.y * g.z > rb.cap) return false;
#define MG_RRB(HASF, MODEL)                                                                                  \
    k_resid_bfp<1, HASF, MODEL><<<g, b, 0, st>>>(Lf.U(0), Lf.U(1), Lf.s[0], Lf.s[1], Lf.f[0], Lf.f[1], Lf.sc, rb,      \
                                             make_levk<double>(Lf.n, Lf.h), op, Lc.U(0), Lc.U(1), Lc.ur[0],      \
                                             Lc.ur[1], Lc.fbuf[0], Lc.fbuf[1], nullptr, nullptr, nullptr,       \
                                             nullptr, nullptr, make_dgpk64(Lf.h), zc)
    if (Lf.model == 0) {
        if (Lf.f[0]) MG_RRB(true, 0);
        else MG_RRB(false, 0);
    } else {
        if (Lf.f[0]) MG_RRB(true, 1);
        else MG_RRB(false, 1);
    }
#undef MG_RRB
    return true;
}

bool launch_resid_norm_bfp(const LevArrays<double> &L, const OpK<double> *op, const RedBuf &rb, cudaStream_t st,
                           float *const *D, bool zero_u)
{
    if (!bfp_eligible(L)) return false;
    const int zc = bfp_planes(L, rb.cap);
    const dim3 b(bfp::THREADS, 1, 1);
    const dim3 g(L.half / bfp::TM, L.n / RR_TJ, (L.n + zc - 1) / zc);
    if ((long long)g.x * g.y * g.z > rb.cap) return false;
#define MG_RNB(HASF, MODEL, ZERO)                                                                             \
    k_resid_bfp<0, HASF, MODEL, ZERO><<<g, b, 0, st>>>(L.U(0), L.U(1), L.s[0], L.s[1], L.f[0], L.f[1], L.sc, rb,           \
                                              make_levk<double>(L.n, L.h), op, nullptr, nullptr, nullptr, nullptr, \
                                              nullptr, nullptr, D ? D[0] : nullptr, D ? D[1] : nullptr, nullptr,  \
                                              nullptr, nullptr, make_dgpk64(L.h), zc)
    if (zero_u && !L.f[0]) {
        if (L.model == 0) MG_RNB(false, 0, true);
        else MG_RNB(false, 1, true);
    } else if (L.model == 0) {
        if (L.f[0]) MG_RNB(true, 0, false);
        else MG_RNB(false, 0, false);
    } else {
        if (L.f[0]) MG_RNB(true, 1, false);
        else MG_RNB(false, 1, false);
    }
#undef MG_RNB
    return true;
}

// the coarse level's FAS source f = L(R u) - (R d + dc) over R d in place
// (R u in Lc.ur, R d in Lc.fbuf, dc from the fine level's scalars); false
// when the coarse level is not eligible
bool launch_coarse_source_bfp(const LevArrays<double> &Lf, const LevArrays<double> &Lc, const OpK<double> *op,
                              const RedBuf &rb, cudaStream_t st)
{
    if (!bfp_eligible(Lc)) return false;
    const int zc = bfp_planes(Lc, rb.cap);
    const dim3 b(bfp::THREADS, 1, 1);
    const dim3 g(Lc.half / bfp::TM, Lc.n / RR_TJ, (Lc.n + zc - 1) / zc);
    if ((long long)g.x * g.y * g.z > rb.cap) return false;
#define MG_CSB(MODEL)                                                                                         \
    k_resid_bfp<2, true, MODEL><<<g, b, 0, st>>>(Lc.ur[0], Lc.ur[1], Lc.s[0], Lc.s[1], nullptr, nullptr, Lc.sc, rb,  \
                                                 make_levk<double>(Lc.n, Lc.h), op, nullptr, nullptr, nullptr,    \
                                                 nullptr, nullptr, nullptr, nullptr, nullptr, Lc.fbuf[0],        \
                                                 Lc.fbuf[1], Lf.sc, make_dgpk64(Lc.h), zc)
    if (Lc.model == 0) MG_CSB(0);
    else MG_CSB(1);
#undef MG_CSB
    return true;
}

}  // namespace mg
