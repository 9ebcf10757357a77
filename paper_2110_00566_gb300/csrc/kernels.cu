// Multigrid kernels of the GB300 MG-GLAM solvers (arXiv:2110.00566,
// Sec. 3.2.1 for the FAS machinery, Sec. 3.2.3 / 3.2.4 for the operators),
// one level per launch.  Colour-split layout and the neighbour gather are
// described in common.cuh, the per-cell bodies are in cells.cuh.  Every
// stencil kernel comes in a plain form (N(u)) and a correction form (CORR:
// N(b + e) - N(b) with a frozen base field b, see op_dN).
#include <algorithm>

#include "cells.cuh"
#include "kernels.cuh"

namespace mg {

namespace {

inline int np2(int x)
{
    int b = 1;
    while (b < x) b <<= 1;
    return b;
}

// 256-thread blocks over (m, j) rows of one colour array
inline dim3 block_mj(int half)
{
    const int bx = std::min(32, np2(half));
    return dim3(bx, 256 / bx, 1);
}

inline dim3 grid_mj(int half, int n, const dim3 &b, int z)
{
    return dim3((half + b.x - 1) / b.x, (n + b.y - 1) / b.y, z);
}

// z extent for reduction kernels: keep the block count within the
// reduction buffer's capacity
inline int red_z(const dim3 &g, int zmax, int cap)
{
    const long long per = (long long)g.x * g.y;
    long long z = cap / std::max<long long>(per, 1);
    return (int)std::max<long long>(1, std::min<long long>(z, zmax));
}

}  // namespace

template <typename T>
OpK<T> make_opk(int model, double alpha, int nkmo, double gamma, double bterm)
{
    OpK<T> o{};
    o.model = model;
    o.nkmo = nkmo;
    o.alpha = (T)alpha;
    o.abs_alpha = (T)(alpha < 0 ? -alpha : alpha);
    o.sgn_alpha = (T)(alpha >= 0 ? 1.0 : -1.0);
    o.alpha2 = (T)(alpha * alpha);
    o.c83 = (T)(8.0 / 3.0);
    o.a75 = (T)(0.75 * alpha);
    o.sgn75 = (T)(alpha >= 0 ? 0.75 : -0.75);
    double bp = 1.0;
    for (int q = 0; q < nkmo - 1; ++q) bp *= bterm;
    o.k1 = (T)(1.0 + gamma * bp);
    o.k2 = (T)((2.0 * nkmo + 1.0) * gamma / 3.0);
    o.k3 = (T)(2.0 * (nkmo - 1) * gamma);
    return o;
}

// per-level constants of the FP64 nDGP update and residual (the level's
// spacing only: the operator's own constants stay in device memory, so that
// captured cycle graphs remain valid when the operator changes)
template <typename T>
static DgpK64 dgp_k64(const LevArrays<T> &L)
{
    return make_dgpk64(L.h);
}

// ---------------------------------------------------------------------------
// smoother: one colour-simultaneous half-sweep (Eq. nonlinear_GS_DGP)
// ---------------------------------------------------------------------------
template <typename T, bool CORR>
__global__ void __launch_bounds__(256)
k_smooth(const T *__restrict__ Uc, const T *__restrict__ Uo, T *__restrict__ Un, const T *__restrict__ Sc,
         const T *__restrict__ Fc, const LevScal *__restrict__ sc, LevK<T> L, const OpK<T> *__restrict__ opp,
         int colour, const T *__restrict__ Bc, const T *__restrict__ Bo)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int i = blockIdx.z;
    if (m >= L.half || j >= L.n) return;
    smooth_cell<T, CORR>(*opp, L, Uc, Uo, Un, Sc, Fc, smooth_cf<T>(sc), colour, Bc, Bo, i, j, m);
}

// two cells of a colour row per thread (rows of even length)
template <typename T, bool CORR>
__global__ void __launch_bounds__(256, 3)
k_smooth2(const T *__restrict__ Uc, const T *__restrict__ Uo, T *__restrict__ Un, const T *__restrict__ Sc,
          const T *__restrict__ Fc, const LevScal *__restrict__ sc, LevK<T> L, const OpK<T> *__restrict__ opp,
          int colour, const T *__restrict__ Bc, const T *__restrict__ Bo, DgpK64 dk)
{
    // the smoother's constants, formed once per block (FP64 adds issue at a
    // small fraction of the integer rate on this GPU)
    __shared__ T cf_s;
    __shared__ NtK nk_s;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        cf_s = smooth_cf<T>(sc);
        if constexpr (sizeof(T) == 8) nk_s = make_ntk(*opp, dk);
    }
    __syncthreads();
    const int mp2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int i = blockIdx.z;
    if (2 * mp2 >= L.half || j >= L.n) return;
    smooth_pair<T, CORR>(*opp, L, Uc, Uo, Un, Sc, Fc, cf_s, nk_s, colour, Bc, Bo, i, j, 2 * mp2, dk);
}

// four cells of an FP32 colour row per thread (rows whose length is a
// multiple of 4, colour arrays below 2^31 elements); a block walks zc
// consecutive planes (z-marching: the rows of planes i and i+1 it read for
// plane i are still in L1 when it updates plane i+1)
template <bool CORR, int MODEL, bool ZM>
__global__ void __launch_bounds__(256, MODEL == 0 ? (ZM ? 3 : 4) : 2) k_smooth4(const float *__restrict__ Uc, const float *__restrict__ Uo, float *__restrict__ Un,
          const float *__restrict__ Sc, const float *__restrict__ Fc, const LevScal *__restrict__ sc, LevK<float> L,
          const OpK<float> *__restrict__ opp, int colour, const float *__restrict__ Bc, const float *__restrict__ Bo,
          int zc)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (4 * q >= L.half || j >= L.n) return;
    if (!ZM) {
        smooth_quad<CORR, MODEL>(*opp, L, Uc, Uo, Un, Sc, Fc, smooth_cf<float>(sc), colour, Bc, Bo, blockIdx.z, j,
                                 4 * q);
        return;
    }
    const int i0 = blockIdx.z * zc, i1 = min(L.n, i0 + zc);
    const float cf = smooth_cf<float>(sc);
    for (int i = i0; i < i1; ++i)
        smooth_quad<CORR, MODEL>(*opp, L, Uc, Uo, Un, Sc, Fc, cf, colour, Bc, Bo, i, j, 4 * q);
}

template <typename T>
bool launch_smooth4(const LevArrays<T> &, const LevK<T> &, const OpK<T> *, int, int, cudaStream_t)
{
    return false;
}

static bool launch_smooth4_bx(const LevArrays<float> &L, const LevK<float> &K, const OpK<float> *op, int colour,
                              int nb, int bx, int zc, cudaStream_t st)
{
    if (L.half % 4 != 0 || L.ncol >= (1LL << 31)) return false;
    zc = std::max(1, zc);
    const dim3 b = bx > 0 ? dim3(bx, 256 / bx, 1) : block_mj(L.half / 4);
    const dim3 g = grid_mj(L.half / 4, L.n, b, (L.n + zc - 1) / zc);
    const float *U0 = L.U(colour), *U1 = L.U(1 - colour);
    float *Un = L.u[nb][colour];
#define MG_SMOOTH4(CORR, MODEL)                                                                              \
    do {                                                                                                      \
        const float *b0 = CORR ? L.base[colour] : nullptr, *b1 = CORR ? L.base[1 - colour] : nullptr;        \
        if (zc > 1)                                                                                           \
            k_smooth4<CORR, MODEL, true><<<g, b, 0, st>>>(U0, U1, Un, L.s[colour], L.f[colour], L.sc, K, op,  \
                                                          colour, b0, b1, zc);                                \
        else                                                                                                  \
            k_smooth4<CORR, MODEL, false><<<g, b, 0, st>>>(U0, U1, Un, L.s[colour], L.f[colour], L.sc, K, op, \
                                                           colour, b0, b1, 1);                                \
    } while (0)
    if (L.base[0]) {
        if (L.model == 0) MG_SMOOTH4(true, 0);
        else if (L.model == 1) MG_SMOOTH4(true, 1);
        else MG_SMOOTH4(true, -1);
    } else {
        if (L.model == 0) MG_SMOOTH4(false, 0);
        else if (L.model == 1) MG_SMOOTH4(false, 1);
        else MG_SMOOTH4(false, -1);
    }
#undef MG_SMOOTH4
    return true;
}

template <>
bool launch_smooth4<float>(const LevArrays<float> &L, const LevK<float> &K, const OpK<float> *op, int colour, int nb,
                           cudaStream_t st)
{
    if (L.qstream > 0 && launch_smooth_stream(L, K, op, colour, nb, L.qstream, st)) return true;
    return launch_smooth4_bx(L, K, op, colour, nb, L.qbx, L.qz, st);
}

bool launch_smooth4_shape(const LevArrays<float> &L, const OpK<float> *op, int colour, int bx, int zc, cudaStream_t st)
{
    return launch_smooth4_bx(L, make_levk<float>(L.n, L.h), op, colour, 1 - L.cur[colour], bx, zc, st);
}

template <typename T>
void launch_smooth(const LevArrays<T> &L, LevArrays<T> *Lw, const OpK<T> *op, int colour, cudaStream_t st)
{
    const int nb = 1 - L.cur[colour];
    const LevK<T> K = make_levk<T>(L.n, L.h);
    if (launch_smooth4<T>(L, K, op, colour, nb, st)) {
        Lw->cur[colour] = nb;
        return;
    }
    if constexpr (sizeof(T) == 8) {
        if (launch_smooth_bfp(L, K, op, colour, nb, st)) {
            Lw->cur[colour] = nb;
            return;
        }
    }
    if (L.half % 2 == 0) {
        const dim3 b = block_mj(L.half / 2);
        const dim3 g = grid_mj(L.half / 2, L.n, b, L.n);
        const DgpK64 dk = dgp_k64(L);
        if (L.base[0])
            k_smooth2<T, true><<<g, b, 0, st>>>(L.U(colour), L.U(1 - colour), L.u[nb][colour], L.s[colour],
                                                L.f[colour], L.sc, K, op, colour, L.base[colour], L.base[1 - colour],
                                                dk);
        else
            k_smooth2<T, false><<<g, b, 0, st>>>(L.U(colour), L.U(1 - colour), L.u[nb][colour], L.s[colour],
                                                 L.f[colour], L.sc, K, op, colour, nullptr, nullptr, dk);
        Lw->cur[colour] = nb;
        return;
    }
    const dim3 b = block_mj(L.half);
    const dim3 g = grid_mj(L.half, L.n, b, L.n);
    if (L.base[0])
        k_smooth<T, true><<<g, b, 0, st>>>(L.U(colour), L.U(1 - colour), L.u[nb][colour], L.s[colour], L.f[colour],
                                           L.sc, K, op, colour, L.base[colour], L.base[1 - colour]);
    else
        k_smooth<T, false><<<g, b, 0, st>>>(L.U(colour), L.U(1 - colour), L.u[nb][colour], L.s[colour],
                                            L.f[colour], L.sc, K, op, colour, nullptr, nullptr);
    Lw->cur[colour] = nb;
}

// one half-sweep with an explicit block shape (bx x 256/bx) into the
// alternate buffer, leaving the buffer state untouched (for the tile-shape
// autotuner)
template <typename T>
void launch_smooth_shape(const LevArrays<T> &L, const OpK<T> *op, int colour, int bx, cudaStream_t st)
{
    const dim3 b(bx, 256 / bx, 1);
    const dim3 g = grid_mj(L.half, L.n, b, L.n);
    const int nb = 1 - L.cur[colour];
    const LevK<T> K = make_levk<T>(L.n, L.h);
    if (L.base[0])
        k_smooth<T, true><<<g, b, 0, st>>>(L.U(colour), L.U(1 - colour), L.u[nb][colour], L.s[colour], L.f[colour],
                                           L.sc, K, op, colour, L.base[colour], L.base[1 - colour]);
    else
        k_smooth<T, false><<<g, b, 0, st>>>(L.U(colour), L.U(1 - colour), L.u[nb][colour], L.s[colour],
                                            L.f[colour], L.sc, K, op, colour, nullptr, nullptr);
}

// finalise a residual pass: c_new = <N>, dc = c_new - c_old, eps^2 of the
// residual with c_new (d_true = d_old + dc)
__device__ __forceinline__ void finish_resid(LevScal *sc, const double (&tot)[4], double cnt, double c_old)
{
    const double c_new = tot[0] / cnt;
    const double dc = c_new - c_old;
    set_c(sc, c_new);
    sc->dc = dc;
    sc->eps2 = (tot[2] + 2.0 * dc * tot[1] + cnt * dc * dc) / cnt;
    sc->sumN = tot[0];
    sc->clamps = tot[3];
}

// ---------------------------------------------------------------------------
// residual norm on one level (both colours); optionally writes -d (old c)
// as FP32 for the correction solve's source
// ---------------------------------------------------------------------------
template <typename T, bool CORR, bool ZERO = false>
__global__ void __launch_bounds__(256)
k_resid_norm(const T *__restrict__ U0, const T *__restrict__ U1, const T *__restrict__ S0,
             const T *__restrict__ S1, const T *__restrict__ F0, const T *__restrict__ F1, LevScal *sc,
             RedBuf rb, LevK<T> L, const OpK<T> *__restrict__ opp, const T *__restrict__ B0,
             const T *__restrict__ B1, float *__restrict__ D0, float *__restrict__ D1, DgpK64 dk)
{
    const OpK<T> op = *opp;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const double c_old = sc->c;
    const double cshift = c_old - sc->fshift;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (m < L.half && j < L.n)
        for (int iz = blockIdx.z; iz < 2 * L.n; iz += gridDim.z)
            resid_cell<T, CORR, -1, ZERO>(op, L, U0, U1, S0, S1, F0, F1, B0, B1, D0, D1, cshift, iz & 1, iz >> 1, j,
                                          m, acc, &dk);
    double tot[4];
    if (grid_sum<4>(acc, rb, tot) && threadIdx.x == 0 && threadIdx.y == 0)
        finish_resid(sc, tot, (double)L.n * L.n * L.n, c_old);
}

template <typename T>
void launch_resid_norm(const LevArrays<T> &L, const OpK<T> *op, const RedBuf &rb, cudaStream_t st,
                       float *const *D, bool zero_u)
{
    // (a zero field takes the zero-field variants, whose norms come out
    // bit-identical to those of the same pass over an explicit zero field)
    if constexpr (sizeof(T) == 8) {
        if (launch_resid_norm_bfp(L, op, rb, st, D, zero_u)) return;
    }
    const dim3 b = block_mj(L.half);
    dim3 g = grid_mj(L.half, L.n, b, 1);
    g.z = red_z(g, 2 * L.n, rb.cap);
    const LevK<T> K = make_levk<T>(L.n, L.h);
    const DgpK64 dk = dgp_k64(L);
    float *d0 = D ? D[0] : nullptr, *d1 = D ? D[1] : nullptr;
    if (zero_u && !L.base[0])
        k_resid_norm<T, false, true><<<g, b, 0, st>>>(L.U(0), L.U(1), L.s[0], L.s[1], L.f[0], L.f[1], L.sc, rb, K,
                                                      op, nullptr, nullptr, d0, d1, dk);
    else if (L.base[0])
        k_resid_norm<T, true><<<g, b, 0, st>>>(L.U(0), L.U(1), L.s[0], L.s[1], L.f[0], L.f[1], L.sc, rb, K, op,
                                               L.base[0], L.base[1], d0, d1, dk);
    else
        k_resid_norm<T, false><<<g, b, 0, st>>>(L.U(0), L.U(1), L.s[0], L.s[1], L.f[0], L.f[1], L.sc, rb, K, op,
                                                nullptr, nullptr, d0, d1, dk);
}

// ---------------------------------------------------------------------------
// fused residual + FAS restriction, one thread per coarse cell (I, J, K)
// ---------------------------------------------------------------------------
template <typename T, bool CORR>
__global__ void __launch_bounds__(256, 2)
k_resid_restrict(const T *__restrict__ U0, const T *__restrict__ U1, const T *__restrict__ S0,
                 const T *__restrict__ S1, const T *__restrict__ F0, const T *__restrict__ F1, LevScal *sc,
                 RedBuf rb, LevK<T> L, const OpK<T> *__restrict__ opp, T *__restrict__ Uc0, T *__restrict__ Uc1,
                 T *__restrict__ URc0, T *__restrict__ URc1, T *__restrict__ RDc0, T *__restrict__ RDc1,
                 const T *__restrict__ B0, const T *__restrict__ B1, DgpK64 dk)
{
    const OpK<T> op = *opp;
    const int nc = L.n / 2;
    const int K = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const double c_old = sc->c;
    const double cshift = c_old - sc->fshift;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (K < nc && J < nc)
        for (int I = blockIdx.z; I < nc; I += gridDim.z)
            rr_cell<T, CORR>(op, L, U0, U1, S0, S1, F0, F1, B0, B1, cshift, Uc0, Uc1, URc0, URc1, RDc0, RDc1, I, J, K,
                             acc, &dk);
    double tot[4];
    if (grid_sum<4>(acc, rb, tot) && threadIdx.x == 0 && threadIdx.y == 0)
        finish_resid(sc, tot, (double)L.n * L.n * L.n, c_old);
}

// four coarse cells per thread (FP32, coarse rows a multiple of 4 long)
template <bool CORR, int MODEL>
__global__ void __launch_bounds__(256, 2) k_resid_restrict4(const float *__restrict__ U0, const float *__restrict__ U1, const float *__restrict__ S0,
                  const float *__restrict__ S1, const float *__restrict__ F0, const float *__restrict__ F1,
                  LevScal *sc, RedBuf rb, LevK<float> L, const OpK<float> *__restrict__ opp, float *__restrict__ Uc0,
                  float *__restrict__ Uc1, float *__restrict__ URc0, float *__restrict__ URc1,
                  float *__restrict__ RDc0, float *__restrict__ RDc1, const float *__restrict__ B0,
                  const float *__restrict__ B1)
{
    const OpK<float> op = *opp;
    const int nc = L.n / 2;
    const int K4 = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const double c_old = sc->c;
    const double cshift = c_old - sc->fshift;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    // a block walks a contiguous run of coarse planes, so that the fine
    // planes shared by consecutive coarse planes are still in L1
    const int chunk = (nc + gridDim.z - 1) / gridDim.z;
    const int I0 = blockIdx.z * chunk, I1 = min(nc, I0 + chunk);
    if (4 * K4 < nc && J < nc)
        for (int I = I0; I < I1; ++I)
            rr_quad<CORR, MODEL>(op, L, U0, U1, S0, S1, F0, F1, B0, B1, cshift, Uc0, Uc1, URc0, URc1, RDc0, RDc1, I,
                                 J, 4 * K4, acc);
    double tot[4];
    if (grid_sum<4>(acc, rb, tot) && threadIdx.x == 0 && threadIdx.y == 0)
        finish_resid(sc, tot, (double)L.n * L.n * L.n, c_old);
}

template <typename T>
bool launch_resid_restrict4(const LevArrays<T> &, LevArrays<T> &, const OpK<T> *, const RedBuf &, cudaStream_t)
{
    return false;
}

template <>
bool launch_resid_restrict4<float>(const LevArrays<float> &Lf, LevArrays<float> &Lc, const OpK<float> *op,
                                   const RedBuf &rb, cudaStream_t st)
{
    const int nc = Lf.n / 2;
    if (nc % 4 != 0 || Lf.ncol >= (1LL << 31)) return false;
    const dim3 b = block_mj(nc / 4);
    dim3 g = grid_mj(nc / 4, nc, b, 1);
    g.z = red_z(g, nc, rb.cap);
    const LevK<float> K = make_levk<float>(Lf.n, Lf.h);
#define MG_RR4(CORR, MODEL)                                                                                       \
    k_resid_restrict4<CORR, MODEL><<<g, b, 0, st>>>(Lf.U(0), Lf.U(1), Lf.s[0], Lf.s[1], Lf.f[0], Lf.f[1], Lf.sc, rb, \
                                                    K, op, Lc.U(0), Lc.U(1), Lc.ur[0], Lc.ur[1], Lc.fbuf[0],      \
                                                    Lc.fbuf[1], CORR ? Lf.base[0] : nullptr,                      \
                                                    CORR ? Lf.base[1] : nullptr)
    if (Lf.base[0]) {
        if (Lf.model == 0) MG_RR4(true, 0);
        else if (Lf.model == 1) MG_RR4(true, 1);
        else MG_RR4(true, -1);
    } else {
        if (Lf.model == 0) MG_RR4(false, 0);
        else if (Lf.model == 1) MG_RR4(false, 1);
        else MG_RR4(false, -1);
    }
#undef MG_RR4
    return true;
}

template <typename T>
void launch_resid_restrict(const LevArrays<T> &Lf, LevArrays<T> &Lc, const OpK<T> *op, const RedBuf &rb,
                           cudaStream_t st)
{
    if constexpr (sizeof(T) == 8) {
        if (launch_resid_restrict_bfp(Lf, Lc, op, rb, st)) return;
    }
    if (launch_resid_restrict4<T>(Lf, Lc, op, rb, st)) return;
    const int nc = Lf.n / 2;
    const dim3 b = block_mj(nc);
    dim3 g = grid_mj(nc, nc, b, 1);
    g.z = red_z(g, nc, rb.cap);
    const LevK<T> K = make_levk<T>(Lf.n, Lf.h);
    const DgpK64 dk = dgp_k64(Lf);
    if (Lf.base[0])
        k_resid_restrict<T, true><<<g, b, 0, st>>>(Lf.U(0), Lf.U(1), Lf.s[0], Lf.s[1], Lf.f[0], Lf.f[1], Lf.sc, rb,
                                                   K, op, Lc.U(0), Lc.U(1), Lc.ur[0], Lc.ur[1], Lc.fbuf[0],
                                                   Lc.fbuf[1], Lf.base[0], Lf.base[1], dk);
    else
        k_resid_restrict<T, false><<<g, b, 0, st>>>(Lf.U(0), Lf.U(1), Lf.s[0], Lf.s[1], Lf.f[0], Lf.f[1], Lf.sc,
                                                    rb, K, op, Lc.U(0), Lc.U(1), Lc.ur[0], Lc.ur[1], Lc.fbuf[0],
                                                    Lc.fbuf[1], nullptr, nullptr, dk);
}

// ---------------------------------------------------------------------------
// coarse FAS source (Eq. general_pde_numerical_coarse), in place over R d;
// finalises c = fshift = <N(Ru)>
// ---------------------------------------------------------------------------
template <typename T, bool CORR>
__global__ void __launch_bounds__(256)
k_coarse_source(const T *__restrict__ UR0, const T *__restrict__ UR1, const T *__restrict__ S0,
                const T *__restrict__ S1, T *F0, T *F1, const LevScal *scf, LevScal *scc, RedBuf rb, LevK<T> L,
                const OpK<T> *__restrict__ opp, const T *__restrict__ B0, const T *__restrict__ B1, DgpK64 dk)
{
    const OpK<T> op = *opp;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const T dcf = (T)scf->dc;
    CsAcc<T> ca;
    if (m < L.half && j < L.n)
        for (int iz = blockIdx.z; iz < 2 * L.n; iz += gridDim.z)
            cs_cell<T, CORR>(op, L, UR0, UR1, S0, S1, F0, F1, B0, B1, dcf, iz & 1, iz >> 1, j, m, ca, &dk);
    double acc[2] = {ca.sum(), (double)ca.cl};
    double tot[2];
    if (grid_sum<2>(acc, rb, tot) && threadIdx.x == 0 && threadIdx.y == 0) {
        const double c = tot[0] / ((double)L.n * L.n * L.n);
        set_c_fshift(scc, c, c);
        scc->dc = 0.0;
        scc->sumN = tot[0];
        scc->clamps = tot[1];
    }
}

template <typename T>
void launch_coarse_source(const LevArrays<T> &Lf, const LevArrays<T> &Lc, const OpK<T> *op, const RedBuf &rb,
                          cudaStream_t st)
{
    if constexpr (sizeof(T) == 8)
        if (launch_coarse_source_bfp(Lf, Lc, op, rb, st)) return;
    const dim3 b = block_mj(Lc.half);
    dim3 g = grid_mj(Lc.half, Lc.n, b, 1);
    g.z = red_z(g, 2 * Lc.n, rb.cap);
    const LevK<T> K = make_levk<T>(Lc.n, Lc.h);
    const DgpK64 dk = dgp_k64(Lc);
    if (Lc.base[0])
        k_coarse_source<T, true><<<g, b, 0, st>>>(Lc.ur[0], Lc.ur[1], Lc.s[0], Lc.s[1], Lc.fbuf[0], Lc.fbuf[1], Lf.sc,
                                                  Lc.sc, rb, K, op, Lc.base[0], Lc.base[1], dk);
    else
        k_coarse_source<T, false><<<g, b, 0, st>>>(Lc.ur[0], Lc.ur[1], Lc.s[0], Lc.s[1], Lc.fbuf[0], Lc.fbuf[1],
                                                   Lf.sc, Lc.sc, rb, K, op, nullptr, nullptr, dk);
}

// ---------------------------------------------------------------------------
// prolongation + correction (Eq. solution_correction)
// ---------------------------------------------------------------------------
// e = u^H - R u^h on the coarse level, in place in the R u buffer: the cycle
// reads that buffer again only after the next restriction has refilled it
template <typename T>
__global__ void __launch_bounds__(256)
k_coarse_e(const T *__restrict__ UH0, const T *__restrict__ UH1, T *RH0, T *RH1, long long ncol)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncol;
         q += (long long)gridDim.x * blockDim.x) {
        RH0[q] = UH0[q] - RH0[q];
        RH1[q] = UH1[q] - RH1[q];
    }
}

// four fine cells per thread (FP32, fine rows a multiple of 4 long)
__global__ void __launch_bounds__(256)
k_prolong4(float *U0, float *U1, const float *__restrict__ UH0, const float *__restrict__ UH1,
           const float *__restrict__ RH0, const float *__restrict__ RH1, int n)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int iz = blockIdx.z;
    if (4 * q >= n / 2 || j >= n) return;
    // the coarse arrays RH hold e = u^H - R u^h (formed by k_coarse_e)
    prolong_quad<true>(U0, U1, RH0, RH1, nullptr, nullptr, n, iz & 1, iz >> 1, j, 4 * q);
}

template <typename T>
bool launch_prolong4(const LevArrays<T> &, const LevArrays<T> &, cudaStream_t)
{
    return false;
}

template <>
bool launch_prolong4<float>(const LevArrays<float> &Lf, const LevArrays<float> &Lc, cudaStream_t st)
{
    if (Lf.half % 4 != 0 || Lf.ncol >= (1LL << 31)) return false;
    const dim3 b = block_mj(Lf.half / 4);
    const dim3 g = grid_mj(Lf.half / 4, Lf.n, b, 2 * Lf.n);
    const long long nc = Lc.ncol;
    const int eb = (int)std::min<long long>((nc + 255) / 256, 152LL * 16);
    k_coarse_e<float><<<eb, 256, 0, st>>>(Lc.U(0), Lc.U(1), Lc.ur[0], Lc.ur[1], nc);
    k_prolong4<<<g, b, 0, st>>>(Lf.U(0), Lf.U(1), Lc.U(0), Lc.U(1), Lc.ur[0], Lc.ur[1], Lf.n);
    return true;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_prolong_e(T *U0, T *U1, const T *__restrict__ E0, const T *__restrict__ E1, int n)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int iz = blockIdx.z;
    if (m >= n / 2 || j >= n) return;
    prolong_cell_e<T>(U0, U1, E0, E1, n, iz & 1, iz >> 1, j, m);
}

template <typename T>
int prolong_kernels(const LevArrays<T> &)
{
    return 2;   // the coarse correction, then the prolongation
}

template <typename T>
void launch_prolong(const LevArrays<T> &Lf, const LevArrays<T> &Lc, cudaStream_t st)
{
    if (launch_prolong4<T>(Lf, Lc, st)) return;
    const long long nc = Lc.ncol;
    const int eb = (int)std::min<long long>((nc + 255) / 256, 152LL * 16);
    k_coarse_e<T><<<eb, 256, 0, st>>>(Lc.U(0), Lc.U(1), Lc.ur[0], Lc.ur[1], nc);
    if constexpr (sizeof(T) == 8) {
        if (launch_prolong_bfp(Lf, Lc, st)) return;
    }
    const dim3 b = block_mj(Lf.half);
    const dim3 g = grid_mj(Lf.half, Lf.n, b, 2 * Lf.n);
    k_prolong_e<T><<<g, b, 0, st>>>(Lf.U(0), Lf.U(1), Lc.ur[0], Lc.ur[1], Lf.n);
}

// ---------------------------------------------------------------------------
// coarsest level: one CTA, FP64 in shared memory
// ---------------------------------------------------------------------------
template <typename T, bool CORR>
__global__ void __launch_bounds__(512)
k_coarsest(T *U0, T *U1, const T *S0, const T *S1, const T *F0, const T *F1, LevScal *sc, int n, double h,
           const OpK<double> *__restrict__ opp, int sweeps, const T *B0, const T *B1)
{
    extern __shared__ double smem[];
    coarsest_block<T, CORR>(U0, U1, S0, S1, F0, F1, sc, n, h, *opp, sweeps, B0, B1, smem);
}

template <typename T>
void launch_coarsest(const LevArrays<T> &L, const OpK<double> *op, int sweeps, cudaStream_t st)
{
    const int n3 = L.n * L.n * L.n;
    const int threads = n3 <= 256 ? 256 : 512;
    const size_t sm = sizeof(double) * 5 * n3;
    if (L.base[0])
        k_coarsest<T, true><<<1, threads, sm, st>>>(L.U(0), L.U(1), L.s[0], L.s[1], L.f[0], L.f[1], L.sc, L.n, L.h,
                                                    op, sweeps, L.base[0], L.base[1]);
    else
        k_coarsest<T, false><<<1, threads, sm, st>>>(L.U(0), L.U(1), L.s[0], L.s[1], L.f[0], L.f[1], L.sc, L.n, L.h,
                                                     op, sweeps, nullptr, nullptr);
}

// ---------------------------------------------------------------------------
// plain restriction of a colour-split field (density and base pyramids)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_restrict_plain(const T *__restrict__ F0, const T *__restrict__ F1, T *__restrict__ C0, T *__restrict__ C1, int nf)
{
    const int nc = nf / 2;
    const int K = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    if (K >= nc || J >= nc) return;
    restrict_cell<T>(F0, F1, C0, C1, nf, blockIdx.z, J, K);
}

template <typename T>
void launch_restrict_plain(T *const fine[2], int nf, T *const coarse[2], cudaStream_t st)
{
    const int nc = nf / 2;
    const dim3 b = block_mj(nc);
    const dim3 g = grid_mj(nc, nc, b, nc);
    k_restrict_plain<T><<<g, b, 0, st>>>(fine[0], fine[1], coarse[0], coarse[1], nf);
}

// ---------------------------------------------------------------------------
// layout conversion, means, element-wise helpers
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_split(const double *__restrict__ nat, int n, T *__restrict__ D0, T *__restrict__ D1, double scale,
        const double *__restrict__ mean)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int i = blockIdx.z;
    if (k >= n || j >= n) return;
    const double mu = mean ? *mean : 0.0;
    const double x = nat[((long long)i * n + j) * n + k];
    const long long si = row_of(i, j, n, n / 2) + (k >> 1);
    (((i + j + k) & 1) ? D1 : D0)[si] = (T)(scale * (x - mu));
}

template <typename T>
void launch_split(const double *nat, int n, T *const dst[2], double scale, const double *mean, cudaStream_t st)
{
    const dim3 b = block_mj(n);
    const dim3 g = grid_mj(n, n, b, n);
    k_split<T><<<g, b, 0, st>>>(nat, n, dst[0], dst[1], scale, mean);
}

template <typename T>
__global__ void __launch_bounds__(256)
k_merge(const T *__restrict__ A0, const T *__restrict__ A1, int n, double *__restrict__ nat,
        const double *__restrict__ mean)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int i = blockIdx.z;
    if (k >= n || j >= n) return;
    const double mu = mean ? *mean : 0.0;
    const long long si = row_of(i, j, n, n / 2) + (k >> 1);
    nat[((long long)i * n + j) * n + k] = (double)(((i + j + k) & 1) ? A1 : A0)[si] - mu;
}

template <typename T>
void launch_merge(T *const src[2], int n, double *nat, const double *mean, cudaStream_t st)
{
    const dim3 b = block_mj(n);
    const dim3 g = grid_mj(n, n, b, n);
    k_merge<T><<<g, b, 0, st>>>(src[0], src[1], n, nat, mean);
}

__global__ void __launch_bounds__(256)
k_mean_nat(const double *__restrict__ x, long long cnt, double *out, RedBuf rb)
{
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) acc[0] += x[q];
    double tot[1];
    if (grid_sum<1>(acc, rb, tot) && threadIdx.x == 0) *out = tot[0] / (double)cnt;
}

void launch_mean_nat(const double *x, long long cnt, double *out_mean, const RedBuf &rb, cudaStream_t st)
{
    const long long nb = std::min<long long>(MAX_RED_BLOCKS / 4, (cnt + 255) / 256);
    k_mean_nat<<<(int)std::max<long long>(1, nb), 256, 0, st>>>(x, cnt, out_mean, rb);
}

__global__ void __launch_bounds__(256)
k_rms_nat(const double *__restrict__ x, long long cnt, double scale, const double *__restrict__ mean, double *out,
          RedBuf rb)
{
    double acc[1] = {0.0};
    const double mu = mean ? *mean : 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) {
        const double y = scale * (x[q] - mu);
        acc[0] += y * y;
    }
    double tot[1];
    if (grid_sum<1>(acc, rb, tot) && threadIdx.x == 0) *out = sqrt(tot[0] / (double)cnt);
}

void launch_rms_nat(const double *x, long long cnt, double scale, const double *mean, double *out, const RedBuf &rb,
                    cudaStream_t st)
{
    const long long nb = std::min<long long>(MAX_RED_BLOCKS / 4, (cnt + 255) / 256);
    k_rms_nat<<<(int)std::max<long long>(1, nb), 256, 0, st>>>(x, cnt, scale, mean, out, rb);
}

template <typename T>
__global__ void __launch_bounds__(256)
k_mean_split(const T *__restrict__ A0, const T *__restrict__ A1, long long ncol, double *out, RedBuf rb)
{
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncol; q += stride)
        acc[0] += (double)A0[q] + (double)A1[q];
    double tot[1];
    if (grid_sum<1>(acc, rb, tot) && threadIdx.x == 0) *out = tot[0] / (2.0 * (double)ncol);
}

template <typename T>
void launch_mean_split(T *const a[2], long long ncol, double *out_mean, const RedBuf &rb, cudaStream_t st)
{
    const long long nb = std::min<long long>(MAX_RED_BLOCKS / 4, (ncol + 255) / 256);
    k_mean_split<T><<<(int)std::max<long long>(1, nb), 256, 0, st>>>(a[0], a[1], ncol, out_mean, rb);
}

template <typename Td, typename Ts>
__global__ void __launch_bounds__(256) k_convert(Td *D0, Td *D1, const Ts *S0, const Ts *S1, long long ncol)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncol; q += stride) {
        D0[q] = (Td)S0[q];
        D1[q] = (Td)S1[q];
    }
}

template <typename Td, typename Ts>
void launch_convert(Td *const dst[2], Ts *const src[2], long long ncol, cudaStream_t st)
{
    const long long nb = std::min<long long>(152 * 16, (ncol + 255) / 256);
    k_convert<Td, Ts><<<(int)std::max<long long>(1, nb), 256, 0, st>>>(dst[0], dst[1], src[0], src[1], ncol);
}

__global__ void __launch_bounds__(256)
k_add_correction(double *U0, double *U1, const float *__restrict__ E0, const float *__restrict__ E1, long long ncol)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncol; q += stride) {
        U0[q] += (double)E0[q];
        U1[q] += (double)E1[q];
    }
}

void launch_add_correction(double *const U[2], float *const E[2], long long ncol, cudaStream_t st)
{
    const long long nb = std::min<long long>(152 * 16, (ncol + 255) / 256);
    k_add_correction<<<(int)std::max<long long>(1, nb), 256, 0, st>>>(U[0], U[1], E[0], E[1], ncol);
}

__global__ void k_set_corr_scalars(LevScal *sc32, const LevScal *__restrict__ sc64, int nlev)
{
    const int l = threadIdx.x;
    if (l >= nlev) return;
    LevScal z{};
    if (l == 0) {
        z.fshift = -sc64->dc;
        z.cf32 = (float)z.fshift;
    }
    sc32[l] = z;
}

void launch_set_corr_scalars(LevScal *sc32, const LevScal *sc64, int nlev32, cudaStream_t st)
{
    k_set_corr_scalars<<<1, 32, 0, st>>>(sc32, sc64, nlev32);
}

// ---------------------------------------------------------------------------
// explicit instantiations
// ---------------------------------------------------------------------------
#define INST(T)                                                                                              \
    template OpK<T> make_opk<T>(int, double, int, double, double);                                         \
    template void launch_smooth<T>(const LevArrays<T> &, LevArrays<T> *, const OpK<T> *, int, cudaStream_t); \
    template void launch_smooth_shape<T>(const LevArrays<T> &, const OpK<T> *, int, int, cudaStream_t);      \
    template void launch_resid_norm<T>(const LevArrays<T> &, const OpK<T> *, const RedBuf &, cudaStream_t,   \
                                       float *const *, bool);                                               \
    template void launch_resid_restrict<T>(const LevArrays<T> &, LevArrays<T> &, const OpK<T> *,              \
                                           const RedBuf &, cudaStream_t);                                   \
    template void launch_coarse_source<T>(const LevArrays<T> &, const LevArrays<T> &, const OpK<T> *,         \
                                          const RedBuf &, cudaStream_t);                                    \
    template void launch_prolong<T>(const LevArrays<T> &, const LevArrays<T> &, cudaStream_t);               \
    template int prolong_kernels<T>(const LevArrays<T> &);                                                  \
    template void launch_coarsest<T>(const LevArrays<T> &, const OpK<double> *, int, cudaStream_t);          \
    template void launch_restrict_plain<T>(T *const[2], int, T *const[2], cudaStream_t);                     \
    template void launch_split<T>(const double *, int, T *const[2], double, const double *, cudaStream_t);   \
    template void launch_merge<T>(T *const[2], int, double *, const double *, cudaStream_t);                 \
    template void launch_mean_split<T>(T *const[2], long long, double *, const RedBuf &, cudaStream_t);
INST(double)
INST(float)
#undef INST
template void launch_convert<float, double>(float *const[2], double *const[2], long long, cudaStream_t);
template void launch_convert<double, float>(double *const[2], float *const[2], long long, cudaStream_t);

}  // namespace mg
