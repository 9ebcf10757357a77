// Particle-mesh pieces of the GB300 MG-GLAM library (Sec. 3.1 of
// arXiv:2110.00566): cloud-in-cell assignment with deterministic fixed-point
// accumulation, and the CIC index used by it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include <cufft.h>

#include "ctx.cuh"
#include "fixsum.cuh"

namespace mg {

// CIC lower cell and weights along one axis: lo = floor(x - 1/2) in FP32
// (the positions are FP32), upper weight dx = x - 1/2 - lo taken exactly in
// FP64.  Positions outside [0, ng) wrap periodically.
__device__ __forceinline__ void cic_axis(float x, int ng, int &i0, int &i1, double &w0, double &w1)
{
    const float t = __fsub_rn(x, 0.5f);
    const int lo = (int)floorf(t);
    const double dx = (double)x - 0.5 - (double)lo;
    int a = lo % ng;
    if (a < 0) a += ng;
    i0 = a;
    i1 = (a + 1 == ng) ? 0 : a + 1;
    w0 = 1.0 - dx;
    w1 = dx;
}

__global__ void __launch_bounds__(256)
k_cic_deposit(const float *__restrict__ pos, long long np, int ng, unsigned long long *__restrict__ acc)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += stride) {
        int i0[3], i1[3];
        double w0[3], w1[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) cic_axis(__ldg(pos + 3 * p + d), ng, i0[d], i1[d], w0[d], w1[d]);
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const double w = __dmul_rn(__dmul_rn(a ? w1[0] : w0[0], b ? w1[1] : w0[1]), c ? w1[2] : w0[2]);
                    const unsigned long long q = (unsigned long long)llrint(w * 4294967296.0);
                    const long long cell = ((long long)(a ? i1[0] : i0[0]) * ng + (b ? i1[1] : i0[1])) * ng +
                                           (c ? i1[2] : i0[2]);
                    atomicAdd(acc + cell, q);
                }
    }
}

__global__ void __launch_bounds__(256)
k_cic_finish(const unsigned long long *__restrict__ acc, long long cnt, double mass, double *__restrict__ delta)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride)
        delta[q] = mass * ((double)acc[q] * (1.0 / 4294967296.0)) - 1.0;
}

__global__ void __launch_bounds__(256)
k_sub_mean(double *__restrict__ x, long long cnt, const double *__restrict__ mean)
{
    const double mu = *mean;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) x[q] -= mu;
}

__global__ void __launch_bounds__(256) k_cic_index(const float *__restrict__ pos, long long np, int ng, int *idx)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 3 * np; q += stride) {
        int i0, i1;
        double w0, w1;
        cic_axis(__ldg(pos + q), ng, i0, i1, w0, w1);
        idx[q] = i0;
    }
}

static int grid1(long long n) { return (int)std::max<long long>(1, std::min<long long>(152 * 16, (n + 255) / 256)); }

struct PmWork {
    unsigned long long *acc = nullptr;
    size_t acc_bytes = 0;
    // Poisson solve for one mesh size: FP32 transforms (r32 -> spec -> r32)
    // inside an FP64 iterative refinement
    int fft_n = 0;
    cufftHandle fwd = 0, inv = 0;
    double *rho = nullptr, *phin = nullptr, *phi = nullptr;
    double *pot = nullptr, *g3 = nullptr;   // the force's potential and -grad of it (3 components)
    float *r32 = nullptr, *table = nullptr;
    cufftComplex *spec = nullptr;
};

// 4 sin^2(pi k / n): minus the eigenvalues of the 1D 3-point Laplacian
__global__ void k_lap_table(float *t, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        const double s = sinpi((double)k / (double)n);
        t[k] = (float)(4.0 * s * s);
    }
}

// Green's function of the 7-point Laplacian on the rfft grid (n, n, n/2+1),
// FP32: Phi_k = scale * rho_k / (-(t[i] + t[j] + t[kz])), zero mode set to 0
__global__ void __launch_bounds__(256)
k_green(cufftComplex *spec, int n, const float *__restrict__ t, float scale)
{
    const int nz = n / 2 + 1;
    const long long total = (long long)n * n * nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += stride) {
        int i, j, kz;
        split3(q, n, nz, i, j, kz);
        cufftComplex v = spec[q];
        const float f = q == 0 ? 0.f : -scale / ((t[i] + t[j]) + t[kz]);
        v.x *= f;
        v.y *= f;
        spec[q] = v;
    }
}

// FP32 copy of coef (rhs - <rhs>), the first right-hand side of the
// refinement (the mean, which the zero mode drops, is taken out before the
// rounding to FP32, so that it cannot swamp the rest)
__global__ void __launch_bounds__(256)
k_rhs32(const double *__restrict__ rhs, const double *__restrict__ mean, double coef, float *__restrict__ r32,
        long long cnt)
{
    const double mu = *mean;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride)
        r32[q] = (float)(coef * (rhs[q] - mu));
}

// u = e (first pass) or u += e, FP64
__global__ void __launch_bounds__(256)
k_add_corr(double *__restrict__ u, const float *__restrict__ e, long long cnt, int first)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride)
        u[q] = first ? (double)e[q] : u[q] + (double)e[q];
}

// the FP64 residual of Lap u = coef (rhs - <rhs>) with the 7-point
// Laplacian (h = 1, periodic), R = coef (rhs - <rhs>) - (sum of the 6
// neighbours - 6 u), written as FP32: the right-hand side of the next
// correction; the Laplacian exact in 64-bit integers
__global__ void __launch_bounds__(256)
k_poisson_resid(const double *__restrict__ u, const double *__restrict__ rhs, const double *__restrict__ mean,
                double coef, float *__restrict__ r32, int n)
{
    const double mu = *mean;
    const long long cnt = (long long)n * n * n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) {
        int i, j, k;
        split3(q, n, n, i, j, k);
        const long long pl = (long long)n * n;
        const long long qip = i + 1 == n ? q - (n - 1) * pl : q + pl, qim = i == 0 ? q + (n - 1) * pl : q - pl;
        const long long qjp = j + 1 == n ? q - (long long)(n - 1) * n : q + n,
                        qjm = j == 0 ? q + (long long)(n - 1) * n : q - n;
        const long long qkp = k + 1 == n ? q - (n - 1) : q + 1, qkm = k == 0 ? q + (n - 1) : q - 1;
        const double v[7] = {u[q], u[qip], u[qim], u[qjp], u[qjm], u[qkp], u[qkm]};
        // Lap u = S6 - 6 u exactly on the integer pipes at the scale of the
        // stencil's largest value (fixsum.cuh: the FP64 pipe is this GPU's
        // narrowest), rounded once; FP64 outside the fixed-point domain
        int ef = 0;
#pragma unroll
        for (int t = 0; t < 7; ++t) ef = max(ef, fx_ef(v[t]));
        ef = fx_zero_scale(ef);
        double lap;
        if (fx_ok(ef)) {
            long long S = -6 * fx_in(v[0], ef);
#pragma unroll
            for (int t = 1; t < 7; ++t) S += fx_in(v[t], ef);
            lap = fx_out(S, ef);
        } else {
            lap = fma(-6.0, v[0], ((v[1] + v[2]) + (v[3] + v[4])) + (v[5] + v[6]));
        }
        r32[q] = (float)fma(coef, rhs[q] - mu, -lap);
    }
}

// the potential of the force at cell q: A + cb Bp (Bp given), rounded as
// written (no contraction)
__device__ __forceinline__ double pot(const double *__restrict__ A, const double *__restrict__ Bp, double cb,
                                      long long q)
{
    const double a = __ldg(A + q);
    return Bp ? __dadd_rn(a, __dmul_rn(cb, __ldg(Bp + q))) : a;
}

// the potential Phi = PhiN + cphi phi (phi given) on the mesh, rounded as
// the per-corner evaluation of the force would round it
__global__ void __launch_bounds__(256)
k_pot(const double *__restrict__ phin, const double *__restrict__ phi, double cphi, double *__restrict__ out,
      long long cnt)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride)
        out[q] = pot(phin, phi, cphi, q);
}

// twice -grad Phi by 3-point differences on the mesh, 2 g_c = Phi(-e_c) -
// Phi(+e_c): the per-corner force's -(Phi(+e_c) - Phi(-e_c)) / 2 without the
// halving, which the kick applies to its factor instead (a power of two
// commutes with every rounding, so the interpolated force is bit-identical
// to evaluating it at the corners)
__global__ void __launch_bounds__(256)
k_force_mesh(const double *__restrict__ P, double *__restrict__ gx, double *__restrict__ gy, double *__restrict__ gz,
             int n)
{
    const long long cnt = (long long)n * n * n, pl = (long long)n * n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) {
        int i, j, k;
        split3(q, n, n, i, j, k);
        const long long qip = i + 1 == n ? q - (n - 1) * pl : q + pl, qim = i == 0 ? q + (n - 1) * pl : q - pl;
        const long long qjp = j + 1 == n ? q - (long long)(n - 1) * n : q + n,
                        qjm = j == 0 ? q + (long long)(n - 1) * n : q - n;
        const long long qkp = k + 1 == n ? q - (n - 1) : q + 1, qkm = k == 0 ? q + (n - 1) : q - 1;
        gx[q] = __dsub_rn(__ldg(P + qim), __ldg(P + qip));
        gy[q] = __dsub_rn(__ldg(P + qjm), __ldg(P + qjp));
        gz[q] = __dsub_rn(__ldg(P + qkm), __ldg(P + qkp));
    }
}

// the force at each particle interpolated from the mesh force with the CIC
// weights, then the leapfrog kick and drift (code units of Sec. 3.1.1):
//   p = p fr + g ck,  x += p cd,  wrap into [0, ng)  (g2 = 2 g from the
// mesh, ck2 = ck / 2: g2 ck2 = g ck exactly).  Phi = PhiN + cphi phi
// when phi is given (nDGP: cphi = 1/2, Eq. poisson_nDGP; Kmouflage: cphi =
// beta c~, Eq. force_Kmo2, whose friction term gives fr = 1 - beta
// (dphibar/da) da_kick; fr = 1 otherwise).  Rounded as written (no
// contraction); the weight of corner (a, b, c) is (w_a w_b) w_c, with w_a w_b
// formed once per (a, b)
__global__ void __launch_bounds__(256)
k_kick_drift(float *__restrict__ pos, float *__restrict__ mom, long long np, int ng, const double *__restrict__ gx,
             const double *__restrict__ gy, const double *__restrict__ gz, double fr, double ck2, double cd)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += stride) {
        int i0[3], i1[3];
        double w0[3], w1[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) cic_axis(pos[3 * p + d], ng, i0[d], i1[d], w0[d], w1[d]);
        double g[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const double wab = __dmul_rn(a ? w1[0] : w0[0], b ? w1[1] : w0[1]);
                const long long rab = ((long long)(a ? i1[0] : i0[0]) * ng + (b ? i1[1] : i0[1])) * ng;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const double w = __dmul_rn(wab, c ? w1[2] : w0[2]);
                    const long long q = rab + (c ? i1[2] : i0[2]);
                    g[0] = __dadd_rn(g[0], __dmul_rn(w, __ldg(gx + q)));
                    g[1] = __dadd_rn(g[1], __dmul_rn(w, __ldg(gy + q)));
                    g[2] = __dadd_rn(g[2], __dmul_rn(w, __ldg(gz + q)));
                }
            }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float pn = (float)__dadd_rn(__dmul_rn((double)mom[3 * p + d], fr), __dmul_rn(g[d], ck2));
            mom[3 * p + d] = pn;
            float x = (float)__dadd_rn((double)pos[3 * p + d], __dmul_rn((double)pn, cd));
            if (x < 0.f) x = __fadd_rn(x, (float)ng);
            if (x >= (float)ng) x = __fsub_rn(x, (float)ng);
            pos[3 * p + d] = x;
        }
    }
}

static PmWork &pmw(mg_ctx *ctx)
{
    if (!ctx->pm) ctx->pm = new PmWork();
    return *ctx->pm;
}

#define MG_CUFFT(call)                                                                               \
    do {                                                                                              \
        cufftResult r_ = (call);                                                                      \
        if (r_ != CUFFT_SUCCESS) {                                                                    \
            set_err(ctx, MG_ERR_CUDA, "cuFFT error %d in %s at %s:%d", (int)r_, #call, __FILE__, __LINE__); \
            throw CudaFail{MG_ERR_CUDA};                                                              \
        }                                                                                             \
    } while (0)

static void pm_release_fft(PmWork &w)
{
    if (w.fwd) cufftDestroy(w.fwd);
    if (w.inv) cufftDestroy(w.inv);
    w.fwd = w.inv = 0;
    for (double *p : {w.rho, w.phin, w.phi, w.pot, w.g3})
        if (p) cudaFree(p);
    for (float *p : {w.r32, w.table})
        if (p) cudaFree(p);
    if (w.spec) cudaFree(w.spec);
    w.rho = w.phin = w.phi = w.pot = w.g3 = nullptr;
    w.r32 = w.table = nullptr;
    w.spec = nullptr;
    w.fft_n = 0;
}

void pm_fft_setup(mg_ctx *ctx, int n)
{
    PmWork &w = pmw(ctx);
    if (w.fft_n == n) return;
    MG_CK(cudaStreamSynchronize(ctx->stream));
    pm_release_fft(w);
    const size_t cells = (size_t)n * n * n, modes = (size_t)n * n * (n / 2 + 1);
    MG_CK(cudaMalloc(&w.rho, sizeof(double) * cells));
    MG_CK(cudaMalloc(&w.phin, sizeof(double) * cells));
    MG_CK(cudaMalloc(&w.phi, sizeof(double) * cells));
    MG_CK(cudaMalloc(&w.pot, sizeof(double) * cells));
    MG_CK(cudaMalloc(&w.g3, sizeof(double) * 3 * cells));
    MG_CK(cudaMalloc(&w.r32, sizeof(float) * cells));
    MG_CK(cudaMalloc(&w.table, sizeof(float) * n));
    MG_CK(cudaMalloc(&w.spec, sizeof(cufftComplex) * modes));
    MG_CUFFT(cufftPlan3d(&w.fwd, n, n, n, CUFFT_R2C));
    MG_CUFFT(cufftPlan3d(&w.inv, n, n, n, CUFFT_C2R));
    MG_CUFFT(cufftSetStream(w.fwd, ctx->stream));
    MG_CUFFT(cufftSetStream(w.inv, ctx->stream));
    k_lap_table<<<(n + 127) / 128, 128, 0, ctx->stream>>>(w.table, n);
    MG_CK(cudaGetLastError());
    MG_CK(cudaMemsetAsync(w.phi, 0, sizeof(double) * cells, ctx->stream));
    w.fft_n = n;
}

// Lap out = coef rhs with the 7-point Green's function by FFT (Sec. 3.1);
// the zero mode is dropped (so the mean of rhs is ignored).  FP64 transforms
// run at the FP64 rate on this GPU, so the solve is FP32 transforms inside
// an FP64 iterative refinement: out = G (coef rhs) in FP32, then twice
// R = coef rhs - Lap out in FP64 and out += G R in FP32; each correction
// carries about 2^-22 of its own size, so two corrections bring out to the
// FP64 solution (relative 1e-15 in L2, measured against FP64 transforms).
// The mean of rhs (the zero mode, which the Green's function drops) is taken
// out in FP64 before any rounding to FP32, and the FP32 transforms leave a
// mean of about 1e-9 of |out| behind, removed at the end (the zero mode of
// the FP64 solution is zero)
void poisson_dev(mg_ctx *ctx, int n, double coef, const double *rhs, double *out)
{
    PmWork &w = pmw(ctx);
    cudaStream_t st = ctx->stream;
    const long long cnt = (long long)n * n * n, modes = (long long)n * n * (n / 2 + 1);
    const float scale = (float)(1.0 / (double)cnt);
    constexpr int CORRECTIONS = 2;
    double *mean_rhs = ctx->dscratch + 1, *mean_out = ctx->dscratch + 2;
    launch_mean_nat(rhs, cnt, mean_rhs, ctx->rb, st);
    k_rhs32<<<grid1(cnt), 256, 0, st>>>(rhs, mean_rhs, coef, w.r32, cnt);
    for (int it = 0; it <= CORRECTIONS; ++it) {
        MG_CUFFT(cufftExecR2C(w.fwd, w.r32, w.spec));
        k_green<<<grid1(modes), 256, 0, st>>>(w.spec, n, w.table, scale);
        MG_CK(cudaGetLastError());
        MG_CUFFT(cufftExecC2R(w.inv, w.spec, w.r32));
        k_add_corr<<<grid1(cnt), 256, 0, st>>>(out, w.r32, cnt, it == 0);
        if (it < CORRECTIONS) k_poisson_resid<<<grid1(cnt), 256, 0, st>>>(out, rhs, mean_rhs, coef, w.r32, n);
        MG_CK(cudaGetLastError());
    }
    launch_mean_nat(out, cnt, mean_out, ctx->rb, st);
    k_sub_mean<<<grid1(cnt), 256, 0, st>>>(out, cnt, mean_out);
    MG_CK(cudaGetLastError());
}

// Lap Phi = (3/2) Omega_m a^-1 delta (Eq. GR_poisson_codeunit)
void newton_potential_dev(mg_ctx *ctx, int n, double a, double om, const double *delta, double *out)
{
    poisson_dev(ctx, n, 1.5 * om / a, delta, out);
}

static double E_lcdm(double a, double om) { return std::sqrt(om * std::pow(a, -3.0) + (1.0 - om)); }

// deposit on device pointers
void cic_deposit_dev(mg_ctx *ctx, int ng, const float *pos, long long np, double *delta)
{
    PmWork &w = pmw(ctx);
    const long long cnt = (long long)ng * ng * ng;
    const size_t bytes = sizeof(unsigned long long) * (size_t)cnt;
    if (w.acc_bytes < bytes) {
        if (w.acc) MG_CK(cudaFree(w.acc));
        w.acc = nullptr;
        w.acc_bytes = 0;
        MG_CK(cudaMalloc(&w.acc, bytes));
        w.acc_bytes = bytes;
    }
    cudaStream_t st = ctx->stream;
    MG_CK(cudaMemsetAsync(w.acc, 0, bytes, st));
    k_cic_deposit<<<grid1(np), 256, 0, st>>>(pos, np, ng, w.acc);
    const double mass = (double)cnt / (double)np;
    k_cic_finish<<<grid1(cnt), 256, 0, st>>>(w.acc, cnt, mass, delta);
    launch_mean_nat(delta, cnt, ctx->dscratch, ctx->rb, st);
    k_sub_mean<<<grid1(cnt), 256, 0, st>>>(delta, cnt, ctx->dscratch);
    MG_CK(cudaGetLastError());
}

}  // namespace mg

using namespace mg;

extern "C" {

void mg_pm_free(mg_ctx *ctx)
{
    if (!ctx || !ctx->pm) return;
    if (ctx->pm->acc) cudaFree(ctx->pm->acc);
    pm_release_fft(*ctx->pm);
    delete ctx->pm;
    ctx->pm = nullptr;
}

int pm_cic_deposit(mg_ctx *ctx, int ng, const float *pos, long long np, double *delta_out)
{
    if (!ctx) return MG_ERR_ARG;
    if (!pos || !delta_out || np < 1 || ng < 2) return set_err(ctx, MG_ERR_ARG, "bad pm_cic_deposit arguments");
    try {
        enter(ctx);
        const size_t pb = sizeof(float) * 3 * (size_t)np, db = sizeof(double) * (size_t)ng * ng * ng;
        const float *dp = (const float *)stage_in(ctx, 0, pos, pb, true);
        double *dd = (double *)stage_in(ctx, 1, delta_out, db, false);
        cic_deposit_dev(ctx, ng, dp, np, dd);
        stage_out(ctx, delta_out, dd, db);
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

int pm_cic_index(mg_ctx *ctx, int ng, const float *pos, long long np, int *idx_out)
{
    if (!ctx) return MG_ERR_ARG;
    if (!pos || !idx_out || np < 1 || ng < 2) return set_err(ctx, MG_ERR_ARG, "bad pm_cic_index arguments");
    try {
        enter(ctx);
        const size_t pb = sizeof(float) * 3 * (size_t)np, ib = sizeof(int) * 3 * (size_t)np;
        const float *dp = (const float *)stage_in(ctx, 0, pos, pb, true);
        int *di = (int *)stage_in(ctx, 1, idx_out, ib, false);
        k_cic_index<<<grid1(3 * np), 256, 0, ctx->stream>>>(dp, np, ng, di);
        MG_CK(cudaGetLastError());
        stage_out(ctx, idx_out, di, ib);
        MG_CK(cudaStreamSynchronize(ctx->stream));
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

int mg_solve_kmouflage_linear(mg_ctx *ctx, const mg_grid *g, const mg_kmo_params *p, const double *delta,
                              double *phi)
{
    if (!ctx) return MG_ERR_ARG;
    if (!g || !p || !delta || !phi) return set_err(ctx, MG_ERR_ARG, "null argument");
    if (g->ng < 2 || g->ng % 2 || p->n < 2 || p->k0 < 0 || !(g->a > 0) || !(g->box_mpch > 0) || !(p->lambda > 0))
        return set_err(ctx, MG_ERR_ARG, "bad Kmouflage parameters");
    try {
        enter(ctx);
        const int n = g->ng;
        const double a = g->a;
        double gam = p->n * p->k0, bp = 1.0;
        for (int q = 0; q < p->n - 1; ++q) {
            gam *= 1.0 / (2.0 * a * a * p->lambda * p->lambda);
            bp *= p->phibar_prime_over_h0 * p->phibar_prime_over_h0;
        }
        const double ct = 2997.92458 * n / g->box_mpch;   // c~ = (c/H0) N / L
        const double coef = 3.0 * p->beta_kmo * p->A_bar * g->omega_m / a / ct / (1.0 + gam * bp);
        const size_t b = sizeof(double) * (size_t)n * n * n;
        const double *dd = (const double *)stage_in(ctx, 0, delta, b, true);
        double *dp = (double *)stage_in(ctx, 1, phi, b, false);
        pm_fft_setup(ctx, n);
        poisson_dev(ctx, n, coef, dd, dp);
        stage_out(ctx, phi, dp, b);
        MG_CK(cudaStreamSynchronize(ctx->stream));
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

int pm_newton_potential(mg_ctx *ctx, int ng, double a, double omega_m, const double *delta, double *phi_out)
{
    if (!ctx) return MG_ERR_ARG;
    if (!delta || !phi_out || ng < 2 || ng % 2 || !(a > 0))
        return set_err(ctx, MG_ERR_ARG, "bad pm_newton_potential arguments");
    try {
        enter(ctx);
        const size_t b = sizeof(double) * (size_t)ng * ng * ng;
        const double *dd = (const double *)stage_in(ctx, 0, delta, b, true);
        double *dp = (double *)stage_in(ctx, 1, phi_out, b, false);
        pm_fft_setup(ctx, ng);
        newton_potential_dev(ctx, ng, a, omega_m, dd, dp);
        stage_out(ctx, phi_out, dp, b);
        MG_CK(cudaStreamSynchronize(ctx->stream));
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

int pm_step(mg_ctx *ctx, pm_state *st, const mg_opts *opts, mg_stats *stats)
{
    if (!ctx) return MG_ERR_ARG;
    if (!st || !st->pos || !st->mom || st->np < 1) return set_err(ctx, MG_ERR_ARG, "bad pm_state");
    if (st->model < 0 || st->model > 2)
        return set_err(ctx, MG_ERR_ARG, "model must be 0 (GR), 1 (nDGP) or 2 (Kmouflage)");
    if (st->model >= 1 ? !valid_ng(st->ng) : (st->ng < 2 || st->ng % 2))
        return set_err(ctx, MG_ERR_ARG, "ng = %d not supported", st->ng);
    if (!(st->a > 0) || !(st->da > 0) || !(st->omega_m > 0) || (st->model == 1 && !(st->dgp.rc_h0 > 0)))
        return set_err(ctx, MG_ERR_ARG, "a, da, omega_m (and rc_h0) must be > 0");
    if (st->model == 2 && (st->kmo.n < 2 || st->kmo.k0 < 0 || !(st->kmo.lambda > 0) || !(st->kmo.A_bar > 0) ||
                           !(st->box_mpch > 0)))
        return set_err(ctx, MG_ERR_ARG, "bad Kmouflage parameters");
    if (!(st->e_a >= 0.0) || !(st->e_mid >= 0.0) || !std::isfinite(st->e_a) || !std::isfinite(st->e_mid))
        return set_err(ctx, MG_ERR_ARG, "e_a, e_mid must be finite and >= 0");
    mg_opts o;
    if (opts)
        o = *opts;
    else
        mg_opts_default(&o);
    int rc = check_opts(ctx, o);
    if (rc) return rc;
    mg_stats loc{};
    try {
        enter(ctx);
        const int n = st->ng;
        const size_t pb = sizeof(float) * 3 * (size_t)st->np, cb = sizeof(double) * (size_t)n * n * n;
        float *dpos = (float *)stage_in(ctx, 0, st->pos, pb, true);
        float *dmom = (float *)stage_in(ctx, 1, st->mom, pb, true);
        pm_fft_setup(ctx, n);
        PmWork &w = pmw(ctx);
        cic_deposit_dev(ctx, n, dpos, st->np, w.rho);
        // Kmouflage: Lap Phi_N = (3/2) A Omega_m a^-1 delta (Eq. kmf_Poission_eqn_codeunit)
        const double Af = st->model == 2 ? st->kmo.A_bar : 1.0;
        newton_potential_dev(ctx, n, st->a, st->omega_m * Af, w.rho, w.phin);
        const double *dphi = nullptr;
        double cphi = 0.5, fr = 1.0;
        if (st->model >= 1) {
            double *phib = w.phi;
            if (st->phi_ws) {
                phib = (double *)stage_in(ctx, 2, st->phi_ws, cb, true);
                o.warm_start = 1;
            } else {
                o.warm_start = 0;
            }
            if (st->model == 1) {
                rc = solve_dgp_dev(ctx, n, st->a, st->omega_m, st->dgp.rc_h0, w.rho, phib, o, &loc);
            } else {
                const mg_grid g{n, st->box_mpch, st->a, st->omega_m};
                rc = solve_kmo_dev(ctx, g, st->kmo, w.rho, phib, o, &loc);
                cphi = st->kmo.beta_kmo * 2997.92458 * n / st->box_mpch;   // beta c~
                fr = 1.0 - st->kmo.beta_kmo * st->dphibar_da * (st->first ? 0.5 * st->da : st->da);
            }
            if (rc < 0) {
                leave(ctx);
                if (stats) *stats = loc;
                return rc;
            }
            dphi = phib;
            if (st->phi_ws) stage_out(ctx, st->phi_ws, phib, cb);
        }
        const double a = st->a, da = st->da, om = st->omega_m;
        const double dak = st->first ? 0.5 * da : da;
        const double am = a + 0.5 * da;
        const bool own_e = st->e_a > 0.0 && st->e_mid > 0.0;   // the caller's expansion history
        const double ck = dak / (a * (own_e ? st->e_a : E_lcdm(a, om)));
        const double cd = da / (std::pow(am, 3.0) * (own_e ? st->e_mid : E_lcdm(am, om)));
        const long long cells = (long long)n * n * n;
        const double *P = w.phin;
        if (dphi) {
            k_pot<<<grid1(cells), 256, 0, ctx->stream>>>(w.phin, dphi, cphi, w.pot, cells);
            P = w.pot;
        }
        k_force_mesh<<<grid1(cells), 256, 0, ctx->stream>>>(P, w.g3, w.g3 + cells, w.g3 + 2 * cells, n);
        k_kick_drift<<<grid1(st->np), 256, 0, ctx->stream>>>(dpos, dmom, st->np, n, w.g3, w.g3 + cells,
                                                             w.g3 + 2 * cells, fr, 0.5 * ck, cd);
        MG_CK(cudaGetLastError());
        stage_out(ctx, st->pos, dpos, pb);
        stage_out(ctx, st->mom, dmom, pb);
        st->a += da;
        st->first = 0;
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    if (stats) *stats = loc;
    return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// CIC deposit for callers that cannot allocate device memory
//
// pm_cic_deposit keeps its fixed-point accumulator and reduction partials in
// memory it allocates on first use.  Some callers cannot let a library call
// cudaMalloc: applications that hand all device memory to their own pool up
// front, and real-time pipelines in which cudaMalloc's implicit device
// synchronisation is not acceptable.  This variant runs the
// same kernels with all of its scratch in one file-scope device array whose
// size is fixed when the library is loaded: the accumulator for meshes up
// to NOALLOC_MAX_NG^3 cells, the reduction partials, the mean and the
// arrival counter (16 MiB + 8 KiB + 256 B on every GPU that loads the
// library, held until the process exits).
// ---------------------------------------------------------------------------
namespace mg {

constexpr int NOALLOC_MAX_NG = 128;
constexpr long long NOALLOC_CELLS = (long long)NOALLOC_MAX_NG * NOALLOC_MAX_NG * NOALLOC_MAX_NG;
constexpr int NOALLOC_BLOCKS = MAX_RED_BLOCKS / 4;   // the mean reduction's largest grid
constexpr size_t NOALLOC_BYTES = sizeof(unsigned long long) * (size_t)NOALLOC_CELLS +
                                 sizeof(double) * (size_t)NOALLOC_BLOCKS + 256;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

static void *g_noalloc_addr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

// device address of the scratch array on the current device, looked up once
// per device (host code only holds a stand-in for the array's name)
static int noalloc_scratch(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MG_ERR_CUDA;
    }
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return MG_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return MG_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return MG_OK;
}

// the accumulator must start at zero for every call, and so must the arrival
// counter of the reduction (it is also reset by the last block of each use)
__global__ void __launch_bounds__(256)
k_noalloc_clear(unsigned long long *__restrict__ acc, long long cnt, unsigned int *counter)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) acc[q] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0u;
}

}  // namespace mg

extern "C" int pm_cic_deposit_noalloc(int ng, const float *pos, long long np, double *delta_out, void *cuda_stream)
{
    using namespace mg;
    if (!pos || !delta_out || np < 1 || ng < 2) return MG_ERR_ARG;
    if (ng > NOALLOC_MAX_NG) return MG_ERR_ARG;      // the scratch holds NOALLOC_MAX_NG^3 cells
    if (!is_device_ptr(pos) || !is_device_ptr(delta_out)) return MG_ERR_ARG;
    void *base = nullptr;
    const int rc = noalloc_scratch(&base);
    if (rc != MG_OK) return rc;
    unsigned char *b = (unsigned char *)base;
    unsigned long long *acc = (unsigned long long *)b;
    double *partials = (double *)(b + sizeof(unsigned long long) * (size_t)NOALLOC_CELLS);
    double *mean = partials + NOALLOC_BLOCKS;
    unsigned int *counter = (unsigned int *)(mean + 1);
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    const long long cnt = (long long)ng * ng * ng;
    // each launch is checked as it is made, with cudaPeekAtLastError, which
    // leaves the error state alone: an error left by the caller's earlier
    // work is neither reported as this call's nor cleared
    k_noalloc_clear<<<grid1(cnt), 256, 0, st>>>(acc, cnt, counter);
    if (cudaPeekAtLastError() != cudaSuccess) return MG_ERR_CUDA;
    k_cic_deposit<<<grid1(np), 256, 0, st>>>(pos, np, ng, acc);
    if (cudaPeekAtLastError() != cudaSuccess) return MG_ERR_CUDA;
    k_cic_finish<<<grid1(cnt), 256, 0, st>>>(acc, cnt, (double)cnt / (double)np, delta_out);
    if (cudaPeekAtLastError() != cudaSuccess) return MG_ERR_CUDA;
    RedBuf rb{partials, counter, NOALLOC_BLOCKS};
    launch_mean_nat(delta_out, cnt, mean, rb, st);
    if (cudaPeekAtLastError() != cudaSuccess) return MG_ERR_CUDA;
    k_sub_mean<<<grid1(cnt), 256, 0, st>>>(delta_out, cnt, mean);
    if (cudaPeekAtLastError() != cudaSuccess) return MG_ERR_CUDA;
    return MG_OK;
}

