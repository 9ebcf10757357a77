// Particle-mesh pieces of the GB300 MG-GLAM library (Sec. 3.1 of
// arXiv:2110.00566): cloud-in-cell assignment with deterministic fixed-point
// accumulation, and the CIC index used by it.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ctx.cuh"

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
};

static PmWork &pmw(mg_ctx *ctx)
{
    if (!ctx->pm) ctx->pm = new PmWork();
    return *ctx->pm;
}

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

int pm_step(mg_ctx *ctx, pm_state *st, const mg_opts *opts, mg_stats *stats)
{
    (void)st;
    (void)opts;
    (void)stats;
    return set_err(ctx, MG_ERR_ARG, "pm_step: not available in this build");
}

int mg_solve_adjoint(mg_ctx *ctx, const mg_grid *g, const mg_dgp_params *p, const mg_opts *opts, const double *phi,
                     const double *delta, const double *dL_dphi, double *dL_ddelta_out, double *dL_drc_out,
                     mg_stats *stats)
{
    (void)g; (void)p; (void)opts; (void)phi; (void)delta; (void)dL_dphi; (void)dL_ddelta_out; (void)dL_drc_out;
    (void)stats;
    return set_err(ctx, MG_ERR_ARG, "mg_solve_adjoint: not available in this build");
}

}  // extern "C"

