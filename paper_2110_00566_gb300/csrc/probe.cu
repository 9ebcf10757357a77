// Throughput probe for the roofline denominators of ALU-bound kernels:
// FP64 and FP32 fused multiply-add rates of this device, measured with
// eight independent FMA chains per thread on a grid of 16 CTAs per SM.
// Accuracy probe of the FP64 square root, quotient and nDGP N(Sigma) that
// the FP64 kernels evaluate, for tests against CUDA's IEEE operations.
#include <algorithm>

#include "cells.cuh"
#include "ctx.cuh"

namespace mg {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T *out, int iters, T a, T b)
{
    T x0 = (T)threadIdx.x, x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
    T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == T(-12345.678)) out[blockIdx.x] = s;   // keeps the chains live
}

template <typename T>
static double probe_one(mg_ctx *ctx, int iters)
{
    int dev = 0, sms = 0;
    MG_CK(cudaGetDevice(&dev));
    MG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 16, threads = 256;
    T *out = (T *)ctx->dscratch;
    k_fma_probe<T><<<blocks, threads, 0, ctx->stream>>>(out, 4, T(0.999), T(1e-3));   // warm-up
    MG_CK(cudaEventRecord(ctx->t0, ctx->stream));
    k_fma_probe<T><<<blocks, threads, 0, ctx->stream>>>(out, iters, T(0.999), T(1e-3));
    MG_CK(cudaEventRecord(ctx->t1, ctx->stream));
    MG_CK(cudaEventSynchronize(ctx->t1));
    float ms = 0.f;
    MG_CK(cudaEventElapsedTime(&ms, ctx->t0, ctx->t1));
    const double fmas = (double)blocks * threads * iters * 16.0 * 8.0;
    return 2.0 * fmas / (ms * 1e-3) / 1e12;
}

// y[q] = f(x[q]) with the kernels' own device functions
__global__ void __launch_bounds__(256)
k_math_probe(const double *__restrict__ x, double *__restrict__ y, long long n, int fn, OpK<double> op, DgpK64 dk)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += stride) {
        const double v = x[q];
        double r;
        if (fn == 0) {
            r = k_sqrt(v);
        } else if (fn == 1) {
            r = k_quot(1.0, v);
        } else {
            // a cell whose stencil has Q = 0 and density term s = v on a level
            // of spacing h = 1: the residual kernels' N
            int cl = 0;
            r = dgp64_N_any(op, dk, make_ntk(op, dk), 0.0, v, cl);
        }
        y[q] = r;
    }
}

}  // namespace mg

extern "C" int mg_probe_fp64_math(mg_ctx *ctx, int fn, const double *x, double *y, long long n, double alpha)
{
    if (!ctx || !x || !y || n < 0 || fn < 0 || fn > 2) return MG_ERR_ARG;
    if (n == 0) return MG_OK;
    if (!mg::is_device_ptr(x) || !mg::is_device_ptr(y))
        return mg::set_err(ctx, MG_ERR_ARG, "mg_probe_fp64_math: x and y must be device pointers");
    if (fn == 2 && !(alpha != 0.0 && alpha == alpha && alpha - alpha == 0.0))
        return mg::set_err(ctx, MG_ERR_ARG, "mg_probe_fp64_math: alpha must be finite and nonzero");
    try {
        mg::enter(ctx);
        mg::OpK<double> op = mg::make_opk<double>(0, alpha, 2, 0.0, 0.0);
        const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
        mg::k_math_probe<<<(unsigned)blocks, 256, 0, ctx->stream>>>(x, y, n, fn, op, mg::make_dgpk64(1.0));
        MG_CK(cudaGetLastError());
        mg::leave(ctx);
    } catch (mg::CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

extern "C" int mg_probe_alu_peaks(mg_ctx *ctx, double *fp64_tflops, double *fp32_tflops)
{
    if (!ctx) return MG_ERR_ARG;
    try {
        mg::enter(ctx);
        if (fp64_tflops) *fp64_tflops = mg::probe_one<double>(ctx, 64);
        if (fp32_tflops) *fp32_tflops = mg::probe_one<float>(ctx, 4096);
        mg::leave(ctx);
    } catch (mg::CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}
