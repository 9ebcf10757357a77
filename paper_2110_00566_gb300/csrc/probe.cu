// Throughput probe for the roofline denominators of ALU-bound kernels:
// FP64 and FP32 fused multiply-add rates of this device, measured with
// eight independent FMA chains per thread on a grid of 16 CTAs per SM.
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

}  // namespace mg

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
