// Differentiable particle-mesh run of the GB300 MG-GLAM library: the
// forward model of Sec. 3.1 / 3.1.1 of arXiv:2110.00566 with the nDGP field
// of Sec. 3.2.3 (Zel'dovich initial conditions from white noise, leapfrog
// steps, binned power spectrum) in FP64 particle state, and its
// hand-written reverse pass: the transposes of the initial-condition map,
// the CIC deposit and interpolation, the central-difference gradient and
// the Green's function, the nDGP adjoint solve of adjoint.cu, with the
// particle states stored every checkpoint_every steps and each segment
// recomputed forward before it is reversed.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cufft.h>

#include "ctx.cuh"
#include "kernels.cuh"

namespace mg {

namespace {

inline int gridp(long long n) { return (int)std::max<long long>(1, std::min<long long>(152 * 16, (n + 255) / 256)); }

constexpr double FIX_SCALE = 1099511627776.0;  // 2^40: fixed point of the deposit
constexpr double FIX_INV = 1.0 / 1099511627776.0;

// CIC lower / upper cell and weights along one axis (cell centres at
// i + 1/2): lo = floor(x - 1/2), upper weight x - 1/2 - lo
__device__ __forceinline__ void cic64(double x, int n, int &i0, int &i1, double &w0, double &w1)
{
    const double t = x - 0.5;
    const double lo = floor(t);
    const double dx = t - lo;
    int a = (int)lo % n;
    if (a < 0) a += n;
    i0 = a;
    i1 = a + 1 == n ? 0 : a + 1;
    w0 = 1.0 - dx;
    w1 = dx;
}

__device__ __forceinline__ long long cell3(int i, int j, int k, int n) { return ((long long)i * n + j) * n + k; }

// signed integer frequency of rfft-grid index i along a full axis
__device__ __forceinline__ int freq(int i, int n) { return i < n / 2 ? i : i - n; }

// --------------------------------------------------------------------------
// initial conditions
// --------------------------------------------------------------------------

// out = m_c in with m_c = i k_c amp / k^2 * scale (k_c = 0 on the Nyquist
// plane of axis c, m = 0 at k = 0); adjoint: out += conj(m_c) in
__global__ void __launch_bounds__(256)
k_ic_spec(const cufftDoubleComplex *__restrict__ in, cufftDoubleComplex *__restrict__ out,
          const double *__restrict__ amp, int n, int c, double kf, double scale, int adjoint)
{
    const int nz = n / 2 + 1;
    const long long total = (long long)n * n * nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += stride) {
        int i_, j_, kz;
        split3(q, n, nz, i_, j_, kz);
        const int mj = freq(j_, n), mi = freq(i_, n);
        const int mc = c == 0 ? mi : (c == 1 ? mj : kz);
        const double kx = kf * mi, ky = kf * mj, kzz = kf * kz;
        const double k2 = kx * kx + ky * ky + kzz * kzz;
        double f = 0.0;
        if (q != 0 && mc != n / 2 && mc != -n / 2) f = kf * mc / k2 * amp[q] * scale;
        const cufftDoubleComplex v = in[q];
        cufftDoubleComplex o;
        if (adjoint) {
            o = out[q];
            o.x += f * v.y;
            o.y -= f * v.x;
        } else {
            o.x = -f * v.y;
            o.y = f * v.x;
        }
        out[q] = o;
    }
}

// x_c = wrap(lattice_c + growth psi_c), p_c = vel psi_c (particle = cell index)
__global__ void __launch_bounds__(256)
k_ic_place(const double *__restrict__ psi, int n, int c, double growth, double vel, double *__restrict__ pos,
           double *__restrict__ mom)
{
    const long long np = (long long)n * n * n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += stride) {
        int i, j, k;
        split3(p, n, n, i, j, k);
        const double q = (c == 0 ? i : (c == 1 ? j : k)) + 0.5;
        const double s = psi[p];
        double x = q + growth * s;
        x = x - (double)n * floor(x / (double)n);
        if (x >= (double)n) x -= (double)n;
        pos[3 * p + c] = x;
        mom[3 * p + c] = vel * s;
    }
}

// psibar_c = growth xbar_c + vel pbar_c on the lattice
__global__ void __launch_bounds__(256)
k_ic_gather(const double *__restrict__ dpos, const double *__restrict__ dmom, long long np, int c, double growth,
            double vel, double *__restrict__ out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += stride)
        out[p] = growth * dpos[3 * p + c] + (dmom ? vel * dmom[3 * p + c] : 0.0);
}

// --------------------------------------------------------------------------
// CIC deposit (64-bit fixed point) and its adjoint
// --------------------------------------------------------------------------

__global__ void __launch_bounds__(256)
k_dep64(const double *__restrict__ pos, long long np, int n, unsigned long long *__restrict__ acc)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += stride) {
        int i0[3], i1[3];
        double w0[3], w1[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) cic64(pos[3 * p + d], n, i0[d], i1[d], w0[d], w1[d]);
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const double w = ((a ? w1[0] : w0[0]) * (b ? w1[1] : w0[1])) * (c ? w1[2] : w0[2]);
                    const unsigned long long q = (unsigned long long)llrint(w * FIX_SCALE);
                    atomicAdd(acc + cell3(a ? i1[0] : i0[0], b ? i1[1] : i0[1], c ? i1[2] : i0[2], n), q);
                }
    }
}

__global__ void __launch_bounds__(256)
k_dep64_finish(const unsigned long long *__restrict__ acc, long long cnt, double mass, double *__restrict__ delta)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride)
        delta[q] = mass * ((double)acc[q] * FIX_INV) - 1.0;
}

// x -= *mean (a device scalar), or x = s * y when y is given
__global__ void __launch_bounds__(256)
k_shift_scale(double *__restrict__ x, const double *__restrict__ y, double s, long long cnt,
              const double *__restrict__ mean)
{
    const double mu = mean ? *mean : 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride)
        x[q] = y ? s * y[q] : x[q] - mu;
}

__global__ void __launch_bounds__(256)
k_add(double *__restrict__ x, const double *__restrict__ y, long long cnt)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) x[q] += y[q];
}

// dpos (+)= mass sum_corners dW/dx dd(corner)
__global__ void __launch_bounds__(256)
k_dep64_adj(const double *__restrict__ pos, long long np, int n, const double *__restrict__ dd, double mass,
            double *__restrict__ dpos, int accum)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += stride) {
        int i0[3], i1[3];
        double w0[3], w1[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) cic64(pos[3 * p + d], n, i0[d], i1[d], w0[d], w1[d]);
        double g[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const double wa = a ? w1[0] : w0[0], wb = b ? w1[1] : w0[1], wc = c ? w1[2] : w0[2];
                    const double v = dd[cell3(a ? i1[0] : i0[0], b ? i1[1] : i0[1], c ? i1[2] : i0[2], n)];
                    g[0] += (a ? v : -v) * (wb * wc);
                    g[1] += (b ? v : -v) * (wa * wc);
                    g[2] += (c ? v : -v) * (wa * wb);
                }
#pragma unroll
        for (int d = 0; d < 3; ++d) dpos[3 * p + d] = (accum ? dpos[3 * p + d] : 0.0) + mass * g[d];
    }
}

// --------------------------------------------------------------------------
// forces: -grad (Phi_N + phi/2) by central differences at the CIC cells
// --------------------------------------------------------------------------

__device__ __forceinline__ double potv(const double *__restrict__ A, const double *__restrict__ B, long long q)
{
    return B ? A[q] + 0.5 * B[q] : A[q];
}

__device__ __forceinline__ void grad_at(const double *__restrict__ A, const double *__restrict__ B, int n, int i,
                                        int j, int k, double (&g)[3])
{
    const int ip = i + 1 == n ? 0 : i + 1, im = i == 0 ? n - 1 : i - 1;
    const int jp = j + 1 == n ? 0 : j + 1, jm = j == 0 ? n - 1 : j - 1;
    const int kp = k + 1 == n ? 0 : k + 1, km = k == 0 ? n - 1 : k - 1;
    g[0] = -(potv(A, B, cell3(ip, j, k, n)) - potv(A, B, cell3(im, j, k, n))) / 2.0;
    g[1] = -(potv(A, B, cell3(i, jp, k, n)) - potv(A, B, cell3(i, jm, k, n))) / 2.0;
    g[2] = -(potv(A, B, cell3(i, j, kp, n)) - potv(A, B, cell3(i, j, km, n))) / 2.0;
}

__device__ __forceinline__ void force_at(const double *__restrict__ A, const double *__restrict__ B, int n,
                                         const double *x, double (&F)[3])
{
    int i0[3], i1[3];
    double w0[3], w1[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) cic64(x[d], n, i0[d], i1[d], w0[d], w1[d]);
    F[0] = F[1] = F[2] = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                const double w = ((a ? w1[0] : w0[0]) * (b ? w1[1] : w0[1])) * (c ? w1[2] : w0[2]);
                double g[3];
                grad_at(A, B, n, a ? i1[0] : i0[0], b ? i1[1] : i0[1], c ? i1[2] : i0[2], g);
                F[0] += w * g[0];
                F[1] += w * g[1];
                F[2] += w * g[2];
            }
}

__global__ void __launch_bounds__(256)
k_force64(const double *__restrict__ A, const double *__restrict__ B, const double *__restrict__ pos, long long np,
          int n, double *__restrict__ F)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += stride) {
        const double x[3] = {pos[3 * p], pos[3 * p + 1], pos[3 * p + 2]};
        double f[3];
        force_at(A, B, n, x, f);
        F[3 * p] = f[0];
        F[3 * p + 1] = f[1];
        F[3 * p + 2] = f[2];
    }
}

// kick p += ck F, drift x += cd p, wrap into [0, n)
__global__ void __launch_bounds__(256)
k_kd64(double *__restrict__ pos, double *__restrict__ mom, long long np, int n, const double *__restrict__ A,
       const double *__restrict__ B, double ck, double cd)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += stride) {
        const double x[3] = {pos[3 * p], pos[3 * p + 1], pos[3 * p + 2]};
        double f[3];
        force_at(A, B, n, x, f);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double pn = mom[3 * p + d] + ck * f[d];
            mom[3 * p + d] = pn;
            double xn = x[d] + cd * pn;
            xn = xn - (double)n * floor(xn / (double)n);
            if (xn >= (double)n) xn -= (double)n;
            pos[3 * p + d] = xn;
        }
    }
}

// adjoint of the force interpolation for cotangents dF: dpos (+)= the weights'
// part sum_c dF_c sum_corners dW/dx g_c, and gb_c += W dF_c at the 8 cells
__global__ void __launch_bounds__(256)
k_force64_adj(const double *__restrict__ A, const double *__restrict__ B, const double *__restrict__ pos,
              long long np, int n, const double *__restrict__ dF, double *__restrict__ dpos, int accum,
              double *__restrict__ gb0, double *__restrict__ gb1, double *__restrict__ gb2)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += stride) {
        int i0[3], i1[3];
        double w0[3], w1[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) cic64(pos[3 * p + d], n, i0[d], i1[d], w0[d], w1[d]);
        const double f0 = dF[3 * p], f1 = dF[3 * p + 1], f2 = dF[3 * p + 2];
        double gx = 0.0, gy = 0.0, gz = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int c = 0; c < 2; ++c) {
                    const double wa = a ? w1[0] : w0[0], wb = b ? w1[1] : w0[1], wc = c ? w1[2] : w0[2];
                    const int i = a ? i1[0] : i0[0], j = b ? i1[1] : i0[1], k = c ? i1[2] : i0[2];
                    double g[3];
                    grad_at(A, B, n, i, j, k, g);
                    const double v = f0 * g[0] + f1 * g[1] + f2 * g[2];
                    gx += (a ? v : -v) * (wb * wc);
                    gy += (b ? v : -v) * (wa * wc);
                    gz += (c ? v : -v) * (wa * wb);
                    const double w = (wa * wb) * wc;
                    const long long q = cell3(i, j, k, n);
                    atomicAdd(gb0 + q, w * f0);
                    atomicAdd(gb1 + q, w * f1);
                    atomicAdd(gb2 + q, w * f2);
                }
        dpos[3 * p] = (accum ? dpos[3 * p] : 0.0) + gx;
        dpos[3 * p + 1] = (accum ? dpos[3 * p + 1] : 0.0) + gy;
        dpos[3 * p + 2] = (accum ? dpos[3 * p + 2] : 0.0) + gz;
    }
}

// dPhi = sum_c (gb_c(+e_c) - gb_c(-e_c)) / 2: the transpose of g_c = -D_c Phi
__global__ void __launch_bounds__(256)
k_div64(const double *__restrict__ gb0, const double *__restrict__ gb1, const double *__restrict__ gb2, int n,
        double *__restrict__ out)
{
    const long long cnt = (long long)n * n * n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) {
        int i, j, k;
        split3(q, n, n, i, j, k);
        const int ip = i + 1 == n ? 0 : i + 1, im = i == 0 ? n - 1 : i - 1;
        const int jp = j + 1 == n ? 0 : j + 1, jm = j == 0 ? n - 1 : j - 1;
        const int kp = k + 1 == n ? 0 : k + 1, km = k == 0 ? n - 1 : k - 1;
        out[q] = ((gb0[cell3(ip, j, k, n)] - gb0[cell3(im, j, k, n)]) +
                  (gb1[cell3(i, jp, k, n)] - gb1[cell3(i, jm, k, n)]) +
                  (gb2[cell3(i, j, kp, n)] - gb2[cell3(i, j, km, n)])) /
                 2.0;
    }
}

// pbar += cd xbar (drift), dF = ck pbar (kick)
__global__ void __launch_bounds__(256)
k_kd64_adj(const double *__restrict__ xb, double *__restrict__ pb, double *__restrict__ dF, long long cnt, double ck,
           double cd)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) {
        const double v = pb[q] + cd * xb[q];
        pb[q] = v;
        dF[q] = ck * v;
    }
}

// --------------------------------------------------------------------------
// binned power spectrum
// --------------------------------------------------------------------------

// bin of the integer wavevector (mi, mj, mz): floor((|m| - 1) nbins /
// (n/2 - 1)) for 1 <= |m| <= n/2, |m| = n/2 in the last bin, else -1;
// sqrt, product and quotient correctly rounded, in this order
__device__ __forceinline__ int pk_bin(int mi, int mj, int mz, int half, int nbins)
{
    const double km = sqrt((double)(mi * mi + mj * mj + mz * mz));
    if (km < 1.0 || km > (double)half) return -1;
    if (km == (double)half) return nbins - 1;
    return (int)floor(__ddiv_rn(__dmul_rn(km - 1.0, (double)nbins), (double)(half - 1)));
}

// block b sums w |delta_k|^2 V/n^6 and w over the modes of bin b (fixed order)
__global__ void __launch_bounds__(256)
k_pk(const cufftDoubleComplex *__restrict__ spec, int n, int nbins, double vscale, double *__restrict__ out)
{
    __shared__ double sh[64];
    const int b = blockIdx.x;
    const int nz = n / 2 + 1, half = n / 2;
    const long long total = (long long)n * n * nz;
    double v[2] = {0.0, 0.0};
    for (long long q = threadIdx.x; q < total; q += blockDim.x) {
        int i_, j_, kz;
        split3(q, n, nz, i_, j_, kz);
        const int mj = freq(j_, n), mi = freq(i_, n);
        if (pk_bin(mi, mj, kz, half, nbins) != b) continue;
        const double w = (kz > 0 && kz < half) ? 2.0 : 1.0;
        const cufftDoubleComplex c = spec[q];
        v[0] += w * (c.x * c.x + c.y * c.y) * vscale;
        v[1] += w;
    }
    block_sum<2>(v, sh);
    if (threadIdx.x == 0) {
        out[2 * b] = v[1] > 0 ? v[0] / v[1] : 0.0;
        out[2 * b + 1] = v[1];
    }
}

// spec *= 2 dP_b V / (n^6 n_b) on the modes of bin b, 0 elsewhere
__global__ void __launch_bounds__(256)
k_pk_adj(cufftDoubleComplex *__restrict__ spec, int n, int nbins, const double *__restrict__ coef)
{
    const int nz = n / 2 + 1, half = n / 2;
    const long long total = (long long)n * n * nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += stride) {
        int i_, j_, kz;
        split3(q, n, nz, i_, j_, kz);
        const int mj = freq(j_, n), mi = freq(i_, n);
        const int b = pk_bin(mi, mj, kz, half, nbins);
        const double f = b >= 0 ? coef[b] : 0.0;
        cufftDoubleComplex c = spec[q];
        c.x *= f;
        c.y *= f;
        spec[q] = c;
    }
}

}  // namespace

// --------------------------------------------------------------------------
// workspace
// --------------------------------------------------------------------------
struct DpmWork {
    int n = 0, nseg = 0, K = 0;
    cufftHandle d2z = 0, z2d = 0;
    cufftDoubleComplex *specA = nullptr, *specB = nullptr;
    unsigned long long *acc = nullptr;
    double *delta = nullptr, *phin = nullptr, *phiw = nullptr, *gb[3] = {}, *dphi = nullptr, *dd = nullptr,
           *tmp = nullptr, *tmp2 = nullptr;
    double *x = nullptr, *p = nullptr, *xb = nullptr, *pb = nullptr, *fb = nullptr;
    double *coef = nullptr, *pkd = nullptr;
    std::vector<double *> ck_x, ck_p, ck_phi, seg_x, seg_phi;
    std::vector<void *> allocs;
};

static void dpm_free(DpmWork *w)
{
    if (!w) return;
    if (w->d2z) cufftDestroy(w->d2z);
    if (w->z2d) cufftDestroy(w->z2d);
    for (void *p : w->allocs) cudaFree(p);
    delete w;
}

void dpm_release(mg_ctx *ctx)
{
    if (ctx && ctx->dpm) {
        dpm_free(ctx->dpm);
        ctx->dpm = nullptr;
    }
}

#define DPM_CUFFT(call)                                                                                \
    do {                                                                                               \
        cufftResult r_ = (call);                                                                       \
        if (r_ != CUFFT_SUCCESS) {                                                                     \
            set_err(ctx, MG_ERR_CUDA, "cuFFT error %d in %s at %s:%d", (int)r_, #call, __FILE__, __LINE__); \
            throw CudaFail{MG_ERR_CUDA};                                                               \
        }                                                                                              \
    } while (0)

template <typename T>
static T *dalloc(mg_ctx *ctx, DpmWork *w, size_t count)
{
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(T) * std::max<size_t>(count, 1));
    if (e != cudaSuccess) {
        fail_cuda(ctx, e, "cudaMalloc(dpm)", __FILE__, __LINE__);
        throw CudaFail{MG_ERR_OOM};
    }
    w->allocs.push_back(p);
    return (T *)p;
}

// the workspace for an n^3 mesh with nseg checkpoints of K steps
static DpmWork &dpm_work(mg_ctx *ctx, int n, int nseg, int K)
{
    DpmWork *w = ctx->dpm;
    if (w && w->n == n && w->nseg >= nseg && w->K >= K) return *w;
    MG_CK(cudaStreamSynchronize(ctx->stream));
    dpm_release(ctx);
    w = new DpmWork();
    ctx->dpm = w;
    w->n = n;
    w->nseg = nseg;
    w->K = K;
    const size_t cells = (size_t)n * n * n, modes = (size_t)n * n * (n / 2 + 1), p3 = 3 * cells;
    w->specA = dalloc<cufftDoubleComplex>(ctx, w, modes);
    w->specB = dalloc<cufftDoubleComplex>(ctx, w, modes);
    w->acc = dalloc<unsigned long long>(ctx, w, cells);
    for (double **m : {&w->delta, &w->phin, &w->phiw, &w->gb[0], &w->gb[1], &w->gb[2], &w->dphi, &w->dd, &w->tmp,
                       &w->tmp2})
        *m = dalloc<double>(ctx, w, cells);
    for (double **m : {&w->x, &w->p, &w->xb, &w->pb, &w->fb}) *m = dalloc<double>(ctx, w, p3);
    w->coef = dalloc<double>(ctx, w, 1024);
    w->pkd = dalloc<double>(ctx, w, 2048);
    for (int s = 0; s < nseg; ++s) {
        w->ck_x.push_back(dalloc<double>(ctx, w, p3));
        w->ck_p.push_back(dalloc<double>(ctx, w, p3));
        w->ck_phi.push_back(dalloc<double>(ctx, w, cells));
    }
    for (int k = 0; k < K; ++k) {
        w->seg_x.push_back(dalloc<double>(ctx, w, p3));
        w->seg_phi.push_back(dalloc<double>(ctx, w, cells));
    }
    DPM_CUFFT(cufftPlan3d(&w->d2z, n, n, n, CUFFT_D2Z));
    DPM_CUFFT(cufftPlan3d(&w->z2d, n, n, n, CUFFT_Z2D));
    DPM_CUFFT(cufftSetStream(w->d2z, ctx->stream));
    DPM_CUFFT(cufftSetStream(w->z2d, ctx->stream));
    return *w;
}

// --------------------------------------------------------------------------
// device-level pieces
// --------------------------------------------------------------------------
struct DpmRun {
    mg_ctx *ctx;
    DpmWork &w;
    dpm_config c;
    double rc;
    mg_opts o;
    long long np, cells;
    double da, mass;
    long long cycles = 0;
    mg_stats last{};
};

static void ic_forward(mg_ctx *ctx, DpmWork &w, const dpm_config &c, const double *amp, const double *noise,
                       double *pos, double *mom)
{
    const int n = c.ng;
    const long long cells = (long long)n * n * n, modes = (long long)n * n * (n / 2 + 1);
    const double kf = 2.0 * 3.14159265358979323846 / c.box_mpch, cell = c.box_mpch / n;
    DPM_CUFFT(cufftExecD2Z(w.d2z, const_cast<double *>(noise), w.specA));
    for (int d = 0; d < 3; ++d) {
        k_ic_spec<<<gridp(modes), 256, 0, ctx->stream>>>(w.specA, w.specB, amp, n, d, kf,
                                                         1.0 / ((double)cells * cell), 0);
        DPM_CUFFT(cufftExecZ2D(w.z2d, w.specB, w.tmp));
        k_ic_place<<<gridp(cells), 256, 0, ctx->stream>>>(w.tmp, n, d, c.growth, c.vel, pos, mom);
    }
    MG_CK(cudaGetLastError());
}

static void ic_adjoint(mg_ctx *ctx, DpmWork &w, const dpm_config &c, const double *amp, const double *dpos,
                       const double *dmom, double *dnoise)
{
    const int n = c.ng;
    const long long cells = (long long)n * n * n, modes = (long long)n * n * (n / 2 + 1);
    const double kf = 2.0 * 3.14159265358979323846 / c.box_mpch, cell = c.box_mpch / n;
    MG_CK(cudaMemsetAsync(w.specB, 0, sizeof(cufftDoubleComplex) * modes, ctx->stream));
    for (int d = 0; d < 3; ++d) {
        k_ic_gather<<<gridp(cells), 256, 0, ctx->stream>>>(dpos, dmom, cells, d, c.growth, c.vel, w.tmp);
        DPM_CUFFT(cufftExecD2Z(w.d2z, w.tmp, w.specA));
        k_ic_spec<<<gridp(modes), 256, 0, ctx->stream>>>(w.specA, w.specB, amp, n, d, kf,
                                                         1.0 / ((double)cells * cell), 1);
    }
    DPM_CUFFT(cufftExecZ2D(w.z2d, w.specB, dnoise));
    MG_CK(cudaGetLastError());
}

static void deposit(mg_ctx *ctx, DpmWork &w, int n, const double *pos, long long np, double *delta)
{
    const long long cells = (long long)n * n * n;
    MG_CK(cudaMemsetAsync(w.acc, 0, sizeof(unsigned long long) * cells, ctx->stream));
    k_dep64<<<gridp(np), 256, 0, ctx->stream>>>(pos, np, n, w.acc);
    k_dep64_finish<<<gridp(cells), 256, 0, ctx->stream>>>(w.acc, cells, (double)cells / (double)np, delta);
    launch_mean_nat(delta, cells, ctx->dscratch, ctx->rb, ctx->stream);
    k_shift_scale<<<gridp(cells), 256, 0, ctx->stream>>>(delta, nullptr, 0.0, cells, ctx->dscratch);
    MG_CK(cudaGetLastError());
}

// P_b into the host array pk (and the counts), from delta
static void power_spectrum(mg_ctx *ctx, DpmWork &w, int n, double box, int nbins, const double *delta, double *pk,
                           double *counts)
{
    DPM_CUFFT(cufftExecD2Z(w.d2z, const_cast<double *>(delta), w.specA));
    const double vscale = box * box * box / ((double)n * n * n * (double)n * n * n);
    k_pk<<<nbins, 256, 0, ctx->stream>>>(w.specA, n, nbins, vscale, w.pkd);
    MG_CK(cudaGetLastError());
    std::vector<double> h(2 * (size_t)nbins);
    MG_CK(cudaMemcpyAsync(h.data(), w.pkd, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, ctx->stream));
    MG_CK(cudaStreamSynchronize(ctx->stream));
    for (int b = 0; b < nbins; ++b) {
        pk[b] = h[2 * b];
        if (counts) counts[b] = h[2 * b + 1];
    }
}

// dL/ddelta from dL/dP (host, nbins) and the bin counts (host)
static void power_spectrum_adjoint(mg_ctx *ctx, DpmWork &w, int n, double box, int nbins, const double *delta,
                                   const double *dpk, const double *counts, double *ddelta)
{
    const long long modes = (long long)n * n * (n / 2 + 1);
    const double vscale = box * box * box / ((double)n * n * n * (double)n * n * n);
    std::vector<double> cf(nbins);
    for (int b = 0; b < nbins; ++b) cf[b] = counts[b] > 0 ? 2.0 * dpk[b] * vscale / counts[b] : 0.0;
    MG_CK(cudaMemcpyAsync(w.coef, cf.data(), sizeof(double) * nbins, cudaMemcpyHostToDevice, ctx->stream));
    DPM_CUFFT(cufftExecD2Z(w.d2z, const_cast<double *>(delta), w.specA));
    k_pk_adj<<<gridp(modes), 256, 0, ctx->stream>>>(w.specA, n, nbins, w.coef);
    MG_CK(cudaGetLastError());
    DPM_CUFFT(cufftExecZ2D(w.z2d, w.specA, ddelta));
    MG_CK(cudaStreamSynchronize(ctx->stream));  // cf lives on the host stack
}

static double E_of(double a, double om) { return std::sqrt(om / (a * a * a) + (1.0 - om)); }

// forward step t from (w.x, w.p) with warm-start field w.phiw (updated)
static int step_forward(DpmRun &R, int t, double *x, double *p)
{
    mg_ctx *ctx = R.ctx;
    DpmWork &w = R.w;
    const int n = R.c.ng;
    const double a = R.c.a_start + t * R.da, om = R.c.omega_m;
    deposit(ctx, w, n, x, R.np, w.delta);
    newton_potential_dev(ctx, n, a, om, w.delta, w.phin);
    const double *phi = nullptr;
    if (R.c.model == 1) {
        mg_stats st{};
        const int rc = solve_dgp_dev(ctx, n, a, om, R.rc, w.delta, w.phiw, R.o, &st);
        R.cycles += st.cycles;
        R.last = st;
        if (rc < 0) return rc;
        phi = w.phiw;
    }
    const double ck = (t == 0 ? 0.5 * R.da : R.da) / (a * E_of(a, om));
    const double am = a + 0.5 * R.da;
    const double cd = R.da / (am * am * am * E_of(am, om));
    k_kd64<<<gridp(R.np), 256, 0, ctx->stream>>>(x, p, R.np, n, w.phin, phi, ck, cd);
    MG_CK(cudaGetLastError());
    return MG_OK;
}

// reverse of step t at positions xs (phis: the step's nDGP field)
static int step_backward(DpmRun &R, int t, const double *xs, const double *phis, double &drc_acc)
{
    mg_ctx *ctx = R.ctx;
    DpmWork &w = R.w;
    cudaStream_t s = ctx->stream;
    const int n = R.c.ng;
    const long long cells = R.cells;
    const double a = R.c.a_start + t * R.da, om = R.c.omega_m;
    const double ck = (t == 0 ? 0.5 * R.da : R.da) / (a * E_of(a, om));
    const double am = a + 0.5 * R.da;
    const double cd = R.da / (am * am * am * E_of(am, om));
    k_kd64_adj<<<gridp(3 * R.np), 256, 0, s>>>(w.xb, w.pb, w.fb, 3 * R.np, ck, cd);
    deposit(ctx, w, n, xs, R.np, w.delta);
    newton_potential_dev(ctx, n, a, om, w.delta, w.phin);
    const double *phi = R.c.model == 1 ? phis : nullptr;
    for (int d = 0; d < 3; ++d) MG_CK(cudaMemsetAsync(w.gb[d], 0, sizeof(double) * cells, s));
    k_force64_adj<<<gridp(R.np), 256, 0, s>>>(w.phin, phi, xs, R.np, n, w.fb, w.xb, 1, w.gb[0], w.gb[1], w.gb[2]);
    k_div64<<<gridp(cells), 256, 0, s>>>(w.gb[0], w.gb[1], w.gb[2], n, w.dphi);
    MG_CK(cudaGetLastError());
    newton_potential_dev(ctx, n, a, om, w.dphi, w.dd);
    if (R.c.model == 1) {
        k_shift_scale<<<gridp(cells), 256, 0, s>>>(w.tmp, w.dphi, 0.5, cells, nullptr);
        double drc = 0.0;
        mg_stats st{};
        const int rc = adjoint_dev(ctx, n, a, om, R.rc, R.o, phis, w.delta, w.tmp, w.tmp2, &drc, &st);
        R.cycles += st.cycles;
        if (rc < 0) return rc;
        drc_acc += drc;
        k_add<<<gridp(cells), 256, 0, s>>>(w.dd, w.tmp2, cells);
    }
    k_dep64_adj<<<gridp(R.np), 256, 0, s>>>(xs, R.np, n, w.dd, (double)cells / (double)R.np, w.xb, 1);
    MG_CK(cudaGetLastError());
    return MG_OK;
}

static int check_cfg(mg_ctx *ctx, const dpm_config *c, bool need_solver)
{
    if (!c) return set_err(ctx, MG_ERR_ARG, "null dpm_config");
    const int n = c->ng;
    if (n < 8 || n % 2) return set_err(ctx, MG_ERR_ARG, "ng = %d: need an even ng >= 8", n);
    if (need_solver && c->model == 1 && !valid_ng(n)) return set_err(ctx, MG_ERR_ARG, "ng = %d not supported", n);
    if (!(c->box_mpch > 0) || !(c->omega_m > 0)) return set_err(ctx, MG_ERR_ARG, "box and omega_m must be > 0");
    if (need_solver) {
        if (c->nsteps < 1 || c->checkpoint_every < 1) return set_err(ctx, MG_ERR_ARG, "nsteps, checkpoint_every >= 1");
        if (!(c->a_start > 0) || !(c->a_end > c->a_start)) return set_err(ctx, MG_ERR_ARG, "need 0 < a_start < a_end");
        if (c->model != 0 && c->model != 1) return set_err(ctx, MG_ERR_ARG, "model must be 0 or 1");
        if (c->nbins < 1 || c->nbins > 1024) return set_err(ctx, MG_ERR_ARG, "nbins in [1, 1024]");
    }
    return MG_OK;
}

}  // namespace mg

using namespace mg;

extern "C" {

// the forward run and, with dL_dnoise_out, the reverse pass seeded with the
// cotangent of P: dL/dP_b = 2 (P_b - target_b) / nbins of the built-in loss
// (target_pk), or the caller's dpk_in
static int run_impl(mg_ctx *ctx, const dpm_config *cfg, const mg_opts *opts, const double *amp, const double *noise,
                    double rc_h0, const double *target_pk, const double *dpk_in, double *pk_out, double *loss_out,
                    double *dL_dnoise_out, double *dL_drc_out, mg_stats *stats)
{
    if (!ctx) return MG_ERR_ARG;
    int rc = check_cfg(ctx, cfg, true);
    if (rc) return rc;
    if (!amp || !noise || !pk_out) return set_err(ctx, MG_ERR_ARG, "null amp, noise or pk_out");
    if (cfg->model == 1 && !(rc_h0 > 0)) return set_err(ctx, MG_ERR_ARG, "rc_h0 must be > 0");
    if (dL_dnoise_out && !target_pk && !dpk_in)
        return set_err(ctx, MG_ERR_ARG, "the gradient needs target_pk or dL/dP");
    mg_opts o;
    if (opts)
        o = *opts;
    else
        mg_opts_default(&o);
    rc = check_opts(ctx, o);
    if (rc) return rc;
    o.warm_start = 1;
    const dpm_config c = *cfg;
    const int n = c.ng, K = c.checkpoint_every, T = c.nsteps;
    const int nseg = (T + K - 1) / K;
    mg_stats loc{};
    try {
        enter(ctx);
        const long long cells = (long long)n * n * n;
        const size_t mb = sizeof(double) * (size_t)cells, ab = sizeof(double) * (size_t)n * n * (n / 2 + 1);
        const double *damp = (const double *)stage_in(ctx, 0, amp, ab, true);
        const double *dnoise = (const double *)stage_in(ctx, 1, noise, mb, true);
        double *dgrad = dL_dnoise_out ? (double *)stage_in(ctx, 2, dL_dnoise_out, mb, false) : nullptr;
        DpmWork &w = dpm_work(ctx, n, dgrad ? nseg : 0, dgrad ? std::min(K, T) : 0);
        pm_fft_setup(ctx, n);
        DpmRun R{ctx, w, c, rc_h0, o, cells, cells, (c.a_end - c.a_start) / T, 1.0};
        cudaStream_t s = ctx->stream;
        const size_t pb = sizeof(double) * 3 * (size_t)cells;
        ic_forward(ctx, w, c, damp, dnoise, w.x, w.p);
        MG_CK(cudaMemsetAsync(w.phiw, 0, mb, s));
        for (int t = 0; t < T && rc >= 0; ++t) {
            if (dgrad && t % K == 0) {
                MG_CK(cudaMemcpyAsync(w.ck_x[t / K], w.x, pb, cudaMemcpyDeviceToDevice, s));
                MG_CK(cudaMemcpyAsync(w.ck_p[t / K], w.p, pb, cudaMemcpyDeviceToDevice, s));
                MG_CK(cudaMemcpyAsync(w.ck_phi[t / K], w.phiw, mb, cudaMemcpyDeviceToDevice, s));
            }
            rc = step_forward(R, t, w.x, w.p);
        }
        if (rc < 0) {
            leave(ctx);
            if (stats) *stats = R.last;
            return rc;
        }
        deposit(ctx, w, n, w.x, cells, w.delta);
        std::vector<double> counts(c.nbins);
        power_spectrum(ctx, w, n, c.box_mpch, c.nbins, w.delta, pk_out, counts.data());
        if (target_pk && loss_out) {
            double L = 0.0;
            for (int b = 0; b < c.nbins; ++b) L += (pk_out[b] - target_pk[b]) * (pk_out[b] - target_pk[b]);
            *loss_out = L / c.nbins;
        }
        if (dgrad) {
            std::vector<double> dpk(c.nbins);
            for (int b = 0; b < c.nbins; ++b)
                dpk[b] = dpk_in ? dpk_in[b] : 2.0 * (pk_out[b] - target_pk[b]) / c.nbins;
            power_spectrum_adjoint(ctx, w, n, c.box_mpch, c.nbins, w.delta, dpk.data(), counts.data(), w.dd);
            k_dep64_adj<<<gridp(cells), 256, 0, s>>>(w.x, cells, n, w.dd, 1.0, w.xb, 0);
            MG_CK(cudaMemsetAsync(w.pb, 0, pb, s));
            double drc = 0.0;
            for (int sg = nseg - 1; sg >= 0 && rc >= 0; --sg) {
                const int t0 = sg * K, t1 = std::min(T, t0 + K);
                MG_CK(cudaMemcpyAsync(w.x, w.ck_x[sg], pb, cudaMemcpyDeviceToDevice, s));
                MG_CK(cudaMemcpyAsync(w.p, w.ck_p[sg], pb, cudaMemcpyDeviceToDevice, s));
                MG_CK(cudaMemcpyAsync(w.phiw, w.ck_phi[sg], mb, cudaMemcpyDeviceToDevice, s));
                for (int t = t0; t < t1 && rc >= 0; ++t) {
                    MG_CK(cudaMemcpyAsync(w.seg_x[t - t0], w.x, pb, cudaMemcpyDeviceToDevice, s));
                    rc = step_forward(R, t, w.x, w.p);
                    MG_CK(cudaMemcpyAsync(w.seg_phi[t - t0], w.phiw, mb, cudaMemcpyDeviceToDevice, s));
                }
                for (int t = t1 - 1; t >= t0 && rc >= 0; --t) rc = step_backward(R, t, w.seg_x[t - t0], w.seg_phi[t - t0], drc);
            }
            if (rc >= 0) {
                ic_adjoint(ctx, w, c, damp, w.xb, w.pb, dgrad);
                stage_out(ctx, dL_dnoise_out, dgrad, mb);
                if (dL_drc_out) *dL_drc_out = c.model == 1 ? drc : 0.0;
            }
        }
        MG_CK(cudaStreamSynchronize(s));
        loc = R.last;
        loc.cycles = (int)std::min<long long>(R.cycles, 0x7fffffff);
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    if (stats) *stats = loc;
    return rc;
}

int dpm_run(mg_ctx *ctx, const dpm_config *cfg, const mg_opts *opts, const double *amp, const double *noise,
            double rc_h0, const double *target_pk, double *pk_out, double *loss_out, double *dL_dnoise_out,
            double *dL_drc_out, mg_stats *stats)
{
    return run_impl(ctx, cfg, opts, amp, noise, rc_h0, target_pk, nullptr, pk_out, loss_out, dL_dnoise_out,
                    dL_drc_out, stats);
}

int dpm_run_vjp(mg_ctx *ctx, const dpm_config *cfg, const mg_opts *opts, const double *amp, const double *noise,
                double rc_h0, const double *dL_dpk, double *pk_out, double *dL_dnoise_out, double *dL_drc_out,
                mg_stats *stats)
{
    if (!ctx) return MG_ERR_ARG;
    if (!dL_dpk || !dL_dnoise_out) return set_err(ctx, MG_ERR_ARG, "null dL_dpk or dL_dnoise_out");
    return run_impl(ctx, cfg, opts, amp, noise, rc_h0, nullptr, dL_dpk, pk_out, nullptr, dL_dnoise_out, dL_drc_out,
                    stats);
}

int dpm_ic(mg_ctx *ctx, const dpm_config *cfg, const double *amp, const double *noise, double *pos_out,
           double *mom_out)
{
    if (!ctx) return MG_ERR_ARG;
    int rc = check_cfg(ctx, cfg, false);
    if (rc) return rc;
    if (!amp || !noise || !pos_out || !mom_out) return set_err(ctx, MG_ERR_ARG, "null argument");
    try {
        enter(ctx);
        const int n = cfg->ng;
        const size_t mb = sizeof(double) * (size_t)n * n * n, ab = sizeof(double) * (size_t)n * n * (n / 2 + 1);
        DpmWork &w = dpm_work(ctx, n, 0, 0);
        const double *damp = (const double *)stage_in(ctx, 0, amp, ab, true);
        const double *dn = (const double *)stage_in(ctx, 1, noise, mb, true);
        double *dp = (double *)stage_in(ctx, 2, pos_out, 3 * mb, false);
        double *dm = (double *)stage_in(ctx, 3, mom_out, 3 * mb, false);
        ic_forward(ctx, w, *cfg, damp, dn, dp, dm);
        stage_out(ctx, pos_out, dp, 3 * mb);
        stage_out(ctx, mom_out, dm, 3 * mb);
        MG_CK(cudaStreamSynchronize(ctx->stream));
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

int dpm_ic_adjoint(mg_ctx *ctx, const dpm_config *cfg, const double *amp, const double *dpos, const double *dmom,
                   double *dnoise_out)
{
    if (!ctx) return MG_ERR_ARG;
    int rc = check_cfg(ctx, cfg, false);
    if (rc) return rc;
    if (!amp || !dpos || !dnoise_out) return set_err(ctx, MG_ERR_ARG, "null argument");
    try {
        enter(ctx);
        const int n = cfg->ng;
        const size_t mb = sizeof(double) * (size_t)n * n * n, ab = sizeof(double) * (size_t)n * n * (n / 2 + 1);
        DpmWork &w = dpm_work(ctx, n, 0, 0);
        const double *damp = (const double *)stage_in(ctx, 0, amp, ab, true);
        const double *dx = (const double *)stage_in(ctx, 1, dpos, 3 * mb, true);
        const double *dm = dmom ? (const double *)stage_in(ctx, 2, dmom, 3 * mb, true) : nullptr;
        double *out = (double *)stage_in(ctx, 3, dnoise_out, mb, false);
        ic_adjoint(ctx, w, *cfg, damp, dx, dm, out);
        stage_out(ctx, dnoise_out, out, mb);
        MG_CK(cudaStreamSynchronize(ctx->stream));
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

int dpm_deposit(mg_ctx *ctx, int ng, const double *pos, long long np, double *delta_out)
{
    if (!ctx) return MG_ERR_ARG;
    if (!pos || !delta_out || np < 1 || ng < 8 || ng % 2) return set_err(ctx, MG_ERR_ARG, "bad dpm_deposit arguments");
    try {
        enter(ctx);
        const size_t mb = sizeof(double) * (size_t)ng * ng * ng, pb = sizeof(double) * 3 * (size_t)np;
        DpmWork &w = dpm_work(ctx, ng, 0, 0);
        const double *dp = (const double *)stage_in(ctx, 0, pos, pb, true);
        double *dd = (double *)stage_in(ctx, 1, delta_out, mb, false);
        deposit(ctx, w, ng, dp, np, dd);
        stage_out(ctx, delta_out, dd, mb);
        MG_CK(cudaStreamSynchronize(ctx->stream));
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

int dpm_deposit_adjoint(mg_ctx *ctx, int ng, const double *pos, long long np, const double *ddelta,
                        double *dpos_out)
{
    if (!ctx) return MG_ERR_ARG;
    if (!pos || !ddelta || !dpos_out || np < 1 || ng < 8 || ng % 2)
        return set_err(ctx, MG_ERR_ARG, "bad dpm_deposit_adjoint arguments");
    try {
        enter(ctx);
        const size_t mb = sizeof(double) * (size_t)ng * ng * ng, pb = sizeof(double) * 3 * (size_t)np;
        const double *dp = (const double *)stage_in(ctx, 0, pos, pb, true);
        const double *dd = (const double *)stage_in(ctx, 1, ddelta, mb, true);
        double *out = (double *)stage_in(ctx, 2, dpos_out, pb, false);
        const double mass = (double)ng * ng * ng / (double)np;
        k_dep64_adj<<<gridp(np), 256, 0, ctx->stream>>>(dp, np, ng, dd, mass, out, 0);
        MG_CK(cudaGetLastError());
        stage_out(ctx, dpos_out, out, pb);
        MG_CK(cudaStreamSynchronize(ctx->stream));
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

int dpm_force(mg_ctx *ctx, int ng, const double *phin, const double *phi, const double *pos, long long np,
              double *force_out)
{
    if (!ctx) return MG_ERR_ARG;
    if (!phin || !pos || !force_out || np < 1 || ng < 8 || ng % 2)
        return set_err(ctx, MG_ERR_ARG, "bad dpm_force arguments");
    try {
        enter(ctx);
        const size_t mb = sizeof(double) * (size_t)ng * ng * ng, pb = sizeof(double) * 3 * (size_t)np;
        const double *A = (const double *)stage_in(ctx, 0, phin, mb, true);
        const double *B = phi ? (const double *)stage_in(ctx, 1, phi, mb, true) : nullptr;
        const double *dp = (const double *)stage_in(ctx, 2, pos, pb, true);
        double *out = (double *)stage_in(ctx, 3, force_out, pb, false);
        k_force64<<<gridp(np), 256, 0, ctx->stream>>>(A, B, dp, np, ng, out);
        MG_CK(cudaGetLastError());
        stage_out(ctx, force_out, out, pb);
        MG_CK(cudaStreamSynchronize(ctx->stream));
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

int dpm_force_adjoint(mg_ctx *ctx, int ng, const double *phin, const double *phi, const double *pos, long long np,
                      const double *dforce, double *dpos_out, double *dphin_out)
{
    if (!ctx) return MG_ERR_ARG;
    if (!phin || !pos || !dforce || !dpos_out || !dphin_out || np < 1 || ng < 8 || ng % 2)
        return set_err(ctx, MG_ERR_ARG, "bad dpm_force_adjoint arguments");
    try {
        enter(ctx);
        const long long cells = (long long)ng * ng * ng;
        const size_t mb = sizeof(double) * (size_t)cells, pb = sizeof(double) * 3 * (size_t)np;
        DpmWork &w = dpm_work(ctx, ng, 0, 0);
        const double *A = (const double *)stage_in(ctx, 0, phin, mb, true);
        const double *B = phi ? (const double *)stage_in(ctx, 1, phi, mb, true) : nullptr;
        const double *dp = (const double *)stage_in(ctx, 2, pos, pb, true);
        const double *df = (const double *)stage_in(ctx, 3, dforce, pb, true);
        double *ox = (double *)stage_in(ctx, 4, dpos_out, pb, false);
        double *op = (double *)stage_in(ctx, 5, dphin_out, mb, false);
        for (int d = 0; d < 3; ++d) MG_CK(cudaMemsetAsync(w.gb[d], 0, mb, ctx->stream));
        k_force64_adj<<<gridp(np), 256, 0, ctx->stream>>>(A, B, dp, np, ng, df, ox, 0, w.gb[0], w.gb[1], w.gb[2]);
        k_div64<<<gridp(cells), 256, 0, ctx->stream>>>(w.gb[0], w.gb[1], w.gb[2], ng, op);
        MG_CK(cudaGetLastError());
        stage_out(ctx, dpos_out, ox, pb);
        stage_out(ctx, dphin_out, op, mb);
        MG_CK(cudaStreamSynchronize(ctx->stream));
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

int dpm_power_spectrum(mg_ctx *ctx, int ng, double box_mpch, int nbins, const double *delta, double *pk_out,
                       double *counts_out)
{
    if (!ctx) return MG_ERR_ARG;
    if (!delta || !pk_out || ng < 8 || ng % 2 || nbins < 1 || nbins > 1024 || !(box_mpch > 0))
        return set_err(ctx, MG_ERR_ARG, "bad dpm_power_spectrum arguments");
    try {
        enter(ctx);
        const size_t mb = sizeof(double) * (size_t)ng * ng * ng;
        DpmWork &w = dpm_work(ctx, ng, 0, 0);
        const double *dd = (const double *)stage_in(ctx, 0, delta, mb, true);
        power_spectrum(ctx, w, ng, box_mpch, nbins, dd, pk_out, counts_out);
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

int dpm_power_spectrum_adjoint(mg_ctx *ctx, int ng, double box_mpch, int nbins, const double *delta,
                               const double *dpk, double *ddelta_out)
{
    if (!ctx) return MG_ERR_ARG;
    if (!delta || !dpk || !ddelta_out || ng < 8 || ng % 2 || nbins < 1 || nbins > 1024 || !(box_mpch > 0))
        return set_err(ctx, MG_ERR_ARG, "bad dpm_power_spectrum_adjoint arguments");
    try {
        enter(ctx);
        const size_t mb = sizeof(double) * (size_t)ng * ng * ng;
        DpmWork &w = dpm_work(ctx, ng, 0, 0);
        const double *dd = (const double *)stage_in(ctx, 0, delta, mb, true);
        double *out = (double *)stage_in(ctx, 1, ddelta_out, mb, false);
        std::vector<double> pk(nbins), counts(nbins);
        power_spectrum(ctx, w, ng, box_mpch, nbins, dd, pk.data(), counts.data());
        power_spectrum_adjoint(ctx, w, ng, box_mpch, nbins, dd, dpk, counts.data(), out);
        stage_out(ctx, ddelta_out, out, mb);
        MG_CK(cudaStreamSynchronize(ctx->stream));
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    return MG_OK;
}

}  // extern "C"
