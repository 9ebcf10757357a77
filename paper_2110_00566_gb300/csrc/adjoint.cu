// Adjoint of the nDGP solve (gradients of a loss of phi with respect to the
// density contrast and to R_c = H0 r_c / c).
//
// With F(phi, s) = Lap phi - Pi N(Sigma(phi) + s) the discrete system of
// mg_solve_dgp (Pi removes the mean; Sec. 3.2.3 operator), s = ks (delta -
// <delta>), ks = (alpha/beta) Omega_m / a, and a cotangent g = dL/dphi, the
// gradient is
//     dL/ds = N'(Sigma) (lambda - <lambda>),  J^T lambda = Pi g,
//     J^T = (Lap - M^T) Pi,   M^T mu = sum_t D_t(kappa_t mu),
// where t runs over the six linear differences of Q (S_x - S_y, S_x - S_z,
// S_y - S_z, C_xy, C_xz, C_yz), D_t is that (symmetric) difference stencil,
// kappa_t = 2 w_t D_t(phi) N'(Sigma) with w_t = 1/(3h^4) or 1/(8h^4), and
// N' = dN/dSigma = 1/sqrt(alpha^2 + 8 Sigma/3) (0 where the root is clamped).
// None of the D_t has a centre coefficient, so the red-black update of the
// forward solver is again the exact local solve; the mean term
// -<lambda> M^T 1 is held fixed during a sweep and recomputed in every
// residual pass, as the compatibility constant is in the forward solve.
// J^T lambda = Pi g is solved by linear (correction-scheme) multigrid with
// the operator rediscretised on each level about R phi.  Then
//     dL/ddelta = ks Pi(N' (lambda - <lambda>)),
//     dL/dR_c  = sum (lambda - <lambda>) [dN/dalpha alpha' + N' ds/dR_c].
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.cuh"

namespace mg {

__device__ __forceinline__ long long nidx(int i, int j, int k, int n) { return ((long long)i * n + j) * n + k; }

// the six linear differences of Q at (i, j, k) of a natural-layout field
__device__ __forceinline__ void q_terms(const double *__restrict__ u, int n, int i, int j, int k, double (&t)[6])
{
    const int ip = wrap_p(i, n), im = wrap_m(i, n), jp = wrap_p(j, n), jm = wrap_m(j, n);
    const int kp = wrap_p(k, n), km = wrap_m(k, n);
    const double Sx = u[nidx(ip, j, k, n)] + u[nidx(im, j, k, n)];
    const double Sy = u[nidx(i, jp, k, n)] + u[nidx(i, jm, k, n)];
    const double Sz = u[nidx(i, j, kp, n)] + u[nidx(i, j, km, n)];
    t[0] = Sx - Sy;
    t[1] = Sx - Sz;
    t[2] = Sy - Sz;
    t[3] = (u[nidx(ip, jp, k, n)] + u[nidx(im, jm, k, n)]) - (u[nidx(ip, jm, k, n)] + u[nidx(im, jp, k, n)]);
    t[4] = (u[nidx(ip, j, kp, n)] + u[nidx(im, j, km, n)]) - (u[nidx(ip, j, km, n)] + u[nidx(im, j, kp, n)]);
    t[5] = (u[nidx(i, jp, kp, n)] + u[nidx(i, jm, km, n)]) - (u[nidx(i, jp, km, n)] + u[nidx(i, jm, kp, n)]);
}

// (M^T mu)(i,j,k) = sum_t D_t(kappa_t mu).  The three face differences
// (S_x - S_y, S_x - S_z, S_y - S_z) meet mu at the same six face neighbours,
// so their kappas are stored combined per face direction:
//   K[0] = kappa_0 + kappa_1 (x faces), K[1] = kappa_2 - kappa_0 (y faces),
//   K[2] = -(kappa_1 + kappa_2) (z faces),
// and K[3..5] = kappa_xy, kappa_xz, kappa_yz (edges, signs by position):
// 18 fused multiply-adds per cell
__device__ __forceinline__ double mt_apply(const double *const *__restrict__ K, const double *__restrict__ mu, int n,
                                           int i, int j, int k)
{
    const int ip = wrap_p(i, n), im = wrap_m(i, n), jp = wrap_p(j, n), jm = wrap_m(j, n);
    const int kp = wrap_p(k, n), km = wrap_m(k, n);
    double r = 0.0;
    auto add = [&](int t, int a, int b, int c) {
        const long long q = nidx(a, b, c, n);
        r = fma(K[t][q], mu[q], r);
    };
    auto sub = [&](int t, int a, int b, int c) {
        const long long q = nidx(a, b, c, n);
        r = fma(-K[t][q], mu[q], r);
    };
    add(0, ip, j, k), add(0, im, j, k), add(1, i, jp, k), add(1, i, jm, k), add(2, i, j, kp), add(2, i, j, km);
    add(3, ip, jp, k), add(3, im, jm, k), sub(3, ip, jm, k), sub(3, im, jp, k);
    add(4, ip, j, kp), add(4, im, j, km), sub(4, ip, j, km), sub(4, im, j, kp);
    add(5, i, jp, kp), add(5, i, jm, km), sub(5, i, jp, km), sub(5, i, jm, kp);
    return r;
}

struct AdjLev {
    int n;
    double h;
    double *phi, *s, *lam[2], *rhs, *K[6], *v, *Np, *dNa, *res;
    int cur;
};

// coefficients of level l: kappa_t, N', dN/dalpha from phi_l and s_l
__global__ void __launch_bounds__(256)
k_adj_coef(const double *__restrict__ phi, const double *__restrict__ s, int n, double h, double alpha,
           double *K0, double *K1, double *K2, double *K3, double *K4, double *K5, double *Np, double *dNa)
{
    const long long cnt = (long long)n * n * n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const double h4 = h * h * h * h, qd = 1.0 / (3.0 * h4), qo = 1.0 / (8.0 * h4);
    const double sg = alpha >= 0 ? 1.0 : -1.0, aa = fabs(alpha);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) {
        int i, j, k;
        split3(q, n, n, i, j, k);
        double t[6];
        q_terms(phi, n, i, j, k, t);
        const double Q = (t[0] * t[0] + t[1] * t[1] + t[2] * t[2]) * qd + (t[3] * t[3] + t[4] * t[4] + t[5] * t[5]) * qo;
        const double sig = Q + s[q];
        const double arg = alpha * alpha + 8.0 / 3.0 * sig;
        double np = 0.0, dna = -0.75;
        if (arg > 0.0) {
            const double r = sqrt(arg);
            np = sg / r;  // dN/dSigma
            // dN/dalpha at fixed Sigma, (3/4)(-1 + sgn(alpha) alpha / r), in
            // the form that does not cancel for Sigma << alpha^2:
            // -(3/4)(8 Sigma / 3) / (r (r + |alpha|))
            dna = -2.0 * sig / (r * (r + aa));
        }
        Np[q] = np;
        dNa[q] = dna;
        // face coefficients combined per direction (see mt_apply)
        K0[q] = 2.0 * qd * (t[0] + t[1]) * np;
        K1[q] = 2.0 * qd * (t[2] - t[0]) * np;
        K2[q] = -2.0 * qd * (t[1] + t[2]) * np;
        K3[q] = 2.0 * qo * t[3] * np;
        K4[q] = 2.0 * qo * t[4] * np;
        K5[q] = 2.0 * qo * t[5] * np;
    }
}

// v = M^T 1
__global__ void __launch_bounds__(256) k_adj_v(AdjLev L)
{
    const int n = L.n;
    const long long cnt = (long long)n * n * n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const double *K[6] = {L.K[0], L.K[1], L.K[2], L.K[3], L.K[4], L.K[5]};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) {
        int i, j, k;
        split3(q, n, n, i, j, k);
        const int ip = wrap_p(i, n), im = wrap_m(i, n), jp = wrap_p(j, n), jm = wrap_m(j, n);
        const int kp = wrap_p(k, n), km = wrap_m(k, n);
        double r = 0.0;
        r += K[0][nidx(ip, j, k, n)] + K[0][nidx(im, j, k, n)] + K[1][nidx(i, jp, k, n)] + K[1][nidx(i, jm, k, n)];
        r += K[2][nidx(i, j, kp, n)] + K[2][nidx(i, j, km, n)];
        r += K[3][nidx(ip, jp, k, n)] + K[3][nidx(im, jm, k, n)] - K[3][nidx(ip, jm, k, n)] - K[3][nidx(im, jp, k, n)];
        r += K[4][nidx(ip, j, kp, n)] + K[4][nidx(im, j, km, n)] - K[4][nidx(ip, j, km, n)] - K[4][nidx(im, j, kp, n)];
        r += K[5][nidx(i, jp, kp, n)] + K[5][nidx(i, jm, km, n)] - K[5][nidx(i, jp, km, n)] - K[5][nidx(i, jm, kp, n)];
        L.v[q] = r;
    }
}

// colour-simultaneous red-black update of J^T lambda = rhs with m = <lambda>
// held fixed: lambda = (S6 - h^2 (rhs + M^T lambda - m v)) / 6.  A thread
// takes one cell of the colour (k = 2 m' + k0 in its row) and copies its
// row neighbour of the other colour into out, so that no warp splits between
// the two (n is even)
__global__ void __launch_bounds__(256)
k_adj_smooth(AdjLev L, const double *__restrict__ in, double *__restrict__ out, const double *__restrict__ mscal,
             int colour)
{
    const int n = L.n, hn = n / 2;
    const long long hc = (long long)n * n * hn;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const double m = *mscal, h2 = L.h * L.h;
    const double *K[6] = {L.K[0], L.K[1], L.K[2], L.K[3], L.K[4], L.K[5]};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < hc; t += stride) {
        int i, j, mm;
        split3(t, n, hn, i, j, mm);
        const int k0 = (colour + i + j) & 1, k = 2 * mm + k0;
        const long long q = nidx(i, j, k, n), qo = nidx(i, j, 2 * mm + 1 - k0, n);
        out[qo] = in[qo];
        const double S6 = in[nidx(wrap_p(i, n), j, k, n)] + in[nidx(wrap_m(i, n), j, k, n)] +
                          in[nidx(i, wrap_p(j, n), k, n)] + in[nidx(i, wrap_m(j, n), k, n)] +
                          in[nidx(i, j, wrap_p(k, n), n)] + in[nidx(i, j, wrap_m(k, n), n)];
        const double mt = mt_apply(K, in, n, i, j, k);
        out[q] = (S6 - h2 * (L.rhs[q] + mt - m * L.v[q])) * (1.0 / 6.0);
    }
}

// the coarsest level's sweeps in one block, lambda in shared memory (two
// buffers of the level's cnt <= ADJ_COARSE_MAX cells): per sweep m =
// <lambda> (a fixed-order block sum), then the two colour half-sweeps of
// k_adj_smooth; lambda is read from and written back to lam; *mslot ends
// with the last sweep's m
constexpr int ADJ_COARSE_MAX = 2048;
__global__ void __launch_bounds__(256) k_adj_coarsest(AdjLev L, double *lam, double *mslot, int sweeps)
{
    extern __shared__ double sbuf[];
    __shared__ double red[32];
    __shared__ double s_m;
    const int n = L.n, cnt = n * n * n, tid = threadIdx.x, nt = blockDim.x;
    double *buf[2] = {sbuf, sbuf + cnt};
    for (int q = tid; q < cnt; q += nt) buf[0][q] = lam[q];
    const double h2 = L.h * L.h;
    const double *K[6] = {L.K[0], L.K[1], L.K[2], L.K[3], L.K[4], L.K[5]};
    int cur = 0;
    for (int sw = 0; sw < sweeps; ++sw) {
        __syncthreads();
        double a[1] = {0.0};
        for (int q = tid; q < cnt; q += nt) a[0] += buf[cur][q];
        block_sum<1>(a, red);
        if (tid == 0) s_m = a[0] / (double)cnt;
        __syncthreads();
        const double m = s_m;
        for (int c = 0; c < 2; ++c) {
            const double *in = buf[cur];
            double *out = buf[1 - cur];
            for (int q = tid; q < cnt; q += nt) {
                const int k = q % n, j = (q / n) % n, i = q / (n * n);
                if (((i + j + k) & 1) != c) {
                    out[q] = in[q];
                    continue;
                }
                const double S6 = in[nidx(wrap_p(i, n), j, k, n)] + in[nidx(wrap_m(i, n), j, k, n)] +
                                  in[nidx(i, wrap_p(j, n), k, n)] + in[nidx(i, wrap_m(j, n), k, n)] +
                                  in[nidx(i, j, wrap_p(k, n), n)] + in[nidx(i, j, wrap_m(k, n), n)];
                const double mt = mt_apply(K, in, n, i, j, k);
                out[q] = (S6 - h2 * (L.rhs[q] + mt - m * L.v[q])) * (1.0 / 6.0);
            }
            __syncthreads();
            cur ^= 1;
        }
    }
    for (int q = tid; q < cnt; q += nt) lam[q] = buf[cur][q];
    if (tid == 0 && sweeps > 0) *mslot = s_m;
}

// res = rhs - J^T lambda with m = *mptr (= <lambda>, or 0 if mptr is
// NULL); out3[0] = sum res^2, out3[1] = <lambda>; writes res
__global__ void __launch_bounds__(256)
k_adj_resid(AdjLev L, const double *__restrict__ lam, const double *__restrict__ mptr, double *res, RedBuf rb,
            double *out3)
{
    const int n = L.n;
    const long long cnt = (long long)n * n * n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const double inv_h2 = 1.0 / (L.h * L.h);
    const double *K[6] = {L.K[0], L.K[1], L.K[2], L.K[3], L.K[4], L.K[5]};
    const double m = mptr ? *mptr : 0.0;
    double acc[2] = {0.0, 0.0};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) {
        int i, j, k;
        split3(q, n, n, i, j, k);
        const double S6 = lam[nidx(wrap_p(i, n), j, k, n)] + lam[nidx(wrap_m(i, n), j, k, n)] +
                          lam[nidx(i, wrap_p(j, n), k, n)] + lam[nidx(i, wrap_m(j, n), k, n)] +
                          lam[nidx(i, j, wrap_p(k, n), n)] + lam[nidx(i, j, wrap_m(k, n), n)];
        const double Av = (S6 - 6.0 * lam[q]) * inv_h2 - mt_apply(K, lam, n, i, j, k) + m * L.v[q];
        const double r = L.rhs[q] - Av;
        res[q] = r;
        acc[0] += r * r;
        acc[1] += lam[q];
    }
    double tot[2];
    if (grid_sum<2>(acc, rb, tot) && threadIdx.x == 0) {
        out3[0] = tot[0];
        out3[1] = tot[1] / (double)cnt;
    }
}

__global__ void __launch_bounds__(256) k_mean_into(const double *__restrict__ x, long long cnt, double *out, RedBuf rb)
{
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) acc[0] += x[q];
    double tot[1];
    if (grid_sum<1>(acc, rb, tot) && threadIdx.x == 0) *out = tot[0] / (double)cnt;
}

// natural-layout 8-cell average and 27/9/3/1 prolongation (Sec. 3.2.1)
__global__ void __launch_bounds__(256) k_restrict_nat(const double *__restrict__ f, int nf, double *c)
{
    const int nc = nf / 2;
    const long long cnt = (long long)nc * nc * nc;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) {
        int I, J, K;
        split3(q, nc, nc, I, J, K);
        double a = 0.0;
        for (int d = 0; d < 8; ++d) a += f[nidx(2 * I + (d >> 2), 2 * J + ((d >> 1) & 1), 2 * K + (d & 1), nf)];
        c[q] = a * 0.125;
    }
}

__global__ void __launch_bounds__(256) k_prolong_nat(double *f, int nf, const double *__restrict__ c)
{
    const int nc = nf / 2;
    const long long cnt = (long long)nf * nf * nf;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) {
        int i, j, k;
        split3(q, nf, nf, i, j, k);
        const int I = i >> 1, J = j >> 1, K = k >> 1;
        const int I2 = (i & 1) ? (I + 1 == nc ? 0 : I + 1) : (I == 0 ? nc - 1 : I - 1);
        const int J2 = (j & 1) ? (J + 1 == nc ? 0 : J + 1) : (J == 0 ? nc - 1 : J - 1);
        const int K2 = (k & 1) ? (K + 1 == nc ? 0 : K + 1) : (K == 0 ? nc - 1 : K - 1);
        const double v = 27.0 * c[nidx(I, J, K, nc)] +
                         9.0 * (c[nidx(I2, J, K, nc)] + c[nidx(I, J2, K, nc)] + c[nidx(I, J, K2, nc)]) +
                         3.0 * (c[nidx(I2, J2, K, nc)] + c[nidx(I2, J, K2, nc)] + c[nidx(I, J2, K2, nc)]) +
                         c[nidx(I2, J2, K2, nc)];
        f[q] += v * (1.0 / 64.0);
    }
}

// gradient pieces: grad_s = N' (lambda - m); dR partial sums
__global__ void __launch_bounds__(256)
k_adj_grad(const double *__restrict__ lam, const double *__restrict__ Np, const double *__restrict__ dNa,
           const double *__restrict__ delta, const double *__restrict__ mscal, long long cnt, double dmean,
           double ks, double alpha_p, double ds_coef, double *out, RedBuf rb, double *dR)
{
    const double m = *mscal;
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride) {
        const double l = lam[q] - m;
        out[q] = ks * Np[q] * l;
        acc[0] += l * (dNa[q] * alpha_p + Np[q] * ds_coef * (delta[q] - dmean));
    }
    double tot[1];
    if (grid_sum<1>(acc, rb, tot) && threadIdx.x == 0) *dR = tot[0];
}

__global__ void __launch_bounds__(256) k_axpy_nat(double *y, const double *__restrict__ x, double a, double b,
                                                  long long cnt, const double *__restrict__ mean)
{
    const double mu = mean ? *mean : 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += stride)
        y[q] = a * y[q] + b * (x[q] - mu);
}

static int g1(long long n) { return (int)std::max<long long>(1, std::min<long long>(1024, (n + 255) / 256)); }

struct AdjWork {
    int n0 = 0;
    std::vector<AdjLev> L;
    std::vector<void *> blocks;
    double *scal = nullptr;   // [0..2]: sums, [8..]: per level m
    RedBuf rb{};
    // one captured cycle (V-cycle, residual pass, copy of its sums to the
    // pinned scratch) for the sweep counts it was captured with
    cudaGraphExec_t cycle = nullptr;
    int cycle_key[3] = {-1, -1, -1};
};

static void adj_free(AdjWork *w)
{
    if (!w) return;
    if (w->cycle) cudaGraphExecDestroy(w->cycle);
    for (void *p : w->blocks) cudaFree(p);
    if (w->scal) cudaFree(w->scal);
    delete w;
}

static AdjWork *adj_alloc(mg_ctx *ctx, int n)
{
    AdjWork *w = new AdjWork();
    w->n0 = n;
    const int nl = (int)level_count(n);
    for (int l = 0; l < nl; ++l) {
        AdjLev a{};
        a.n = n >> l;
        a.h = (double)(1 << l);
        const size_t cnt = (size_t)a.n * a.n * a.n;
        double *b = nullptr;
        MG_CK(cudaMalloc(&b, sizeof(double) * cnt * 17));
        w->blocks.push_back(b);
        a.phi = b;
        a.s = b + cnt;
        a.lam[0] = b + 2 * cnt;
        a.lam[1] = b + 3 * cnt;
        a.rhs = b + 4 * cnt;
        for (int t = 0; t < 6; ++t) a.K[t] = b + (5 + t) * cnt;
        a.v = b + 11 * cnt;
        a.Np = b + 12 * cnt;
        a.dNa = b + 13 * cnt;
        a.res = b + 14 * cnt;
        a.cur = 0;
        w->L.push_back(a);
    }
    MG_CK(cudaMalloc(&w->scal, sizeof(double) * (64 + 4 * MAX_RED_BLOCKS) + 256));
    MG_CK(cudaMemset(w->scal, 0, sizeof(double) * (64 + 4 * MAX_RED_BLOCKS) + 256));
    w->rb.partials = w->scal + 64;
    w->rb.counter = (unsigned int *)(w->rb.partials + 4 * MAX_RED_BLOCKS);
    w->rb.cap = MAX_RED_BLOCKS;
    return w;
}

// one linear V-cycle on level l for J^T e = rhs_l (e in lam[cur])
static void adj_vcycle(mg_ctx *ctx, AdjWork &w, int l, const mg_opts &o)
{
    cudaStream_t s = ctx->stream;
    AdjLev &A = w.L[l];
    const long long cnt = (long long)A.n * A.n * A.n;
    double *mslot = w.scal + 8 + l;
    auto sweep = [&]() {
        for (int c = 0; c < 2; ++c) {
            k_adj_smooth<<<g1(cnt / 2), 256, 0, s>>>(A, A.lam[A.cur], A.lam[1 - A.cur], mslot, c);
            A.cur ^= 1;
        }
    };
    const bool coarsest = l + 1 == (int)w.L.size();
    const int sweeps = coarsest ? o.coarse_sweeps : o.pre;
    if (coarsest && cnt <= ADJ_COARSE_MAX) {
        // (2 sweeps per sweep flip A.cur twice: the result stays in A.lam[A.cur])
        k_adj_coarsest<<<1, 256, 2 * sizeof(double) * cnt, s>>>(A, A.lam[A.cur], mslot, sweeps);
        return;
    }
    for (int q = 0; q < sweeps; ++q) {
        k_mean_into<<<g1(cnt), 256, 0, s>>>(A.lam[A.cur], cnt, mslot, w.rb);
        sweep();
    }
    if (coarsest) return;
    // residual (m = <lambda> of the current field), restrict as the coarse rhs
    k_mean_into<<<g1(cnt), 256, 0, s>>>(A.lam[A.cur], cnt, mslot, w.rb);
    k_adj_resid<<<g1(cnt), 256, 0, s>>>(A, A.lam[A.cur], mslot, A.res, w.rb, w.scal);
    AdjLev &C = w.L[l + 1];
    const long long cc = (long long)C.n * C.n * C.n;
    k_restrict_nat<<<g1(cc), 256, 0, s>>>(A.res, A.n, C.rhs);
    MG_CK(cudaMemsetAsync(C.lam[C.cur], 0, sizeof(double) * cc, s));
    MG_CK(cudaMemsetAsync(w.scal + 8 + l + 1, 0, sizeof(double), s));
    adj_vcycle(ctx, w, l + 1, o);
    k_prolong_nat<<<g1(cnt), 256, 0, s>>>(A.lam[A.cur], A.n, C.lam[C.cur]);
    for (int q = 0; q < o.post; ++q) {
        k_mean_into<<<g1(cnt), 256, 0, s>>>(A.lam[A.cur], cnt, mslot, w.rb);
        sweep();
    }
}

void adj_release(mg_ctx *ctx)
{
    if (ctx && ctx->adj) {
        adj_free((AdjWork *)ctx->adj);
        ctx->adj = nullptr;
    }
}

// the adjoint solve on device arrays (validated arguments): dL/ddelta into
// dout, dL/dR_c into *drc; CUDA failures throw CudaFail
int adjoint_dev(mg_ctx *ctx, int n, double a, double om, double Rc, const mg_opts &o, const double *dphi,
                const double *ddel, const double *dg, double *dout, double *drc, mg_stats *st)
{
    mg_stats loc{};
    cudaStream_t s = ctx->stream;
    const long long cnt = (long long)n * n * n;
    const size_t b = sizeof(double) * (size_t)cnt;
    // workspace (one per context, reallocated when the size changes)
    AdjWork *w = (AdjWork *)ctx->adj;
    if (w && w->n0 != n) {
        MG_CK(cudaStreamSynchronize(s));
        adj_free(w);
        w = nullptr;
        ctx->adj = nullptr;
    }
    if (!w) {
        w = adj_alloc(ctx, n);
        ctx->adj = w;
    }
    // background scalars (Eq. beta_dgp) and their R_c derivatives
    const double oma = om / (a * a * a), ol = 1.0 - om;
    const double B0 = (oma + 2.0 * ol) / std::sqrt(oma + ol);   // beta = 1 + Rc B0
    const double beta = 1.0 + Rc * B0, beta_p = B0;
    const double alpha = 3.0 * beta * a * a / (Rc * Rc);
    const double alpha_p = 3.0 * a * a * (beta_p / (Rc * Rc) - 2.0 * beta / (Rc * Rc * Rc));
    const double ks = (alpha / beta) * om / a;
    const double ks_p = ((alpha_p * beta - alpha * beta_p) / (beta * beta)) * om / a;
    double *dscr = w->scal;
    // level 0: phi, s = ks (delta - <delta>), rhs = Pi g
    AdjLev &A0 = w->L[0];
    MG_CK(cudaMemcpyAsync(A0.phi, dphi, b, cudaMemcpyDeviceToDevice, s));
    k_mean_into<<<g1(cnt), 256, 0, s>>>(ddel, cnt, dscr + 4, w->rb);
    MG_CK(cudaMemsetAsync(A0.s, 0, b, s));
    k_axpy_nat<<<g1(cnt), 256, 0, s>>>(A0.s, ddel, 0.0, ks, cnt, dscr + 4);
    k_mean_into<<<g1(cnt), 256, 0, s>>>(dg, cnt, dscr + 5, w->rb);
    MG_CK(cudaMemsetAsync(A0.rhs, 0, b, s));
    k_axpy_nat<<<g1(cnt), 256, 0, s>>>(A0.rhs, dg, 0.0, 1.0, cnt, dscr + 5);
    for (size_t l = 0; l < w->L.size(); ++l) {
        AdjLev &L = w->L[l];
        const long long c = (long long)L.n * L.n * L.n;
        if (l > 0) {
            k_restrict_nat<<<g1(c), 256, 0, s>>>(w->L[l - 1].phi, w->L[l - 1].n, L.phi);
            k_restrict_nat<<<g1(c), 256, 0, s>>>(w->L[l - 1].s, w->L[l - 1].n, L.s);
        }
        k_adj_coef<<<g1(c), 256, 0, s>>>(L.phi, L.s, L.n, L.h, alpha, L.K[0], L.K[1], L.K[2], L.K[3], L.K[4],
                                         L.K[5], L.Np, L.dNa);
        k_adj_v<<<g1(c), 256, 0, s>>>(L);
    }
    MG_CK(cudaMemsetAsync(A0.lam[A0.cur], 0, b, s));
    MG_CK(cudaMemsetAsync(dscr + 8, 0, sizeof(double) * 32, s));
    // reference norm: rms(Pi g)
    k_adj_resid<<<g1(cnt), 256, 0, s>>>(A0, A0.lam[A0.cur], nullptr, A0.res, w->rb, dscr);
    double h3[3];
    MG_CK(cudaMemcpyAsync(h3, dscr, sizeof h3, cudaMemcpyDeviceToHost, s));
    MG_CK(cudaStreamSynchronize(s));
    const double ref = std::sqrt(h3[0] / (double)cnt);
    loc.eps_ref = ref;
    loc.eps[0] = ref;
    loc.n_eps = 1;
    int cyc = 0;
    bool conv = ref <= o.atol || ref == 0.0;
    // every sweep flips a level's buffer twice, so a cycle leaves the buffer
    // state as it found it and one captured cycle replays every cycle
    auto record = [&]() {
        adj_vcycle(ctx, *w, 0, o);
        k_mean_into<<<g1(cnt), 256, 0, s>>>(A0.lam[A0.cur], cnt, dscr + 8, w->rb);
        k_adj_resid<<<g1(cnt), 256, 0, s>>>(A0, A0.lam[A0.cur], dscr + 8, A0.res, w->rb, dscr);
        MG_CK(cudaMemcpyAsync(ctx->hpin, dscr, sizeof h3, cudaMemcpyDeviceToHost, s));
    };
    const int key[3] = {o.pre, o.post, o.coarse_sweeps};
    if (o.use_graph && (!w->cycle || std::memcmp(key, w->cycle_key, sizeof key) != 0)) {
        if (w->cycle) {
            MG_CK(cudaGraphExecDestroy(w->cycle));
            w->cycle = nullptr;
        }
        cudaGraph_t g = nullptr;
        MG_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        record();
        MG_CK(cudaStreamEndCapture(s, &g));
        MG_CK(cudaGraphInstantiate(&w->cycle, g, 0));
        MG_CK(cudaGraphDestroy(g));
        std::memcpy(w->cycle_key, key, sizeof key);
    }
    while (!conv && cyc < o.max_cycles) {
        if (o.use_graph)
            MG_CK(cudaGraphLaunch(w->cycle, s));
        else
            record();
        ++cyc;
        MG_CK(cudaStreamSynchronize(s));
        std::memcpy(h3, ctx->hpin, sizeof h3);
        const double eps = std::sqrt(h3[0] / (double)cnt);
        if (loc.n_eps < 65) loc.eps[loc.n_eps++] = eps;
        if (!std::isfinite(eps)) {
            if (st) *st = loc;
            return set_err(ctx, MG_ERR_NONFINITE, "adjoint: non-finite residual");
        }
        conv = eps <= o.rtol * ref + o.atol;
    }
    // gradients
    double hmean[2];
    MG_CK(cudaMemcpyAsync(hmean, dscr + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
    MG_CK(cudaStreamSynchronize(s));
    k_mean_into<<<g1(cnt), 256, 0, s>>>(A0.lam[A0.cur], cnt, dscr + 8, w->rb);
    k_adj_grad<<<g1(cnt), 256, 0, s>>>(A0.lam[A0.cur], A0.Np, A0.dNa, ddel, dscr + 8, cnt, hmean[0], ks, alpha_p,
                                       ks_p, dout, w->rb, dscr + 6);
    k_mean_into<<<g1(cnt), 256, 0, s>>>(dout, cnt, dscr + 7, w->rb);
    k_axpy_nat<<<g1(cnt), 256, 0, s>>>(dout, dout, 0.0, 1.0, cnt, dscr + 7);
    double hdr = 0.0;
    MG_CK(cudaMemcpyAsync(&hdr, dscr + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
    MG_CK(cudaStreamSynchronize(s));
    if (drc) *drc = hdr;
    loc.cycles = cyc;
    const int rc = conv ? MG_OK : MG_WARN_NOT_CONVERGED;
    loc.status = rc;
    if (st) *st = loc;
    return rc;
}

}  // namespace mg

using namespace mg;

extern "C" int mg_solve_adjoint(mg_ctx *ctx, const mg_grid *g, const mg_dgp_params *p, const mg_opts *opts,
                                const double *phi, const double *delta, const double *dL_dphi,
                                double *dL_ddelta_out, double *dL_drc_out, mg_stats *stats)
{
    if (!ctx) return MG_ERR_ARG;
    if (!g || !p || !phi || !delta || !dL_dphi || !dL_ddelta_out) return set_err(ctx, MG_ERR_ARG, "null argument");
    if (!valid_ng(g->ng)) return set_err(ctx, MG_ERR_ARG, "ng = %d is not 2^k or 3*2^k in [8, 1536]", g->ng);
    if (!(g->a > 0) || !(g->omega_m > 0) || !(p->rc_h0 > 0)) return set_err(ctx, MG_ERR_ARG, "bad parameters");
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
        const int n = g->ng;
        const size_t b = sizeof(double) * (size_t)n * n * n;
        const double *dphi = (const double *)stage_in(ctx, 0, phi, b, true);
        const double *ddel = (const double *)stage_in(ctx, 1, delta, b, true);
        const double *dg = (const double *)stage_in(ctx, 2, dL_dphi, b, true);
        double *dout = (double *)stage_in(ctx, 3, dL_ddelta_out, b, false);
        double hdr = 0.0;
        rc = adjoint_dev(ctx, n, g->a, g->omega_m, p->rc_h0, o, dphi, ddel, dg, dout, &hdr, &loc);
        if (rc >= 0) {
            stage_out(ctx, dL_ddelta_out, dout, b);
            if (dL_drc_out) *dL_drc_out = hdr;
        }
        leave(ctx);
    } catch (CudaFail &f) {
        return f.code;
    }
    if (stats) *stats = loc;
    return rc;
}
