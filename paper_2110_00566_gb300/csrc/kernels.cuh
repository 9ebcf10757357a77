// Launchers of the multigrid kernels (kernels.cu), templated on the storage
// type T (double or float).  All launches go to the given stream.  A level
// whose base[] arrays are set runs the correction form (unknown e, frozen
// base field b, operator N(b + e) - N(b)) used inside the mixed-precision
// solve; otherwise the plain operator N(u).
#pragma once
#include "common.cuh"

namespace mg {

// arrays of one level, colour-split (index 0/1 = colour)
template <typename T>
struct LevArrays {
    int n, half;
    long long ncol;      // elements per colour array = n*n*n/2
    double h;
    T *u[2][2];          // [buffer][colour]
    int cur[2];          // current buffer of each colour
    T *s[2];             // density term
    T *f[2];             // active FAS source f' (nullptr on a finest level)
    T *fbuf[2];          // storage behind f
    T *ur[2];            // R u saved for the correction
    T *base[2];          // correction form: base field (nullptr: plain form)
    LevScal *sc;         // this level's device scalars
    int model = -1;      // operator of the uploaded OpK (0 nDGP, 1 Kmouflage), -1 unknown
    int qbx = 0;         // FP32 four-cell smoother: threads along a row (autotuned; 0 = default)
    int qstream = 0;     // FP32 streaming smoother variant (autotuned; <= 0: the gathering kernel)
    int qz = 1;          // FP32 four-cell smoother: planes per block (autotuned)
    T *U(int colour) const { return u[cur[colour]][colour]; }
};

template <typename T> OpK<T> make_opk(int model, double alpha, int nkmo, double gamma, double bterm);


template <typename T>
void launch_smooth(const LevArrays<T> &L, LevArrays<T> *Lw, const OpK<T> *op, int colour, cudaStream_t st);
template <typename T>
void launch_smooth_shape(const LevArrays<T> &L, const OpK<T> *op, int colour, int bx, cudaStream_t st);
// FP32 four-cell half-sweep with bx threads along a row (256 / bx rows) and
// zc planes per block into the alternate buffer, leaving the buffer state
// untouched (autotuner); false when the level does not use the four-cell
// kernel
bool launch_smooth4_shape(const LevArrays<float> &L, const OpK<float> *op, int colour, int bx, int zc,
                          cudaStream_t st);
// FP64 nDGP half-sweep with the stencil staged once per block in shared
// memory as block fixed point (smooth_bfp.cu), into buffer nb; false when
// the level is not eligible (correction form, Kmouflage, half % 32 != 0 or
// n % 8 != 0)
bool launch_smooth_bfp(const LevArrays<double> &L, const LevK<double> &K, const OpK<double> *op, int colour, int nb,
                       cudaStream_t st);
// FP64 nDGP residual passes with the stencil staged in shared memory as
// block fixed point (resid_bfp.cu): the fused residual/restriction into the
// coarse level Lc, and the residual norm (with D set, -d as FP32); false when
// the level is not eligible (as launch_smooth_bfp)
bool launch_resid_restrict_bfp(const LevArrays<double> &Lf, LevArrays<double> &Lc, const OpK<double> *op,
                               const RedBuf &rb, cudaStream_t st);
bool launch_resid_norm_bfp(const LevArrays<double> &L, const OpK<double> *op, const RedBuf &rb, cudaStream_t st,
                           float *const *D, bool zero_u);
// the coarse level's FAS source (Eq. general_pde_numerical_coarse) on the
// block-staged kernel (resid_bfp.cu); false when the coarse level is not
// eligible
bool launch_coarse_source_bfp(const LevArrays<double> &Lf, const LevArrays<double> &Lc, const OpK<double> *op,
                              const RedBuf &rb, cudaStream_t st);
// FP64 prolongation of the coarse correction held in Lc.ur (formed by the
// coarse-correction pass) with the coarse planes staged in shared memory as
// block fixed point (prolong_bfp.cu); false when the fine level is not
// eligible (n < 128, rows not a multiple of 64 long)
bool launch_prolong_bfp(const LevArrays<double> &Lf, const LevArrays<double> &Lc, cudaStream_t st);
// streaming FP32 four-cell half-sweep (shared-memory plane ring fed by bulk
// asynchronous copies) for n = 256 and 512: variants 1 .. stream_variants()
// (ring depth and planes per block); false when the level is not eligible
int stream_variants();
void stream_setup();   // shared-memory limits of the streaming kernels (once)
bool stream_eligible(const LevArrays<float> &L);
bool launch_smooth_stream(const LevArrays<float> &L, const LevK<float> &K, const OpK<float> *op, int colour, int nb,
                          int variant, cudaStream_t st);
// the streaming kernel's timeout flag (1 if a bounded wait gave up since the
// last reset, -1 on a CUDA error); synchronises the stream
int stream_timeout_flag(cudaStream_t st, bool reset);
// residual norm; with D set also writes -d (with the old c) as FP32,
// colour-split; zero_u: the level's u is known to be zero everywhere (the
// same result from the source alone, without the stencil)
template <typename T>
void launch_resid_norm(const LevArrays<T> &L, const OpK<T> *op, const RedBuf &rb, cudaStream_t st,
                       float *const *D = nullptr, bool zero_u = false);
template <typename T>
void launch_resid_restrict(const LevArrays<T> &Lf, LevArrays<T> &Lc, const OpK<T> *op, const RedBuf &rb,
                           cudaStream_t st);
template <typename T>
void launch_coarse_source(const LevArrays<T> &Lf, const LevArrays<T> &Lc, const OpK<T> *op, const RedBuf &rb,
                          cudaStream_t st);
template <typename T>
void launch_prolong(const LevArrays<T> &Lf, const LevArrays<T> &Lc, cudaStream_t st);
// kernels launch_prolong launches for the fine level Lf (1 or 2)
template <typename T>
int prolong_kernels(const LevArrays<T> &Lf);
template <typename T>
void launch_coarsest(const LevArrays<T> &L, const OpK<double> *op, int sweeps, cudaStream_t st);
template <typename T>
void launch_restrict_plain(T *const fine[2], int nf, T *const coarse[2], cudaStream_t st);

// natural FP64 <-> colour-split T
template <typename T>
void launch_split(const double *nat, int n, T *const dst[2], double scale, const double *mean, cudaStream_t st);
template <typename T>
void launch_merge(T *const src[2], int n, double *nat, const double *mean, cudaStream_t st);
// mean of a natural FP64 array -> *out_mean (device)
void launch_mean_nat(const double *x, long long cnt, double *out_mean, const RedBuf &rb, cudaStream_t st);
// mean of a colour-split array -> *out_mean (device)
template <typename T>
void launch_mean_split(T *const a[2], long long ncol, double *out_mean, const RedBuf &rb, cudaStream_t st);
// rms of scale * (x - mean) for a natural FP64 array -> *out (device)
void launch_rms_nat(const double *x, long long cnt, double scale, const double *mean, double *out, const RedBuf &rb,
                    cudaStream_t st);

// element-wise helpers on colour-split arrays
template <typename Td, typename Ts>
void launch_convert(Td *const dst[2], Ts *const src[2], long long ncol, cudaStream_t st);
// U += (double) E
void launch_add_correction(double *const U[2], float *const E[2], long long ncol, cudaStream_t st);
// correction pyramid scalars: all zero except fshift of level 0 = -dc of
// the FP64 defect pass (the defect's compatibility shift)
void launch_set_corr_scalars(LevScal *sc32, const LevScal *sc64, int nlev32, cudaStream_t st);

}  // namespace mg
