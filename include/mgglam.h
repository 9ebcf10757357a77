/*
 * mgglam.h -- C-ABI of libmgglam.so, the GB300 (sm_103a) implementation of
 * the MG-GLAM derivative-coupling field solvers of Hernandez-Aguayo et al.,
 * "Fast full N-body simulations of generic modified gravity: derivative
 * coupling models" (arXiv:2110.00566).
 *
 * Conventions for every call below
 * --------------------------------
 *  - Code units of the paper's Sec. 3.1.1: a mesh of ng^3 cells of size
 *    h = 1 on the finest level; positions x~ in [0, ng); potentials
 *    Phi~ = (ng/(H0 L))^2 Phi; the nDGP field phi~ in the same unit; the
 *    Kmouflage field phi~ = c~ phi (Eq. Kmo_unit), c~ = (c/H0) ng / L.
 *  - Mesh arrays are C-ordered (i, j, k) with k fastest, ng^3 elements, cell
 *    (i, j, k) centred at (i+1/2, j+1/2, k+1/2).  Particle arrays are np x 3.
 *  - Pointers may be device pointers on the context's device or host
 *    pointers (pageable or pinned); the library detects which with
 *    cudaPointerGetAttributes and stages host data through its own device
 *    workspace.  All arrays are owned by the caller; the library owns only
 *    the workspace inside mg_ctx (level pyramids, staging and reduction
 *    buffers, CUDA graphs), allocated on first use for a given mesh size
 *    and precision and kept until mg_ctx_destroy.
 *  - Calls are issued on the context's stream.  Calls that return a
 *    statistics record synchronise that stream before returning; the
 *    others return once the work is queued (device pointers) or done (host
 *    pointers).  One context must not be used from two host threads at once.
 *  - Return value: MG_OK (0), a warning (> 0: the result is valid), or an
 *    error (< 0: the outputs are unspecified); mg_last_error_string() gives
 *    the detail of the last error or warning.
 */
#ifndef MGGLAM_H
#define MGGLAM_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------- */
#define MG_OK                   0
#define MG_WARN_NOT_CONVERGED   1   /* max_cycles reached; phi still returned */
#define MG_ERR_ARG             -1   /* null pointer, unsupported size, bad option */
#define MG_ERR_CUDA            -2   /* a CUDA runtime or cuFFT call failed */
#define MG_ERR_TIMEOUT         -3   /* a bounded device-side wait gave up */
#define MG_ERR_NONFINITE       -4   /* NaN/Inf in an input or a residual norm */
#define MG_ERR_OOM             -5   /* device workspace allocation failed */

/* ---- context ---------------------------------------------------------- */
typedef struct mg_ctx mg_ctx;

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to
 * issue all work on, or NULL to let the context create its own.
 * Errors: MG_ERR_ARG (out == NULL), MG_ERR_CUDA (bad device). */
int mg_ctx_create(mg_ctx **out, int device, void *cuda_stream);

/* Free the workspace and the context (a NULL argument is ignored). */
void mg_ctx_destroy(mg_ctx *ctx);

/* Detail of the last error or warning of this context (never NULL). */
const char *mg_last_error_string(const mg_ctx *ctx);

/* Device bytes currently held by the context's workspace. */
long long mg_ctx_workspace_bytes(const mg_ctx *ctx);

/* on != 0: bracket every finest-level smoother launch of the following
 * solves with CUDA events (recorded inside the captured cycle graphs) and
 * report their summed device time in mg_stats.fine_smooth_ms.  Returns
 * MG_OK or MG_ERR_ARG (ctx == NULL). */
int mg_ctx_set_profiling(mg_ctx *ctx, int on);

/* Choice of the FP32 half-sweep kernel on the 256^3 and 512^3 levels of the
 * mixed-precision solve: 0 (default) = autotuned per level on first use
 * between the gathering kernel (rows read through L1/L2) and the streaming
 * kernel (planes staged in shared memory by bulk asynchronous copies);
 * -1 = gathering kernel only; k >= 1 = streaming variant k (ring depth and
 * planes per block; at most mg_fp32_smoother_variants()).  Both kernels
 * give bit-identical fields.  Resets the tuning and the cached cycle graphs.
 * Errors: MG_ERR_ARG. */
int mg_ctx_set_fp32_smoother(mg_ctx *ctx, int choice);
int mg_fp32_smoother_variants(void);

/* Pins the gathering FP32 half-sweep's shape on levels of size n (the
 * autotuner otherwise picks it on first use): bx threads along a row
 * (8, 16, 32 or 64, with 4 bx <= n/2; 256 / bx rows per block) and zc
 * consecutive planes per block (zc >= 1); bx = 0 removes the pin.  For
 * profiling and reproducible launch configurations; the streaming kernel
 * is still tried against it under mg_ctx_set_fp32_smoother(0).  Resets the
 * tuning and the cached cycle graphs.  Errors: MG_ERR_ARG. */
int mg_ctx_set_fp32_smoother_shape(mg_ctx *ctx, int n, int bx, int zc);

/* Measured FP64 and FP32 fused multiply-add throughput of the context's
 * device in TFLOP/s (an FMA counts 2), from eight independent FMA chains
 * per thread on 16 CTAs per SM: the denominator for kernels bound by plain
 * ALU arithmetic.  Either output may be NULL.  Blocks until done.  (The
 * paper has no counterpart; this is measurement support.) */
int mg_probe_alu_peaks(mg_ctx *ctx, double *fp64_tflops, double *fp32_tflops);

/* Accuracy probe of the FP64 arithmetic the FP64 nDGP kernels use in place
 * of CUDA's IEEE square root and division (those issue many instructions on
 * this GPU's narrow FP64 pipe): y[q] = f(x[q]) for q < n, with
 *   fn = 0: the square root (one Heron step on a single-precision
 *           reciprocal-square-root estimate; relative error below 2^-43 for
 *           positive normal x),
 *   fn = 1: the reciprocal 1/x (single-precision estimate and one corrected
 *           quotient; relative error below 2^-43 for positive normal x below
 *           2^1022),
 *   fn = 2: N(Sigma) of Eq. DGP, the Vainshtein term, at Sigma = x[q] for the
 *           given alpha, N = (3/4)[-alpha + sgn(alpha) sqrt(alpha^2 + 8 Sigma/3)],
 *           as the kernels evaluate it (a cell with Q = 0 and density term
 *           Sigma): an FP32 estimate of the rationalised form
 *           2 sgn(alpha) Sigma / (|alpha| + sqrt(...)) refined by one FP64
 *           Newton step on Eq. dgp_quadratic_eom, (2/3) N^2 + alpha N = Sigma
 *           (relative error about 2^-44 where the root's square root is at
 *           least |alpha|/2), else the rationalised form in FP64 with the
 *           square root and reciprocal of fn 0 and 1 (arguments below zero
 *           give -(3/4) alpha).
 * x, y: device arrays of n doubles on the context's device (host pointers
 * are rejected); alpha: finite and nonzero (read for fn = 2 only).  Queued
 * on the context's stream.  Errors: MG_ERR_ARG, MG_ERR_CUDA.  (The paper has
 * no counterpart; this is test support for the kernels' arithmetic.) */
int mg_probe_fp64_math(mg_ctx *ctx, int fn, const double *x, double *y, long long n, double alpha);

/* ---- problem description (Sec. 3.1.1, 3.2.3, 3.2.4) ------------------- */
typedef struct {
    int ng;            /* cells per side: 2^k or 3 * 2^k, 8 <= ng <= 1536
                          (levels halve to a 4^3 or 6^3 coarsest mesh, Sec.
                          3.2.1; above 1536 MG_ERR_ARG)                       */
    double box_mpch;   /* box side L in Mpc/h                                  */
    double a;          /* scale factor                                         */
    double omega_m;    /* present-day matter density parameter                 */
} mg_grid;

/* nDGP: R_c = H0 r_c / c (Sec. 3.2.3); beta_DGP(a) of Eq. beta_dgp for the
 * LCDM-matched background and alpha = 3 beta a^2 / R_c^2 are derived. */
typedef struct {
    double rc_h0;
} mg_dgp_params;

/* Kmouflage, K(X) = -1 + X + K0 X^n, A = exp(beta phi) (Sec. 2.2, 3.2.4):
 * gamma = n K0 (1/(2 a^2 lambda^2))^(n-1) is derived; lambda, the
 * background phibar'/H0 and A(phibar) are inputs, which
 * mg_kmo_background computes. */
typedef struct {
    int n;                        /* exponent, n >= 2                          */
    double k0;                    /* K0 >= 0                                   */
    double beta_kmo;              /* coupling beta_Kmo                         */
    double lambda;                /* lambda of Lambda^4/M_Pl^2 = H0^2 lambda^2 */
    double phibar_prime_over_h0;  /* phibar' / H0 (conformal-time derivative)  */
    double A_bar;                 /* A(phibar)                                 */
} mg_kmo_params;

/* ---- Kmouflage background (Sec. 3.2.4, background solver) ------------- */

/* Model and cosmology of the background solve.  Omega_r is that of photons
 * at t_cmb plus n_eff massless neutrino species (Omega_gamma from the
 * black-body density over 3 (100 h km/s/Mpc)^2 / (8 pi G)). */
typedef struct {
    int n;              /* K(X) = -1 + X + K0 X^n, n >= 2                      */
    double k0;          /* K0 >= 0                                            */
    double beta_kmo;    /* A(phi) = exp(beta phi)                             */
    double omega_m, h;  /* Omega_m; H0 = 100 h km/s/Mpc                       */
    double t_cmb;       /* K (0: no radiation)                                */
    double n_eff;       /* massless neutrino species                          */
    double a_ini;       /* start of the integration, 0 < a_ini < 1            */
    double phi_ini;     /* phibar at a_ini                                    */
    double dphi_ini;    /* d phibar / d ln a at a_ini                         */
    double rtol;        /* local relative error per step of the integrator    */
    double h0_tol;      /* |H(a=1)/H0 - 1| accepted by the lambda shooting    */
} mg_kmo_background_params;

/* Defaults: n = 2, K0 = 1, beta = 0.2, Omega_m = 0.3089, h = 0.6774,
 * t_cmb = 2.7255, n_eff = 3.046, a_ini = 1e-5 (z = 1e5), phi_ini =
 * dphi_ini = 1e-30, rtol = 1e-12, h0_tol = 1e-12.  Errors: MG_ERR_ARG. */
int mg_kmo_background_defaults(mg_kmo_background_params *p);

/*
 * HOST.  The background of the Kmouflage model: the field equation (Eq.
 * kmf_background_eom2) integrated in N = ln a from a_ini with an adaptive
 * Dormand-Prince 5(4) Runge-Kutta pair, the conformal Hubble rate at each
 * point taken from the Friedmann equation (Eq. kmf_background_Friedmann,
 * a polynomial in (H/H0)^2 solved by Newton's method on its LCDM-connected
 * branch) and its derivative from the acceleration equation a''/a =
 * -(4 pi G/3)(rho + 3p) with the scalar's energy density and pressure.
 * lambda: if lambda_in > 0 it is used as given; otherwise it is found by
 * shooting (Illinois regula falsi) so that H(a = 1) = H0 to h0_tol.
 * a: na > 0 host scale factors, each in [a_ini, 100], any order.
 * out: host, na x 5 doubles, row i for a[i]:
 *   [H/H0, phibar, d phibar / d a, A(phibar), phibar'/H0]
 * (phibar' the conformal-time derivative: the mg_kmo_params input).
 * lambda_out: host scalar (may be NULL).
 * Returns MG_OK, MG_WARN_NOT_CONVERGED (the shooting did not reach h0_tol;
 * the table is that of the last lambda), MG_ERR_ARG or MG_ERR_NONFINITE
 * (the Friedmann equation lost its real root, or the integrator failed).
 */
int mg_kmo_background(const mg_kmo_background_params *p, double lambda_in, int na,
                      const double *a, double *out, double *lambda_out);

/* ---- solver options ---------------------------------------------------- */
#define MG_CYCLE_V 0
#define MG_CYCLE_F 1
#define MG_CYCLE_W 2
#define MG_PREC_FP64  0   /* every level in FP64                             */
#define MG_PREC_MIXED 1   /* FP32 FAS cycles on the correction, FP64
                             finest-level defect, norms and coarsest solve   */

typedef struct {
    int pre, post;        /* red-black sweeps before / after the coarse-grid
                             correction on every level (paper: 2 and 2)       */
    int max_cycles;       /* <= 64                                            */
    int cycle;            /* MG_CYCLE_V / _F / _W (Sec. 3.2.1)                */
    int precision;        /* MG_PREC_FP64 / MG_PREC_MIXED                     */
    double rtol, atol;    /* stop when eps <= rtol * eps_ref + atol, eps =
                             rms of the finest residual (Sec. 3.2.1)         */
    int warm_start;       /* 1: phi holds the initial guess; 0: start at 0    */
    int coarse_sweeps;    /* red-black sweeps on the coarsest level           */
    int use_graph;        /* 1: replay each cycle from a captured CUDA graph  */
    int inner_cycles;     /* MIXED: FP32 cycles per FP64 defect correction;
                             0: chosen per correction from the observed
                             convergence rate (1..4)                         */
} mg_opts;

/* pre = post = 2, max_cycles = 30, V, FP64, rtol = 1e-8, atol = 0,
 * warm_start = 0, coarse_sweeps = 16, use_graph = 1, inner_cycles = 0. */
void mg_opts_default(mg_opts *o);

typedef struct {
    int cycles;              /* cycles run (FP64: V/F/W cycles; MIXED: FP32
                                inner cycles in total)                         */
    int status;              /* the call's return code                          */
    double eps_ref;          /* nDGP: rms(Omega_m a^-1 delta / beta);
                                Kmouflage: rms(3 beta A Omega_m a^-1 delta/c~)  */
    double eps[65];          /* eps[0] initial, then after each measured cycle
                                (FP64: the norm pass is skipped on cycles
                                predicted far from the tolerance; MIXED: after
                                each defect correction)                         */
    int n_eps;               /* entries of eps[] written                        */
    double c_final;          /* <N(phi)>, the compatibility constant            */
    double mean_shift;       /* mean removed from phi (gauge <phi> = 0)          */
    long long sqrt_clamps;   /* nDGP cells whose sqrt argument was clamped at 0 */
    double ms;               /* wall time of the solve on the stream (ms)       */
    long long cell_updates;  /* smoother cell-updates summed over all levels    */
    long long kernel_launches;      /* CUDA kernels launched by the solve       */
    double fine_smooth_ms;          /* with profiling on: summed device time of
                                       the finest-level smoother launches (ms)  */
    long long fine_smooth_launches; /* ... and their number                     */
} mg_stats;

typedef struct {
    mg_grid g;
    mg_dgp_params p;
    const double *delta;     /* ng^3 density contrast                            */
    double *phi;             /* ng^3 output (and guess if warm_start)            */
} mg_instance;

/* ---- the hot path ------------------------------------------------------ */

/*
 * nDGP scalar field (Eq. dgp_eom_code in the form of Eq. DGP):
 *   Lap phi = (3/4)[-alpha + sqrt(alpha^2 + 8 Sigma / 3)],
 *   Sigma = traceless (d_i d_j phi)^2 + (alpha / beta) Omega_m a^-1 delta,
 * discretised as the paper's L^h with the 19-point Sigma_ijk (Sec. 3.2.3)
 * and solved by FAS multigrid (Sec. 3.2.1) with the colour-simultaneous
 * red-black update of Eq. nonlinear_GS_DGP.  delta - <delta> is used; the
 * periodic system is made compatible by L(u) = Lap u - N(u) + <N(u)>, and
 * the result has <phi> = 0.
 * count >= 1 independent instances (sizes may differ).  count > 1 with
 * precision MG_PREC_MIXED, device-resident delta/phi and pre + post even is
 * the batched form: one persistent cooperative kernel runs the whole
 * mixed-precision solve of every instance, walking the tiles of all
 * instances still iterating in each phase; an instance leaves the work
 * lists when it meets its tolerance.  Other count > 1 calls solve the
 * instances one after another.  stats: `count` records (or NULL).
 * Returns MG_OK, MG_WARN_NOT_CONVERGED, MG_ERR_ARG, MG_ERR_CUDA,
 * MG_ERR_NONFINITE or MG_ERR_OOM.
 */
int mg_solve_dgp(mg_ctx *ctx, int count, const mg_instance *inst,
                 const mg_opts *opts, mg_stats *stats);

/*
 * Kmouflage field (Eq. kmo_eom1 in the split form of Eq.
 * kmf_eqn_codeunit_final, divided by c~):
 *   Lap phi = [3 beta A Omega_m a^-1 delta / c~ - 2 (n-1) gamma (G^2)^(n-2) T]
 *             / [1 + gamma (phibar'/H0)^(2(n-1)) + (2n+1) gamma/3 (G^2)^(n-1)],
 * G the central-difference gradient, T the 19-point
 * hat-nabla^i hat-nabla^j phi nabla_i phi nabla_j phi (cross terms with
 * 1/(8h^4)).  Same multigrid, options and errors as mg_solve_dgp.
 */
int mg_solve_kmouflage(mg_ctx *ctx, const mg_grid *g, const mg_kmo_params *p,
                       const mg_opts *opts, const double *delta, double *phi,
                       mg_stats *stats);

/*
 * Linear-theory Kmouflage field (Eq. kmf_eqn_codeunit_lin): the gradient
 * term of the denominator and the T term dropped,
 *   Lap phi = 3 beta A Omega_m a^-1 (delta - <delta>) / [c~ (1 + gamma (phibar'/H0)^(2(n-1)))],
 * solved by FFT with the 7-point Green's function (the multigrid Laplacian;
 * FP32 transforms inside an FP64 refinement, as pm_newton_potential);
 * the screening-off reference for mg_solve_kmouflage.  ng even >= 2.
 * Errors: MG_ERR_ARG, MG_ERR_CUDA, MG_ERR_OOM.
 */
int mg_solve_kmouflage_linear(mg_ctx *ctx, const mg_grid *g, const mg_kmo_params *p,
                              const double *delta, double *phi);

/*
 * Cloud-in-cell density contrast (Sec. 3.1): each of the np particles
 * (FP32 positions in [0, ng), np x 3) carries (ng^3/np) mean cell masses
 * spread over the 8 cells around it; delta_out = rho/rho_bar - 1 (ng^3,
 * FP64, mean removed).  The lower cell per axis is floor(x - 1/2) taken in
 * FP32.  Deterministic: weights are summed as 32.32 fixed point in 64-bit
 * integers.  Errors: MG_ERR_ARG (bad sizes, positions outside [0, ng) are
 * wrapped, never rejected), MG_ERR_CUDA, MG_ERR_OOM.
 */
int pm_cic_deposit(mg_ctx *ctx, int ng, const float *pos, long long np,
                   double *delta_out);

/*
 * pm_cic_deposit for callers that cannot allocate device memory:
 * applications whose device memory all belongs to their own pool, and
 * pipelines that cannot afford the device synchronisation of cudaMalloc.
 * The paper has no counterpart; this is a deployment variant of the CIC
 * deposit above with the same result (same kernels, same fixed-point sums).
 *  - Allocates nothing: no mg_ctx, no cudaMalloc/cudaFree, no allocating
 *    library call.  Its scratch (fixed-point accumulator, reduction
 *    partials, mean, counter) is one static device array of 16 MiB + 8 KiB
 *    + 256 B that every GPU loading the library holds until process exit.
 *  - ng <= 128 (the array holds 128^3 cells): larger ng returns MG_ERR_ARG,
 *    as do ng < 2, np < 1, NULL or host pointers.  pos (np x 3 FP32 in
 *    [0, ng)) and delta_out (ng^3 FP64) must be device arrays of the
 *    current device; work is queued on cuda_stream (a cudaStream_t, NULL =
 *    legacy default stream) and the call returns without synchronising.
 *  - The first call on a device (the current one) looks up the array's
 *    device address with cudaGetSymbolAddress.
 *  - Every call shares the one array, which keeps the last call's contents
 *    (each call clears what must start at zero): calls whose work overlaps
 *    on the GPU (other streams, other threads) race and corrupt each other.
 * Returns MG_OK, MG_ERR_ARG or MG_ERR_CUDA.
 */
int pm_cic_deposit_noalloc(int ng, const float *pos, long long np,
                           double *delta_out, void *cuda_stream);

/* Lower CIC cell per axis, floor(x - 1/2) mod ng, as used by
 * pm_cic_deposit (np x 3 int32 output); for checking the indexing. */
int pm_cic_index(mg_ctx *ctx, int ng, const float *pos, long long np,
                 int *idx_out);

/* Newtonian potential on the mesh (Sec. 3.1; Eq. GR_poisson_codeunit):
 * Lap Phi = (3/2) Omega_m a^-1 delta with the 7-point Laplacian, solved by
 * FFT with the Green's function -1/sum_d 4 sin^2(pi k_d/ng); the k = 0 mode
 * is set to zero (the mean of delta is ignored).  The transforms run in
 * FP32 (cuFFT) inside an FP64 iterative refinement (two corrections from
 * FP64 residuals of the 7-point system), which returns the FP64 solution to
 * about 1e-15 relative.  delta, phi_out: ng^3 FP64 (ng even). */
int pm_newton_potential(mg_ctx *ctx, int ng, double a, double omega_m,
                        const double *delta, double *phi_out);

/*
 * Particle-mesh state for pm_step: positions x~ (FP32, np x 3, in [0, ng))
 * at scale factor a, momenta p~ (FP32, np x 3) at a - da/2 (at a itself
 * when first != 0).  model 0 = GR (Newtonian force only), 1 = nDGP
 * (Phi = Phi_N + phi/2, Eq. poisson_nDGP), 2 = Kmouflage (Eqs. force_Kmo2,
 * kmf_Poission_eqn_codeunit: Lap Phi_N = (3/2) A Omega_m a^-1 delta,
 * Phi = Phi_N + beta c~ phi~, and the friction term -beta (dphibar/da) p~,
 * with the background inputs kmo (at a) and dphibar_da).  The expansion
 * rate is e_a, e_mid when both are set (the Kmouflage background of
 * mg_kmo_background), else LCDM's.  phi_ws: ng^3 FP64 device or host buffer
 * carrying the field between steps as a warm start (may be NULL; then each
 * solve starts from zero).
 */
typedef struct {
    float *pos, *mom;
    long long np;
    int ng;
    double box_mpch, omega_m, a, da;
    int model;
    int first;
    mg_dgp_params dgp;
    double *phi_ws;
    mg_kmo_params kmo;   /* model 2: the Kmouflage parameters at a           */
    double dphibar_da;   /* model 2: d phibar / d a at a                       */
    double e_a, e_mid;   /* H/H0 at a and at a + da/2 for the kick and drift;
                            0 (either) = LCDM's from omega_m                   */
} pm_state;

/*
 * One leapfrog step in a (code-unit equations of motion of Sec. 3.1.1 with
 * the drift sign of Eq. force_Kmo1): CIC density, FFT Poisson solve of
 * Lap Phi_N = (3/2) Omega_m a^-1 delta with the 7-point Green's function,
 * the nDGP field (model 1), 3-point gradient of Phi at the 8 CIC cells
 * (formed once per mesh cell) interpolated to each particle, kick p += g da/(a E(a)) (da/2 if first),
 * drift x += p da/(a_m^3 E(a_m)) with a_m = a + da/2, wrap into [0, ng);
 * E = H/H0 (e_a, e_mid when set).
 * Updates pos, mom, a (+= da) and first (= 0).  stats: the nDGP solve.
 */
int pm_step(mg_ctx *ctx, pm_state *st, const mg_opts *opts, mg_stats *stats);

/*
 * Adjoint of the nDGP solve: given the forward solution phi for delta and
 * a cotangent g = dLoss/dphi, solves J^T lambda = g (J the Jacobian of the
 * discrete operator of mg_solve_dgp, restricted to zero-mean fields) by a
 * linear multigrid on J^T and returns dLoss/ddelta = (dN/ddelta)^T lambda
 * (ng^3) and dLoss/dR_c (one FP64 scalar written to a HOST pointer).  Both
 * outputs are exact gradients of the discrete solution map at the given
 * tolerance.  dL_drc_out may be NULL.
 */
int mg_solve_adjoint(mg_ctx *ctx, const mg_grid *g, const mg_dgp_params *p,
                     const mg_opts *opts, const double *phi, const double *delta,
                     const double *dL_dphi, double *dL_ddelta_out,
                     double *dL_drc_out, mg_stats *stats);

/* ---- differentiable particle-mesh run ------------------------------------
 * The forward model (Sec. 3.1 and 3.1.1 with the nDGP field of Sec. 3.2.3)
 * and its hand-written reverse pass, in FP64 particle state:
 *   white noise w (ng^3) -> linear density delta_L(k) = amp(k) FFT(w)(k)
 *   -> Zel'dovich displacement psi(k) = i k delta_L(k) / k^2 in mesh cells
 *   (the Nyquist component of k dropped) -> one particle per cell on the
 *   lattice (i + 1/2, j + 1/2, k + 1/2): x = lattice + growth psi wrapped
 *   into [0, ng), p = vel psi;
 *   nsteps kick-drift-kick steps of constant da from a_start to a_end, the
 *   first with a half kick, each: delta = CIC(x) (mean removed), Phi_N by
 *   the 7-point Green's function, phi by mg_solve_dgp (model 1, warm
 *   started from the previous step), Phi = Phi_N + phi/2, force -grad Phi by
 *   central differences at the 8 CIC cells interpolated with the CIC
 *   weights, p += F da_k/(a E(a)), x += p da/(a_m^3 E(a_m)), wrap;
 *   P_b = <|FFT(CIC(x_T))|^2> L^3/ng^6 over the modes of bin b,
 *   b = floor((|m| - 1) nbins / (ng/2 - 1)) for integer wavevectors
 *   1 <= |m| <= ng/2 (|m| = ng/2 in the last bin), and the loss
 *   L = mean_b (P_b - target_b)^2.
 * amp is given on the rfft grid (ng, ng, ng/2+1): sqrt(P(k) / V_cell).
 * Particle arrays are (np, 3) FP64 in lattice order; meshes ng^3 FP64.
 * Arrays may be host or device pointers (copied in and out as needed)
 * unless marked HOST.  Errors: MG_ERR_ARG, MG_ERR_CUDA, MG_ERR_OOM, and the
 * solves' codes. */
typedef struct {
    int ng;                /* mesh cells per side = particles per side       */
    double box_mpch;       /* L                                              */
    double omega_m;
    double a_start, a_end; /* the run's scale factors                        */
    int nsteps;            /* leapfrog steps (>= 1)                          */
    int checkpoint_every;  /* steps between stored states for the reverse
                              pass (>= 1): memory ~ nsteps/checkpoint_every
                              particle states + checkpoint_every meshes     */
    int nbins;             /* P(k) bins (>= 1)                               */
    int model;             /* 0 GR, 1 nDGP                                   */
    double growth;         /* D(a_start): displacement factor of the ICs     */
    double vel;            /* momentum factor of the ICs, a^2 E D f          */
} dpm_config;

/* Runs the model from noise; writes P (HOST, nbins) and, with target_pk
 * (HOST, nbins) given, the loss (HOST scalar).  With dL_dnoise_out given,
 * also runs the reverse pass (needs target_pk): dL/dw (ng^3) and, when
 * dL_drc_out (HOST) is given, dL/dR_c.  stats (or NULL): the last forward
 * nDGP solve; stats->cycles holds the total number of solver cycles. */
int dpm_run(mg_ctx *ctx, const dpm_config *cfg, const mg_opts *opts, const double *amp,
            const double *noise, double rc_h0, const double *target_pk, double *pk_out,
            double *loss_out, double *dL_dnoise_out, double *dL_drc_out, mg_stats *stats);

/* The vector-Jacobian product of the run for any loss of the caller's on
 * P: the forward run (P written to pk_out, HOST, nbins) and the reverse pass
 * seeded with dL_dpk (HOST, nbins: dL/dP_b) instead of the built-in loss's
 * 2 (P_b - target_b) / nbins, giving dL/dw (ng^3) and, when dL_drc_out
 * (HOST) is given, dL/dR_c (0 for GR).  The forward run is deterministic, so
 * a forward call with dpm_run and this call see the same P.  Errors as
 * dpm_run; dL_dpk and dL_dnoise_out must not be NULL. */
int dpm_run_vjp(mg_ctx *ctx, const dpm_config *cfg, const mg_opts *opts, const double *amp,
                const double *noise, double rc_h0, const double *dL_dpk, double *pk_out,
                double *dL_dnoise_out, double *dL_drc_out, mg_stats *stats);

/* The pieces, each with its adjoint (vector-Jacobian product), for
 * checking.  dpm_ic: positions and momenta from noise; dpm_ic_adjoint:
 * dL/dw from dL/dx and dL/dp. */
int dpm_ic(mg_ctx *ctx, const dpm_config *cfg, const double *amp, const double *noise,
           double *pos_out, double *mom_out);
int dpm_ic_adjoint(mg_ctx *ctx, const dpm_config *cfg, const double *amp, const double *dpos,
                   const double *dmom, double *dnoise_out);
/* delta = (ng^3/np) sum of CIC weights - 1, mean removed; the weights are
 * summed in 64-bit fixed point (2^-40), so the result is deterministic.
 * The adjoint writes dL/dx = sum over the 8 cells of dW/dx (ng^3/np) dL/ddelta. */
int dpm_deposit(mg_ctx *ctx, int ng, const double *pos, long long np, double *delta_out);
int dpm_deposit_adjoint(mg_ctx *ctx, int ng, const double *pos, long long np, const double *ddelta,
                        double *dpos_out);
/* F = CIC interpolation of -grad (Phi_N + phi/2) (phi may be NULL); the
 * adjoint writes dL/dx (the interpolation weights' part) and dL/dPhi_N
 * (dL/dphi is half of it). */
int dpm_force(mg_ctx *ctx, int ng, const double *phin, const double *phi, const double *pos,
              long long np, double *force_out);
int dpm_force_adjoint(mg_ctx *ctx, int ng, const double *phin, const double *phi, const double *pos,
                      long long np, const double *dforce, double *dpos_out, double *dphin_out);
/* P_b (HOST, nbins) and the bins' full-grid mode counts (HOST, or NULL);
 * the adjoint writes dL/ddelta for dL/dP (HOST, nbins). */
int dpm_power_spectrum(mg_ctx *ctx, int ng, double box_mpch, int nbins, const double *delta,
                       double *pk_out, double *counts_out);
int dpm_power_spectrum_adjoint(mg_ctx *ctx, int ng, double box_mpch, int nbins, const double *delta,
                               const double *dpk, double *ddelta_out);

/* ---- kernel-level entry points (one multigrid step each) ---------------
 * For checking each kernel against a reference implementation.  Natural
 * layout FP64 in and out on the context's device (or host); `precision`
 * selects the FP64 (0) or FP32 (1) kernel (inputs are rounded to FP32 on
 * the way in for 1).  The FP64 nDGP kernels (here and in every FP64 solve)
 * form the stencil's signed sums and the quadratic form of its differences
 * exactly in integer arithmetic and round each once to binary64, so their
 * results are at least as accurate as an all-FP64 evaluation; a stencil
 * whose largest value lies outside [2^-453, 2^506] in magnitude (NaN,
 * infinity, extreme magnitudes; an all-zero stencil excepted, which is
 * exact either way) takes FP64 arithmetic.  The operator is given
 * explicitly:                                                             */
typedef struct {
    int model;        /* 0 = nDGP, 1 = Kmouflage                             */
    double alpha;     /* nDGP alpha                                          */
    int nkmo;         /* Kmouflage n                                         */
    double gamma;     /* Kmouflage gamma                                     */
    double bterm;     /* Kmouflage (phibar'/H0)^2                            */
} mg_op_params;

/* One colour-simultaneous half-sweep of Eq. nonlinear_GS_DGP on an n^3
 * level of spacing h with compatibility constant c: cells of `colour`
 * ((i+j+k) mod 2) get (sum of face neighbours - h^2 (N - c + f)) / 6, the
 * other colour is copied.  f may be NULL (zero). */
int mg_op_smooth(mg_ctx *ctx, const mg_op_params *op, int precision, int n,
                 double h, const double *u_in, const double *s, const double *f,
                 double c, int colour, double *u_out);

/* The FP32 correction-form half-sweep used inside MG_PREC_MIXED: with a
 * frozen base field b, the unknown correction e is updated on `colour` as
 * e = (sum of face neighbours of e - h^2 (dN - c + f)) / 6 with
 * dN = N(b + e) - N(b) evaluated without cancellation; the other colour is
 * copied.  The same update as mg_op_smooth applied to u = b + e. */
int mg_op_smooth_corr(mg_ctx *ctx, const mg_op_params *op, int n, double h,
                      const double *e_in, const double *base, const double *s,
                      const double *f, double c, int colour, double *e_out);

/* Fused residual and FAS restriction (Sec. 3.2.1): with c_new = <N(u)>,
 * d = Lap u - N + c_new - f; writes R u and R d ((n/2)^3 each, 8-cell
 * averages), c_new and eps = rms(d) (host scalars). */
int mg_op_resid_restrict(mg_ctx *ctx, const mg_op_params *op, int precision,
                         int n, double h, const double *u, const double *s,
                         const double *f, double *Ru, double *Rd,
                         double *c_out, double *eps_out);

/* Coarse FAS source (Eq. general_pde_numerical_coarse): on an n^3 coarse
 * level, f = L^H(Ru) - Rd with L^H including its own c = <N^H(Ru)>;
 * writes f and c (host scalar). */
int mg_op_coarse_source(mg_ctx *ctx, const mg_op_params *op, int precision,
                        int n, double h, const double *Ru, const double *Rd,
                        const double *s, double *f_out, double *c_out);

/* Correction (Eq. solution_correction): u_fine += P(uc - urc) with the
 * 27/9/3/1 over 64 prolongation; n = fine size. */
int mg_op_prolong_add(mg_ctx *ctx, int precision, int n, double *u_fine,
                      const double *uc, const double *urc);

/* Coarsest-level solve: `sweeps` times { c = <N(u)>; red-black sweep },
 * in FP64 in shared memory (n^3 <= 512). */
int mg_op_coarsest(mg_ctx *ctx, const mg_op_params *op, int n, double h,
                   double *u, const double *s, const double *f, int sweeps);

#ifdef __cplusplus
}
#endif
#endif /* MGGLAM_H */
