/*
 * Plain FP64 CPU oracle for the MG-GLAM derivative-coupling field solvers
 * (Hernandez-Aguayo et al. 2021, arXiv:2110.00566).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker, not the product: only
 * tests/, __graft_entry__.smoke() and the cpu_baseline / reference leg of
 * bench.py may load it.  It shares no source, header, table or helper with
 * the CUDA path under paper_2110_00566_gb300/csrc.
 *
 * Everything is written to be read against the paper by eye: natural C-order
 * arrays idx = (i*n + j)*n + k (k fastest), periodic wrap by an explicit
 * modulo, one cell at a time, FP64 throughout, no blocking or fusion.
 * OpenMP only parallelises loops over i-planes whose iterations are
 * independent (the colour-simultaneous smoother writes to a separate output
 * array), so results do not depend on the thread count; every reduction is a
 * plain sequential sum.
 *
 * Sources of each function:
 *   Sec. 3.2.1 (Eqs. general_pde .. solution_correction): residual d = L(u)-f,
 *     global residual eps = rms(d), black/red Gauss-Seidel, FAS coarse
 *     equation S^H = L^H(R u) - R d, 8-child restriction, 27/9/3/1 over 64
 *     prolongation, V/F/W cycles down to a 4^3 coarsest mesh.
 *   Sec. 3.2.3 (Eqs. operator_split, dgp_quadratic_eom, DGP, the discrete
 *     L^h and Sigma_ijk, nonlinear_GS_DGP): the nDGP operator and update.
 *   Sec. 3.2.4 (Eqs. kmo_eom1, kmf_eqn_codeunit_final, the discrete gradient
 *     and the discrete hat-nabla^i hat-nabla^j phi nabla_i phi nabla_j phi):
 *     the Kmouflage operator and update.
 *   Sec. 3.1 (GLAM): cloud-in-cell assignment and interpolation.
 *
 * Readings where the paper is silent (the same readings as the GPU path):
 *   - compatibility: on a periodic mesh sum(Lap u) = 0 but the discrete
 *     nonlinear term need not average to zero, so each level's operator is
 *     L(u) = Lap u - N(u) + c with c = <N(u)>, recomputed in every residual
 *     pass and held fixed during the smoothing that follows;
 *   - the 12 edge neighbours of the 19-point stencil have the same colour, so
 *     each colour is updated simultaneously (all reads from before the
 *     half-sweep); colour 0 = (i+j+k) even goes first;
 *   - coarsest level: coarse_sweeps sweeps, each preceded by c = <N(u)>;
 *   - Kmouflage off-diagonal coefficient: 1/(8h^4) (the printed 1/(2h^4)
 *     is inconsistent with the diagonal 1/(12h^4) and the continuum form);
 *   - sqrt of a negative argument: clamped at 0 (counted).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* indexing                                                             */
/* ------------------------------------------------------------------ */
static long wrap(long i, long n) { return ((i % n) + n) % n; }
static long IX(long i, long j, long k, long n)
{
    return (wrap(i, n) * n + wrap(j, n)) * n + wrap(k, n);
}

/* ------------------------------------------------------------------ */
/* the two model operators                                              */
/* ------------------------------------------------------------------ */
typedef struct {
    int model;      /* 0 = nDGP (Vainshtein), 1 = Kmouflage                  */
    double alpha;   /* nDGP: alpha = 3 beta_DGP a^2 / R_c^2 (Sec. 3.2.3)       */
    int nkmo;       /* Kmouflage: exponent n of K(X) = -1 + X + K0 X^n      */
    double gamma;   /* Kmouflage: gamma = n K0 (1/(2 a^2 lambda^2))^(n-1)    */
    double bterm;   /* Kmouflage: (phibar'/H0)^2                              */
} orc_op;

/*
 * nDGP: Sigma_ijk exactly as printed in Sec. 3.2.3 (the discrete L^h):
 *   (2/3h^4)[Dxx^2+Dyy^2+Dzz^2] - (2/3h^4)[DxxDyy + DxxDzz + DyyDzz]
 *   + (1/8h^4)[Cxy^2 + Cxz^2 + Cyz^2] + s,
 * with Dxx = u(i+1)+u(i-1)-2u(i) (no 1/h^2), Cxy the 4-point cross
 * difference, and s = (alpha/beta) Omega_m a^-1 delta (restricted on coarse
 * levels).
 */
double orc_dgp_sigma(const double *u, long n, double h,
                     long i, long j, long k, double s)
{
    const double c = u[IX(i, j, k, n)];
    const double dxx = u[IX(i + 1, j, k, n)] + u[IX(i - 1, j, k, n)] - 2.0 * c;
    const double dyy = u[IX(i, j + 1, k, n)] + u[IX(i, j - 1, k, n)] - 2.0 * c;
    const double dzz = u[IX(i, j, k + 1, n)] + u[IX(i, j, k - 1, n)] - 2.0 * c;
    const double cxy = u[IX(i + 1, j + 1, k, n)] + u[IX(i - 1, j - 1, k, n)]
                     - u[IX(i + 1, j - 1, k, n)] - u[IX(i - 1, j + 1, k, n)];
    const double cxz = u[IX(i + 1, j, k + 1, n)] + u[IX(i - 1, j, k - 1, n)]
                     - u[IX(i + 1, j, k - 1, n)] - u[IX(i - 1, j, k + 1, n)];
    const double cyz = u[IX(i, j + 1, k + 1, n)] + u[IX(i, j - 1, k - 1, n)]
                     - u[IX(i, j + 1, k - 1, n)] - u[IX(i, j - 1, k + 1, n)];
    const double h4 = h * h * h * h;
    double sig = 2.0 / (3.0 * h4) * (dxx * dxx + dyy * dyy + dzz * dzz);
    sig -= 2.0 / (3.0 * h4) * dxx * dyy;
    sig -= 2.0 / (3.0 * h4) * dxx * dzz;
    sig -= 2.0 / (3.0 * h4) * dyy * dzz;
    sig += 1.0 / (8.0 * h4) * (cxy * cxy + cxz * cxz + cyz * cyz);
    return sig + s;
}

/*
 * nDGP: Lap u = (3/4)[-alpha + sign(alpha) sqrt(alpha^2 + 8 Sigma/3)]
 * (Eq. DGP; sign(0) = +1).  Evaluated in the algebraically identical
 * rationalised form 2 sign(alpha) Sigma / (|alpha| + sqrt(...)), which does
 * not cancel when Sigma << alpha^2.  A negative sqrt argument is clamped to
 * zero, giving -(3/4) alpha as the literal form does.
 */
double orc_dgp_N(double sigma, double alpha, long *clamps)
{
    const double arg = alpha * alpha + 8.0 * sigma / 3.0;
    const double sgn = alpha >= 0.0 ? 1.0 : -1.0;
    if (arg < 0.0) {
        if (clamps) (*clamps)++;
        return -0.75 * alpha;
    }
    return 2.0 * sgn * sigma / (fabs(alpha) + sqrt(arg));
}

/* integer power with x^0 = 1 (also at x = 0) */
static double ipow(double x, int p)
{
    double r = 1.0;
    for (int q = 0; q < p; ++q) r *= x;
    return r;
}

/*
 * Kmouflage (Sec. 3.2.4, Eq. kmf_eqn_codeunit_final divided by c~):
 *   Lap u = [ s + Sigma_2 / c~ ] / Sigma_1,   s = 3 beta A Omega_m a^-1 delta / c~
 *   Sigma_1 = 1 + gamma b^(n-1) + ((2n+1) gamma / 3) (G^2)^(n-1)
 *   Sigma_2 / c~ = -2 (n-1) gamma (G^2)^(n-2) T
 * G_a = (u(a+1) - u(a-1)) / 2h, G^2 = sum_a G_a^2, and
 * T = hat-nabla^i hat-nabla^j u nabla_i u nabla_j u in the printed 19-point
 * form: diagonal terms with 1/(12 h^4), cross terms with 1/(8 h^4).
 */
double orc_kmo_N(const orc_op *op, const double *u, long n, double h,
                 long i, long j, long k, double s)
{
    const double xp = u[IX(i + 1, j, k, n)], xm = u[IX(i - 1, j, k, n)];
    const double yp = u[IX(i, j + 1, k, n)], ym = u[IX(i, j - 1, k, n)];
    const double zp = u[IX(i, j, k + 1, n)], zm = u[IX(i, j, k - 1, n)];
    const double dx = xp - xm, dy = yp - ym, dz = zp - zm;
    const double cxy = u[IX(i + 1, j + 1, k, n)] + u[IX(i - 1, j - 1, k, n)]
                     - u[IX(i + 1, j - 1, k, n)] - u[IX(i - 1, j + 1, k, n)];
    const double cxz = u[IX(i + 1, j, k + 1, n)] + u[IX(i - 1, j, k - 1, n)]
                     - u[IX(i + 1, j, k - 1, n)] - u[IX(i - 1, j, k + 1, n)];
    const double cyz = u[IX(i, j + 1, k + 1, n)] + u[IX(i, j - 1, k - 1, n)]
                     - u[IX(i, j + 1, k - 1, n)] - u[IX(i, j - 1, k + 1, n)];
    const double h2 = h * h, h4 = h2 * h2;
    double T = 0.0;
    T += dx * dx * (2.0 * xp + 2.0 * xm - yp - ym - zp - zm) / (12.0 * h4);
    T += dy * dy * (2.0 * yp + 2.0 * ym - xp - xm - zp - zm) / (12.0 * h4);
    T += dz * dz * (2.0 * zp + 2.0 * zm - xp - xm - yp - ym) / (12.0 * h4);
    T += cxy * dx * dy / (8.0 * h4);
    T += cxz * dx * dz / (8.0 * h4);
    T += cyz * dy * dz / (8.0 * h4);
    const double G2 = (dx * dx + dy * dy + dz * dz) / (4.0 * h2);
    const int nn = op->nkmo;
    const double sigma1 = 1.0 + op->gamma * ipow(op->bterm, nn - 1)
                        + (2.0 * nn + 1.0) * op->gamma / 3.0 * ipow(G2, nn - 1);
    const double sigma2 = -2.0 * (nn - 1) * op->gamma * ipow(G2, nn - 2) * T;
    return (s + sigma2) / sigma1;
}

/* N(u) at one cell for either model: the nonlinear right-hand side of
 * Lap u = N(u). */
static double cell_N(const orc_op *op, const double *u, long n, double h,
                     long i, long j, long k, double s, long *clamps)
{
    if (op->model == 0)
        return orc_dgp_N(orc_dgp_sigma(u, n, h, i, j, k, s), op->alpha, clamps);
    return orc_kmo_N(op, u, n, h, i, j, k, s);
}

/* ------------------------------------------------------------------ */
/* per-level operations                                                 */
/* ------------------------------------------------------------------ */

/* N(u) at every cell. */
void orc_N_field(const orc_op *op, const double *u, const double *s, long n,
                 double h, double *Nout, long *clamps)
{
    long cl = 0;
#pragma omp parallel for reduction(+ : cl) schedule(static)
    for (long i = 0; i < n; ++i)
        for (long j = 0; j < n; ++j)
            for (long k = 0; k < n; ++k) {
                long c = 0;
                Nout[IX(i, j, k, n)] = cell_N(op, u, n, h, i, j, k, s[IX(i, j, k, n)], &c);
                cl += c;
            }
    if (clamps) *clamps += cl;
}

/* plain sequential mean */
double orc_mean(const double *x, long count)
{
    double acc = 0.0;
    for (long q = 0; q < count; ++q) acc += x[q];
    return acc / (double)count;
}

/*
 * One colour-simultaneous half-sweep (Eq. nonlinear_GS_DGP; the same update
 * for Kmouflage).  For every cell of the given colour ((i+j+k) mod 2), with
 * every neighbour taken from u_in:
 *   u_out = u - (L(u) - f) / (dL/du),  dL/du = -6/h^2,
 * which, because N does not depend on the centre value, equals
 *   u_out = (sum of the 6 face neighbours - h^2 (N - c + f)) / 6.
 * Cells of the other colour are copied.  f may be NULL (zero).
 */
void orc_smooth(const orc_op *op, const double *u_in, double *u_out,
                const double *s, const double *f, long n, double h, double c,
                int colour)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i)
        for (long j = 0; j < n; ++j)
            for (long k = 0; k < n; ++k) {
                const long q = IX(i, j, k, n);
                if (((i + j + k) & 1) != colour) {
                    u_out[q] = u_in[q];
                    continue;
                }
                const double N = cell_N(op, u_in, n, h, i, j, k, s[q], NULL);
                const double fq = f ? f[q] : 0.0;
                const double lap_u = (u_in[IX(i + 1, j, k, n)] + u_in[IX(i - 1, j, k, n)]
                                    + u_in[IX(i, j + 1, k, n)] + u_in[IX(i, j - 1, k, n)]
                                    + u_in[IX(i, j, k + 1, n)] + u_in[IX(i, j, k - 1, n)]
                                    - 6.0 * u_in[q]) / (h * h);
                const double L = lap_u - N + c;
                u_out[q] = u_in[q] - (L - fq) / (-6.0 / (h * h));
            }
}

/*
 * Residual (Eqs. general_pde_numerical .. residual_d): with N computed at
 * every cell and c = <N>, d = Lap u - N + c - f.  Returns c; writes eps =
 * rms(d) (the global residual of Sec. 3.2.1) if eps != NULL.
 */
double orc_residual(const orc_op *op, const double *u, const double *s,
                    const double *f, long n, double h, double *d, double *eps,
                    long *clamps)
{
    const long cnt = n * n * n;
    double *N = (double *)malloc(sizeof(double) * cnt);
    orc_N_field(op, u, s, n, h, N, clamps);
    const double c = orc_mean(N, cnt);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i)
        for (long j = 0; j < n; ++j)
            for (long k = 0; k < n; ++k) {
                const long q = IX(i, j, k, n);
                const double lap_u = (u[IX(i + 1, j, k, n)] + u[IX(i - 1, j, k, n)]
                                    + u[IX(i, j + 1, k, n)] + u[IX(i, j - 1, k, n)]
                                    + u[IX(i, j, k + 1, n)] + u[IX(i, j, k - 1, n)]
                                    - 6.0 * u[q]) / (h * h);
                d[q] = lap_u - N[q] + c - (f ? f[q] : 0.0);
            }
    if (eps) {
        double acc = 0.0;
        for (long q = 0; q < cnt; ++q) acc += d[q] * d[q];
        *eps = sqrt(acc / (double)cnt);
    }
    free(N);
    return c;
}

/* Restriction: arithmetic average of the 8 fine cells of each coarse cell
 * (Sec. 3.2.1, after Eq. general_pde_numerical_coarse). nf = fine size. */
void orc_restrict(const double *fine, long nf, double *coarse)
{
    const long nc = nf / 2;
#pragma omp parallel for schedule(static)
    for (long I = 0; I < nc; ++I)
        for (long J = 0; J < nc; ++J)
            for (long K = 0; K < nc; ++K) {
                double acc = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        for (int cc = 0; cc < 2; ++cc)
                            acc += fine[IX(2 * I + a, 2 * J + b, 2 * K + cc, nf)];
                coarse[IX(I, J, K, nc)] = acc / 8.0;
            }
}

/*
 * Correction (Eq. solution_correction): u_fine += P(uc - urc), where P gives
 * a fine cell 27/64 of its parent coarse cell, 9/64 of each of the 3 coarse
 * cells sharing a face with the parent on the fine cell's side, 3/64 of each
 * of the 3 sharing an edge, and 1/64 of the one sharing a vertex.
 */
void orc_prolong_add(double *u_fine, long nf, const double *uc, const double *urc)
{
    const long nc = nf / 2;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < nf; ++i)
        for (long j = 0; j < nf; ++j)
            for (long k = 0; k < nf; ++k) {
                const long I = i / 2, J = j / 2, K = k / 2;
                const long si = (i % 2) ? 1 : -1, sj = (j % 2) ? 1 : -1, sk = (k % 2) ? 1 : -1;
                double acc = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        for (int cc = 0; cc < 2; ++cc) {
                            /* a = 0: parent along x (weight 3), a = 1: neighbour (weight 1) */
                            const double w = (a ? 1.0 : 3.0) * (b ? 1.0 : 3.0) * (cc ? 1.0 : 3.0) / 64.0;
                            const long q = IX(I + a * si, J + b * sj, K + cc * sk, nc);
                            acc += w * (uc[q] - urc[q]);
                        }
                u_fine[IX(i, j, k, nf)] += acc;
            }
}

/* ------------------------------------------------------------------ */
/* the multigrid solve                                                  */
/* ------------------------------------------------------------------ */
typedef struct {
    int pre, post;          /* smoothing sweeps before / after the coarse correction */
    int max_cycles;
    int cycle;              /* 0 = V, 1 = F, 2 = W                             */
    int coarse_sweeps;      /* sweeps on the coarsest level                    */
    double rtol, atol;      /* stop when eps <= rtol * eps_ref + atol          */
} orc_opts;

typedef struct {
    int cycles;
    double eps_ref;
    double eps[65];         /* eps[0] = initial, eps[q] after cycle q          */
    double c_final;         /* <N> of the returned field                       */
    double mean_shift;      /* <u> removed by the gauge fix                    */
    long sqrt_clamps;
} orc_stats;

typedef struct {
    long n;
    double h;
    double *u, *s, *f, *ur, *tmp, *rd;
    double c;
} lev_t;

typedef struct {
    const orc_op *op;
    const orc_opts *o;
    int nlev;
    lev_t *L;
    long clamps;
} mg_t;

static void smooth_level(mg_t *m, int l)
{
    lev_t *v = &m->L[l];
    for (int colour = 0; colour < 2; ++colour) {
        orc_smooth(m->op, v->u, v->tmp, v->s, v->f, v->n, v->h, v->c, colour);
        double *t = v->u; v->u = v->tmp; v->tmp = t;
    }
}

static void cycle(mg_t *m, int l, int type)
{
    lev_t *v = &m->L[l];
    const long cnt = v->n * v->n * v->n;
    if (l == m->nlev - 1) {
        for (int it = 0; it < m->o->coarse_sweeps; ++it) {
            double *N = v->rd;  /* scratch */
            orc_N_field(m->op, v->u, v->s, v->n, v->h, N, NULL);
            v->c = orc_mean(N, cnt);
            smooth_level(m, l);
        }
        return;
    }
    for (int p = 0; p < m->o->pre; ++p) smooth_level(m, l);

    /* residual d^h with c = <N(u)>, then the FAS coarse problem
     * (Eq. general_pde_numerical_coarse): u^H_0 = R u (also kept as R u for
     * the correction), S^H = L^H(R u) - R d^h. */
    v->c = orc_residual(m->op, v->u, v->s, v->f, v->n, v->h, v->rd, NULL, NULL);
    lev_t *w = &m->L[l + 1];
    const long cntc = w->n * w->n * w->n;
    orc_restrict(v->u, v->n, w->ur);
    memcpy(w->u, w->ur, sizeof(double) * cntc);
    double *Rd = w->rd;
    orc_restrict(v->rd, v->n, Rd);
    /* L^H(R u) with its own c^H = <N^H(R u)> */
    double *LH = w->tmp;
    w->c = orc_residual(m->op, w->ur, w->s, NULL, w->n, w->h, LH, NULL, NULL);
    for (long q = 0; q < cntc; ++q) w->f[q] = LH[q] - Rd[q];

    const int visits = (type == 2) ? 2 : 1;
    for (int vv = 0; vv < visits; ++vv) cycle(m, l + 1, type);
    if (type == 1) cycle(m, l + 1, 0);   /* F-cycle: an F then a V visit */

    orc_prolong_add(v->u, v->n, w->u, w->ur);
    for (int p = 0; p < m->o->post; ++p) smooth_level(m, l);
}

/* Level sizes: halve while the size is even and the half is still >= 4
 * (Sec. 3.2.1: coarsest mesh 4^3 for N = 2^l; 6^3 for N = 3*2^l). */
int orc_num_levels(long n)
{
    int nl = 1;
    while (n % 2 == 0 && n / 2 >= 4) { n /= 2; ++nl; }
    return nl;
}

/*
 * Full solve of L(u) = 0 on the finest level (f = 0), given the finest
 * density term s0 (already mean-subtracted and scaled) and eps_ref for the
 * relative stopping rule.  u: in = initial guess, out = solution with <u> = 0.
 * Returns the number of cycles run (0 if already converged).
 */
int orc_mg_solve(const orc_op *op, long n, const double *s0, double eps_ref,
                 const orc_opts *o, double *u, orc_stats *st)
{
    mg_t m;
    m.op = op; m.o = o; m.clamps = 0;
    m.nlev = orc_num_levels(n);
    m.L = (lev_t *)calloc((size_t)m.nlev, sizeof(lev_t));
    long nl = n;
    for (int l = 0; l < m.nlev; ++l) {
        lev_t *v = &m.L[l];
        v->n = nl;
        v->h = (double)(1L << l);
        const long cnt = nl * nl * nl;
        v->u = (double *)calloc((size_t)cnt, sizeof(double));
        v->s = (double *)calloc((size_t)cnt, sizeof(double));
        v->f = (l == 0) ? NULL : (double *)calloc((size_t)cnt, sizeof(double));
        v->ur = (double *)calloc((size_t)cnt, sizeof(double));
        v->tmp = (double *)calloc((size_t)cnt, sizeof(double));
        v->rd = (double *)calloc((size_t)cnt, sizeof(double));
        nl /= 2;
    }
    const long cnt0 = n * n * n;
    memcpy(m.L[0].u, u, sizeof(double) * cnt0);
    memcpy(m.L[0].s, s0, sizeof(double) * cnt0);
    for (int l = 1; l < m.nlev; ++l) orc_restrict(m.L[l - 1].s, m.L[l - 1].n, m.L[l].s);

    lev_t *v0 = &m.L[0];
    double eps;
    v0->c = orc_residual(op, v0->u, v0->s, NULL, n, 1.0, v0->rd, &eps, NULL);
    st->eps_ref = eps_ref;
    st->eps[0] = eps;
    int cyc = 0;
    if (!(eps <= o->rtol * eps_ref + o->atol)) {
        for (cyc = 1; cyc <= o->max_cycles && cyc < 65; ++cyc) {
            cycle(&m, 0, o->cycle);
            v0->c = orc_residual(op, v0->u, v0->s, NULL, n, 1.0, v0->rd, &eps, NULL);
            st->eps[cyc] = eps;
            if (eps <= o->rtol * eps_ref + o->atol) break;
        }
        if (cyc > o->max_cycles) cyc = o->max_cycles;
    }
    st->cycles = cyc;
    /* gauge: the equations contain only differences of u */
    const double mu = orc_mean(v0->u, cnt0);
    for (long q = 0; q < cnt0; ++q) u[q] = v0->u[q] - mu;
    st->mean_shift = mu;
    long cl = 0;
    st->c_final = orc_residual(op, u, v0->s, NULL, n, 1.0, v0->rd, NULL, &cl);
    st->sqrt_clamps = cl;
    for (int l = 0; l < m.nlev; ++l) {
        free(m.L[l].u); free(m.L[l].s); free(m.L[l].f);
        free(m.L[l].ur); free(m.L[l].tmp); free(m.L[l].rd);
    }
    free(m.L);
    return cyc;
}

/* ------------------------------------------------------------------ */
/* particle-mesh pieces (Sec. 3.1)                                      */
/* ------------------------------------------------------------------ */

/*
 * CIC index and weight along one axis for a position x in [0, n) (code
 * units, cell i has its centre at i + 1/2): the lower cell is
 * floor(x - 1/2), taken in FP32 as the positions are FP32, and the upper
 * weight is the distance from the lower cell's centre.
 */
void orc_cic_axis(float x, long n, long *i0, long *i1, double *w0, double *w1)
{
    const float t = x - 0.5f;
    const long lo = (long)floorf(t);
    const double dx = (double)x - 0.5 - (double)lo;
    *i0 = wrap(lo, n);
    *i1 = wrap(lo + 1, n);
    *w0 = 1.0 - dx;
    *w1 = dx;
}

/*
 * Density contrast by cloud-in-cell assignment: every particle carries mass
 * (n/np_side)^3 in units of the mean cell mass and spreads it over the 8
 * nearest cell centres with weights wx*wy*wz; delta = rho/rho_bar - 1.
 * pos: np x 3 FP32 code-unit positions in [0, n).  Sequential in particle
 * order.  Also returns the lower-cell indices if idx != NULL (np x 3).
 */
void orc_cic_deposit(const float *pos, long np, long n, double mass,
                     double *delta, long *idx)
{
    const long cnt = n * n * n;
    for (long q = 0; q < cnt; ++q) delta[q] = 0.0;
    for (long p = 0; p < np; ++p) {
        long i0[3], i1[3];
        double w0[3], w1[3];
        for (int d = 0; d < 3; ++d) {
            orc_cic_axis(pos[3 * p + d], n, &i0[d], &i1[d], &w0[d], &w1[d]);
            if (idx) idx[3 * p + d] = i0[d];
        }
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int c = 0; c < 2; ++c) {
                    const double w = (a ? w1[0] : w0[0]) * (b ? w1[1] : w0[1]) * (c ? w1[2] : w0[2]);
                    delta[((a ? i1[0] : i0[0]) * n + (b ? i1[1] : i0[1])) * n + (c ? i1[2] : i0[2])] += mass * w;
                }
    }
    for (long q = 0; q < cnt; ++q) delta[q] -= 1.0;
}

/*
 * Force on each particle from a potential Phi on the mesh: the three-point
 * central difference g = -(Phi(i+1) - Phi(i-1)) / 2 at the 8 cells around
 * the particle, interpolated with the same CIC weights (GLAM keeps no force
 * mesh).  acc: np x 3.
 */
void orc_cic_force(const double *phi, long n, const float *pos, long np, double *acc)
{
#pragma omp parallel for schedule(static)
    for (long p = 0; p < np; ++p) {
        long i0[3], i1[3];
        double w0[3], w1[3];
        for (int d = 0; d < 3; ++d)
            orc_cic_axis(pos[3 * p + d], n, &i0[d], &i1[d], &w0[d], &w1[d]);
        double g[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int c = 0; c < 2; ++c) {
                    const double w = (a ? w1[0] : w0[0]) * (b ? w1[1] : w0[1]) * (c ? w1[2] : w0[2]);
                    const long i = a ? i1[0] : i0[0], j = b ? i1[1] : i0[1], k = c ? i1[2] : i0[2];
                    g[0] += w * -(phi[IX(i + 1, j, k, n)] - phi[IX(i - 1, j, k, n)]) / 2.0;
                    g[1] += w * -(phi[IX(i, j + 1, k, n)] - phi[IX(i, j - 1, k, n)]) / 2.0;
                    g[2] += w * -(phi[IX(i, j, k + 1, n)] - phi[IX(i, j, k - 1, n)]) / 2.0;
                }
        acc[3 * p + 0] = g[0];
        acc[3 * p + 1] = g[1];
        acc[3 * p + 2] = g[2];
    }
}
