// Kmouflage background cosmology (Sec. 3.2.4, background solver): host code.
//
// The background is two ordinary differential equations in N = ln a (the
// field and its N-derivative), a scalar problem with no data parallelism,
// so it runs on the host inside the library and hands the device solvers
// their per-step inputs (lambda, phibar'/H0, A(phibar), dphibar/da, H/H0).
//
// Notation: phi is the dimensionless background field (phi / M_Pl), r its
// derivative d phi / dN, h = (conformal Hubble rate / H0)^2, and
// X = h r^2 / (2 lambda^2 a^2) the background kinetic variable of the
// model K(X) = -1 + X + K0 X^n (Eq. kmf_model_K_function).
//
// Friedmann (Eq. kmf_background_Friedmann times a^2 / H0^2, with
// a phidot = H r and 8 pi G rho_{m0} = 3 Omega_m H0^2): the scalar's terms
// (1/3) K_X h r^2 - (1/3) lambda^2 a^2 K collect to
// h r^2 / 6 + lambda^2 a^2 / 3 + (2n-1)/3 K0 lambda^2 a^2 X^n, so
//     D h - B - C h^n = 0,   D = 1 - r^2/6,
//     B = Omega_r a^-2 + A Omega_m a^-1 + lambda^2 a^2 / 3,
//     C = (2n-1)/3 K0 lambda^2 a^2 (r^2 / (2 lambda^2 a^2))^n.
// The left side is concave in h; Newton's method from the C = 0 root B/D
// climbs monotonically to the smallest root (the LCDM-connected branch).
//
// Acceleration: a''/a = -(4 pi G / 3)(rho + 3p), with the scalar's
// rho = M_Pl^2 (K_X phidot^2 - lambda^2 H0^2 K) and p = M_Pl^2 lambda^2 H0^2 K,
// in conformal time over H0^2:
//     H'/H0^2 = -Omega_r a^-2 - (1/2) A Omega_m a^-1
//               + (lambda^2 a^2 / 3) (1 - 2X - (n+1) K0 X^n).
// (The printed Eq. kmf_background_Raychaudhuri has twice these scalar terms,
// which contradicts its own Friedmann equation in the K = -1 limit.)
//
// Field (Eq. kmf_background_eom2), with K_X + 2X K_XX = 1 + n(2n-1) K0 X^(n-1)
// and K_X - X K_XX = 1 + n(2-n) K0 X^(n-1):
//     (K_X + 2X K_XX)(h r' + (H'/H0^2) r) + 2 (K_X - X K_XX) h r
//         + 3 beta A Omega_m e^-N = 0.
//
// Integrator: the Dormand-Prince 5(4) embedded pair (J. R. Dormand and
// P. J. Prince, J. Comput. Appl. Math. 6 (1980) 19), fifth-order solution,
// step size from the fourth-order error estimate.  lambda: Illinois
// regula falsi (M. Dowell and P. Jarratt, BIT 11 (1971) 168) on
// h(a = 1) - 1, which increases with lambda.
#include "mgglam.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace {

struct Bg {
    int n;
    double k0, beta, om, orad, lam;
};

double ipow(double x, int k)
{
    double r = 1.0;
    for (int i = 0; i < k; ++i)
        r *= x;
    return r;
}

// Omega_r: photons (rho = a_rad T^4 / c^2, a_rad = 4 sigma / c) over the
// critical density 3 H0^2 / (8 pi G), times 1 + n_eff (7/8)(4/11)^(4/3).
double omega_rad(double hub, double t_cmb, double n_eff)
{
    const double sigma_sb = 5.670374419e-8, c = 299792458.0, G = 6.67430e-11, mpc = 3.0856775814913673e22;
    const double a_rad = 4.0 * sigma_sb / c;
    const double rho_g = a_rad * std::pow(t_cmb, 4.0) / (c * c);
    const double H0 = hub * 1.0e5 / mpc;
    const double rho_c = 3.0 * H0 * H0 / (8.0 * M_PI * G);
    return rho_g / rho_c * (1.0 + n_eff * 0.875 * std::pow(4.0 / 11.0, 4.0 / 3.0));
}

// h from the Friedmann polynomial; false when it has no real root.
bool hubble2(const Bg &p, double a, double phi, double r, double &h)
{
    const double l2a2 = p.lam * p.lam * a * a;
    const double B = p.orad / (a * a) + std::exp(p.beta * phi) * p.om / a + l2a2 / 3.0;
    const double D = 1.0 - r * r / 6.0;
    if (!(D > 0.0))
        return false;
    const double C = (2 * p.n - 1) / 3.0 * p.k0 * l2a2 * ipow(r * r / (2.0 * l2a2), p.n);
    double x = B / D;
    if (C == 0.0) {
        h = x;
        return std::isfinite(x);
    }
    for (int it = 0; it < 200; ++it) {
        const double xn1 = ipow(x, p.n - 1);
        const double f = D * x - B - C * xn1 * x;
        const double fp = D - p.n * C * xn1;
        if (!(fp > 0.0))
            return false;
        const double dx = -f / fp;
        x += dx;
        if (std::fabs(dx) <= 4e-16 * x) {
            h = x;
            return std::isfinite(x);
        }
    }
    return false;
}

struct Deriv {
    double dphi, dr, h;
};

bool rhs(const Bg &p, double N, double phi, double r, Deriv &d)
{
    const double a = std::exp(N);
    double h;
    if (!hubble2(p, a, phi, r, h))
        return false;
    const double l2a2 = p.lam * p.lam * a * a;
    const double X = h * r * r / (2.0 * l2a2);
    const double Xn1 = ipow(X, p.n - 1);
    const double A = std::exp(p.beta * phi);
    const double hp = -p.orad / (a * a) - 0.5 * A * p.om / a + l2a2 / 3.0 * (1.0 - 2.0 * X - (p.n + 1) * p.k0 * Xn1 * X);
    const double c2 = 1.0 + p.n * (2 * p.n - 1) * p.k0 * Xn1;
    const double c1 = 1.0 + p.n * (2 - p.n) * p.k0 * Xn1;
    d.dphi = r;
    d.dr = -(c2 * hp * r + 2.0 * c1 * h * r + 3.0 * p.beta * A * p.om / a) / (c2 * h);
    d.h = h;
    return std::isfinite(d.dr);
}

// Dormand-Prince 5(4) coefficients.
constexpr double C2 = 1.0 / 5, C3 = 3.0 / 10, C4 = 4.0 / 5, C5 = 8.0 / 9;
constexpr double A21 = 1.0 / 5;
constexpr double A31 = 3.0 / 40, A32 = 9.0 / 40;
constexpr double A41 = 44.0 / 45, A42 = -56.0 / 15, A43 = 32.0 / 9;
constexpr double A51 = 19372.0 / 6561, A52 = -25360.0 / 2187, A53 = 64448.0 / 6561, A54 = -212.0 / 729;
constexpr double A61 = 9017.0 / 3168, A62 = -355.0 / 33, A63 = 46732.0 / 5247, A64 = 49.0 / 176,
                 A65 = -5103.0 / 18656;
constexpr double B1 = 35.0 / 384, B3 = 500.0 / 1113, B4 = 125.0 / 192, B5 = -2187.0 / 6784, B6 = 11.0 / 84;
// fifth- minus fourth-order weights
constexpr double E1 = 71.0 / 57600, E3 = -71.0 / 16695, E4 = 71.0 / 1920, E5 = -17253.0 / 339200,
                 E6 = 22.0 / 525, E7 = -1.0 / 40;

struct State {
    double N, phi, r;
};

// Advance s to N_end with adaptive steps; false on failure.
bool integrate_to(const Bg &p, State &s, double N_end, double rtol, double &dt)
{
    const double atol = 1e-30;
    Deriv k1, k2, k3, k4, k5, k6, k7;
    if (!rhs(p, s.N, s.phi, s.r, k1))
        return false;
    for (long step = 0; s.N < N_end; ++step) {
        if (step > 2000000)
            return false;
        const bool last = s.N + dt >= N_end;
        const double hs = last ? N_end - s.N : dt;
        auto stage = [&](double c, double a1, double a2, double a3, double a4, double a5, Deriv &k) {
            return rhs(p, s.N + c * hs,
                       s.phi + hs * (a1 * k1.dphi + a2 * k2.dphi + a3 * k3.dphi + a4 * k4.dphi + a5 * k5.dphi),
                       s.r + hs * (a1 * k1.dr + a2 * k2.dr + a3 * k3.dr + a4 * k4.dr + a5 * k5.dr), k);
        };
        bool ok = stage(C2, A21, 0, 0, 0, 0, k2) && stage(C3, A31, A32, 0, 0, 0, k3) &&
                  stage(C4, A41, A42, A43, 0, 0, k4) && stage(C5, A51, A52, A53, A54, 0, k5) &&
                  stage(1.0, A61, A62, A63, A64, A65, k6);
        double phi1 = 0, r1 = 0, err = INFINITY;
        if (ok) {
            phi1 = s.phi + hs * (B1 * k1.dphi + B3 * k3.dphi + B4 * k4.dphi + B5 * k5.dphi + B6 * k6.dphi);
            r1 = s.r + hs * (B1 * k1.dr + B3 * k3.dr + B4 * k4.dr + B5 * k5.dr + B6 * k6.dr);
            ok = rhs(p, s.N + hs, phi1, r1, k7);
        }
        if (ok) {
            const double ep = hs * (E1 * k1.dphi + E3 * k3.dphi + E4 * k4.dphi + E5 * k5.dphi + E6 * k6.dphi +
                                    E7 * k7.dphi);
            const double er = hs * (E1 * k1.dr + E3 * k3.dr + E4 * k4.dr + E5 * k5.dr + E6 * k6.dr + E7 * k7.dr);
            const double sp = atol + rtol * std::max(std::fabs(s.phi), std::fabs(phi1));
            const double sr = atol + rtol * std::max(std::fabs(s.r), std::fabs(r1));
            err = std::sqrt(0.5 * ((ep / sp) * (ep / sp) + (er / sr) * (er / sr)));
        }
        if (ok && err <= 1.0) {
            s.N = last ? N_end : s.N + hs;
            s.phi = phi1;
            s.r = r1;
            k1 = k7;
            const double fac = err > 0.0 ? std::min(5.0, 0.9 * std::pow(err, -0.2)) : 5.0;
            if (!last)
                dt = hs * fac;
        } else {
            const double fac = std::isfinite(err) ? std::max(0.2, 0.9 * std::pow(err, -0.2)) : 0.25;
            dt = hs * fac;
            if (!(dt > 1e-14))
                return false;
        }
    }
    return true;
}

// h(a = 1) - 1 for a given lambda; false on failure.
bool h_today(Bg p, const mg_kmo_background_params *q, double lam, double &g)
{
    p.lam = lam;
    State s{std::log(q->a_ini), q->phi_ini, q->dphi_ini};
    double dt = 1e-3;
    if (!integrate_to(p, s, 0.0, q->rtol, dt))
        return false;
    double h;
    if (!hubble2(p, 1.0, s.phi, s.r, h))
        return false;
    g = h - 1.0;
    return true;
}

}  // namespace

extern "C" int mg_kmo_background_defaults(mg_kmo_background_params *p)
{
    if (!p)
        return MG_ERR_ARG;
    p->n = 2;
    p->k0 = 1.0;
    p->beta_kmo = 0.2;
    p->omega_m = 0.3089;
    p->h = 0.6774;
    p->t_cmb = 2.7255;
    p->n_eff = 3.046;
    p->a_ini = 1e-5;
    p->phi_ini = 1e-30;
    p->dphi_ini = 1e-30;
    p->rtol = 1e-12;
    p->h0_tol = 1e-12;
    return MG_OK;
}

extern "C" int mg_kmo_background(const mg_kmo_background_params *q, double lambda_in, int na, const double *a,
                                 double *out, double *lambda_out)
{
    if (!q || na <= 0 || !a || !out)
        return MG_ERR_ARG;
    if (q->n < 2 || q->n > 16 || !(q->k0 >= 0.0) || !std::isfinite(q->k0) || !std::isfinite(q->beta_kmo) ||
        !(q->omega_m > 0.0 && q->omega_m < 1.0) || !(q->h > 0.0) || !(q->t_cmb >= 0.0) || !(q->n_eff >= 0.0) ||
        !(q->a_ini > 0.0 && q->a_ini < 1.0) || !std::isfinite(q->phi_ini) || !std::isfinite(q->dphi_ini) ||
        !(q->rtol >= 1e-14 && q->rtol <= 1e-3) || !(q->h0_tol > 0.0) || !std::isfinite(lambda_in))
        return MG_ERR_ARG;
    for (int i = 0; i < na; ++i)
        if (!(a[i] >= q->a_ini && a[i] <= 100.0))
            return MG_ERR_ARG;
    Bg p{q->n, q->k0, q->beta_kmo, q->omega_m, omega_rad(q->h, q->t_cmb, q->n_eff), 0.0};
    if (!(1.0 - p.om - p.orad > 0.0))
        return MG_ERR_ARG;

    int rc = MG_OK;
    double lam = lambda_in;
    if (!(lam > 0.0)) {
        // bracket the root of g(lambda) = h(1) - 1 from the LCDM value, then Illinois
        double l0 = std::sqrt(3.0 * (1.0 - p.om - p.orad)), g0;
        if (!h_today(p, q, l0, g0))
            return MG_ERR_NONFINITE;
        double l1 = l0, g1 = g0;
        const double fac = g0 > 0.0 ? 1.0 / 1.1 : 1.1;
        int tries = 0;
        while (g1 * g0 > 0.0 && std::fabs(g1) > q->h0_tol) {
            l0 = l1;
            g0 = g1;
            l1 *= fac;
            if (++tries > 200 || !h_today(p, q, l1, g1))
                return MG_ERR_NONFINITE;
        }
        lam = l1;
        double g = g1;
        for (int it = 0; it < 200 && std::fabs(g) > q->h0_tol && g0 != g1; ++it) {
            lam = (l0 * g1 - l1 * g0) / (g1 - g0);
            if (!h_today(p, q, lam, g))
                return MG_ERR_NONFINITE;
            if (g * g1 < 0.0) {       // the root lies between lam and l1
                l0 = l1;
                g0 = g1;
            } else {                  // l0 retained again: halve its value
                g0 *= 0.5;
            }
            l1 = lam;
            g1 = g;
        }
        if (std::fabs(g) > q->h0_tol)
            rc = MG_WARN_NOT_CONVERGED;
    }
    p.lam = lam;

    std::vector<int> order(na);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int x, int y) { return a[x] < a[y]; });
    State s{std::log(q->a_ini), q->phi_ini, q->dphi_ini};
    double dt = 1e-3;
    for (int idx : order) {
        const double N = std::log(a[idx]);
        if (N > s.N && !integrate_to(p, s, N, q->rtol, dt))
            return MG_ERR_NONFINITE;
        double h;
        if (!hubble2(p, a[idx], s.phi, s.r, h))
            return MG_ERR_NONFINITE;
        double *o = out + 5 * (size_t)idx;
        o[0] = std::sqrt(h) / a[idx];
        o[1] = s.phi;
        o[2] = s.r / a[idx];
        o[3] = std::exp(p.beta * s.phi);
        o[4] = std::sqrt(h) * s.r;
    }
    if (lambda_out)
        *lambda_out = lam;
    return rc;
}
