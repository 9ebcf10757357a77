"""FP64 oracle of the Kmouflage background cosmology (Sec. 3.2.4, the
background solver): the scalar's field equation, the modified Friedmann
equation and the acceleration equation, integrated in N = ln a, with the
coupling scale lambda fixed by shooting on H(a = 1) = H0.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  scipy's DOP853
integrator and Brent root finder serve as library steps; the physics is
written out below from the paper's equations.

Units: phi is the dimensionless field (phi / M_Pl), h = (conformal Hubble
rate / H0)^2, an over-ring is d/dN.  The model is K(X) = -1 + X + K0 X^n
(Eq. kmf_model_K_function), A(phi) = exp(beta phi), and on the background
X = phidot^2 / (2 H0^2 lambda^2) = h ring(phi)^2 / (2 lambda^2 a^2)
(the definition of X below Eq. kmouflage_eom with a phidot = H ring(phi)).

Readings (each pinned in tests/test_oracle_background.py):
* Friedmann: Eq. kmf_background_Friedmann multiplied by a^2 / H0^2,
  h = Omega_r a^-2 + A Omega_m a^-1 + (1/3) K_X h ring(phi)^2
      - (1/3) lambda^2 a^2 K(X),
  solved for h at fixed (a, phi, ring(phi)) as the smallest root above the
  K0 = 0 value (the branch continuous with LCDM).  The printed rewritten
  form (Eq. kmf_background_Friedmann2) is not used: it drops a square on
  ring(phi) and a factor a^2 in its last term.
* Acceleration: conformal-time form of a''/a = -(4 pi G / 3)(rho + 3p) with
  the scalar's rho = M_Pl^2 (K_X phidot^2 - lambda^2 H0^2 K) and
  p = M_Pl^2 lambda^2 H0^2 K, i.e.
  H'/H0^2 = -Omega_r a^-2 - (1/2) A Omega_m a^-1 - (1/6) K_X h ring(phi)^2
            - (1/3) lambda^2 a^2 K(X).
  The printed Eq. kmf_background_Raychaudhuri carries twice these scalar
  terms; its K = -1 limit would give a''/a = 2 Lambda / 3 instead of the
  Lambda / 3 its own Friedmann equation implies.
* Field equation: Eq. kmf_background_eom2 as printed (derived again from
  Eq. kmf_background_eom with the conformal-time identities below it).
* Radiation: photons at T_cmb plus n_eff massless neutrinos, each adding
  (7/8)(4/11)^(4/3) of the photon density.
* Initial conditions: phi = ring(phi) = 1e-30 at a_ini = 1e-5 (z = 1e5).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

# SI constants (CODATA 2018) for the radiation density.
SIGMA_SB = 5.670374419e-8       # W m^-2 K^-4
C_LIGHT = 299792458.0           # m s^-1
G_NEWTON = 6.67430e-11          # m^3 kg^-1 s^-2
MPC_M = 3.0856775814913673e22   # m


def omega_radiation(h, t_cmb=2.7255, n_eff=3.046):
    """Omega_r of photons at t_cmb plus n_eff massless neutrino species.
    rho_gamma = 4 sigma T^4 / c^3 (mass density); rho_crit = 3 H0^2 / (8 pi G)."""
    rho_gamma = 4.0 * SIGMA_SB * t_cmb ** 4 / C_LIGHT ** 3
    H0 = 100.0 * h * 1e3 / MPC_M
    rho_crit = 3.0 * H0 * H0 / (8.0 * math.pi * G_NEWTON)
    return rho_gamma / rho_crit * (1.0 + n_eff * 7.0 / 8.0 * (4.0 / 11.0) ** (4.0 / 3.0))


@dataclass
class Background:
    n: int = 2
    k0: float = 1.0
    beta: float = 0.2
    omega_m: float = 0.3089
    h: float = 0.6774
    t_cmb: float = 2.7255
    n_eff: float = 3.046
    a_ini: float = 1e-5
    phi_ini: float = 1e-30
    dphi_ini: float = 1e-30

    @property
    def omega_r(self):
        return omega_radiation(self.h, self.t_cmb, self.n_eff)


def K(X, bg):
    return -1.0 + X + bg.k0 * X ** bg.n


def K_X(X, bg):
    return 1.0 + bg.n * bg.k0 * X ** (bg.n - 1)


def K_XX(X, bg):
    return bg.n * (bg.n - 1) * bg.k0 * X ** (bg.n - 2)


def friedmann_residual(hh, N, phi, dphi, lam, bg):
    """h minus the right-hand side of the Friedmann equation (times a^2/H0^2)."""
    a = math.exp(N)
    X = hh * dphi * dphi / (2.0 * lam * lam * a * a)
    rhs = (bg.omega_r / (a * a) + math.exp(bg.beta * phi) * bg.omega_m / a
           + K_X(X, bg) * hh * dphi * dphi / 3.0 - lam * lam * a * a * K(X, bg) / 3.0)
    return hh - rhs


def hubble2(N, phi, dphi, lam, bg):
    """h = (H/H0)^2 from the Friedmann equation: Brent's method on its
    residual between the K0 = 0 root and the residual's maximum."""
    a = math.exp(N)
    B = bg.omega_r / (a * a) + math.exp(bg.beta * phi) * bg.omega_m / a + lam * lam * a * a / 3.0
    D = 1.0 - dphi * dphi / 6.0
    lo = B / D
    if bg.k0 == 0.0 or dphi == 0.0:
        return lo
    # residual = D h - B - C h^n with C > 0: its maximum is at (D / (n C))^(1/(n-1))
    X1 = dphi * dphi / (2.0 * lam * lam * a * a)
    C = (2 * bg.n - 1) / 3.0 * bg.k0 * lam * lam * a * a * X1 ** bg.n
    hi = (D / (bg.n * C)) ** (1.0 / (bg.n - 1))
    flo = friedmann_residual(lo, N, phi, dphi, lam, bg)
    if flo >= 0.0:
        return lo
    if friedmann_residual(hi, N, phi, dphi, lam, bg) < 0.0:
        raise ArithmeticError("Friedmann equation has no real root")
    return brentq(friedmann_residual, lo, hi, args=(N, phi, dphi, lam, bg), xtol=1e-300, rtol=1e-15,
                  maxiter=500)


def hubble_prime(N, phi, dphi, hh, lam, bg):
    """H'/H0^2 (conformal time) from the acceleration equation."""
    a = math.exp(N)
    X = hh * dphi * dphi / (2.0 * lam * lam * a * a)
    return (-bg.omega_r / (a * a) - 0.5 * math.exp(bg.beta * phi) * bg.omega_m / a
            - K_X(X, bg) * hh * dphi * dphi / 6.0 - lam * lam * a * a * K(X, bg) / 3.0)


def rhs(N, y, lam, bg):
    """d/dN (phi, ring(phi)) from Eq. kmf_background_eom2."""
    phi, dphi = y
    hh = hubble2(N, phi, dphi, lam, bg)
    hp = hubble_prime(N, phi, dphi, hh, lam, bg)
    a = math.exp(N)
    X = hh * dphi * dphi / (2.0 * lam * lam * a * a)
    kx, kxx = K_X(X, bg), K_XX(X, bg)
    c2 = kx + 2.0 * X * kxx
    coupling = 3.0 * bg.beta * math.exp(bg.beta * phi) * bg.omega_m * math.exp(-N)
    ddphi = -(c2 * hp * dphi + 2.0 * (kx - X * kxx) * hh * dphi + coupling) / (c2 * hh)
    return [dphi, ddphi]


def integrate(lam, bg, N_end=0.0, dense=False, rtol=1e-12, atol=1e-30):
    return solve_ivp(rhs, (math.log(bg.a_ini), N_end), [bg.phi_ini, bg.dphi_ini], method="DOP853",
                     args=(lam, bg), rtol=rtol, atol=atol, dense_output=dense)


def h_today(lam, bg):
    sol = integrate(lam, bg)
    phi, dphi = sol.y[:, -1]
    return hubble2(0.0, phi, dphi, lam, bg)


def shoot_lambda(bg, tol=1e-13):
    """lambda such that H(a = 1) = H0: Brent's method on h(a = 1) - 1, bracketed
    around the LCDM value sqrt(3 (1 - Omega_m - Omega_r))."""
    lam0 = math.sqrt(3.0 * (1.0 - bg.omega_m - bg.omega_r))
    lo, hi = 0.5 * lam0, 2.0 * lam0
    while h_today(lo, bg) > 1.0:
        lo *= 0.5
    while h_today(hi, bg) < 1.0:
        hi *= 2.0
    return brentq(lambda l: h_today(l, bg) - 1.0, lo, hi, xtol=1e-300, rtol=tol, maxiter=200)


def solve(bg: Background, a_out, lam=None):
    """Background at the scale factors a_out: lambda and a (len, 5) table of
    [H/H0, phibar, dphibar/da, A(phibar), phibar'/H0] (phibar' the conformal
    time derivative)."""
    if lam is None:
        lam = shoot_lambda(bg)
    a_out = np.asarray(a_out, dtype=np.float64)
    N_end = max(0.0, float(np.log(a_out.max())))
    sol = integrate(lam, bg, N_end=N_end, dense=True)
    out = np.empty((a_out.size, 5))
    for i, a in enumerate(a_out):
        N = math.log(a)
        phi, dphi = sol.sol(N)
        hh = hubble2(N, phi, dphi, lam, bg)
        out[i] = [math.sqrt(hh) / a, phi, dphi / a, math.exp(bg.beta * phi), math.sqrt(hh) * dphi]
    return lam, out
