"""Pins of the Kmouflage background oracle (oracle/background.py) against
closed forms and invariants that do not depend on the oracle itself:

* the radiation density of a 2.7255 K black body and the massless-neutrino
  ratio (textbook values);
* the uncoupled limit beta = 0, where the system is LCDM with radiation:
  lambda^2 = 3 (1 - Omega_m - Omega_r) and H(a) in closed form;
* the coupled-quintessence matter era (K0 = 0, no radiation), whose exact
  attractor is ring(phi) = -2 beta (the cubic (x + 2 beta)(x^2 - 6) = 0 of
  the fixed point of the three equations);
* d(h)/dN along the solution, with h taken from the Friedmann equation,
  equals 2 H'/H0^2 from the acceleration equation (the two equations and
  the field equation are consistent only together: a dropped or mis-signed
  term in any of them breaks this);
* the paper's qualitative statements on the models it ran (Sec. 4.1): the
  background field is negative and falls with time, A < 1 at late times,
  and H(a = 1) = H0 after the shooting."""
import math

import numpy as np
import pytest

from oracle import background as ob


def test_radiation_density():
    bg = ob.Background(h=1.0, n_eff=0.0)
    assert bg.omega_r == pytest.approx(2.4730e-5, rel=3e-4)          # Omega_gamma h^2 at 2.7255 K
    ratio = ob.omega_radiation(0.6774) / ob.omega_radiation(0.6774, n_eff=0.0)
    assert ratio == pytest.approx(1.0 + 3.046 * 0.2271, rel=1e-4)          # textbook 0.2271 per species


@pytest.mark.parametrize("n,k0", [(2, 1.0), (3, 10.0)])
def test_uncoupled_limit_is_lcdm(n, k0):
    bg = ob.Background(n=n, k0=k0, beta=0.0)
    a = np.array([1e-5, 1e-3, 0.02, 0.3, 1.0, 1.5])
    lam, tab = ob.solve(bg, a)
    om, orad = bg.omega_m, bg.omega_r
    assert lam ** 2 == pytest.approx(3.0 * (1.0 - om - orad), rel=1e-11)
    E = np.sqrt(orad / a ** 4 + om / a ** 3 + (1.0 - om - orad))
    np.testing.assert_allclose(tab[:, 0], E, rtol=1e-11)
    assert np.abs(tab[:, 1]).max() < 1e-20
    np.testing.assert_array_equal(tab[:, 3], 1.0)


@pytest.mark.parametrize("beta", [0.1, 0.3])
def test_coupled_matter_era_attractor(beta):
    bg = ob.Background(k0=0.0, beta=beta, t_cmb=0.0, a_ini=1e-10)
    lam = math.sqrt(3.0 * (1.0 - bg.omega_m))
    a = np.array([1e-3, 3e-3])
    _, tab = ob.solve(bg, a, lam=lam)
    ring = tab[:, 2] * a                                   # d phi / dN
    np.testing.assert_allclose(ring, -2.0 * beta, rtol=2e-5)
    # h (1 - ring^2 / 6) = A Omega_m / a there
    h = (tab[:, 0] * a) ** 2
    np.testing.assert_allclose(h * (1.0 - ring ** 2 / 6.0) * a / (tab[:, 3] * bg.omega_m), 1.0, rtol=2e-5)


@pytest.mark.parametrize("n,k0,beta", [(2, 1.0, 0.2), (3, 1.0, 0.2), (2, 100.0, 0.3)])
def test_friedmann_derivative_matches_acceleration(n, k0, beta):
    bg = ob.Background(n=n, k0=k0, beta=beta)
    lam = ob.shoot_lambda(bg)
    sol = ob.integrate(lam, bg, N_end=0.2, dense=True)

    def h_at(N):
        phi, dphi = sol.sol(N)
        return ob.hubble2(N, phi, dphi, lam, bg)

    d = 1e-4
    for N in (-9.0, -6.0, -3.0, -1.0, 0.0):
        fd = (h_at(N + d) - h_at(N - d)) / (2 * d)
        phi, dphi = sol.sol(N)
        hp = ob.hubble_prime(N, phi, dphi, h_at(N), lam, bg)
        assert fd == pytest.approx(2.0 * hp, rel=2e-7), N
        if N >= -3.0:
            # the scalar's part of d h / dN is not negligible here (so the test sees the field equation)
            hp0 = ob.hubble_prime(N, phi, 0.0, h_at(N), lam, bg)
            assert abs(hp - hp0) > 1e-3 * abs(hp)


def test_shooting_and_paper_statements():
    a = np.array([0.1, 0.3, 0.6, 1.0])
    res = {}
    for k0 in (1.0, 10.0, 100.0):
        bg = ob.Background(n=2, k0=k0, beta=0.2)
        lam, tab = ob.solve(bg, a)
        assert tab[-1, 0] == pytest.approx(1.0, abs=1e-11)
        assert (tab[:, 1] < 0).all() and (np.diff(tab[:, 1]) < 0).all()
        assert (tab[:, 2] < 0).all() and (tab[:, 3] < 1.0).all()
        res[k0] = tab[-1, 1]
    # a stiffer kinetic function screens the background field more
    assert abs(res[1.0]) > abs(res[10.0]) > abs(res[100.0])
