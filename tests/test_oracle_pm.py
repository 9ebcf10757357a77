"""Pins of the oracle's particle-mesh pieces (Sec. 3.1, 3.1.1 of
arXiv:2110.00566): cloud-in-cell assignment, the FFT Poisson solve, force
interpolation and the leapfrog step."""
import numpy as np
import pytest

from paper_2110_00566_gb300 import inputs


def lap7(u):
    out = -6.0 * u
    for ax in range(3):
        out = out + np.roll(u, 1, ax) + np.roll(u, -1, ax)
    return out


def test_cic_mass_and_placement(orc):
    """CIC (Sec. 3.1): each particle's 8 weights sum to one, so delta has
    zero mean; a particle at a cell centre puts all its mass in that cell,
    one at a cell corner splits it equally over 8 cells."""
    ng, nps = 8, 4
    pos = np.array([[2.5, 3.5, 4.5], [1.0, 1.0, 1.0]], dtype=np.float32)
    delta, idx = orc.cic_deposit(pos, ng, nps)
    m = (ng / nps) ** 3
    assert delta[2, 3, 4] == pytest.approx(m - 1.0)
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                assert delta[a, b, c] == pytest.approx(m / 8 - 1.0)
    assert idx[0].tolist() == [2, 3, 4] and idx[1].tolist() == [0, 0, 0]
    pos, _ = inputs.zeldovich(16, 32, 64.0, inputs.pk_cutoff(), 1.0, seed=3)
    delta, _ = orc.cic_deposit(pos, 32, 16)
    assert abs(delta.mean()) < 1e-13


def test_cic_indices_exact(orc):
    """The lower CIC cell is floor(x - 1/2), decided in FP32 on the FP32
    positions; checked against numpy float32 arithmetic, including
    positions at and next to cell centres and the periodic seam."""
    ng = 16
    rng = np.random.default_rng(5)
    pos = rng.uniform(0, ng, (4000, 3)).astype(np.float32)
    edge = np.array([0.0, 0.5, np.nextafter(np.float32(0.5), np.float32(0)), 15.5,
                     np.nextafter(np.float32(16.0), np.float32(0)), 7.5, 7.499999], dtype=np.float32)
    pos[: len(edge)] = edge[:, None]
    _, idx = orc.cic_deposit(pos, ng, 8)
    lo = np.floor(pos - np.float32(0.5)).astype(np.int64) % ng
    assert np.array_equal(idx, lo)


def test_fft_poisson_inverts_the_7_point_laplacian(orc):
    """Sec. 3.1: the discrete Poisson equation is solved exactly by the FFT
    with the 7-point Green's function; the zero mode is dropped."""
    rhs = inputs.white_noise(16, 8)
    phi = orc.fft_poisson(rhs)
    np.testing.assert_allclose(lap7(phi), rhs - rhs.mean(), atol=1e-12)
    assert abs(phi.mean()) < 1e-14


def test_total_momentum_conserved(orc):
    """CIC assignment, a symmetric Green's function, an antisymmetric
    3-point gradient and CIC interpolation with the same weights make the
    self-consistent forces sum to zero over all particles."""
    ng, nps = 16, 8
    pos, _ = inputs.zeldovich(nps, ng, 64.0, inputs.pk_cutoff(), 1.0, seed=9)
    delta, _ = orc.cic_deposit(pos, ng, nps)
    phi = orc.newton_potential(delta, 1.0, 0.3)
    acc = orc.cic_force(phi, pos)
    tot = acc.sum(axis=0)
    assert np.abs(tot).max() < 1e-12 * np.abs(acc).sum()


def _plane_wave_growth(orc, model, rc=1.0, steps=100, a0=0.01, ng=32):
    nps = ng
    q = inputs.cell_centres(ng)
    Q = np.stack(np.meshgrid(q, q, q, indexing="ij"), -1).reshape(-1, 3)
    k = 2 * np.pi / ng
    A0 = 0.005
    om = 0.3
    f0 = inputs.growth_rate_lcdm(a0, om)
    disp = A0 * np.sin(k * Q[:, 0])
    pos = Q.copy()
    pos[:, 0] += disp
    pos = np.mod(pos, ng).astype(np.float32)
    mom = np.zeros_like(pos)
    mom[:, 0] = (a0 ** 2 * orc.E_lcdm(a0, om) * f0 * disp).astype(np.float32)
    da = (1.0 - a0) / steps
    a = a0
    phi = None
    for s in range(steps):
        pos, mom, phi = orc.pm_step(pos, mom, ng, nps, om, a, da, model, rc, first=(s == 0),
                                    phi_guess=phi, opts=orc.Opts(rtol=1e-9))
        a += da
    # the last drift leaves x at a = 1 (momenta half a step ahead)
    d = np.mod(pos[:, 0].astype(np.float64) - Q[:, 0] + ng / 2, ng) - ng / 2
    amp = 2.0 * np.mean(d * np.sin(k * Q[:, 0]))
    return amp / A0


def test_linear_growth_lcdm(orc):
    """A small plane wave (64 cells per wavelength) evolved from z = 99 to 0
    with 200 constant-da leapfrog steps (GR forces only) grows as the LCDM
    linear growth factor.  The 2.5% band covers the two known discrete
    effects, both measured to shrink with resolution: the first steps span
    a large fraction of a (da/a ~ 0.5), and the CIC deposit, CIC
    interpolation and 3-point gradient each damp the force by ~k^2/12."""
    ratio = _plane_wave_growth(orc, model=0, steps=200, ng=64)
    expect = inputs.growth_lcdm(1.0, 0.3) / inputs.growth_lcdm(0.01, 0.3)
    assert ratio == pytest.approx(expect, rel=0.025)
    assert ratio < expect


def _growth_ode(orc, om, rc, a0, dgp):
    from scipy.integrate import solve_ivp

    def rhs(N, y):
        a = np.exp(N)
        oma = om * a ** -3 / (om * a ** -3 + 1 - om)
        g = 1.0 + (1.0 / (3.0 * orc.beta_dgp(a, om, rc)) if dgp else 0.0)
        return [y[1], -(2 - 1.5 * oma) * y[1] + 1.5 * oma * g * y[0]]

    sol = solve_ivp(rhs, [np.log(a0), 0.0], [a0, a0], rtol=1e-10, atol=1e-14)
    return sol.y[0, -1] / a0


def test_linear_growth_ndgp(orc):
    """With the nDGP field solved every step the wave grows as Eq. Dp, whose
    source carries 1 + 1/(3 beta_DGP) (Eq. dgp_linear).  The discrete
    effects of the PM scheme cancel in the nDGP/GR ratio, which must match
    the ratio of the two growth ODE solutions to 0.5%."""
    om, rc, a0 = 0.3, 1.0, 0.01
    expect = _growth_ode(orc, om, rc, a0, True) / _growth_ode(orc, om, rc, a0, False)
    got = _plane_wave_growth(orc, model=1, rc=rc) / _plane_wave_growth(orc, model=0)
    assert got == pytest.approx(expect, rel=0.005)
    assert got > 1.05                      # enhanced growth, beta > 0


def _kmo_pars(beta=0.2, dphibar_da=0.0, A_bar=1.02, bp=0.3):
    return dict(n=2, k0=1.0, beta=beta, lam=1.0, phibar_prime_over_h0=bp, A_bar=A_bar, dphibar_da=dphibar_da)


def _wave_load(ng, amp):
    """One particle per cell, displaced by a small x plane wave."""
    q = np.arange(ng) + 0.5
    X, Y, Z = np.meshgrid(q, q, q, indexing="ij")
    x = X + amp * np.sin(2 * np.pi * X / ng)
    pos = np.stack([x % ng, Y, Z], -1).reshape(-1, 3).astype(np.float32)
    return pos, np.zeros_like(pos)


def test_kmo_step_reduces_to_gr_without_coupling(orc):
    """beta = 0 and A = 1: the Kmouflage step is the GR step, bit for bit."""
    ng = 16
    pos, mom = _wave_load(ng, 0.2)
    k = _kmo_pars(beta=0.0, dphibar_da=0.7, A_bar=1.0)
    p0, m0, _ = orc.pm_step(pos, mom, ng, ng, 0.3, 0.5, 0.01, model=0, first=True)
    p2, m2, _ = orc.pm_step(pos, mom, ng, ng, 0.3, 0.5, 0.01, model=2, first=True, kmo=k, box_mpch=64.0)
    assert np.array_equal(p0, p2) and np.array_equal(m0, m2)


def test_kmo_linear_force_ratio(orc):
    """In the linear regime the Kmouflage kick is A (1 + 2 beta^2 / K1) times
    the GR kick, K1 = 1 + gamma (phibar'/H0)^(2(n-1)): the fifth-force to
    Newtonian ratio the paper derives from Eqs. kmf_eqn_codeunit_lin and
    kmf_Poission_eqn_codeunit (force ratio with the mass variation)."""
    ng = 32
    pos, mom = _wave_load(ng, 1e-3)
    k = _kmo_pars(beta=0.4, A_bar=1.05, bp=0.5)
    a = 0.5
    _, m0, _ = orc.pm_step(pos, mom, ng, ng, 0.3, a, 0.01, model=0, first=True)
    _, m2, _ = orc.pm_step(pos, mom, ng, ng, 0.3, a, 0.01, model=2, first=True, kmo=k, box_mpch=64.0,
                           opts=orc.Opts(rtol=1e-12, max_cycles=60))
    K1 = 1.0 + orc.gamma_kmo(2, k["k0"], a, k["lam"]) * k["phibar_prime_over_h0"] ** 2
    expect = k["A_bar"] * (1.0 + 2.0 * k["beta"] ** 2 / K1)
    sel = np.abs(m0[:, 0]) > 0.5 * np.abs(m0[:, 0]).max()
    ratio = m2[sel, 0] / m0[sel, 0]
    assert np.allclose(ratio, expect, rtol=1e-4)


def test_kmo_friction_on_a_uniform_load(orc):
    """No density contrast: no force, and the momenta decay by the friction
    factor 1 - beta (dphibar/da) da of Eq. force_Kmo2."""
    ng = 16
    pos, _ = _wave_load(ng, 0.0)
    mom = np.full_like(pos, 0.25)
    k = _kmo_pars(beta=0.3, dphibar_da=-0.8)
    _, m2, _ = orc.pm_step(pos, mom, ng, ng, 0.3, 0.5, 0.02, model=2, kmo=k, box_mpch=64.0)
    assert np.allclose(m2, np.float32(0.25 * (1.0 - 0.3 * (-0.8) * 0.02)), rtol=1e-6, atol=1e-7)
