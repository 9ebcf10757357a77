"""Pins of the FP64 oracle's nDGP solver against what the paper and the
mathematics fix, independently of the oracle's own code.

Each test names the passage of arXiv:2110.00566 it pins.
"""
import numpy as np
import pytest

from paper_2110_00566_gb300 import inputs


def lap7(u, h=1.0):
    """7-point periodic Laplacian by array rolls (independent of the oracle)."""
    out = -6.0 * u
    for ax in range(3):
        out = out + np.roll(u, 1, ax) + np.roll(u, -1, ax)
    return out / h ** 2


# ---------------------------------------------------------------- background

def test_beta_alpha_closed_form(orc):
    """Eq. beta_dgp at a=1, Omega_m=0.3, H0 r_c = 1: Omega_rc = 1/4, so
    beta = 1 + (0.3 + 1.4) / (2 sqrt(0.25)) = 2.7 and alpha = 3 beta = 8.1."""
    assert orc.beta_dgp(1.0, 0.3, 1.0) == pytest.approx(2.7, rel=1e-15)
    assert orc.alpha_dgp(1.0, 0.3, 1.0) == pytest.approx(8.1, rel=1e-15)
    # large r_c: beta grows like 1/sqrt(Omega_rc) (GR limit, Sec. 2.1)
    assert orc.beta_dgp(1.0, 0.3, 100.0) == pytest.approx(1.0 + 1.7 * 100.0, rel=1e-12)


# ------------------------------------------------------------ cell operator

def test_N_solves_the_quadratic(orc):
    """Eq. DGP is the root of Eq. dgp_quadratic_eom, (2/3) x^2 + alpha x -
    Sigma = 0, on the branch with x -> 0 as Sigma -> 0 (sign(alpha) rule)."""
    rng = np.random.default_rng(0)
    for alpha in (8.1, 0.3, -2.0):
        for sig in rng.uniform(-0.3 * alpha ** 2, 50.0, 40):
            x, cl = orc.dgp_N(sig, alpha)
            assert cl == 0
            res = 2.0 / 3.0 * x * x + alpha * x - sig
            assert abs(res) <= 1e-12 * (abs(sig) + alpha ** 2)
            # the other root is -(3/2) alpha - x; the chosen one is nearer 0
            assert abs(x) <= abs(-1.5 * alpha - x) + 1e-12
        # literal printed form agrees where it does not cancel
        sig = 3.0 * alpha ** 2
        lit = 0.75 * (-alpha + np.sign(alpha) * np.sqrt(alpha ** 2 + 8.0 * sig / 3.0))
        assert orc.dgp_N(sig, alpha)[0] == pytest.approx(lit, rel=1e-13)
    # small Sigma: linear limit Sigma / alpha
    assert orc.dgp_N(1e-12, 8.1)[0] == pytest.approx(1e-12 / 8.1, rel=1e-12)
    # negative sqrt argument: clamped and counted
    x, cl = orc.dgp_N(-10.0, 1.0)
    assert cl == 1 and x == -0.75


def _rand_field(n, seed):
    return inputs.white_noise(n, seed)


def test_sigma_independent_of_centre(orc):
    """Footnote to Eq. nonlinear_GS_DGP: the discrete Sigma does not depend
    on the centre value u_ijk (a sign slip in a -2u term would break this)."""
    u = _rand_field(8, 11)
    for (i, j, k) in [(0, 0, 0), (3, 5, 7), (7, 1, 2)]:
        s0 = orc.dgp_sigma(u, 1.0, i, j, k, 0.25)
        v = u.copy()
        v[i, j, k] += 3.7
        assert orc.dgp_sigma(v, 1.0, i, j, k, 0.25) == pytest.approx(s0, rel=1e-12, abs=1e-12)


def test_sigma_rewritten_identity(orc):
    """The printed (2/3h^4)[Dxx^2 + ... - DxxDyy - ...] equals
    [(Sx-Sy)^2 + (Sx-Sz)^2 + (Sy-Sz)^2]/(3h^4), with S_a the pair sums of
    the face neighbours, since D_aa - D_bb = S_a - S_b."""
    u = _rand_field(8, 12)
    h = 2.0
    for (i, j, k) in [(1, 2, 3), (0, 7, 4), (6, 6, 6)]:
        g = lambda a, b, c: u[(i + a) % 8, (j + b) % 8, (k + c) % 8]
        Sx, Sy, Sz = g(1, 0, 0) + g(-1, 0, 0), g(0, 1, 0) + g(0, -1, 0), g(0, 0, 1) + g(0, 0, -1)
        Cxy = g(1, 1, 0) + g(-1, -1, 0) - g(1, -1, 0) - g(-1, 1, 0)
        Cxz = g(1, 0, 1) + g(-1, 0, -1) - g(1, 0, -1) - g(-1, 0, 1)
        Cyz = g(0, 1, 1) + g(0, -1, -1) - g(0, 1, -1) - g(0, -1, 1)
        Q = ((Sx - Sy) ** 2 + (Sx - Sz) ** 2 + (Sy - Sz) ** 2) / (3 * h ** 4) \
            + (Cxy ** 2 + Cxz ** 2 + Cyz ** 2) / (8 * h ** 4)
        assert orc.dgp_sigma(u, h, i, j, k, 0.0) == pytest.approx(Q, rel=1e-12)


def _manufactured(n, m=(1, 2, 3), A=0.7):
    """u = A[s1 s2 + s2 s3 + s3 s1], s_a = sin(k_a x_a), k_a = 2 pi m_a / n,
    at cell centres, with its exact Hessian."""
    x = inputs.cell_centres(n)
    k = [2 * np.pi * mm / n for mm in m]
    X = np.meshgrid(x, x, x, indexing="ij")
    s = [np.sin(k[a] * X[a]) for a in range(3)]
    c = [np.cos(k[a] * X[a]) for a in range(3)]
    u = A * (s[0] * s[1] + s[1] * s[2] + s[2] * s[0])
    H = np.zeros((3, 3) + u.shape)
    H[0, 0] = -k[0] ** 2 * A * (s[0] * s[1] + s[2] * s[0])
    H[1, 1] = -k[1] ** 2 * A * (s[0] * s[1] + s[1] * s[2])
    H[2, 2] = -k[2] ** 2 * A * (s[1] * s[2] + s[2] * s[0])
    H[0, 1] = H[1, 0] = k[0] * k[1] * A * c[0] * c[1]
    H[1, 2] = H[2, 1] = k[1] * k[2] * A * c[1] * c[2]
    H[0, 2] = H[2, 0] = k[0] * k[2] * A * c[0] * c[2]
    return u, H, k


def test_sigma_second_order_consistent(orc):
    """Sec. 3.2.3: the discrete Sigma approximates the traceless part
    sum_ij (d_i d_j u - delta_ij Lap u / 3)^2 to O(h^2): the error falls by
    ~4 per halving of the cell (which fixes the 2/3 and 1/8 coefficients)."""
    errs = []
    for n in (32, 64, 128):
        u, H, _ = _manufactured(n)
        tr = H[0, 0] + H[1, 1] + H[2, 2]
        cont = sum(H[a, b] ** 2 for a in range(3) for b in range(3)) - tr ** 2 / 3.0
        disc = np.array([[[orc.dgp_sigma(u, 1.0, i, j, k, 0.0) for k in range(n)]
                          for j in range(n)] for i in range(n)])
        errs.append(np.sqrt(np.mean((disc - cont) ** 2)) / np.sqrt(np.mean(cont ** 2)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.7 < r1 < 4.2 and 3.85 < r2 < 4.15, errs


# ---------------------------------------------------- smoother and residual

def test_smoother_is_the_local_exact_solve(orc):
    """Eq. nonlinear_GS_DGP with dL/du = -6/h^2: with every other cell held
    at its old value, the updated value zeroes L(u) - f at that cell."""
    n, h, alpha, c = 8, 2.0, 1.7, 0.013
    u = 0.3 * _rand_field(n, 21)
    s = 0.5 * _rand_field(n, 22)
    f = 0.05 * _rand_field(n, 23)
    op = orc.dgp_op(alpha)
    out = orc.smooth(op, u, s, f, h, c, colour=1)
    for (i, j, k) in [(0, 0, 1), (3, 4, 0), (7, 7, 7), (2, 2, 3)]:
        assert (i + j + k) % 2 == 1
        v = u.copy()
        v[i, j, k] = out[i, j, k]
        N = orc.dgp_N(orc.dgp_sigma(v, h, i, j, k, s[i, j, k]), alpha)[0]
        L = lap7(v, h)[i, j, k] - N + c
        assert abs(L - f[i, j, k]) < 1e-12 * (1 + abs(f[i, j, k]))
    # the other colour is untouched
    par = np.add.outer(np.add.outer(np.arange(n), np.arange(n)), np.arange(n)) % 2
    assert np.array_equal(out[par == 0], u[par == 0])


def test_residual_definition(orc):
    """Eqs. general_pde_numerical .. residual_d with the compatibility
    constant: d = Lap u - N + <N> - f and eps = rms(d)."""
    n, h, alpha = 8, 1.0, 8.1
    u = 0.2 * _rand_field(n, 31)
    s = 2.0 * _rand_field(n, 32)
    f = 0.1 * _rand_field(n, 33)
    op = orc.dgp_op(alpha)
    Nf, _ = orc.N_field(op, u, s, h)
    d, c, eps = orc.residual(op, u, s, f, h)
    assert c == pytest.approx(Nf.mean(), rel=1e-13)
    np.testing.assert_allclose(d, lap7(u, h) - Nf + Nf.mean() - f, rtol=0, atol=1e-13)
    assert eps == pytest.approx(np.sqrt(np.mean(d ** 2)), rel=1e-13)


# ------------------------------------------------ restriction / prolongation

def test_restriction_is_the_8_cell_average(orc):
    f = _rand_field(8, 41)
    r = orc.restrict(f)
    np.testing.assert_allclose(r, f.reshape(4, 2, 4, 2, 4, 2).mean(axis=(1, 3, 5)), atol=1e-15)


def test_prolongation_weights(orc):
    """Sec. 3.2.1 prolongation: weights 27/64, 9/64, 3/64, 1/64 sum to one
    (a constant correction is reproduced), linear fields are reproduced
    exactly away from the periodic seam (it is trilinear interpolation
    between coarse centres), and a single coarse spike spreads with exactly
    the printed weights."""
    nc = 8
    z = np.zeros((2 * nc,) * 3)
    zc = np.zeros((nc,) * 3)
    out = orc.prolong_add(z, np.full((nc,) * 3, 2.5), zc)
    np.testing.assert_allclose(out, 2.5, atol=1e-15)
    Xc = (np.arange(nc) * 2 + 1.0)
    lin_c = (0.3 * Xc[:, None, None] - 0.2 * Xc[None, :, None] + 0.7 * Xc[None, None, :])
    out = orc.prolong_add(z, lin_c, zc)
    xf = np.arange(2 * nc) + 0.5
    lin_f = 0.3 * xf[:, None, None] - 0.2 * xf[None, :, None] + 0.7 * xf[None, None, :]
    inner = (slice(1, -1),) * 3
    np.testing.assert_allclose(out[inner], lin_f[inner], atol=1e-12)
    spike = np.zeros((nc,) * 3)
    spike[3, 3, 3] = 64.0
    out = orc.prolong_add(z, spike, zc)
    # fine cells (6..7) are children of coarse 3: weight 27
    assert out[6, 7, 6] == pytest.approx(27.0)
    # fine cell 8 has parent 4 and neighbour 3 along x (on its low side): 9
    assert out[8, 6, 7] == pytest.approx(9.0)
    assert out[8, 8, 7] == pytest.approx(3.0)
    assert out[8, 8, 8] == pytest.approx(1.0)
    assert out[9, 7, 7] == 0.0        # parent 4, neighbour 5: no weight from 3
    assert out.sum() == pytest.approx(64.0 * 8)


# ----------------------------------------------------------- full solves

def test_exact_discrete_1d_solution(orc, paper):
    """Sec. 4.2.2 with Eq. sine_nDGP: delta = -(a beta/(Omega_m N^2))
    sin(2 pi x/N).  For a 1D field Sigma = (2/3)(Lap u)^2 + s, so the exact
    discrete solution of Eq. DGP is the linear one,
    u = sin(2 pi x/N) / (N^2 (2 - 2 cos(2 pi/N))), whose continuum limit is
    the paper's sin(2 pi x/N)/(4 pi^2).  Checked along each axis."""
    a, om, rc = 1.0, 0.3, 1.0
    beta = orc.beta_dgp(a, om, rc)
    for n in (16, 32):
        for axis in range(3):
            delta = -(a * beta / (om * n * n)) * inputs.sine_pattern(n, 1, axis)
            u, st = orc.dgp_solve(delta, a, om, rc, orc.Opts(rtol=1e-13, max_cycles=40))
            exact = inputs.sine_pattern(n, 1, axis) / (n * n * (2 - 2 * np.cos(2 * np.pi / n)))
            assert np.abs(u - exact).max() < 1e-10 * np.abs(exact).max()
            assert st.eps[-1] <= 1e-13 * st.eps_ref
    # the paper's continuum amplitude 1/(4 pi^2) is approached at O(h^2)
    amp = lambda n: 1.0 / (n * n * (2 - 2 * np.cos(2 * np.pi / n)))
    printed = paper["ndgp_sine_test"]["continuum_amplitude"]
    assert abs(amp(64) - printed) < 1e-3 * printed
    assert abs(amp(64) - printed) < abs(amp(32) - printed) / 3.9


def test_uniform_density(orc, paper):
    """Sec. 4.2.1: delta = 0 with a U[-0.05, 0.05] initial guess relaxes to
    a constant field (zero after the gauge fix)."""
    n = 16
    lo, hi = paper["uniform_test"]["initial_guess_range"]
    u0 = inputs.uniform_guess(n, seed=1, half_width=hi)
    assert u0.min() >= lo and u0.max() <= hi
    u, st = orc.dgp_solve(np.zeros((n,) * 3), 1.0, 0.3, 1.0, orc.Opts(rtol=0.0, atol=1e-13), u0)
    assert np.abs(u).max() < 1e-12
    assert st.eps[0] > 1e-3


def test_linear_limit(orc):
    """Eq. dgp_linear: for small delta the nonlinear terms vanish and
    Lap phi = Omega_m a^-1 delta / beta.  The MG solution approaches the FFT
    solution of the discrete linear equation with a relative difference
    proportional to the amplitude (slope 1)."""
    n, a, om, rc = 16, 1.0, 0.3, 1.0
    beta = orc.beta_dgp(a, om, rc)
    base = inputs.white_noise(n, 7)
    diffs = []
    for eps_amp in (1e-1, 1e-2, 1e-3):
        delta = eps_amp * base
        u, _ = orc.dgp_solve(delta, a, om, rc, orc.Opts(rtol=1e-13, max_cycles=40))
        lin = orc.fft_poisson(om / (a * beta) * (delta - delta.mean()))
        diffs.append(np.linalg.norm(u - lin) / np.linalg.norm(lin))
    assert 7.0 < diffs[0] / diffs[1] < 13.0 and 7.0 < diffs[1] / diffs[2] < 13.0, diffs
    assert diffs[2] < 1e-2


def _newton_solve(orc, op, s0, n):
    """Brute-force Newton on the discrete system F(u) = d(u) = 0 plus the
    gauge row <u> = 0: dense central-difference Jacobian, least squares."""
    u = np.zeros((n,) * 3)
    F = lambda v: orc.residual(op, v, s0, None, 1.0)[0].ravel()
    for _ in range(30):
        r = F(u)
        if np.abs(r).max() < 1e-14 * max(1.0, np.abs(s0).max()):
            break
        J = np.empty((n ** 3, n ** 3))
        hstep = 1e-5
        for q in range(n ** 3):
            e = np.zeros(n ** 3)
            e[q] = hstep
            J[:, q] = (F(u + e.reshape(u.shape)) - F(u - e.reshape(u.shape))) / (2 * hstep)
        A = np.vstack([J, np.full((1, n ** 3), 1.0 / n ** 3)])
        b = -np.concatenate([r, [u.mean()]])
        du = np.linalg.lstsq(A, b, rcond=None)[0]
        u = u + du.reshape(u.shape)
    return u


@pytest.mark.parametrize("seed,rms,rc", [(1, 0.3, 1.0), (2, 1.0, 5.0), (3, 3.0, 10.0), (4, 10.0, 10.0)])
def test_mg_matches_brute_force_newton(orc, seed, rms, rc):
    """The FAS V-cycles (Sec. 3.2.1) converge to the root of the discrete
    nDGP system found by a dense Newton solve on an 8^3 mesh."""
    n, a, om = 8, 1.0, 0.3
    delta = inputs.white_noise(n, 100 + seed)
    delta = rms * delta / delta.std()
    s0, eps_ref, alpha, _ = orc.dgp_source(delta, a, om, rc)
    op = orc.dgp_op(alpha)
    un = _newton_solve(orc, op, s0, n)
    u, st = orc.mg_solve(op, s0, eps_ref, orc.Opts(rtol=1e-14, max_cycles=60))
    assert np.linalg.norm(u - un) < 1e-10 * np.linalg.norm(un)
    # genuinely nonlinear: differs from the linear solution
    lin = orc.fft_poisson(s0 / alpha)
    assert np.linalg.norm(u - lin) > 1e-4 * np.linalg.norm(lin)


def test_invariants(orc):
    """Shift symmetry and lattice symmetries of the discrete system: a
    constant added to the guess, an axis permutation or an even periodic
    roll of delta give the transformed solution; a cycle started at the
    solution stays there (FAS fixed point)."""
    n, a, om, rc = 16, 1.0, 0.3, 1.0
    delta = 2.0 * inputs.white_noise(n, 5)
    opts = orc.Opts(rtol=1e-13, max_cycles=40)
    u, _ = orc.dgp_solve(delta, a, om, rc, opts)
    scale = np.abs(u).max()
    u2, _ = orc.dgp_solve(delta, a, om, rc, opts, u0=u + 3.0)
    assert np.abs(u2 - u).max() < 1e-11 * scale
    up, _ = orc.dgp_solve(delta.transpose(2, 0, 1).copy(), a, om, rc, opts)
    assert np.abs(up - u.transpose(2, 0, 1)).max() < 1e-11 * scale
    ur, _ = orc.dgp_solve(np.roll(delta, (2, 4, 6), (0, 1, 2)).copy(), a, om, rc, opts)
    assert np.abs(ur - np.roll(u, (2, 4, 6), (0, 1, 2))).max() < 1e-11 * scale
    u3, st = orc.dgp_solve(delta, a, om, rc, orc.Opts(rtol=0.0, atol=0.0, max_cycles=1), u0=u)
    assert np.abs(u3 - u).max() < 1e-12 * scale


def test_cycle_types_agree(orc):
    """V, F and W cycles (Sec. 3.2.1, Fig. multigrid_cycles) reach the same
    discrete solution; F and W need no more cycles than V."""
    n = 16
    delta = 2.0 * inputs.white_noise(n, 9)
    sols = {}
    for cyc in (0, 1, 2):
        sols[cyc] = orc.dgp_solve(delta, 1.0, 0.3, 1.0, orc.Opts(rtol=1e-12, cycle=cyc, max_cycles=40))
    for cyc in (1, 2):
        assert np.abs(sols[cyc][0] - sols[0][0]).max() < 1e-9 * np.abs(sols[0][0]).max()
        assert sols[cyc][1].cycles <= sols[0][1].cycles


def test_sphere_shape(orc, paper):
    """Sec. 4.2.3 (Eqs. phir_in, phir_out with R_c^2 in place of the printed
    R_c, which is what Eq. dgp_eom_code gives; identical at R_c = 1): top
    hat delta = 0.5, R = 0.1 N at the mesh centre.  dphi/dr along the axes
    agrees with the closed form near the centre to a few per cent (the
    closed form ignores the periodic images)."""
    n, a, om = 64, 1.0, 0.3
    t = paper["ndgp_sphere_test"]
    R = t["R_over_Ng"] * n
    delta = inputs.tophat_sphere(n, R, t["delta"])
    for rc in t["H0_rc"]:
        u, _ = orc.dgp_solve(delta, a, om, rc, orc.Opts(rtol=1e-10))
        beta = orc.beta_dgp(a, om, rc)
        dm = t["delta"] - delta.mean()    # the solver sees delta - <delta>

        def dphidr(r):
            d = dm if r <= R else dm * R ** 3 / r ** 3
            return 0.75 * beta / rc ** 2 * (np.sqrt(1 + 8 * om * rc ** 2 / (9 * beta ** 2) * d) - 1) * r

        c = n // 2
        # r = distance from the mesh centre (a cell corner) of cell centre c+m
        for m in (1, 2, 3, 5, 7):
            # along the x axis through cells (c+m, c, c) and (c+m-1, c, c):
            # the difference quotient sits at x = c + m, y = z = 1/2 off axis
            g = u[c + m, c, c] - u[c + m - 1, c, c]
            r = np.sqrt(m ** 2 + 0.5)
            expect = dphidr(r) * m / r
            assert g == pytest.approx(expect, rel=0.08), (rc, m, g, expect)


# ------------------------------------------------------- reference gradient

def test_reference_gradient_matches_finite_differences(orc):
    """The oracle's dense-Jacobian gradient of L = <g, phi> equals central
    differences of the oracle's own solution map, in delta along random
    directions and in R_c (strongly nonlinear field, 8^3)."""
    n, a, om, rc = 8, 1.0, 0.3, 1.0
    delta = 3.0 * inputs.white_noise(n, 201)
    g = inputs.white_noise(n, 202)
    dd, dr, phi = orc.dgp_gradient(delta, a, om, rc, g)
    opts = orc.Opts(rtol=1e-14, max_cycles=80)
    L = lambda d, r: float(np.sum(g * orc.dgp_solve(d, a, om, r, opts)[0]))
    for seed in (203, 204, 205):
        v = inputs.white_noise(n, seed)
        eps = 1e-4
        fd = (L(delta + eps * v, rc) - L(delta - eps * v, rc)) / (2 * eps)
        assert float(np.sum(dd * v)) == pytest.approx(fd, rel=1e-6, abs=1e-10)
    fd = (L(delta, rc * (1 + 1e-5)) - L(delta, rc * (1 - 1e-5))) / (2e-5 * rc)
    assert dr == pytest.approx(fd, rel=1e-5)


def test_reference_gradient_linear_limit(orc):
    """For small delta the solution map is the linear Poisson solve
    Lap phi = Omega_m a^-1 Pi delta / beta, whose Green's function is
    symmetric, so dL/ddelta = (Omega_m/(a beta)) Pi G(Pi g)."""
    n, a, om, rc = 8, 1.0, 0.3, 2.0
    delta = 1e-7 * inputs.white_noise(n, 206)
    g = inputs.white_noise(n, 207)
    dd, _, _ = orc.dgp_gradient(delta, a, om, rc, g)
    beta = orc.beta_dgp(a, om, rc)
    ref = om / (a * beta) * orc.fft_poisson(g - g.mean())
    ref -= ref.mean()
    assert np.abs(dd - ref).max() < 1e-6 * np.abs(ref).max()
