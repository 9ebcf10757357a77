"""Pins of the FP64 oracle of the differentiable particle-mesh chain
(oracle/dpm.py): each piece against the oracle's C code or a closed form,
the sparse nDGP Jacobian against central differences of the C residual, the
implicit-function adjoint against the dense finite-difference gradient, and
the whole-chain gradient against central differences of the loss."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import dpm
from paper_2110_00566_gb300 import inputs

torch = pytest.importorskip("torch")


def grid_positions(n, npart, seed):
    """Positions exactly representable in FP32, so the C oracle (FP32
    positions) and the FP64 chain see the same particles."""
    u = inputs.uniform01(seed, 3 * npart).reshape(npart, 3)
    return np.ascontiguousarray((np.floor(u * n * 1024) / 1024.0) % n)


def test_cic_density_matches_c_oracle():
    n, npart = 8, 512
    x = grid_positions(n, npart, 11)
    ref, _ = oracle.cic_deposit(x.astype(np.float32), n, 8)
    got = dpm.cic_density(torch.from_numpy(x), n).numpy()
    assert np.abs(got - ref).max() < 1e-13


def test_newton_matches_c_oracle():
    n = 16
    d = inputs.white_noise(n, 12)
    d -= d.mean()
    ref = oracle.newton_potential(d, 0.5, 0.3)
    got = dpm.newton(torch.from_numpy(d), 0.5, 0.3).numpy()
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_force_matches_c_oracle():
    n, npart = 8, 300
    x = grid_positions(n, npart, 13)
    phi = inputs.white_noise(n, 14)
    ref = oracle.cic_force(phi, x.astype(np.float32))
    got = dpm.force(torch.from_numpy(phi), torch.from_numpy(x)).numpy()
    assert np.abs(got - ref).max() < 1e-13


def test_zeldovich_divergence_is_minus_delta():
    """i k . psi(k) = -delta_L(k) on modes with no Nyquist component, and the
    lattice plus displacement matches the input generator's load."""
    n, box = 16, 64.0
    pk = inputs.pk_cutoff()
    amp = inputs.pk_amplitude(n, box, pk)
    w = inputs.white_noise(n, 15)
    cfg = dpm.DpmConfig(ng=n, box=box, omega_m=0.3, a_start=0.1, a_end=1.0, nsteps=1, growth=1.0, vel=0.0)
    x, _ = dpm.zeldovich(torch.from_numpy(w), amp, cfg)
    q = (np.arange(n) + 0.5)
    lat = np.stack(np.meshgrid(q, q, q, indexing="ij"), -1).reshape(-1, 3)
    psi = (x.numpy() - lat + n / 2) % n - n / 2
    m = np.fft.fftfreq(n) * n
    mz = np.fft.rfftfreq(n) * n
    kf = 2 * np.pi / box
    cell = box / n
    div = sum(1j * kf * mm * np.fft.rfftn(psi[:, c].reshape(n, n, n)) * cell
              for c, mm in enumerate((m[:, None, None], m[None, :, None], mz[None, None, :])))
    dl = np.fft.rfftn(w) * amp
    ok = ((np.abs(m)[:, None, None] != n // 2) & (np.abs(m)[None, :, None] != n // 2)
          & (mz[None, None, :] != n // 2))
    assert np.abs(div + dl)[ok].max() < 1e-10 * np.abs(dl).max()
    gen, _ = inputs.zeldovich(n, n, box, pk, 1.0, 0, noise=w)
    dx = (x.numpy() - gen + n / 2) % n - n / 2
    assert np.abs(dx).max() < 1e-5   # the generator rounds to FP32


def test_power_spectrum_plane_wave():
    """A single cosine of integer wavevector m0: its power sits in the bin of
    |m0| and equals 2 (A n^3 / 2)^2 V / n^6 over the mode count of that bin."""
    n, box, nbins = 16, 100.0, 8
    m0 = np.array([3, 1, 0])
    i = np.arange(n)
    X = np.meshgrid(i, i, i, indexing="ij")
    A = 0.7
    d = A * np.cos(2 * np.pi * (m0[0] * X[0] + m0[1] * X[1] + m0[2] * X[2]) / n)
    pk, cnt = dpm.power_spectrum(torch.from_numpy(d), box, nbins)
    kmag = np.sqrt((m0 ** 2).sum())
    b = int(np.floor((kmag - 1.0) * nbins / (n // 2 - 1)))
    # brute-force mode count of that bin over the full grid
    full = 0
    for v in itertools.product(range(-n // 2 + 1, n // 2 + 1), repeat=3):
        km = np.sqrt(sum(t * t for t in v))
        if 1.0 <= km <= n // 2:
            bb = nbins - 1 if km == n // 2 else int(np.floor((km - 1.0) * nbins / (n // 2 - 1)))
            full += bb == b
    assert cnt[b] == full
    expect = 2 * (A * n ** 3 / 2) ** 2 * box ** 3 / n ** 6 / full
    assert pk[b].item() == pytest.approx(expect, rel=1e-12)
    others = np.delete(pk.numpy(), b)
    assert np.abs(others).max() < 1e-20


def _dgp_state(n, seed, amp=2.0, rc=1.0):
    d = amp * inputs.white_noise(n, seed)
    phi, _ = oracle.dgp_solve(d, 1.0, 0.3, rc, oracle.Opts(rtol=1e-13, max_cycles=60))
    return d, phi


def test_sparse_jacobian_matches_residual_differences():
    n = 8
    d, phi = _dgp_state(n, 21)
    v = inputs.white_noise(n, 22)
    s0, _, alpha, _ = oracle.dgp_source(d, 1.0, 0.3, 1.0)
    F = lambda u: oracle.residual(oracle.dgp_op(alpha), u, s0, None, 1.0)[0]
    eps = 1e-6
    fd = (F(phi + eps * v) - F(phi - eps * v)) / (2 * eps)
    jv = dpm.dgp_jacobian_apply(phi, d, 1.0, 0.3, 1.0, v)
    assert np.abs(jv - fd).max() < 1e-7 * np.abs(fd).max()


@pytest.mark.parametrize("rc", [1.0, 3.0])
def test_implicit_adjoint_matches_dense_gradient(rc):
    n = 8
    d, _ = _dgp_state(n, 23, rc=rc)
    g = inputs.white_noise(n, 24)
    dd_ref, dr_ref, phi = oracle.dgp_gradient(d, 1.0, 0.3, rc, g)
    dd, dr = dpm.dgp_adjoint(phi, d, 1.0, 0.3, rc, g)
    assert np.abs(dd - dd_ref).max() < 1e-6 * np.abs(dd_ref).max()
    assert dr == pytest.approx(dr_ref, rel=1e-6)


def small_case(n=8, steps=3, model=1):
    box = 32.0 * n / 8
    cfg = dpm.DpmConfig(ng=n, box=box, omega_m=0.3, a_start=0.2, a_end=1.0, nsteps=steps, nbins=6,
                        model=model, growth=0.2, vel=0.2 * 0.2 ** 2 * float(oracle.E_lcdm(0.2, 0.3)))
    amp = inputs.pk_amplitude(n, box, inputs.pk_cutoff())
    w = inputs.white_noise(n, 31)
    tgt = 0.8 * dpm.loss(torch.from_numpy(inputs.white_noise(n, 32)), torch.tensor(1.0, dtype=torch.float64),
                         amp, cfg, np.zeros(cfg.nbins))[1].detach().numpy()
    return cfg, amp, w, tgt


@pytest.mark.parametrize("model", [0, 1])
def test_chain_gradient_matches_finite_differences(model):
    cfg, amp, w, tgt = small_case(model=model)
    rc = 1.5
    L, gw, gr, _ = dpm.gradient(w, rc, amp, cfg, tgt)

    def Lf(ww, r):
        with torch.no_grad():
            return dpm.loss(torch.from_numpy(ww), torch.tensor(r, dtype=torch.float64), amp, cfg, tgt)[0].item()

    for seed in (41, 42, 43):
        v = inputs.white_noise(cfg.ng, seed)
        v /= np.linalg.norm(v)
        eps = 1e-5
        fd = (Lf(w + eps * v, rc) - Lf(w - eps * v, rc)) / (2 * eps)
        assert float(np.sum(gw * v)) == pytest.approx(fd, rel=2e-5, abs=1e-9 * abs(L))
    if model == 1:
        fd = (Lf(w, rc * (1 + 1e-5)) - Lf(w, rc * (1 - 1e-5))) / (2e-5 * rc)
        assert gr == pytest.approx(fd, rel=2e-5)
    else:
        assert gr == 0.0


@pytest.mark.parametrize("model", [0, 1])
def test_steps_match_pm_step(model):
    """Two leapfrog steps of the FP64 chain against the oracle's FP32-state
    PM step (the pinned particle-mesh code) from the same particles."""
    n = 16
    cfg = dpm.DpmConfig(ng=n, box=64.0, omega_m=0.3, a_start=0.3, a_end=0.5, nsteps=2, model=model)
    pos, mom = inputs.zeldovich(n, n, 64.0, inputs.pk_cutoff(), 0.5, 51, vel_factor=0.05)
    x, p = dpm.run_steps(torch.from_numpy(pos.astype(np.float64)), torch.from_numpy(mom.astype(np.float64)),
                         torch.tensor(1.0, dtype=torch.float64), cfg, 0, 2)
    po, mo = pos, mom
    a = 0.3
    for t in range(2):
        po, mo, _ = oracle.pm_step(po, mo, n, n, 0.3, a, 0.1, model=model, rc_h0=1.0, first=(t == 0),
                                   opts=oracle.Opts(rtol=1e-12, max_cycles=60))
        a += 0.1
    dx = (x.numpy() - po + n / 2) % n - n / 2
    assert np.abs(dx).max() < 2e-5
    assert np.abs(p.numpy() - mo).max() < 2e-5 * max(1.0, np.abs(mo).max())
