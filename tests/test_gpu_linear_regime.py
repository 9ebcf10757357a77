"""The FP64 nDGP path in the linear regime (Sec. 2, the linearised nDGP
equation with its beta factor; Eq. DGP): where Sigma << alpha^2 the
Vainshtein term N = (3/4)[-alpha + sgn(alpha) sqrt(alpha^2 + 8 Sigma/3)] is
~Sigma/alpha, and any error relative to alpha in the square root would
dominate it.  These tests pin, on the GPU and through the C-ABI:

* the FP64 square root and quotient the kernels use in place of CUDA's IEEE
  operations, against torch's (IEEE, correctly rounded) sqrt and division:
  relative error below 2^-43;
* N(Sigma) as the kernels evaluate it, against the oracle's N, to 1e-13
  relative at every amplitude from 1e-20 to 1e6;
* the smoother's and the residual's N part at an amplitude of 1e-6 against
  the oracle, relative to N itself (not to the stencil's sums);
* the linear limit (pin P3 of the oracle): delta = eps * white noise for
  eps in {1e-2, 1e-4, 1e-6}; the FP64 and mixed-precision solves match the
  oracle's to 1e-6 relative L2, the difference from the FFT solution of
  Lap u = Omega_m a^-1 delta / beta falls in proportion to eps, and at
  eps = 1e-6 it is below 1e-6."""
import numpy as np
import pytest

import oracle
from paper_2110_00566_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2110_00566_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0)
    yield c
    c.close()


def _log_uniform(n, lo, hi, seed):
    u = np.random.default_rng(seed).random(n)
    return np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * u)


def test_fp64_sqrt_and_quotient_bounds(B, ctx):
    """k_sqrt and k_quot against IEEE sqrt and 1/x over the whole positive
    normal range and densely over [1, 4): relative error below 2^-43."""
    xs = np.concatenate([_log_uniform(200000, 1e-300, 1e300, 1), _log_uniform(200000, 1.0, 4.0, 2),
                         np.array([1.0, 2.0, 3.0, 4.0, 0.5, 65.61, 8.1 ** 2 + 1e-12, np.nextafter(1.0, 2.0),
                                   np.nextafter(2.0, 1.0), 2.0 ** -1022, 2.0 ** 1021])])
    x = torch.from_numpy(xs).cuda()
    y = torch.empty_like(x)
    ctx.probe_fp64_math(0, x, y)
    ref = torch.sqrt(x)
    err_s = float(((y - ref).abs() / ref).max())
    ctx.probe_fp64_math(1, x, y)
    ref = 1.0 / x
    err_q = float(((y - ref).abs() / ref).max())
    assert err_s < 2.0 ** -43, err_s
    assert err_q < 2.0 ** -43, err_q
    # zeros: sqrt(+-0) = +-0
    z = torch.tensor([0.0, -0.0], dtype=torch.float64, device="cuda")
    yz = torch.empty_like(z)
    ctx.probe_fp64_math(0, z, yz)
    assert float(yz.abs().max()) == 0.0


@pytest.mark.parametrize("alpha", [8.1, 0.37, -2.5])
def test_fp64_N_relative_at_every_amplitude(B, ctx, alpha):
    """N(Sigma) as the FP64 kernels evaluate it, against the oracle's N (the
    rationalised form with a correctly rounded square root): 1e-13 relative
    for |Sigma| from 1e-20 to 1e6 of either sign (where the square-root
    argument stays positive)."""
    mags = _log_uniform(4000, 1e-20, 1e6, 3)
    sig = np.concatenate([mags, -mags])
    arg = alpha * alpha + 8.0 * sig / 3.0
    sig = sig[arg > 1e-3 * alpha * alpha]
    x = torch.from_numpy(sig).cuda()
    y = torch.empty_like(x)
    ctx.probe_fp64_math(2, x, y, alpha)
    got = y.cpu().numpy()
    ref = np.array([oracle.dgp_N(s, alpha)[0] for s in sig])
    rel = np.abs(got - ref) / np.abs(ref)
    assert rel.max() < 1e-13, (rel.max(), sig[rel.argmax()])
    # the clamp: a negative argument gives -(3/4) alpha
    xc = torch.tensor([-(alpha * alpha) * 3.0 / 8.0 * 1.5], dtype=torch.float64, device="cuda")
    yc = torch.empty_like(xc)
    ctx.probe_fp64_math(2, xc, yc, alpha)
    assert float(yc[0]) == -0.75 * alpha


@pytest.mark.parametrize("n,h", [(16, 1.0), (32, 2.0), (64, 1.0), (128, 4.0)])
def test_smoother_and_residual_N_at_small_amplitude(B, ctx, n, h):
    """The FP64 smoother and fused residual/restriction at amplitude 1e-6
    (density term) and 1e-9 (field): the N part of the update and of the
    residual against the oracle, measured relative to N, not to the
    stencil's sums."""
    alpha = 8.1
    o = oracle.dgp_op(alpha)
    b = B.op_params(0, alpha, 2, 0.0, 0.0)
    u = 1e-9 * inputs.white_noise(n, 50)
    s = 1e-6 * inputs.white_noise(n, 51)
    Nf, _ = oracle.N_field(o, u, s, h)
    c = float(Nf.mean())
    for colour in (0, 1):
        ref = oracle.smooth(o, u, s, None, h, c, colour)
        out = np.empty_like(u)
        B.mg_op_smooth(ctx, b, 0, n, h, u, s, None, c, colour, out)
        # the update is S6/6 - h^2 (N - c)/6: S6/6 carries one rounding
        tol = 1e-12 * h * h * np.abs(Nf - c).max() / 6.0 + 1e-15 * np.abs(u).max()
        assert np.abs(out - ref).max() < tol, (colour, np.abs(out - ref).max(), tol)
    d, cr, eps = oracle.residual(o, u, s, None, h)
    Ru = np.empty((n // 2,) * 3)
    Rd = np.empty((n // 2,) * 3)
    cg, eg = B.mg_op_resid_restrict(ctx, b, 0, n, h, u, s, None, Ru, Rd)
    scale = np.abs(Nf).max()
    lap = 12.0 * np.abs(u).max() / h ** 2 * 2.2e-16
    assert np.abs(Rd - oracle.restrict(d)).max() < 1e-12 * scale + 4 * lap
    assert abs(cg - cr) < 1e-12 * scale
    assert abs(eg - eps) < 1e-11 * eps


@pytest.fixture(scope="module")
def linear_case():
    n, a, om, rc = 32, 1.0, 0.3, 1.0
    base = inputs.white_noise(n, 7)
    beta = oracle.beta_dgp(a, om, rc)
    out = {}
    for eps_amp in (1e-2, 1e-4, 1e-6):
        delta = eps_amp * base
        ref, st = oracle.dgp_solve(delta, a, om, rc, oracle.Opts(rtol=1e-10, max_cycles=40))
        lin = oracle.fft_poisson(om / (a * beta) * (delta - delta.mean()))
        out[eps_amp] = (delta, ref, lin)
    return dict(n=n, a=a, om=om, rc=rc, cases=out)


@pytest.mark.parametrize("prec", [0, 1])
def test_linear_limit_solves(B, ctx, linear_case, prec):
    """P3 on the GPU path: the FP64 (prec 0) and mixed-precision (prec 1)
    solves of delta = eps * white noise against the oracle (1e-6 relative
    L2 at every eps) and against the FFT solution of the linearised
    equation (slope 1 in eps; below 1e-6 at eps = 1e-6)."""
    L = linear_case
    n = L["n"]
    diffs = []
    for eps_amp, (delta, ref, lin) in sorted(L["cases"].items(), reverse=True):
        d = torch.from_numpy(delta).cuda()
        phi = torch.zeros_like(d)
        rc, st = B.mg_solve_dgp(ctx, [dict(ng=n, box_mpch=64.0, a=L["a"], omega_m=L["om"], rc_h0=L["rc"],
                                           delta=d, phi=phi)],
                                B.opts(rtol=1e-10, max_cycles=60, precision=prec))
        assert rc == 0, (eps_amp, rc)
        got = phi.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 1e-6, (eps_amp, prec, err)
        diffs.append(np.linalg.norm(got - lin) / np.linalg.norm(lin))
    # diffs at eps = 1e-2, 1e-4, 1e-6: O(eps)
    assert 50.0 < diffs[0] / diffs[1] < 200.0, diffs
    assert diffs[2] < 1e-6, diffs
