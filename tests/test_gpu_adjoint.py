"""GPU parity of the adjoint nDGP solve (mg_solve_adjoint): gradients of
L = <g, phi> with respect to delta and R_c against the FP64 oracle's
dense-Jacobian reference gradient (8^3, 12^3 -- whose coarsest level is
6^3 -- and 16^3), and against central differences of the GPU's own forward
solve (32^3)."""
import numpy as np
import pytest

import oracle
from paper_2110_00566_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import B, ctx, config1_delta  # noqa: E402,F401


def adjoint_gpu(B, ctx, delta, phi, g, a, om, rc, **kw):
    n = delta.shape[0]
    out = np.empty_like(delta)
    code, drc, st = B.mg_solve_adjoint(ctx, n, float(n), a, om, rc, phi, delta, g, out,
                                       B.opts(rtol=1e-12, max_cycles=60, **kw))
    assert code == 0, st.eps_list()
    return out, drc, st


@pytest.mark.parametrize("n,amp,rc", [(8, 3.0, 1.0), (12, 2.0, 1.0), (16, 1.0, 1.0), (16, 2.0, 5.0)])
def test_adjoint_matches_oracle_reference(B, ctx, n, amp, rc):
    a, om = 1.0, 0.3
    delta = amp * inputs.white_noise(n, 300 + n)
    g = inputs.white_noise(n, 400 + n)
    dd_ref, dr_ref, phi = oracle.dgp_gradient(delta, a, om, rc, g)
    dd, dr, st = adjoint_gpu(B, ctx, delta, phi, g, a, om, rc)
    assert np.abs(dd - dd_ref).max() < 1e-6 * np.abs(dd_ref).max()
    assert dr == pytest.approx(dr_ref, rel=1e-6)


def test_adjoint_matches_finite_differences_of_the_gpu_solve(B, ctx):
    n, a, om, rc = 32, 1.0, 0.3, 1.0
    delta = config1_delta()
    g = inputs.white_noise(n, 501)

    def L(d, r):
        phi = np.zeros_like(d)
        B.mg_solve_dgp(ctx, [dict(ng=n, a=a, omega_m=om, rc_h0=r, delta=d, phi=phi)],
                       B.opts(rtol=1e-13, max_cycles=60))
        return float(np.sum(g * phi)), phi

    L0, phi = L(delta, rc)
    dd, dr, st = adjoint_gpu(B, ctx, delta, phi, g, a, om, rc)
    for seed in (502, 503, 504, 505):
        v = inputs.white_noise(n, seed)
        eps = 1e-4
        fd = (L(delta + eps * v, rc)[0] - L(delta - eps * v, rc)[0]) / (2 * eps)
        assert float(np.sum(dd * v)) == pytest.approx(fd, rel=1e-5)
    fd = (L(delta, rc * (1 + 1e-5))[0] - L(delta, rc * (1 - 1e-5))[0]) / (2e-5 * rc)
    assert dr == pytest.approx(fd, rel=1e-5)
    # the adjoint solve converges like the forward one (a handful of cycles)
    assert st.cycles <= 20


def test_autograd_function(B, ctx):
    """The autograd wrapper's backward equals mg_solve_adjoint, and a loss
    gradient along a direction matches central differences of the forward."""
    n, a, om = 16, 1.0, 0.3
    dev = torch.device("cuda", 0)
    delta = torch.from_numpy(2.0 * inputs.white_noise(n, 601)).to(dev).requires_grad_(True)
    rc = torch.tensor(1.5, dtype=torch.float64, requires_grad=True)
    g = torch.from_numpy(inputs.white_noise(n, 602)).to(dev)
    Fn = B.autograd_solve()
    o = B.opts(rtol=1e-13, max_cycles=60)
    phi = Fn.apply(delta, rc, ctx, a, om, float(n), o)
    loss = (g * phi).sum()
    loss.backward()
    dd = delta.grad.cpu().numpy()
    ref = np.empty((n,) * 3)
    _, drc, _ = B.mg_solve_adjoint(ctx, n, float(n), a, om, 1.5, phi.detach(), delta.detach(), g, ref, o)
    assert np.abs(dd - ref).max() < 1e-12 * np.abs(ref).max()
    assert rc.grad.item() == pytest.approx(drc, rel=1e-12)
    v = torch.from_numpy(inputs.white_noise(n, 603)).to(dev)
    with torch.no_grad():
        lp = (g * Fn.apply(delta + 1e-4 * v, rc, ctx, a, om, float(n), o)).sum().item()
        lm = (g * Fn.apply(delta - 1e-4 * v, rc, ctx, a, om, float(n), o)).sum().item()
    assert float((delta.grad * v).sum()) == pytest.approx((lp - lm) / 2e-4, rel=1e-5)
