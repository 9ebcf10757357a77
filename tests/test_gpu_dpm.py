"""GPU parity of the differentiable particle-mesh run (dpm_* entry points)
against the FP64 oracle of oracle/dpm.py: each piece and its adjoint (the
adjoints against torch.autograd vector-Jacobian products of the oracle's
pieces), the whole run's loss and gradients against the oracle's gradient,
and the gradient against central differences of the GPU forward run."""
import numpy as np
import pytest

import oracle
from oracle import dpm as odpm
from paper_2110_00566_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import B, ctx  # noqa: E402,F401


def cfgs(B, n=16, steps=4, K=2, nbins=8, model=1, box=None):
    box = box or 4.0 * n
    a0 = 0.2
    D = inputs.growth_lcdm(a0, 0.3)
    vel = a0 * a0 * float(oracle.E_lcdm(a0, 0.3)) * D * inputs.growth_rate_lcdm(a0, 0.3)
    oc = odpm.DpmConfig(ng=n, box=box, omega_m=0.3, a_start=a0, a_end=1.0, nsteps=steps, nbins=nbins,
                        model=model, growth=D, vel=vel)
    gc = B.make_dpm_config(n, box, 0.3, a0, 1.0, steps, K, nbins, model, D, vel)
    amp = inputs.pk_amplitude(n, box, inputs.pk_cutoff())
    return oc, gc, amp


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def wrapdiff(x, y, n):
    return (x - y + n / 2) % n - n / 2


def test_ic_and_adjoint(B, ctx):
    oc, gc, amp = cfgs(B)
    n = oc.ng
    w = inputs.white_noise(n, 701)
    pos, mom = np.empty((n ** 3, 3)), np.empty((n ** 3, 3))
    B.dpm_ic(ctx, gc, amp, w, pos, mom)
    wt = torch.tensor(w, requires_grad=True)
    x, p = odpm.zeldovich(wt, amp, oc)
    assert np.abs(wrapdiff(pos, x.detach().numpy(), n)).max() < 1e-12
    assert np.abs(mom - p.detach().numpy()).max() < 1e-12 * max(1.0, np.abs(mom).max())
    dx = np.stack([inputs.white_noise(n, 703 + c).reshape(-1) for c in range(3)], 1)
    dp = np.stack([inputs.white_noise(n, 706 + c).reshape(-1) for c in range(3)], 1)
    ref = torch.autograd.grad((x * torch.from_numpy(dx)).sum() + (p * torch.from_numpy(dp)).sum(), wt)[0].numpy()
    got = np.empty((n, n, n))
    B.dpm_ic_adjoint(ctx, gc, amp, dx, dp, got)
    assert rel(got, ref) < 1e-12


def test_deposit_and_adjoint(B, ctx):
    n, npart = 16, 16 ** 3
    x = np.ascontiguousarray(inputs.uniform01(711, 3 * npart).reshape(npart, 3) * n)
    got = np.empty((n, n, n))
    B.dpm_deposit(ctx, n, x, got)
    xt = torch.tensor(x, requires_grad=True)
    d = odpm.cic_density(xt, n)
    assert np.abs(got - d.detach().numpy()).max() < 1e-10
    dd = inputs.white_noise(n, 712)
    ref = torch.autograd.grad((d * torch.from_numpy(dd)).sum(), xt)[0].numpy()
    out = np.empty_like(x)
    B.dpm_deposit_adjoint(ctx, n, x, dd, out)
    assert rel(out, ref) < 1e-12


def test_force_and_adjoint(B, ctx):
    n, npart = 16, 3000
    x = np.ascontiguousarray(inputs.uniform01(721, 3 * npart).reshape(npart, 3) * n)
    phin, phi = inputs.white_noise(n, 722), inputs.white_noise(n, 723)
    got = np.empty_like(x)
    B.dpm_force(ctx, n, phin, phi, x, got)
    xt = torch.tensor(x, requires_grad=True)
    pt = torch.tensor(phin, requires_grad=True)
    F = odpm.force(pt + 0.5 * torch.from_numpy(phi), xt)
    assert rel(got, F.detach().numpy()) < 1e-13
    dF = np.stack([inputs.white_noise(20, 724 + c).reshape(-1)[:npart] for c in range(3)], 1)
    gx, gp = torch.autograd.grad((F * torch.from_numpy(dF)).sum(), (xt, pt))
    ox, op = np.empty_like(x), np.empty((n, n, n))
    B.dpm_force_adjoint(ctx, n, phin, phi, x, dF, ox, op)
    assert rel(ox, gx.numpy()) < 1e-12
    assert rel(op, gp.numpy()) < 1e-12


def test_power_spectrum_and_adjoint(B, ctx):
    n, box, nbins = 16, 64.0, 8
    d = inputs.white_noise(n, 731)
    pk, cnt = B.dpm_power_spectrum(ctx, n, box, nbins, d)
    dt = torch.tensor(d, requires_grad=True)
    ref, rcnt = odpm.power_spectrum(dt, box, nbins)
    assert np.array_equal(cnt, rcnt)
    assert rel(pk, ref.detach().numpy()) < 1e-13
    dpk = inputs.normal(732, nbins)
    gref = torch.autograd.grad((ref * torch.from_numpy(dpk)).sum(), dt)[0].numpy()
    out = np.empty((n, n, n))
    B.dpm_power_spectrum_adjoint(ctx, n, box, nbins, d, dpk, out)
    assert rel(out, gref) < 1e-12


def target_for(oc, amp):
    wt = torch.from_numpy(inputs.white_noise(oc.ng, 742))
    with torch.no_grad():
        return 0.8 * odpm.loss(wt, torch.tensor(1.0, dtype=torch.float64), amp, oc, np.zeros(oc.nbins))[1].numpy()


@pytest.mark.parametrize("model,K", [(1, 2), (0, 3)])
def test_run_matches_oracle_gradient(B, ctx, model, K):
    """The whole run at 16^3 (4 steps, checkpoints every K): loss, P(k) and
    dL/dw, dL/dR_c against the oracle's FP64 reference gradient."""
    oc, gc, amp = cfgs(B, model=model, K=K)
    n, rc = oc.ng, 1.3
    w = inputs.white_noise(n, 741)
    tgt = target_for(oc, amp)
    L, gw, gr, pk_ref = odpm.gradient(w, rc, amp, oc, tgt, oracle.Opts(rtol=1e-12, max_cycles=60))
    out = np.empty((n, n, n))
    o = B.opts(rtol=1e-12, max_cycles=60)
    pk, loss, drc, st = B.dpm_run(ctx, gc, amp, w, rc, tgt, out, o=o)
    assert rel(pk, pk_ref) < 1e-10
    assert loss == pytest.approx(L, rel=1e-9)
    assert rel(out, gw) < 1e-7
    if model == 1:
        assert drc == pytest.approx(gr, rel=1e-6)
    else:
        assert drc == 0.0


def test_run_gradient_matches_gpu_finite_differences(B, ctx):
    """Central differences of the GPU forward run at 32^3.  The loss is only
    piecewise smooth (the CIC weights have kinks at the cell centres, which
    particles cross inside any finite step), so the agreement is limited to
    the fraction of crossings: 5e-3 here (the exact comparison is the one
    against the oracle's gradient above)."""
    oc, gc, amp = cfgs(B, n=32, steps=6, K=3, nbins=12)
    n, rc = oc.ng, 2.0
    w = inputs.white_noise(n, 751)
    tgt = target_for(oc, amp)
    o = B.opts(rtol=1e-12, max_cycles=60)
    out = np.empty((n, n, n))
    _, L0, drc, _ = B.dpm_run(ctx, gc, amp, w, rc, tgt, out, o=o)

    def Lf(ww, r):
        return B.dpm_run(ctx, gc, amp, np.ascontiguousarray(ww), r, tgt, o=o)[1]

    for seed in (752, 753, 754, 755):
        v = inputs.white_noise(n, seed)
        v /= np.linalg.norm(v)
        eps = 1e-5
        fd = (Lf(w + eps * v, rc) - Lf(w - eps * v, rc)) / (2 * eps)
        assert float(np.sum(out * v)) == pytest.approx(fd, rel=5e-3, abs=1e-9 * abs(L0))
    fd = (Lf(w, rc * (1 + 1e-5)) - Lf(w, rc * (1 - 1e-5))) / (2e-5 * rc)
    assert drc == pytest.approx(fd, rel=5e-3)


def test_checkpoint_interval_does_not_change_the_gradient(B, ctx):
    n = 16
    outs = []
    for K in (1, 3, 5):
        oc, gc, amp = cfgs(B, n=n, steps=5, K=K)
        w = inputs.white_noise(n, 761)
        tgt = target_for(oc, amp)
        out = np.empty((n, n, n))
        _, L, drc, _ = B.dpm_run(ctx, gc, amp, w, 1.0, tgt, out, o=B.opts(rtol=1e-12, max_cycles=60))
        outs.append((L, drc, out))
    for L, drc, out in outs[1:]:
        assert L == outs[0][0]
        assert rel(out, outs[0][2]) < 1e-12
        assert drc == pytest.approx(outs[0][1], rel=1e-12)


def test_autograd_pm_with_a_loss_of_the_callers(B, ctx):
    """The run behind torch.autograd.Function (binding.autograd_pm, backward by
    dpm_run_vjp): a loss the library does not know -- a weighted squared
    log-ratio of P to a target -- differentiated by loss.backward() against
    the oracle's FP64 autograd gradient of the same loss at 16^3 (dL/dw to
    1e-7, dL/dR_c to 1e-6), and the built-in MSE through the same Function
    against dpm_run's own gradient."""
    oc, gc, amp = cfgs(B, model=1, K=2)
    n, rc = oc.ng, 1.3
    w = inputs.white_noise(n, 741)
    tgt = torch.from_numpy(target_for(oc, amp))
    wts = torch.linspace(1.0, 2.0, oc.nbins, dtype=torch.float64)
    o = B.opts(rtol=1e-12, max_cycles=60)
    Fn = B.autograd_pm()
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    rt = torch.tensor(rc, dtype=torch.float64, requires_grad=True)
    pk = Fn.apply(wt, rt, ctx, gc, amp, o)
    L = (wts.cuda() * torch.log(pk / tgt.cuda()) ** 2).sum()
    L.backward()
    # the oracle: the same loss on its own P by torch autograd
    wo = torch.tensor(w, requires_grad=True)
    ro = torch.tensor(rc, dtype=torch.float64, requires_grad=True)
    delta, _, _ = odpm.forward(wo, ro, amp, oc, oracle.Opts(rtol=1e-12, max_cycles=60))
    pko, _ = odpm.power_spectrum(delta, oc.box, oc.nbins)
    Lo = (wts * torch.log(pko / tgt) ** 2).sum()
    Lo.backward()
    assert float(L) == pytest.approx(float(Lo), rel=1e-9)
    assert rel(wt.grad.cpu().numpy(), wo.grad.numpy()) < 1e-7
    assert float(rt.grad) == pytest.approx(float(ro.grad), rel=1e-6)
    # the built-in MSE through the Function equals dpm_run's gradient
    wt.grad = None
    rt.grad = None
    pk = Fn.apply(wt, rt, ctx, gc, amp, o)
    ((pk - tgt.cuda()) ** 2).mean().backward()
    ref = np.empty((n, n, n))
    _, _, drc, _ = B.dpm_run(ctx, gc, amp, w, rc, tgt.numpy(), ref, o=o)
    assert rel(wt.grad.cpu().numpy(), ref) < 1e-12
    assert float(rt.grad) == pytest.approx(drc, rel=1e-12)
