"""Error paths of the C ABI on the GPU: every entry point turns malformed
arguments into MG_ERR_ARG before touching the device, non-finite inputs into
MG_ERR_NONFINITE (detected in the first residual, with no fault), and the
context stays usable afterwards."""
import numpy as np
import pytest

from paper_2110_00566_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import B, ctx  # noqa: E402,F401


def _code(fn, *args, **kw):
    with pytest.raises(Exception) as e:
        fn(*args, **kw)
    return getattr(e.value, "code", None)


def test_solver_argument_and_input_errors(B, ctx):
    n = 16
    delta = inputs.white_noise(n, 201)
    phi = np.zeros_like(delta)
    # no instances; an unsupported mesh; a non-positive R_c
    assert _code(B.mg_solve_dgp, ctx, []) == B.MG_ERR_ARG
    assert _code(B.mg_solve_dgp, ctx, [dict(ng=10, a=1.0, omega_m=0.3, rc_h0=1.0, delta=np.zeros((10,) * 3),
                                            phi=np.zeros((10,) * 3))]) == B.MG_ERR_ARG
    assert _code(B.mg_solve_dgp, ctx, [dict(ng=n, a=1.0, omega_m=0.3, rc_h0=0.0, delta=delta, phi=phi)]) == \
        B.MG_ERR_ARG
    # a mesh above the supported 1536^3, rejected on the host before any
    # array is read (the arrays passed are the small ones)
    assert _code(B.mg_solve_dgp, ctx, [dict(ng=2048, a=1.0, omega_m=0.3, rc_h0=1.0, delta=delta, phi=phi)]) == \
        B.MG_ERR_ARG
    # an unknown cycle type; odd pre + post with several device instances is
    # not the batched form: the instances are solved one after another
    two = [dict(ng=n, a=1.0, omega_m=0.3, rc_h0=1.0, delta=torch.from_numpy(delta).cuda(),
                phi=torch.zeros((n,) * 3, dtype=torch.float64, device="cuda")) for _ in range(2)]
    code, st = B.mg_solve_dgp(ctx, two, B.opts(precision=B.MG_PREC_MIXED, pre=1, post=2))
    assert code == 0 and torch.equal(two[0]["phi"], two[1]["phi"])
    assert _code(B.mg_solve_dgp, ctx, [dict(ng=n, a=1.0, omega_m=0.3, rc_h0=1.0, delta=delta, phi=phi)],
                 B.opts(cycle=7)) == B.MG_ERR_ARG
    # a non-finite density, in both precisions
    bad = delta.copy()
    bad[1, 2, 3] = np.inf
    for prec in (B.MG_PREC_FP64, B.MG_PREC_MIXED):
        assert _code(B.mg_solve_dgp, ctx, [dict(ng=n, a=1.0, omega_m=0.3, rc_h0=1.0, delta=bad, phi=phi)],
                     B.opts(precision=prec)) == B.MG_ERR_NONFINITE
    # Kmouflage: exponent below 2, lambda <= 0, a NaN density
    kp = (n, 32.0, 1.0, 0.3)
    assert _code(B.mg_solve_kmouflage, ctx, *kp, 1, 1.0, 0.2, 1.4, -0.1, 0.9, delta, phi) == B.MG_ERR_ARG
    assert _code(B.mg_solve_kmouflage, ctx, *kp, 2, 1.0, 0.2, 0.0, -0.1, 0.9, delta, phi) == B.MG_ERR_ARG
    bad[1, 2, 3] = np.nan
    assert _code(B.mg_solve_kmouflage, ctx, *kp, 2, 1.0, 0.2, 1.4, -0.1, 0.9, bad, phi) == B.MG_ERR_NONFINITE
    # the context still solves
    code, st = B.mg_solve_dgp(ctx, [dict(ng=n, a=1.0, omega_m=0.3, rc_h0=1.0, delta=delta, phi=phi)])
    assert code == 0 and st[0].eps[st[0].n_eps - 1] <= 1e-8 * st[0].eps_ref


def test_particle_mesh_argument_errors(B, ctx):
    ng = 16
    pos = np.ascontiguousarray(inputs.uniform01(211, 30).reshape(10, 3).astype(np.float32) * ng)
    mom = np.zeros_like(pos)
    out = np.empty((ng,) * 3)
    assert _code(B.pm_cic_deposit, ctx, 1, pos, np.empty((1, 1, 1))) == B.MG_ERR_ARG
    assert _code(B.pm_cic_deposit, ctx, ng, pos[:0], out) == B.MG_ERR_ARG
    for kw in (dict(model=3), dict(model=1, rc_h0=-1.0), dict(model=0, hubble=(-1.0, 1.0))):
        st = B.make_pm_state(pos, mom, ng, 32.0, 0.3, 0.5, 0.01, **kw)
        assert _code(B.pm_step, ctx, st) == B.MG_ERR_ARG
    # a Kmouflage step without its background parameters (lambda = 0)
    st = B.make_pm_state(pos, mom, ng, 32.0, 0.3, 0.5, 0.01, model=2,
                         kmo=dict(n=2, k0=1.0, beta=0.2, lam=0.0, phibar_prime_over_h0=0.0, A_bar=1.0, dphibar_da=0.0))
    assert _code(B.pm_step, ctx, st) == B.MG_ERR_ARG
    # positions at and beyond the box edge are wrapped, never rejected
    edge = np.array([[0.0, 0.0, 0.0], [ng, ng, ng], [-0.25, ng + 0.25, 3.0]], dtype=np.float32)
    B.pm_cic_deposit(ctx, ng, edge, out)
    assert np.isfinite(out).all()


def test_differentiable_run_argument_errors(B, ctx):
    n = 16
    amp = np.ones((n, n, n // 2 + 1))
    noise = inputs.white_noise(n, 221)
    for cfg in (B.make_dpm_config(6, 32.0, 0.3, 0.1, 1.0, 4),          # mesh below 8
                B.make_dpm_config(n, 32.0, 0.3, 0.5, 0.5, 4),          # a_end <= a_start
                B.make_dpm_config(n, 32.0, 0.3, 0.1, 1.0, 4, nbins=0),
                B.make_dpm_config(n, 32.0, 0.3, 0.1, 1.0, 0)):         # no steps
        assert _code(B.dpm_run, ctx, cfg, amp, noise, 1.0) == B.MG_ERR_ARG
    cfg = B.make_dpm_config(n, 32.0, 0.3, 0.1, 1.0, 4)
    assert _code(B.dpm_run, ctx, cfg, amp, noise, 0.0) == B.MG_ERR_ARG                     # R_c <= 0
    assert _code(B.dpm_run, ctx, cfg, amp, noise, 1.0, dnoise_out=np.empty_like(noise)) == B.MG_ERR_ARG
