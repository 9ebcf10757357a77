"""GPU parity of the mixed-precision form: the FP32 correction smoother
against the oracle's FP64 N(b + e) - N(b), and full mixed solves against
the FP64 oracle solution (1e-6 relative L2 on phi, the stated target; the
FP64 defect must reach the same 1e-8 relative residual as the plain
solve)."""
import numpy as np
import pytest

import oracle
from paper_2110_00566_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import B, ctx, MODELS, ops, config1_delta, l2  # noqa: E402,F401


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def lap6(e):
    out = np.zeros_like(e)
    for ax in range(3):
        out = out + np.roll(e, 1, ax) + np.roll(e, -1, ax)
    return out


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("n,h", [(16, 1.0), (24, 2.0), (128, 1.0), (256, 2.0)])
def test_correction_smoother(B, ctx, name, n, h):
    """A correction 1e-4 the size of the base field: a naive FP32
    N(b+e) - N(b) would lose ~3 digits; the expanded form keeps FP32
    relative accuracy in the update.  The density term stays in the
    physical range (delta >= -1 keeps alpha^2 + 8 Sigma/3 >= alpha(alpha -
    8 Omega_m/(3 a beta)) > 0): at the sqrt-clamp boundary dN/dSigma = 1/r
    is singular and no difference form is well conditioned."""
    o, b_, amp = ops(B, name)
    base = f32(amp * inputs.white_noise(n, 60))
    e = f32(1e-4 * amp * inputs.white_noise(n, 61))
    s = f32(np.maximum(0.7 * inputs.white_noise(n, 62), -0.5))
    f = f32(1e-4 * inputs.white_noise(n, 63))
    c = 3e-6
    for colour in (0, 1):
        N1, _ = oracle.N_field(o, base + e, s, h)
        N0, _ = oracle.N_field(o, base, s, h)
        upd = (lap6(e) - h * h * ((N1 - N0) - c + f)) / 6.0
        par = np.add.outer(np.add.outer(np.arange(n), np.arange(n)), np.arange(n)) % 2
        ref = np.where(par == colour, upd, e)
        out = np.empty_like(e)
        B.mg_op_smooth_corr(ctx, b_, n, h, e, base, s, f, c, colour, out)
        err = np.abs(out - ref).max() / np.abs(ref).max()
        assert err < 2e-5, (colour, err)


@pytest.mark.parametrize("rc", [1.0, 5.0])
def test_mixed_solve_ndgp(B, ctx, rc):
    delta = config1_delta()
    ref, rst = oracle.dgp_solve(delta, 1.0, 0.3, rc, oracle.Opts(rtol=1e-10, max_cycles=40))
    phi = np.zeros_like(delta)
    code, st = B.mg_solve_dgp(ctx, [dict(ng=32, a=1.0, omega_m=0.3, rc_h0=rc, delta=delta, phi=phi)],
                              B.opts(rtol=1e-8, precision=B.MG_PREC_MIXED, max_cycles=40))
    st = st[0]
    assert code == 0, st.eps_list()
    assert st.eps[st.n_eps - 1] <= 1e-8 * st.eps_ref
    assert l2(phi, ref) < 1e-6, l2(phi, ref)


def test_mixed_solve_ragged(B, ctx):
    delta = 1.5 * inputs.white_noise(24, 3)
    ref, _ = oracle.dgp_solve(delta, 1.0, 0.3, 1.0, oracle.Opts(rtol=1e-11, max_cycles=40))
    phi = np.zeros_like(delta)
    code, st = B.mg_solve_dgp(ctx, [dict(ng=24, a=1.0, omega_m=0.3, rc_h0=1.0, delta=delta, phi=phi)],
                              B.opts(rtol=1e-10, precision=B.MG_PREC_MIXED, max_cycles=60))
    assert code == 0 and l2(phi, ref) < 1e-8, l2(phi, ref)


@pytest.mark.parametrize("nk,k0", [(2, 1.0), (3, 1.0)])
def test_mixed_solve_kmouflage(B, ctx, nk, k0):
    n, box, a, om = 32, 64.0, 1.0, 0.3
    delta = 30.0 * config1_delta()
    lam = np.sqrt(3 * (1 - om))
    ref, _ = oracle.kmo_solve(delta, a, om, box, nk, k0, 0.2, lam, -1e-3, np.exp(-0.02),
                              oracle.Opts(rtol=1e-10, max_cycles=40))
    phi = np.zeros_like(delta)
    code, st = B.mg_solve_kmouflage(ctx, n, box, a, om, nk, k0, 0.2, lam, -1e-3, np.exp(-0.02), delta, phi,
                                    B.opts(rtol=1e-8, precision=B.MG_PREC_MIXED, max_cycles=60))
    assert code == 0, st.eps_list()
    assert l2(phi, ref) < 1e-6, l2(phi, ref)


@pytest.mark.parametrize("model,n", [("dgp", 256), ("kmo", 256), ("dgp", 512)])
def test_streaming_smoother_is_bit_identical(B, model, n):
    """The streaming FP32 half-sweep (planes staged in shared memory by bulk
    asynchronous copies) and the gathering one run the same per-quad
    arithmetic: a whole mixed-precision solve gives the same bits with the
    gathering kernel and with every streaming variant."""
    box = 0.5 * n
    pos, _ = inputs.zeldovich(n // 2, n, box, inputs.pk_cutoff(0.96, 5.0, 0.8), 1.0, seed=12)
    c = B.Context(0)
    try:
        d = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
        B.pm_cic_deposit(c, n, torch.from_numpy(pos).cuda(), d)
        o = B.opts(rtol=1e-8, precision=B.MG_PREC_MIXED, max_cycles=40)
        ref = None
        for choice in [-1] + list(range(1, B.fp32_smoother_variants() + 1)):
            c.set_fp32_smoother(choice)
            phi = torch.zeros_like(d)
            if model == "dgp":
                code, _ = B.mg_solve_dgp(c, [dict(ng=n, box_mpch=box, a=1.0, omega_m=0.3, rc_h0=1.0, delta=d,
                                                  phi=phi)], o)
            else:
                code, _ = B.mg_solve_kmouflage(c, n, box, 1.0, 0.3, 2, 1.0, 0.2, float(np.sqrt(2.1)), -0.15, 0.88,
                                               d, phi, o)
            assert code == 0, choice
            if ref is None:
                ref = phi
            else:
                assert torch.equal(phi, ref), choice
        with pytest.raises(B.MGError):
            c.set_fp32_smoother(B.fp32_smoother_variants() + 1)
    finally:
        c.close()


def test_pinned_smoother_shapes_are_bit_identical(B):
    """Pinned block shapes and planes per block of the gathering FP32
    half-sweep (z-marching on and off) give the same bits as the autotuned
    choice; bad shapes are rejected."""
    n, box = 256, 128.0
    pos, _ = inputs.zeldovich(n // 2, n, box, inputs.pk_cutoff(0.96, 5.0, 0.8), 1.0, seed=13)
    c = B.Context(0)
    try:
        d = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
        B.pm_cic_deposit(c, n, torch.from_numpy(pos).cuda(), d)
        o = B.opts(rtol=1e-8, precision=B.MG_PREC_MIXED, max_cycles=40)
        c.set_fp32_smoother(-1)
        ref = None
        for bx, zc in [(0, 1), (8, 1), (32, 2), (32, 8), (16, 3)]:
            c.set_fp32_smoother_shape(n, bx, zc)
            phi = torch.zeros_like(d)
            code, _ = B.mg_solve_dgp(c, [dict(ng=n, box_mpch=box, a=1.0, omega_m=0.3, rc_h0=1.0, delta=d, phi=phi)], o)
            assert code == 0
            if ref is None:
                ref = phi
            else:
                assert torch.equal(phi, ref), (bx, zc)
        for bad in [(n, 12, 1), (n, 64, 0), (16, 8, 1)]:
            with pytest.raises(B.MGError):
                c.set_fp32_smoother_shape(*bad)
    finally:
        c.close()


@pytest.mark.parametrize("model,precision,n", [("dgp", "fp64", 64), ("dgp", "mixed", 64), ("dgp", "fp64", 128),
                                               ("dgp", "mixed", 128), ("kmo", "fp64", 128), ("kmo", "mixed", 128)])
def test_cold_start_defect_is_bit_identical(B, ctx, model, precision, n):
    """A solve from phi = 0 evaluates its first defect from the source alone
    (the stencil of a zero field vanishes; at 128^3 and more the staged norm
    pass skips the staging); it must give the same bits as a warm start from
    an explicit zero field, which runs the full stencil."""
    delta = 2.0 * inputs.white_noise(n, 14)
    prec = B.MG_PREC_FP64 if precision == "fp64" else B.MG_PREC_MIXED
    outs = []
    for warm in (0, 1):
        phi = np.zeros_like(delta)
        o = B.opts(rtol=1e-9, precision=prec, max_cycles=40, warm_start=warm)
        if model == "dgp":
            code, st = B.mg_solve_dgp(ctx, [dict(ng=n, a=1.0, omega_m=0.3, rc_h0=1.0, delta=delta, phi=phi)], o)
            st = st[0]
        else:
            code, st = B.mg_solve_kmouflage(ctx, n, 2.0 * n, 1.0, 0.3, 2, 1.0, 0.2, float(np.sqrt(2.1)), -1e-3,
                                            np.exp(-0.02), 30.0 * delta, phi, o)
        assert code == 0
        outs.append((phi, st.eps_list()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]
