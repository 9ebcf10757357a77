"""GPU parity: every multigrid kernel and the full solves of the CUDA path
against the FP64 CPU oracle on the same seeded inputs, called through the
C-ABI.  Tolerances: FP64 kernels 1e-12 (max-norm, relative), FP32 kernels
2e-5 (inputs are rounded to FP32 on the way in); full solves 1e-6 relative
L2 on phi (the stated target); CIC indices bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2110_00566_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-5}


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


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


MODELS = {
    "dgp": dict(model=0, alpha=1.7, nkmo=0, gamma=0.0, bterm=0.0, amp=1.0),
    "kmo2": dict(model=1, alpha=0.0, nkmo=2, gamma=0.8, bterm=0.3, amp=1.0),
    "kmo3": dict(model=1, alpha=0.0, nkmo=3, gamma=0.5, bterm=0.2, amp=0.7),
}


def ops(B, name):
    m = MODELS[name]
    o = oracle.OrcOp(m["model"], m["alpha"], m["nkmo"], m["gamma"], m["bterm"])
    b = B.op_params(m["model"], m["alpha"], max(m["nkmo"], 2), m["gamma"], m["bterm"])
    return o, b, m["amp"]


def fields(n, seed, amp):
    u = amp * inputs.white_noise(n, seed)
    s = 0.7 * inputs.white_noise(n, seed + 1)
    f = 0.2 * inputs.white_noise(n, seed + 2)
    return u, s, f


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,h", [(16, 1.0), (24, 4.0), (8, 2.0), (64, 2.0), (192, 1.0)])
def test_smooth_half_sweep(B, ctx, name, prec, n, h):
    o, b, amp = ops(B, name)
    u, s, f = fields(n, 10, amp)
    for colour in (0, 1):
        for ff in (None, f):
            ref = oracle.smooth(o, u, s, ff, h, 0.031, colour)
            out = np.empty_like(u)
            B.mg_op_smooth(ctx, b, prec, n, h, u, s, ff, 0.031, colour, out)
            assert rel(out, ref) < TOL[prec], (colour, rel(out, ref))


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,h", [(16, 1.0), (24, 2.0), (64, 1.0), (128, 2.0)])
def test_residual_restriction(B, ctx, name, prec, n, h):
    o, b, amp = ops(B, name)
    u, s, f = fields(n, 20, amp)
    for ff in (None, f):
        d, c, eps = oracle.residual(o, u, s, ff, h)
        Ru = np.empty((n // 2,) * 3)
        Rd = np.empty((n // 2,) * 3)
        cg, eg = B.mg_op_resid_restrict(ctx, b, prec, n, h, u, s, ff, Ru, Rd)
        # d = (S6 - 6u)/h^2 - N + c - f: its rounding scale
        scale = np.abs(d).max() + 12.0 * np.abs(u).max() / h ** 2
        assert rel(Ru, oracle.restrict(u)) < TOL[prec]
        assert np.abs(Rd - oracle.restrict(d)).max() < TOL[prec] * scale
        assert abs(cg - c) <= TOL[prec] * scale
        assert abs(eg - eps) <= TOL[prec] * scale


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("prec", [0, 1])
def test_coarse_source(B, ctx, name, prec):
    o, b, amp = ops(B, name)
    n, h = 12, 2.0
    Ru, s, Rd = fields(n, 30, amp)
    LH, cH, _ = oracle.residual(o, Ru, s, None, h)
    ref = LH - Rd
    out = np.empty_like(Ru)
    cg = B.mg_op_coarse_source(ctx, b, prec, n, h, Ru, Rd, s, out)
    scale = np.abs(LH).max() + 12.0 * np.abs(Ru).max() / h ** 2 + np.abs(Rd).max()
    assert np.abs(out - ref).max() < TOL[prec] * scale
    assert abs(cg - cH) <= TOL[prec] * scale


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("n", [128, 256])
def test_coarse_source_staged(B, ctx, name, n):
    # coarse levels of 128^3 and more take the block-staged FP64 kernel
    o, b, amp = ops(B, name)
    h = 2.0
    Ru, s, Rd = fields(n, 31, amp)
    LH, cH, _ = oracle.residual(o, Ru, s, None, h)
    ref = LH - Rd
    out = np.empty_like(Ru)
    cg = B.mg_op_coarse_source(ctx, b, 0, n, h, Ru, Rd, s, out)
    scale = np.abs(LH).max() + 12.0 * np.abs(Ru).max() / h ** 2 + np.abs(Rd).max()
    assert np.abs(out - ref).max() < TOL[0] * scale
    assert abs(cg - cH) <= TOL[0] * scale


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [8, 16, 24])
def test_prolongation(B, ctx, prec, n):
    uf = inputs.white_noise(n, 40)
    uc = inputs.white_noise(n // 2, 41)
    urc = inputs.white_noise(n // 2, 42)
    ref = oracle.prolong_add(uf, uc, urc)
    out = uf.copy()
    B.mg_op_prolong_add(ctx, prec, n, out, uc, urc)
    assert rel(out, ref) < TOL[prec]


@pytest.mark.parametrize("n,scale", [(128, 1.0), (256, 1.0), (128, 1e-300), (128, 1e300)])
def test_prolongation_staged(B, ctx, n, scale):
    # fine levels of 128^3 and more take the block-staged FP64 prolongation:
    # the fixed-point path, and at 1e-300 (exponents below its domain) the
    # FP64 path; 1e300 stays in the fixed-point domain
    uf = scale * inputs.white_noise(n, 43)
    uc = scale * inputs.white_noise(n // 2, 44)
    urc = scale * inputs.white_noise(n // 2, 45)
    ref = oracle.prolong_add(uf, uc, urc)
    out = uf.copy()
    B.mg_op_prolong_add(ctx, 0, n, out, uc, urc)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("n", [4, 6])
def test_coarsest(B, ctx, name, n):
    o, b, amp = ops(B, name)
    u, s, f = fields(n, 50, 0.3 * amp)
    h = 16.0
    ref = u.copy()
    for _ in range(7):
        N, _ = oracle.N_field(o, ref, s, h)
        c = N.mean()
        ref = oracle.smooth(o, ref, s, f, h, c, 0)
        ref = oracle.smooth(o, ref, s, f, h, c, 1)
    out = u.copy()
    B.mg_op_coarsest(ctx, b, n, h, out, s, f, 7)
    assert rel(out, ref) < 1e-11


# ------------------------------------------------------------ full solves

def config1_delta(n=32, box=64.0, seed=1):
    pos, _ = inputs.powerlaw_particles(n, n, box, seed=seed)
    delta, _ = oracle.cic_deposit(pos, n, n)
    return delta


def dgp_gpu(B, ctx, delta, a, om, rc, **kw):
    n = delta.shape[0]
    phi = np.zeros_like(delta)
    rcode, st = B.mg_solve_dgp(ctx, [dict(ng=n, box_mpch=float(n), a=a, omega_m=om, rc_h0=rc, delta=delta,
                                          phi=phi)], B.opts(**kw))
    return phi, rcode, st[0]


def l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("rc", [1.0, 5.0])
def test_solve_config1_fp64(B, ctx, rc):
    """32^3 config-1 workload (power-law Zel'dovich load, rms delta ~ 1),
    V(2,2) to 1e-8: phi within 1e-6 relative L2 of the oracle."""
    delta = config1_delta()
    ref, rst = oracle.dgp_solve(delta, 1.0, 0.3, rc, oracle.Opts(rtol=1e-8))
    phi, code, st = dgp_gpu(B, ctx, delta, 1.0, 0.3, rc, rtol=1e-8)
    assert code == 0
    assert l2(phi, ref) < 1e-6
    assert abs(st.cycles - rst.cycles) <= 1
    assert st.eps[st.n_eps - 1] <= 1e-8 * st.eps_ref
    assert abs(st.eps_ref - rst.eps_ref) < 1e-12 * rst.eps_ref
    assert abs(st.c_final - rst.c_final) < 1e-9 * max(abs(rst.c_final), 1e-12) + 1e-14
    # tight tolerance: both converge to the same discrete solution
    ref2, _ = oracle.dgp_solve(delta, 1.0, 0.3, rc, oracle.Opts(rtol=1e-12, max_cycles=40))
    phi2, _, _ = dgp_gpu(B, ctx, delta, 1.0, 0.3, rc, rtol=1e-12, max_cycles=40)
    assert l2(phi2, ref2) < 1e-10


def test_solve_ragged_and_cycles(B, ctx):
    """3 * 2^k mesh (24^3, coarsest 6^3) and the F and W cycles."""
    delta = 1.5 * inputs.white_noise(24, 3)
    for cyc in (0, 1, 2):
        ref, _ = oracle.dgp_solve(delta, 1.0, 0.3, 1.0, oracle.Opts(rtol=1e-11, cycle=cyc, max_cycles=40))
        phi, code, _ = dgp_gpu(B, ctx, delta, 1.0, 0.3, 1.0, rtol=1e-11, cycle=cyc, max_cycles=40)
        assert code == 0 and l2(phi, ref) < 1e-9, (cyc, l2(phi, ref))


@pytest.mark.parametrize("nk,k0", [(2, 1.0), (3, 1.0), (2, 0.5)])
def test_solve_kmouflage(B, ctx, nk, k0):
    """Kmouflage (n, K0) of the paper's models, beta = 0.2, synthetic
    background: lambda^2 = 3(1 - Omega_m), phibar'/H0 = -1e-3, A = e^-0.02."""
    n, box, a, om = 32, 64.0, 1.0, 0.3
    delta = 30.0 * config1_delta()
    lam = np.sqrt(3 * (1 - om))
    pars = (box, nk, k0, 0.2, lam, -1e-3, np.exp(-0.02))
    ref, rst = oracle.kmo_solve(delta, a, om, *pars, oracle.Opts(rtol=1e-10, max_cycles=40))
    phi = np.zeros_like(delta)
    code, st = B.mg_solve_kmouflage(ctx, n, box, a, om, nk, k0, 0.2, lam, -1e-3, np.exp(-0.02), delta, phi,
                                    B.opts(rtol=1e-10, max_cycles=40))
    assert code == 0 and l2(phi, ref) < 1e-8, l2(phi, ref)
    assert abs(st.cycles - rst.cycles) <= 1


def test_uniform_and_warm_start(B, ctx):
    n = 16
    z = np.zeros((n,) * 3)
    phi = inputs.uniform_guess(n, 1)
    code, st = B.mg_solve_dgp(ctx, [dict(ng=n, a=1.0, omega_m=0.3, rc_h0=1.0, delta=z, phi=phi)],
                              B.opts(rtol=0.0, atol=1e-13, warm_start=1))
    assert code == 0 and np.abs(phi).max() < 1e-12
    delta = config1_delta(16, 32.0, 2)
    ref, _ = oracle.dgp_solve(delta, 1.0, 0.3, 1.0, oracle.Opts(rtol=1e-12, max_cycles=40))
    phi = ref.copy()
    code, st = B.mg_solve_dgp(ctx, [dict(ng=n, a=1.0, omega_m=0.3, rc_h0=1.0, delta=delta, phi=phi)],
                              B.opts(rtol=1e-8, warm_start=1))
    assert code == 0 and st[0].cycles == 0 and l2(phi, ref) < 1e-13


def test_device_and_host_pointers_agree_and_are_deterministic(B, ctx):
    delta = config1_delta()
    phi_h, _, _ = dgp_gpu(B, ctx, delta, 1.0, 0.3, 1.0)
    d = torch.from_numpy(delta).cuda()
    outs = []
    for _ in range(2):
        p = torch.zeros_like(d)
        B.mg_solve_dgp(ctx, [dict(ng=32, a=1.0, omega_m=0.3, rc_h0=1.0, delta=d, phi=p)], B.opts())
        torch.cuda.synchronize()
        outs.append(p.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], phi_h)
    p = torch.zeros_like(d)
    B.mg_solve_dgp(ctx, [dict(ng=32, a=1.0, omega_m=0.3, rc_h0=1.0, delta=d, phi=p)], B.opts(use_graph=0))
    assert np.array_equal(p.cpu().numpy(), phi_h)


@pytest.mark.parametrize("graph", [1, 0])
def test_profiling_events(B, ctx, graph):
    """With profiling on, every finest-level half-sweep is bracketed by
    events (graph nodes when captured): 2 (pre + post) launches per cycle."""
    delta = config1_delta()
    ctx.set_profiling(True)
    try:
        _, _, st = dgp_gpu(B, ctx, delta, 1.0, 0.3, 1.0, use_graph=graph)
    finally:
        ctx.set_profiling(False)
    assert st.fine_smooth_launches == st.cycles * 2 * (2 + 2)
    assert 0.0 < st.fine_smooth_ms < st.ms
    assert st.kernel_launches > st.fine_smooth_launches


def test_errors(B, ctx):
    z = np.zeros((20,) * 3)
    with pytest.raises(B.MGError) as e:
        B.mg_solve_dgp(ctx, [dict(ng=20, a=1.0, omega_m=0.3, rc_h0=1.0, delta=z, phi=z.copy())])
    assert e.value.code == B.MG_ERR_ARG
    bad = np.zeros((16,) * 3)
    bad[3, 4, 5] = np.nan
    with pytest.raises(B.MGError) as e:
        B.mg_solve_dgp(ctx, [dict(ng=16, a=1.0, omega_m=0.3, rc_h0=1.0, delta=bad, phi=np.zeros_like(bad))])
    assert e.value.code == B.MG_ERR_NONFINITE
    delta = config1_delta(16, 32.0, 2)
    code, st = B.mg_solve_dgp(ctx, [dict(ng=16, a=1.0, omega_m=0.3, rc_h0=1.0, delta=delta,
                                         phi=np.zeros_like(delta))], B.opts(max_cycles=1, rtol=1e-12))
    assert code == B.MG_WARN_NOT_CONVERGED and st[0].cycles == 1


# ------------------------------------------------------------ CIC

def test_cic_parity(B, ctx):
    ng, nps = 32, 16
    pos, _ = inputs.zeldovich(nps, ng, 64.0, inputs.pk_cutoff(), 1.0, seed=5)
    edge = np.array([0.0, 0.5, np.nextafter(np.float32(0.5), np.float32(0)), 31.5,
                     np.nextafter(np.float32(32.0), np.float32(0)), 7.5, 7.499999], dtype=np.float32)
    pos[: len(edge)] = edge[:, None]
    ref, idx = oracle.cic_deposit(pos, ng, nps)
    out = np.empty((ng,) * 3)
    B.pm_cic_deposit(ctx, ng, pos, out)
    assert np.abs(out - ref).max() < 1e-8
    gidx = np.empty((pos.shape[0], 3), dtype=np.int32)
    B.pm_cic_index(ctx, ng, pos, gidx)
    assert np.array_equal(gidx.astype(np.int64), idx)
    out2 = np.empty_like(out)
    B.pm_cic_deposit(ctx, ng, pos, out2)
    assert np.array_equal(out, out2)


@pytest.mark.parametrize("n,nk", [(16, 2), (32, 3)])
def test_kmouflage_linear_solve(B, ctx, n, nk):
    """The linear-theory Kmouflage field (Eq. kmf_eqn_codeunit_lin) against
    the oracle's FFT solution, and the full solve approaching it for a small
    density field."""
    a, om, L = 1.0, 0.3, float(n)
    pars = (nk, 10.0, 0.2, 1.0, 0.3, 1.0)
    delta = 50.0 * inputs.white_noise(n, 95)
    ref = oracle.kmo_linear_solve(delta, a, om, L, *pars)
    out = np.empty_like(delta)
    B.mg_solve_kmouflage_linear(ctx, n, L, a, om, *pars, delta, out)
    assert l2(out, ref) < 1e-12
    full = np.zeros_like(delta)
    B.mg_solve_kmouflage(ctx, n, L, a, om, *pars, 0.01 * delta, full, B.opts(rtol=1e-12, max_cycles=60))
    assert l2(full, 0.01 * ref) < 1e-4
