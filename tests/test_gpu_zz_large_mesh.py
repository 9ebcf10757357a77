"""The largest power-of-two mesh below the supported 1536^3: a 1024^3 nDGP
solve (8x the benchmark's cells, nine levels) in FP64 and in mixed
precision, with its own context so that its ~100 GB of workspace is
released at the end.  The oracle cannot solve or even hold this mesh in
seconds, so the checks are the ones that hold at any size: both solves
converge to the requested eps/eps_ref < 1e-8 on their FP64 residual norm,
phi is finite with zero mean (the gauge of the output), and the two solves
agree to the stated 1e-6 relative L2.  The density is seeded white noise
(rms 2) drawn on the device by torch's generator.  Collected last."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import B  # noqa: E402,F401


def test_1024_fp64_and_mixed_solves(B):
    n = 1024
    g = torch.Generator(device="cuda").manual_seed(1024)
    delta = 2.0 * torch.randn((n,) * 3, generator=g, dtype=torch.float64, device="cuda")
    c = B.Context(0)
    try:
        sols = []
        for prec in (B.MG_PREC_FP64, B.MG_PREC_MIXED):
            phi = torch.zeros_like(delta)
            code, st = B.mg_solve_dgp(c, [dict(ng=n, box_mpch=512.0, a=1.0, omega_m=0.3, rc_h0=1.0, delta=delta,
                                               phi=phi)], B.opts(rtol=1e-8, precision=prec, max_cycles=40))
            assert code == 0, (prec, st[0].eps_list())
            eps = st[0].eps_list()
            assert eps[-1] <= 1e-8 * st[0].eps_ref, (prec, eps[-1] / st[0].eps_ref)
            assert bool(torch.isfinite(phi).all())
            scale = float(phi.abs().max())
            assert abs(float(phi.mean())) < 1e-12 * scale
            sols.append(phi)
        rel = float(torch.linalg.vector_norm(sols[1] - sols[0]) / torch.linalg.vector_norm(sols[0]))
        assert rel < 1e-6, rel
    finally:
        c.close()
        torch.cuda.empty_cache()
