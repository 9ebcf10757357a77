"""Invariants of the discrete nDGP and Kmouflage systems on the GPU path (the oracle's
pins P7, here on the CUDA solve): the periodic mesh has no preferred
origin and no preferred axis, so a periodic shift or an axis permutation of
delta shifts or permutes phi, and the mean-subtracted source makes phi
independent of a constant added to delta.  The block-staged kernels tile
the mesh with fixed tiles and scales, so the two solves round differently;
both are converged far below the comparison tolerance (1e-10 relative
residual, compared at 1e-8).  Meshes: 48^3 (per-thread kernels) and 128^3
(block-staged FP64 kernels), FP64 and mixed precision, nDGP and Kmouflage
(n = 2)."""
import numpy as np
import pytest

from paper_2110_00566_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import B, ctx  # noqa: E402,F401


def l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def solve(B, ctx, delta, prec, model="dgp"):
    n = delta.shape[0]
    phi = np.zeros_like(delta)
    o = B.opts(rtol=1e-10, precision=prec, max_cycles=60)
    if model == "dgp":
        code, st = B.mg_solve_dgp(ctx, [dict(ng=n, box_mpch=float(n), a=1.0, omega_m=0.3, rc_h0=1.0, delta=delta,
                                             phi=phi)], o)
        st = st[0]
    else:
        code, st = B.mg_solve_kmouflage(ctx, n, 2.0 * n, 1.0, 0.3, 2, 1.0, 0.2, float(np.sqrt(2.1)), -1e-3,
                                        np.exp(-0.02), delta, phi, o)
    assert code == 0, st.eps_list()
    return phi


@pytest.mark.parametrize("model", ["dgp", "kmo"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [48, 128])
def test_shift_permutation_and_offset(B, ctx, n, prec, model):
    amp = 3.0 if model == "dgp" else 30.0
    d = np.ascontiguousarray(amp * inputs.white_noise(n, 91))
    ref = solve(B, ctx, d, prec, model)
    # periodic shifts by odd and even offsets (an odd shift swaps the colours)
    for sh in [(1, 0, 0), (0, 3, 0), (0, 0, 5), (2, 7, 11)]:
        got = solve(B, ctx, np.ascontiguousarray(np.roll(d, sh, axis=(0, 1, 2))), prec, model)
        assert l2(np.roll(got, [-x for x in sh], axis=(0, 1, 2)), ref) < 1e-8, sh
    # axis permutations (the stencil's k-fastest split layout is not symmetric in the axes)
    for perm in [(1, 0, 2), (0, 2, 1), (2, 0, 1)]:
        got = solve(B, ctx, np.ascontiguousarray(np.transpose(d, perm)), prec, model)
        assert l2(np.transpose(got, np.argsort(perm)), ref) < 1e-8, perm
    # a constant added to delta: the source is mean-subtracted
    got = solve(B, ctx, d + 0.75, prec, model)
    assert l2(got, ref) < 1e-8
