"""The FP64 nDGP kernels sum their stencil exactly in 64-bit fixed point on
the integer pipe and form the quadratic form of the differences exactly in
128-bit integers, with FP64 arithmetic as the fallback outside the range
those integers cover (the largest value of a stencil between 2^-453 and
2^506) and a general shift where a stencil's exponents span 32 binades or
more.  Each branch is checked against the oracle here.

The operator is scale-covariant: with u -> lam u, alpha -> lam alpha,
s -> lam^2 s, f -> lam f and c -> lam c, N and the smoother's new value scale
by lam exactly, so one field at several scales drives every branch:
lam = 1 (fixed point, near shifts), lam = 1e150 (fixed point at the top of
its range), lam = 1e-140 (FP64 fallback below it), and a field whose
magnitudes spread over 12 decades (fixed point, general shifts).  Meshes of
64^3 and more run the smoother whose blocks stage their stencil planes in
shared memory at one block-wide fixed-point scale; the smaller ones the
kernel whose threads convert their own stencils.  Above the
range (2^506) lies only a few binades' window before the operator's squares
overflow binary64 in any arithmetic, so it has no case here."""
import numpy as np
import pytest

import oracle
from paper_2110_00566_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import B, ctx, rel  # noqa: E402,F401

ALPHA = 1.7


def case(n, seed, lam, spread):
    u = inputs.white_noise(n, seed)
    if spread:
        u = u * 10.0 ** (-12.0 * inputs.uniform01(seed + 7, n ** 3).reshape((n,) * 3))
    s = 0.7 * inputs.white_noise(n, seed + 1)
    f = 0.2 * inputs.white_noise(n, seed + 2)
    return lam * u, lam * lam * s, lam * f


@pytest.mark.parametrize("lam,spread", [(1.0, False), (1e150, False), (1e-140, False), (1.0, True)])
@pytest.mark.parametrize("n,h", [(16, 1.0), (24, 4.0), (64, 2.0), (128, 1.0)])
def test_fp64_smoother_branches(B, ctx, lam, spread, n, h):
    o = oracle.OrcOp(0, ALPHA * lam, 0, 0.0, 0.0)
    b = B.op_params(0, ALPHA * lam, 2, 0.0, 0.0)
    u, s, f = case(n, 31, lam, spread)
    for colour in (0, 1):
        for ff in (None, f):
            ref = oracle.smooth(o, u, s, ff, h, 0.031 * lam, colour)
            out = np.empty_like(u)
            B.mg_op_smooth(ctx, b, 0, n, h, u, s, ff, 0.031 * lam, colour, out)
            assert rel(out, ref) < 1e-12, (colour, rel(out, ref))


@pytest.mark.parametrize("lam,spread", [(1.0, False), (1e150, False), (1e-140, False), (1.0, True)])
@pytest.mark.parametrize("n", [16, 128])
def test_fp64_residual_branches(B, ctx, lam, spread, n):
    h = 2.0
    o = oracle.OrcOp(0, ALPHA * lam, 0, 0.0, 0.0)
    b = B.op_params(0, ALPHA * lam, 2, 0.0, 0.0)
    u, s, f = case(n, 41, lam, spread)
    for ff in (None, f):
        d, c, eps = oracle.residual(o, u, s, ff, h)
        Ru = np.empty((n // 2,) * 3)
        Rd = np.empty((n // 2,) * 3)
        cg, eg = B.mg_op_resid_restrict(ctx, b, 0, n, h, u, s, ff, Ru, Rd)
        scale = np.abs(d).max() + 12.0 * np.abs(u).max() / h ** 2
        assert rel(Ru, oracle.restrict(u)) < 1e-14
        assert np.abs(Rd - oracle.restrict(d)).max() < 1e-13 * scale
        assert abs(cg - c) <= 1e-13 * scale
        assert abs(eg - eps) <= 1e-12 * scale


def test_scale_covariance_of_the_fixed_point_update(B, ctx):
    """The fixed-point update at lam = 2^500 is the lam = 1 update times lam,
    bit for bit: every FP64 step sees its operands scaled by a power of two
    (the integer part of the arithmetic is scale-free up to the power of two
    in its exponent; the
    square root's seed is formed from the mantissa and the exponent's parity,
    so it scales exactly by powers of four)."""
    n, h = 16, 1.0
    outs = []
    for lam in (1.0, 2.0 ** 500):
        b = B.op_params(0, ALPHA * lam, 2, 0.0, 0.0)
        u, s, f = case(n, 51, lam, False)
        out = np.empty_like(u)
        B.mg_op_smooth(ctx, b, 0, n, h, u, s, f, 0.031 * lam, 0, out)
        outs.append(out / lam)
    # a power-of-two scale leaves every rounding unchanged
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("n", [64, 128])
def test_block_fixed_point_with_a_nonfinite_and_a_rising_scale(B, ctx, n):
    """The block-staged FP64 smoother where a block's running scale rises
    along its planes (a field growing by 10^6 across the mesh in i: the
    staged planes are shifted down to the new scale) and where one value is
    infinite (that block's later planes take the FP64 gather form): every
    finite result against the oracle, the infinite neighbourhood non-finite
    in both."""
    h = 1.0
    o = oracle.OrcOp(0, ALPHA, 0, 0.0, 0.0)
    b = B.op_params(0, ALPHA, 2, 0.0, 0.0)
    u, s, f = case(n, 61, 1.0, False)
    grow = 10.0 ** (6.0 * np.arange(n) / n)
    u = u * grow[:, None, None]
    for colour in (0, 1):
        ref = oracle.smooth(o, u, s, f, h, 0.031, colour)
        out = np.empty_like(u)
        B.mg_op_smooth(ctx, b, 0, n, h, u, s, f, 0.031, colour, out)
        # error relative to the largest |u| of the three planes around each
        # updated plane (the block's scale is that of its staged planes)
        pm = np.abs(u).reshape(n, -1).max(axis=1)
        scale = np.maximum(np.maximum(pm, np.roll(pm, 1)), np.roll(pm, -1))
        err = np.abs(out - ref).reshape(n, -1).max(axis=1)
        assert (err <= 1e-12 * scale).all(), (err / scale).max()
    # the infinite value in a cell of the colour not updated (a face
    # neighbour of updated cells): the printed Sigma of the oracle also has
    # centre terms, which cancel algebraically but give inf - inf at an
    # infinite centre, where the GPU's form has none
    v = u.copy()
    v[n // 2, 5, 8] = np.inf
    ref = oracle.smooth(o, v, s, f, h, 0.031, 0)
    out = np.empty_like(v)
    B.mg_op_smooth(ctx, b, 0, n, h, v, s, f, 0.031, 0, out)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(out))
    scale = np.abs(ref[fin]).max()
    assert np.abs(out[fin] - ref[fin]).max() <= 1e-12 * scale
