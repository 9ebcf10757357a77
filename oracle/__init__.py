"""Plain FP64 CPU oracle for the MG-GLAM derivative-coupling solvers.

TEST INFRASTRUCTURE ONLY.  The oracle is the checker the CUDA path is
compared against.  Only tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference leg of ``bench.py`` import it; the product package
never does.  It shares no code with the CUDA path: the cell-level arithmetic
lives in ``mg_oracle.c`` (plain C loops, FP64), and this module adds the
paper's closed-form background quantities, the FFT Poisson solve (numpy FFT
as a library primitive) and the particle-mesh step, each citing the passage
of arXiv:2110.00566 it follows.

Arrays are numpy float64 of shape (n, n, n), C order, index (i, j, k) with
k fastest; cell (i, j, k) has its centre at (i+1/2, j+1/2, k+1/2) in code
units (cell size h = 1 on the finest mesh, Sec. 3.1.1).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

C_OVER_H0_MPCH = 2997.92458   # c / H0 in Mpc/h (c = 299792.458 km/s, H0 = 100 h km/s/Mpc)

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _declare(_lib)
    return _lib


class OrcOp(C.Structure):
    _fields_ = [("model", C.c_int), ("alpha", C.c_double), ("nkmo", C.c_int),
                ("gamma", C.c_double), ("bterm", C.c_double)]


class OrcOpts(C.Structure):
    _fields_ = [("pre", C.c_int), ("post", C.c_int), ("max_cycles", C.c_int),
                ("cycle", C.c_int), ("coarse_sweeps", C.c_int),
                ("rtol", C.c_double), ("atol", C.c_double)]


class OrcStats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("eps_ref", C.c_double),
                ("eps", C.c_double * 65), ("c_final", C.c_double),
                ("mean_shift", C.c_double), ("sqrt_clamps", C.c_long)]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_fp = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def _declare(L):
    P = C.POINTER
    L.orc_dgp_sigma.restype = C.c_double
    L.orc_dgp_sigma.argtypes = [_dp, C.c_long, C.c_double, C.c_long, C.c_long, C.c_long, C.c_double]
    L.orc_dgp_N.restype = C.c_double
    L.orc_dgp_N.argtypes = [C.c_double, C.c_double, P(C.c_long)]
    L.orc_kmo_N.restype = C.c_double
    L.orc_kmo_N.argtypes = [P(OrcOp), _dp, C.c_long, C.c_double, C.c_long, C.c_long, C.c_long, C.c_double]
    L.orc_N_field.restype = None
    L.orc_N_field.argtypes = [P(OrcOp), _dp, _dp, C.c_long, C.c_double, _dp, P(C.c_long)]
    L.orc_mean.restype = C.c_double
    L.orc_mean.argtypes = [_dp, C.c_long]
    L.orc_smooth.restype = None
    L.orc_smooth.argtypes = [P(OrcOp), _dp, _dp, _dp, C.c_void_p, C.c_long, C.c_double, C.c_double, C.c_int]
    L.orc_residual.restype = C.c_double
    L.orc_residual.argtypes = [P(OrcOp), _dp, _dp, C.c_void_p, C.c_long, C.c_double, _dp,
                               P(C.c_double), P(C.c_long)]
    L.orc_restrict.restype = None
    L.orc_restrict.argtypes = [_dp, C.c_long, _dp]
    L.orc_prolong_add.restype = None
    L.orc_prolong_add.argtypes = [_dp, C.c_long, _dp, _dp]
    L.orc_num_levels.restype = C.c_int
    L.orc_num_levels.argtypes = [C.c_long]
    L.orc_mg_solve.restype = C.c_int
    L.orc_mg_solve.argtypes = [P(OrcOp), C.c_long, _dp, C.c_double, P(OrcOpts), _dp, P(OrcStats)]
    L.orc_cic_deposit.restype = None
    L.orc_cic_deposit.argtypes = [_fp, C.c_long, C.c_long, C.c_double, _dp, C.c_void_p]
    L.orc_cic_force.restype = None
    L.orc_cic_force.argtypes = [_dp, C.c_long, _fp, C.c_long, _dp]


# ---------------------------------------------------------------------------
# background quantities (closed forms of Sec. 2.1 and Sec. 3.2.3-3.2.4)
# ---------------------------------------------------------------------------

def E_lcdm(a, omega_m):
    """H(a)/H0 for flat LCDM (Eq. H_lcdm); nDGP is tuned to this history."""
    return np.sqrt(omega_m * a ** -3 + (1.0 - omega_m))


def beta_dgp(a, omega_m, rc_h0):
    """beta_DGP(a) for the LCDM-matched nDGP background (Eq. beta_dgp), with
    Omega_rc = 1/(4 R_c^2) and R_c = r_c H0 / c (Sec. 3.2.3)."""
    omega_rc = 1.0 / (4.0 * rc_h0 ** 2)
    om_a = omega_m * a ** -3
    ol = 1.0 - omega_m
    return 1.0 + (om_a + 2.0 * ol) / (2.0 * np.sqrt(omega_rc * (om_a + ol)))


def alpha_dgp(a, omega_m, rc_h0):
    """alpha = 3 beta_DGP a^2 / R_c^2 (Sec. 3.2.3, after Eq. dgp_quadratic_eom)."""
    return 3.0 * beta_dgp(a, omega_m, rc_h0) * a * a / rc_h0 ** 2


def c_tilde(ng, box_mpch):
    """Code-unit speed of light c~ = (N_g / (H0 L)) c (Sec. 3.1.1)."""
    return C_OVER_H0_MPCH * ng / box_mpch


def gamma_kmo(n, k0, a, lam):
    """gamma = n K0 (1/(2 a^2 lambda^2))^(n-1) (Sec. 3.2.4, after Eq. kmo_eom)."""
    return n * k0 * (1.0 / (2.0 * a * a * lam * lam)) ** (n - 1)


# ---------------------------------------------------------------------------
# thin wrappers over the C oracle
# ---------------------------------------------------------------------------

def _c(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def dgp_op(alpha):
    return OrcOp(0, float(alpha), 0, 0.0, 0.0)


def kmo_op(n, gamma, bterm):
    return OrcOp(1, 0.0, int(n), float(gamma), float(bterm))


def dgp_sigma(u, h, i, j, k, s):
    u = _c(u)
    return lib().orc_dgp_sigma(u.ravel(), u.shape[0], float(h), i, j, k, float(s))


def dgp_N(sigma, alpha):
    cl = C.c_long(0)
    v = lib().orc_dgp_N(float(sigma), float(alpha), C.byref(cl))
    return v, cl.value


def N_field(op, u, s, h):
    u, s = _c(u), _c(s)
    out = np.empty_like(u)
    cl = C.c_long(0)
    lib().orc_N_field(C.byref(op), u.ravel(), s.ravel(), u.shape[0], float(h), out.ravel(), C.byref(cl))
    return out, cl.value


def smooth(op, u, s, f, h, c, colour):
    """One colour-simultaneous half-sweep; returns the new field."""
    u, s = _c(u), _c(s)
    out = np.empty_like(u)
    fp = None if f is None else _c(f)
    lib().orc_smooth(C.byref(op), u.ravel(), out.ravel(), s.ravel(),
                     None if fp is None else fp.ctypes.data, u.shape[0], float(h), float(c), int(colour))
    return out


def residual(op, u, s, f, h):
    """Returns (d, c, eps) with c = <N(u)> and d = Lap u - N + c - f."""
    u, s = _c(u), _c(s)
    d = np.empty_like(u)
    fp = None if f is None else _c(f)
    eps = C.c_double(0.0)
    cl = C.c_long(0)
    c = lib().orc_residual(C.byref(op), u.ravel(), s.ravel(), None if fp is None else fp.ctypes.data,
                           u.shape[0], float(h), d.ravel(), C.byref(eps), C.byref(cl))
    return d, c, eps.value


def restrict(fine):
    fine = _c(fine)
    n = fine.shape[0]
    out = np.empty((n // 2,) * 3)
    lib().orc_restrict(fine.ravel(), n, out.ravel())
    return out


def prolong_add(u_fine, uc, urc):
    out = _c(u_fine).copy()
    lib().orc_prolong_add(out.ravel(), out.shape[0], _c(uc).ravel(), _c(urc).ravel())
    return out


def num_levels(n):
    return lib().orc_num_levels(int(n))


@dataclass
class Opts:
    pre: int = 2
    post: int = 2
    max_cycles: int = 30
    cycle: int = 0            # 0 = V, 1 = F, 2 = W
    coarse_sweeps: int = 16
    rtol: float = 1e-8
    atol: float = 0.0

    def c(self):
        return OrcOpts(self.pre, self.post, self.max_cycles, self.cycle, self.coarse_sweeps,
                       self.rtol, self.atol)


@dataclass
class Stats:
    cycles: int
    eps_ref: float
    eps: list = field(default_factory=list)
    c_final: float = 0.0
    mean_shift: float = 0.0
    sqrt_clamps: int = 0


def mg_solve(op, s0, eps_ref, opts: Opts = None, u0=None):
    """Generic FAS multigrid solve of Lap u = N(u) - <N(u)> on the finest
    level (Sec. 3.2.1).  s0: finest density term (mean-subtracted, scaled)."""
    opts = opts or Opts()
    s0 = _c(s0)
    n = s0.shape[0]
    u = np.zeros_like(s0) if u0 is None else _c(u0).copy()
    st = OrcStats()
    lib().orc_mg_solve(C.byref(op), n, s0.ravel(), float(eps_ref), C.byref(opts.c()), u.ravel(), C.byref(st))
    stats = Stats(st.cycles, st.eps_ref, list(st.eps[: st.cycles + 1]), st.c_final, st.mean_shift, st.sqrt_clamps)
    return u, stats


def dgp_source(delta, a, omega_m, rc_h0):
    """Finest-level density term of the nDGP equation in code units
    (Eq. dgp_eom_code): s = (alpha/beta) Omega_m a^-1 (delta - <delta>), and
    the reference scale eps_ref = rms(Omega_m a^-1 delta / beta)."""
    delta = _c(delta)
    beta = beta_dgp(a, omega_m, rc_h0)
    alpha = alpha_dgp(a, omega_m, rc_h0)
    dm = delta - lib().orc_mean(delta.ravel(), delta.size)
    s0 = (alpha / beta) * omega_m / a * dm
    eps_ref = float(np.sqrt(np.mean((omega_m / (a * beta) * dm) ** 2)))
    return s0, eps_ref, alpha, beta


def dgp_solve(delta, a, omega_m, rc_h0, opts: Opts = None, u0=None):
    """nDGP scalar field phi~ (code units) for a density contrast delta."""
    s0, eps_ref, alpha, _ = dgp_source(delta, a, omega_m, rc_h0)
    return mg_solve(dgp_op(alpha), s0, eps_ref, opts, u0)


def kmo_source(delta, a, omega_m, ng, box_mpch, beta_kmo, A_bar):
    """Finest-level Kmouflage density term: the right-hand side of Eq.
    kmf_eqn_codeunit_final divided by c~, 3 beta A(phibar) Omega_m a^-1 delta
    / c~ (dA/dphi = beta A for A = exp(beta phi)); eps_ref = rms of it."""
    delta = _c(delta)
    ct = c_tilde(ng, box_mpch)
    dm = delta - lib().orc_mean(delta.ravel(), delta.size)
    s0 = 3.0 * beta_kmo * A_bar * omega_m / a * dm / ct
    eps_ref = float(np.sqrt(np.mean(s0 ** 2)))
    return s0, eps_ref


def kmo_solve(delta, a, omega_m, box_mpch, n, k0, beta_kmo, lam, phibar_prime_over_h0, A_bar,
              opts: Opts = None, u0=None):
    """Kmouflage field phi~ = c~ phi (Eq. Kmo_unit) for a density contrast."""
    ng = delta.shape[0]
    s0, eps_ref = kmo_source(delta, a, omega_m, ng, box_mpch, beta_kmo, A_bar)
    op = kmo_op(n, gamma_kmo(n, k0, a, lam), phibar_prime_over_h0 ** 2)
    return mg_solve(op, s0, eps_ref, opts, u0)


def kmo_linear_solve(delta, a, omega_m, box_mpch, n, k0, beta_kmo, lam, phibar_prime_over_h0, A_bar):
    """Linear-theory Kmouflage field (Eq. kmf_eqn_codeunit_lin): the gradient
    term of Sigma_1 and Sigma_2 dropped,
        Lap phi~ = 3 beta A Omega_m a^-1 delta / [c~ (1 + gamma (phibar'^2/H0^2)^(n-1))],
    solved with the 7-point Green's function (the multigrid Laplacian)."""
    ng = delta.shape[0]
    s0, _ = kmo_source(delta, a, omega_m, ng, box_mpch, beta_kmo, A_bar)
    k1 = 1.0 + gamma_kmo(n, k0, a, lam) * (phibar_prime_over_h0 ** 2) ** (n - 1)
    return fft_poisson(s0 / k1)


# ---------------------------------------------------------------------------
# particle-mesh pieces (Sec. 3.1, 3.1.1)
# ---------------------------------------------------------------------------

def cic_deposit(pos, ng, np_side):
    """delta on the mesh by cloud-in-cell (Sec. 3.1); pos: (np, 3) float32
    code-unit positions in [0, ng).  Returns (delta, lower-cell indices)."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    npart = pos.shape[0]
    delta = np.empty((ng,) * 3)
    idx = np.empty((npart, 3), dtype=np.int64)
    mass = (ng / np_side) ** 3
    lib().orc_cic_deposit(pos.ravel(), npart, ng, mass, delta.ravel(), idx.ctypes.data)
    return delta, idx


def cic_force(phi, pos):
    """-grad phi by 3-point differences at the 8 CIC cells, interpolated to
    the particles with the CIC weights (Sec. 3.1)."""
    phi = _c(phi)
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    acc = np.empty((pos.shape[0], 3))
    lib().orc_cic_force(phi.ravel(), phi.shape[0], pos.ravel(), pos.shape[0], acc.ravel())
    return acc


def laplacian_eigenvalues(ng):
    """Eigenvalues of the 7-point periodic Laplacian on the rfftn grid:
    -sum_d 4 sin^2(pi k_d / N)."""
    k = np.fft.fftfreq(ng) * ng
    kz = np.fft.rfftfreq(ng) * ng
    sx = 4.0 * np.sin(np.pi * k / ng) ** 2
    sz = 4.0 * np.sin(np.pi * kz / ng) ** 2
    return -(sx[:, None, None] + sx[None, :, None] + sz[None, None, :])


def fft_poisson(rhs):
    """Solve Lap_h Phi = rhs on the periodic mesh with the discrete (7-point)
    Green's function; the k = 0 mode is set to zero (Sec. 3.1: GLAM solves
    the discrete analogue of the Poisson equation by FFT)."""
    ng = rhs.shape[0]
    rk = np.fft.rfftn(rhs)
    lam = laplacian_eigenvalues(ng)
    lam[0, 0, 0] = 1.0
    pk = rk / lam
    pk[0, 0, 0] = 0.0
    return np.fft.irfftn(pk, s=rhs.shape, axes=(0, 1, 2))


def newton_potential(delta, a, omega_m):
    """Phi_N~ from Lap Phi~ = (3/2) Omega_m a^-1 delta (Eq. GR_poisson_codeunit)."""
    return fft_poisson(1.5 * omega_m / a * _c(delta))


def _wrap32(x, ng):
    x = x.astype(np.float32)
    x = np.where(x < 0, x + np.float32(ng), x).astype(np.float32)
    x = np.where(x >= ng, x - np.float32(ng), x).astype(np.float32)
    return x


def pm_step(pos, mom, ng, np_side, omega_m, a, da, model=1, rc_h0=1.0, first=False,
            phi_guess=None, opts: Opts = None, kmo=None, box_mpch=None, hubble=None):
    """One leapfrog step in the scale factor (Sec. 3.1.1 code-unit equations
    of motion, with the drift sign of Eq. force_Kmo1):
        dp~/da = -(H0/adot) grad~ Phi~,   dx~/da = H0/(a^2 adot) p~,
    H0/adot = 1/(a E(a)).  Positions at a, momenta at a - da/2 (a - 0 when
    first=True) are advanced to a + da and a + da/2.  Phi = Phi_N + phi/2 for
    nDGP (Eq. poisson_nDGP), Phi_N for GR (model 0).  Kmouflage (model 2,
    Eqs. force_Kmo2 and kmf_Poission_eqn_codeunit): Lap Phi_N = (3/2) A
    Omega_m a^-1 delta, Phi = Phi_N + beta c~ phi~ with phi~ the Kmouflage
    field, and the friction term dp~/da = -beta (dphibar/da) p~ taken in the
    kick as the factor 1 - beta (dphibar/da) da_kick; kmo = dict(n, k0, beta,
    lam, phibar_prime_over_h0, A_bar, dphibar_da), the background inputs at
    a, and box_mpch the box (for c~).  hubble = (E(a), E(a + da/2)), the
    model's own H/H0 (the Kmouflage background), replaces LCDM's E in
    H0/adot = 1/(a E).  FP32 state, FP64 force.
    Returns (pos, mom, phi)."""
    delta, _ = cic_deposit(pos, ng, np_side)
    phi = None
    fr = 1.0
    dak = 0.5 * da if first else da
    if model == 2:
        k = kmo
        phin = newton_potential(delta, a, omega_m * k["A_bar"])
        phi, _ = kmo_solve(delta, a, omega_m, box_mpch, k["n"], k["k0"], k["beta"], k["lam"],
                           k["phibar_prime_over_h0"], k["A_bar"], opts, phi_guess)
        phin = phin + (k["beta"] * c_tilde(ng, box_mpch)) * phi
        fr = 1.0 - k["beta"] * k["dphibar_da"] * dak
    else:
        phin = newton_potential(delta, a, omega_m)
    if model == 1:
        phi, _ = dgp_solve(delta, a, omega_m, rc_h0, opts, phi_guess)
        phin = phin + 0.5 * phi
    acc = cic_force(phin, pos)
    am = a + 0.5 * da
    E_a, E_m = hubble if hubble is not None else (E_lcdm(a, omega_m), E_lcdm(am, omega_m))
    mom = (mom.astype(np.float64) * fr + acc * (dak / (a * E_a))).astype(np.float32)
    pos = (pos.astype(np.float64) + mom.astype(np.float64) * (da / (am ** 3 * E_m)))
    return _wrap32(pos, ng), mom, phi


# ---------------------------------------------------------------------------
# reference gradient of the nDGP solution map (brute force, small meshes)
# ---------------------------------------------------------------------------

def dgp_gradient(delta, a, omega_m, rc_h0, g, opts: Opts = None, step=1e-6):
    """Gradient of L = <g, phi(delta, R_c)> for the discrete nDGP solve
    (Sec. 3.2.3 operator with the compatibility projection, gauge <phi> = 0):
    the dense Jacobians J = dF/dphi and B = dF/ddelta of the residual map
    F(phi, delta) are taken by central differences of the oracle's own
    residual at the converged phi, and J^T lambda = Pi g is solved with the
    constant null direction pinned by adding 11^T/n^3 (J^T maps zero-mean
    fields to zero-mean fields and 1 to 0).  Then dL/ddelta = -B^T lambda and
    dL/dR_c = -lambda . dF/dR_c (dF/dR_c by central differences as well).
    Returns (dL/ddelta, dL/dR_c, phi).  Cost O(n^6) memory: small n only."""
    delta = _c(delta)
    n = delta.shape[0]
    N = n ** 3
    phi, _ = dgp_solve(delta, a, omega_m, rc_h0, opts or Opts(rtol=1e-13, max_cycles=60))

    def F(u, d, rc):
        s0, _, alpha, _ = dgp_source(d, a, omega_m, rc)
        return residual(dgp_op(alpha), u, s0, None, 1.0)[0].ravel()

    su = step * max(1.0, np.abs(phi).max())
    sd = step * max(1.0, np.abs(delta).max())
    J = np.empty((N, N))
    Bm = np.empty((N, N))
    for q in range(N):
        e = np.zeros(N)
        e[q] = 1.0
        e = e.reshape(delta.shape)
        J[:, q] = (F(phi + su * e, delta, rc_h0) - F(phi - su * e, delta, rc_h0)) / (2 * su)
        Bm[:, q] = (F(phi, delta + sd * e, rc_h0) - F(phi, delta - sd * e, rc_h0)) / (2 * sd)
    gp = g.ravel() - g.mean()
    lam = np.linalg.solve(J.T + np.full((N, N), 1.0 / N), gp)
    dd = -(Bm.T @ lam)
    sr = step * rc_h0
    dFdr = (F(phi, delta, rc_h0 + sr) - F(phi, delta, rc_h0 - sr)) / (2 * sr)
    return dd.reshape(delta.shape), float(-(lam @ dFdr)), phi
