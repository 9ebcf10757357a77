"""Differentiable particle-mesh chain with the nDGP solve: FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only tests/,
``__graft_entry__.smoke()`` and bench.py's CPU legs use it.

The forward model of the adjoint workload, each piece after arXiv:2110.00566:

* initial conditions: unit white noise w -> linear density
  delta_L(k) = A(k) w(k) (A = sqrt(P/V_cell), given) -> Zel'dovich
  displacement psi(k) = i k delta_L(k) / k^2 (the Nyquist component of k
  dropped), in mesh cells; particles on the lattice (q + 1/2) at
  x = q + D psi, momenta p = V psi (code units, Sec. 3.1.1);
* T leapfrog steps of constant da from a_start (Sec. 3.1.1 equations of
  motion, kick-drift-kick with the first half kick):
  delta = CIC(x) (Sec. 3.1), Phi_N from the 7-point Green's function
  (Eq. GR_poisson_codeunit), phi from the nDGP multigrid solve (Eq.
  dgp_eom_code), Phi = Phi_N + phi / 2 (Eq. poisson_nDGP), the force -grad
  Phi by central differences interpolated with the CIC weights;
  p += -(H0/adot) grad Phi da, x += H0/(a^2 adot) p da (H0/adot = 1/(a E));
* the binned power spectrum of CIC(x_T) in nbins linear bins from the
  fundamental to the Nyquist wavenumber, and the loss
  L = mean_b (P_b - P_target,b)^2.

Gradients of L with respect to the white noise and R_c = r_c H0 / c come
from reverse-mode automatic differentiation (torch.autograd, used as a
library primitive, FP64 on the CPU) through every piece except the nDGP
solve, whose backward is the implicit-function adjoint: with
F(phi, delta, R_c) = L(phi) the discrete residual of the oracle's C code and
J = dF/dphi written out as a sparse matrix from the stencil,
    J^T lambda = Pi dL/dphi   (zero-mean lambda),
    dL/ddelta = -(dF/ddelta)^T lambda,  dL/dR_c = -lambda . dF/dR_c,
the last by central differences of the oracle's residual in R_c.  The
sparse J is pinned against central differences of the oracle's residual
(tests/test_oracle_dpm.py).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

from . import (Opts, alpha_dgp, beta_dgp, dgp_op, dgp_solve, dgp_source, E_lcdm, residual)


@dataclass
class DpmConfig:
    ng: int                 # mesh cells per side = particles per side
    box: float              # Mpc/h
    omega_m: float
    a_start: float
    a_end: float
    nsteps: int
    nbins: int = 32
    model: int = 1          # 0 GR, 1 nDGP
    growth: float = 1.0     # D(a_start) applied to the displacement
    vel: float = 0.0        # momentum factor a^2 E D f at a_start


# ---------------------------------------------------------------------------
# pieces
# ---------------------------------------------------------------------------

def _freq(n):
    m = np.fft.fftfreq(n) * n
    mz = np.fft.rfftfreq(n) * n
    return m, mz


def zeldovich(w, amp, cfg: DpmConfig):
    """Particles (n^3, 3) and momenta from white noise w (n, n, n) tensor."""
    n = cfg.ng
    m, mz = _freq(n)
    kf = 2.0 * np.pi / cfg.box
    kx = torch.from_numpy((kf * m)[:, None, None] * np.ones((1, n, n // 2 + 1)))
    ky = torch.from_numpy((kf * m)[None, :, None] * np.ones((n, 1, n // 2 + 1)))
    kz = torch.from_numpy((kf * mz)[None, None, :] * np.ones((n, n, 1)))
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k2[0, 0, 0] = 1.0
    nyq = n // 2
    dk = torch.fft.rfftn(w) * torch.from_numpy(amp)
    cell = cfg.box / n
    psi = []
    for kc, mc in ((kx, m[:, None, None]), (ky, m[None, :, None]), (kz, mz[None, None, :])):
        keep = torch.from_numpy(np.broadcast_to(np.abs(mc) != nyq, kc.shape).copy())
        kc = torch.where(keep, kc, torch.zeros_like(kc))
        spec = (1j * kc / k2) * dk
        psi.append(torch.fft.irfftn(spec, s=(n, n, n)) / cell)
    psi = torch.stack([p.reshape(-1) for p in psi], dim=1)
    q = torch.arange(n, dtype=torch.float64) + 0.5
    qx, qy, qz = torch.meshgrid(q, q, q, indexing="ij")
    lat = torch.stack([qx.reshape(-1), qy.reshape(-1), qz.reshape(-1)], dim=1)
    x = torch.remainder(lat + cfg.growth * psi, float(n))
    return x, cfg.vel * psi


def _cic(x, n):
    """Lower cells, upper cells and weights per axis: lo = floor(x - 1/2),
    upper weight x - 1/2 - lo (Sec. 3.1, cell centres at i + 1/2)."""
    t = x - 0.5
    lo = torch.floor(t.detach())
    dx = t - lo
    i0 = torch.remainder(lo.long(), n)
    i1 = torch.remainder(i0 + 1, n)
    return i0, i1, 1.0 - dx, dx


def _corners():
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                yield a, b, c


def cic_density(x, n):
    """delta = (n^3 / n_p) * sum of CIC weights - 1, mean removed."""
    i0, i1, w0, w1 = _cic(x, n)
    I = (i0, i1)
    W = (w0, w1)
    rho = torch.zeros(n ** 3, dtype=torch.float64)
    for a, b, c in _corners():
        idx = (I[a][:, 0] * n + I[b][:, 1]) * n + I[c][:, 2]
        w = W[a][:, 0] * W[b][:, 1] * W[c][:, 2]
        rho = rho.index_add(0, idx, w)
    delta = rho * (n ** 3 / x.shape[0]) - 1.0
    return (delta - delta.mean()).reshape(n, n, n)


def _lap_eigs(n):
    m, mz = _freq(n)
    sx = 4.0 * np.sin(np.pi * m / n) ** 2
    sz = 4.0 * np.sin(np.pi * mz / n) ** 2
    lam = -(sx[:, None, None] + sx[None, :, None] + sz[None, None, :])
    lam[0, 0, 0] = 1.0
    return lam


def newton(delta, a, omega_m):
    """Lap Phi = (3/2) Omega_m a^-1 delta with the 7-point Green's function."""
    n = delta.shape[0]
    spec = torch.fft.rfftn(delta) * torch.from_numpy(1.5 * omega_m / a / _lap_eigs(n))
    spec = spec * torch.from_numpy(_zero_mode_mask(n))
    return torch.fft.irfftn(spec, s=(n, n, n))


def _zero_mode_mask(n):
    msk = np.ones((n, n, n // 2 + 1))
    msk[0, 0, 0] = 0.0
    return msk


def force(Phi, x):
    """-grad Phi (central differences) interpolated to x with CIC weights."""
    n = Phi.shape[0]
    g = [-(torch.roll(Phi, -1, d) - torch.roll(Phi, 1, d)).reshape(-1) / 2.0 for d in range(3)]
    i0, i1, w0, w1 = _cic(x, n)
    I = (i0, i1)
    W = (w0, w1)
    F = torch.zeros_like(x)
    for a, b, c in _corners():
        idx = (I[a][:, 0] * n + I[b][:, 1]) * n + I[c][:, 2]
        w = W[a][:, 0] * W[b][:, 1] * W[c][:, 2]
        F = F + w[:, None] * torch.stack([g[d][idx] for d in range(3)], dim=1)
    return F


def power_spectrum(delta, box, nbins):
    """Binned P(k) = <|delta_k|^2> V / n^6 over the modes with
    1 <= |m| <= n/2 (m the integer wavevector), nbins linear bins in |m|;
    bin b = floor((|m| - 1) * nbins / (n/2 - 1)), |m| = n/2 in the last bin.
    Modes 0 < m_z < n/2 of the half spectrum count twice."""
    n = delta.shape[0]
    b, wt = pk_bins(n, nbins)
    dk = torch.fft.rfftn(delta)
    p = (dk.real ** 2 + dk.imag ** 2) * (box ** 3 / float(n) ** 6)
    sel = b >= 0
    bt = torch.from_numpy(b[sel])
    num = torch.zeros(nbins, dtype=torch.float64).index_add(0, bt, (p * torch.from_numpy(wt))[torch.from_numpy(sel)])
    cnt = np.zeros(nbins)
    np.add.at(cnt, b[sel], wt[sel])
    den = torch.from_numpy(np.where(cnt > 0, cnt, 1.0))
    return num / den, cnt


def pk_bins(n, nbins):
    m, mz = _freq(n)
    m2 = (m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2)
    kmag = np.sqrt(m2)
    half = n // 2
    b = np.floor(((kmag - 1.0) * nbins) / (half - 1)).astype(np.int64)
    b = np.where(kmag == half, nbins - 1, b)
    b = np.where((kmag < 1.0) | (kmag > half), -1, b)
    wt = np.where((mz[None, None, :] > 0) & (mz[None, None, :] < half), 2.0, 1.0) * np.ones_like(m2)
    return b, wt


# ---------------------------------------------------------------------------
# the nDGP solve with its implicit-function backward
# ---------------------------------------------------------------------------

def _shift(n, di, dj, dk):
    """Sparse S with (S u)[i, j, k] = u[i + di, j + dj, k + dk] (periodic)."""
    N = n ** 3
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    rows = ((i * n + j) * n + k).ravel()
    cols = ((((i + di) % n) * n + (j + dj) % n) * n + (k + dk) % n).ravel()
    return sp.csr_matrix((np.ones(N), (rows, cols)), shape=(N, N))


def dgp_linear_terms(n):
    """The six linear differences t of Q with their weights (h = 1):
    Sx - Sy, Sx - Sz, Sy - Sz (1/3) and Cxy, Cxz, Cyz (1/8)."""
    S = lambda a, b, c: _shift(n, a, b, c)
    Sx, Sy, Sz = S(1, 0, 0) + S(-1, 0, 0), S(0, 1, 0) + S(0, -1, 0), S(0, 0, 1) + S(0, 0, -1)
    Cxy = S(1, 1, 0) + S(-1, -1, 0) - S(1, -1, 0) - S(-1, 1, 0)
    Cxz = S(1, 0, 1) + S(-1, 0, -1) - S(1, 0, -1) - S(-1, 0, 1)
    Cyz = S(0, 1, 1) + S(0, -1, -1) - S(0, 1, -1) - S(0, -1, 1)
    lap = Sx + Sy + Sz - 6.0 * sp.identity(n ** 3, format="csr")
    return lap, [(Sx - Sy, 1.0 / 3.0), (Sx - Sz, 1.0 / 3.0), (Sy - Sz, 1.0 / 3.0),
                 (Cxy, 1.0 / 8.0), (Cxz, 1.0 / 8.0), (Cyz, 1.0 / 8.0)]


def dgp_jacobian_parts(phi, delta, a, omega_m, rc_h0):
    """(A, Np, ks) with F(phi + v) - F(phi) = A v + <Np dQ v> + O(v^2):
    A = Lap - diag(Np) dQ (sparse; dQ = sum_t 2 w_t diag(t phi) t),
    Np = dN/dSigma = 1 / sqrt(alpha^2 + 8 Sigma / 3) (0 where clamped), and
    ks = dSigma/d(delta - <delta>) = (alpha / beta) Omega_m / a.  The full
    Jacobian is J = A + 1 (Np . dQ) / n^3, i.e. J v = Lap v - Pi(Np dQ v)."""
    n = phi.shape[0]
    lap, terms = dgp_linear_terms(n)
    u = phi.ravel()
    s0, _, alpha, beta = dgp_source(delta, a, omega_m, rc_h0)
    Q = sum(w * (t @ u) ** 2 for t, w in terms)
    arg = alpha * alpha + 8.0 * (Q + s0.ravel()) / 3.0
    Np = np.where(arg > 0, 1.0 / np.sqrt(np.maximum(arg, 1e-300)), 0.0)
    dQ = sum(sp.diags(2.0 * w * (t @ u)) @ t for t, w in terms)
    A = lap - sp.diags(Np) @ dQ
    return A.tocsr(), dQ.tocsr(), Np, (alpha / beta) * omega_m / a


def dgp_jacobian_apply(phi, delta, a, omega_m, rc_h0, v):
    """J v of the residual map (for pinning against finite differences)."""
    A, dQ, Np, _ = dgp_jacobian_parts(phi, delta, a, omega_m, rc_h0)
    t = Np * (dQ @ v.ravel())
    return (A @ v.ravel() + t.mean()).reshape(phi.shape)


def dgp_adjoint(phi, delta, a, omega_m, rc_h0, g, rc_step=1e-6):
    """(dL/ddelta, dL/dR_c) for L with dL/dphi = g at the solution phi."""
    n = phi.shape[0]
    N = n ** 3
    A, dQ, Np, ks = dgp_jacobian_parts(phi, delta, a, omega_m, rc_h0)
    gp = g.ravel() - g.mean()
    # for zero-mean lambda, J^T lambda = A^T lambda; pin the mean by a border
    one = np.ones((N, 1))
    K = sp.bmat([[A.T, sp.csr_matrix(one)], [sp.csr_matrix(one.T), sp.csr_matrix((1, 1))]], format="csc")
    sol = spla.spsolve(K, np.concatenate([gp, [0.0]]))
    lam = sol[:N]
    t = Np * lam
    dd = ks * (t - t.mean())

    def F(rc):
        s0, _, alpha, _ = dgp_source(delta, a, omega_m, rc)
        return residual(dgp_op(alpha), phi, s0, None, 1.0)[0].ravel()

    h = rc_step * rc_h0
    dFdr = (F(rc_h0 + h) - F(rc_h0 - h)) / (2.0 * h)
    return dd.reshape(phi.shape), float(-(lam @ dFdr))


class _DGPSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, delta, rc, a, omega_m, opts):
        d = delta.detach().numpy()
        phi, _ = dgp_solve(d, a, omega_m, float(rc.detach()), opts)
        ctx.a, ctx.om = a, omega_m
        ctx.save_for_backward(delta.detach(), rc.detach(), torch.from_numpy(phi))
        return torch.from_numpy(phi)

    @staticmethod
    def backward(ctx, gphi):
        delta, rc, phi = ctx.saved_tensors
        dd, dr = dgp_adjoint(phi.numpy(), delta.numpy(), ctx.a, ctx.om, float(rc), gphi.numpy())
        return torch.from_numpy(dd), torch.tensor(dr, dtype=torch.float64), None, None, None


def dgp_field(delta, rc, a, omega_m, opts: Opts):
    return _DGPSolve.apply(delta, rc, a, omega_m, opts)


# ---------------------------------------------------------------------------
# the whole chain
# ---------------------------------------------------------------------------

def forward(w, rc, amp, cfg: DpmConfig, opts: Opts = None, keep=None):
    """Final CIC density of the T-step run from white noise w (tensor);
    rc a 0-d tensor.  keep (a list) receives (x_t, p_t) before each step."""
    x, p = zeldovich(w, amp, cfg)
    x, p = run_steps(x, p, rc, cfg, 0, cfg.nsteps, opts, keep)
    return cic_density(x, cfg.ng), x, p


def run_steps(x, p, rc, cfg: DpmConfig, t0, t1, opts: Opts = None, keep=None):
    """Steps t0 .. t1-1 of the leapfrog (positions at a_t, momenta at
    a_t - da/2, or at a_start before the first half kick)."""
    opts = opts or Opts(rtol=1e-12, max_cycles=60)
    n = cfg.ng
    da = (cfg.a_end - cfg.a_start) / cfg.nsteps
    for t in range(t0, t1):
        if keep is not None:
            keep.append((x.detach().clone(), p.detach().clone()))
        a = cfg.a_start + t * da
        delta = cic_density(x, n)
        Phi = newton(delta, a, cfg.omega_m)
        if cfg.model == 1:
            Phi = Phi + 0.5 * dgp_field(delta, rc, a, cfg.omega_m, opts)
        kick = (0.5 * da if t == 0 else da) / (a * E_lcdm(a, cfg.omega_m))
        p = p + kick * force(Phi, x)
        am = a + 0.5 * da
        x = torch.remainder(x + (da / (am ** 3 * E_lcdm(am, cfg.omega_m))) * p, float(n))
    return x, p


def loss(w, rc, amp, cfg: DpmConfig, target, opts: Opts = None):
    """(L, P) with L = mean_b (P_b - target_b)^2."""
    delta, _, _ = forward(w, rc, amp, cfg, opts)
    pk, _ = power_spectrum(delta, cfg.box, cfg.nbins)
    return ((pk - torch.as_tensor(target)) ** 2).mean(), pk


def gradient(w, rc_h0, amp, cfg: DpmConfig, target, opts: Opts = None):
    """(L, dL/dw, dL/dR_c, P) in FP64."""
    wt = torch.tensor(np.asarray(w, dtype=np.float64), requires_grad=True)
    rt = torch.tensor(float(rc_h0), dtype=torch.float64, requires_grad=True)
    L, pk = loss(wt, rt, amp, cfg, target, opts)
    L.backward()
    rg = 0.0 if rt.grad is None else float(rt.grad)
    return float(L.detach()), wt.grad.numpy().copy(), rg, pk.detach().numpy()
