"""Seeded synthetic inputs for the solver and particle-mesh workloads.

This module only makes inputs: random numbers, Gaussian random fields,
Zel'dovich particle loads and simple analytic density patterns.  It contains
none of the solver's arithmetic (no operator, smoother, deposit, Poisson
solve or time step), so both the CUDA path and the CPU oracle can be fed from
it without sharing any of the method.

Random numbers: SplitMix64 (Steele, Lea & Flood 2014) used as a
counter-based generator -- the q-th draw of stream ``seed`` is
mix64(seed * 0x9E3779B97F4A7C15 + (q + 1) * 0x9E3779B97F4A7C15) -- then
Box-Muller in FP64 for normal deviates.  White noise is drawn in real space
in C order (i, j, k), k fastest.

Units: Mpc/h for lengths and h/Mpc for wavenumbers inside this module;
particle positions are returned in mesh code units (Sec. 3.1.1 of
arXiv:2110.00566: x~ = (N_g / L) x), as float32 in [0, N_g).
"""
from __future__ import annotations

import numpy as np

_trapz = getattr(np, "trapezoid", None) or getattr(np, "trapz")

_GOLD = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of SplitMix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLD
        q = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = base + q * _GOLD
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform deviates in (0, 1]: ((x >> 11) + 1) * 2^-53."""
    x = splitmix64(seed, count, offset)
    return ((x >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal deviates by Box-Muller from consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def white_noise(n: int, seed: int) -> np.ndarray:
    return normal(seed, n ** 3).reshape(n, n, n)


# ---------------------------------------------------------------------------
# power spectra and LCDM growth (used only to shape the initial field)
# ---------------------------------------------------------------------------

def tophat_window(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x > 1e-6
    xs = x[nz]
    out[nz] = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs ** 3
    return out


def sigma_R(pk, R=8.0):
    """sigma(R) of a spectrum with a top-hat window (numerical quadrature)."""
    lk = np.linspace(np.log(1e-5), np.log(1e3), 20001)
    k = np.exp(lk)
    integrand = pk(k) * tophat_window(k * R) ** 2 * k ** 3 / (2.0 * np.pi ** 2)
    return float(np.sqrt(_trapz(integrand, lk)))


def pk_cutoff(ns=0.96, kc=5.0, sigma8=0.8):
    """P(k) = A k^ns exp(-k/kc), A fixed by sigma_8 at z = 0."""
    shape = lambda k: np.power(k, ns) * np.exp(-k / kc)
    amp = (sigma8 / sigma_R(shape)) ** 2
    return lambda k: amp * shape(k)


def growth_lcdm(a, omega_m):
    """LCDM linear growth D(a), D(1) = 1: D ~ E(a) int_0^a da'/(a' E(a'))^3."""
    def raw(aa):
        x = np.linspace(1e-8, aa, 200001)
        E = np.sqrt(omega_m * x ** -3 + 1.0 - omega_m)
        return np.sqrt(omega_m * aa ** -3 + 1.0 - omega_m) * _trapz(1.0 / (x * E) ** 3, x)
    return raw(a) / raw(1.0)


def growth_rate_lcdm(a, omega_m, eps=1e-4):
    """f = dln D / dln a by central differences of growth_lcdm."""
    lo, hi = a * np.exp(-eps), a * np.exp(eps)
    return (np.log(growth_lcdm(hi, omega_m)) - np.log(growth_lcdm(lo, omega_m))) / (2 * eps)


# ---------------------------------------------------------------------------
# Gaussian fields and Zel'dovich loads
# ---------------------------------------------------------------------------

def _kgrid(n, box):
    k = 2.0 * np.pi * np.fft.fftfreq(n, d=box / n)
    kz = 2.0 * np.pi * np.fft.rfftfreq(n, d=box / n)
    return k[:, None, None], k[None, :, None], kz[None, None, :]


def pk_amplitude(n, box, pk):
    """sqrt(P(|k|) / V_cell) on the rfftn grid (n, n, n/2 + 1) of an n^3
    lattice of side box, zero at k = 0: the factor that turns the FFT of
    unit white noise into a field with spectrum pk."""
    kx, ky, kz = _kgrid(n, box)
    kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    kk[0, 0, 0] = 1.0
    amp = np.sqrt(pk(kk) / (box / n) ** 3)
    amp[0, 0, 0] = 0.0
    return np.ascontiguousarray(amp)


def linear_field_k(n, box, pk, seed, noise=None):
    """Fourier modes (numpy rfftn convention) of a Gaussian field with
    spectrum pk on an n^3 lattice of side box: FFT(white noise) *
    sqrt(P(k) / V_cell); the k = 0 mode is zero."""
    w = white_noise(n, seed) if noise is None else np.asarray(noise, dtype=np.float64)
    return np.fft.rfftn(w) * pk_amplitude(n, box, pk)


def linear_field(n, box, pk, seed):
    return np.fft.irfftn(linear_field_k(n, box, pk, seed), s=(n, n, n), axes=(0, 1, 2))


def zeldovich(np_side, ng, box, pk, growth, seed, noise=None, vel_factor=0.0):
    """Particles on a lattice displaced by growth * psi with div psi = -delta
    (Zel'dovich approximation).  Lattice points sit at (q + 1/2) ng/np_side
    in mesh units, so an undisplaced load deposits a uniform density.
    Returns float32 positions (np_side^3, 3) in [0, ng) and float32 momenta
    vel_factor * psi (mesh units), where vel_factor = a^2 E(a) D(a) f(a)
    gives the code-unit momentum p~ of the growing mode."""
    dk = linear_field_k(np_side, box, pk, seed, noise)
    kx, ky, kz = _kgrid(np_side, box)
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k2[0, 0, 0] = 1.0
    nyq = np.pi * np_side / box
    cell = box / ng
    disp = []
    for kc in (kx, ky, kz):
        kc = np.where(np.isclose(np.abs(kc), nyq), 0.0, kc)
        psi = np.fft.irfftn(1j * kc / k2 * dk, s=(np_side,) * 3, axes=(0, 1, 2))
        disp.append(psi / cell)          # Mpc/h -> mesh cells
    q = (np.arange(np_side) + 0.5) * (ng / np_side)
    qx, qy, qz = np.meshgrid(q, q, q, indexing="ij")
    pos = np.stack([qx + growth * disp[0], qy + growth * disp[1], qz + growth * disp[2]], axis=-1)
    pos = np.mod(pos, ng).reshape(-1, 3)
    pos32 = pos.astype(np.float32)
    pos32[pos32 >= ng] -= np.float32(ng)
    mom = (vel_factor * np.stack(disp, axis=-1)).reshape(-1, 3).astype(np.float32)
    return np.ascontiguousarray(pos32), np.ascontiguousarray(mom)


def powerlaw_particles(np_side, ng, box, seed, index=-2.0, rms=1.0):
    """Config-1 style load: a power-law spectrum P ~ k^index from the
    fundamental mode to Nyquist, scaled so that the realised linear density
    on the particle lattice has the given rms, then Zel'dovich-displaced."""
    kf, kn = 2 * np.pi / box, np.pi * np_side / box
    shape = lambda k: np.where((k >= kf * 0.999) & (k <= kn * np.sqrt(3.0)), np.power(k, index), 0.0)
    d = np.fft.irfftn(linear_field_k(np_side, box, shape, seed), s=(np_side,) * 3, axes=(0, 1, 2))
    scale = rms / float(np.sqrt(np.mean(d ** 2)))
    pk = lambda k: shape(k) * scale ** 2
    return zeldovich(np_side, ng, box, pk, 1.0, seed)


# ---------------------------------------------------------------------------
# analytic patterns for the paper's code tests (Sec. 4.2)
# ---------------------------------------------------------------------------

def cell_centres(n):
    return np.arange(n) + 0.5


def sine_pattern(n, waves=1, axis=0):
    """sin(2 pi K x / n) at cell centres, varying along one axis."""
    x = cell_centres(n)
    s = np.sin(2.0 * np.pi * waves * x / n)
    shape = [1, 1, 1]
    shape[axis] = n
    return np.broadcast_to(s.reshape(shape), (n, n, n)).copy()


def tophat_sphere(n, radius, value, centre=None):
    """value inside a sphere of the given radius (mesh units) around the mesh
    centre (a cell corner, Sec. 4.2.3), zero outside."""
    c = n / 2.0 if centre is None else centre
    x = cell_centres(n) - c
    r2 = x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
    return np.where(r2 <= radius ** 2, float(value), 0.0)


def uniform_guess(n, seed, half_width=0.05):
    """Initial guess uniform in [-half_width, half_width] (Sec. 4.2.1)."""
    return (uniform01(seed, n ** 3) * 2.0 - 1.0).reshape(n, n, n) * half_width
