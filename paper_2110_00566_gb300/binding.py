"""Thin ctypes binding of libmgglam.so (include/mgglam.h).

Argument marshalling only: every step of the solvers runs in the CUDA
library.  Functions carry the C names and accept torch tensors (CUDA or
CPU) or numpy arrays for the array arguments; CPU arrays are staged by the
library itself.  The library is loaded on first use; if it is missing or
cannot be loaded, an ImportError is raised -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmgglam.so")

MG_OK = 0
MG_WARN_NOT_CONVERGED = 1
MG_ERR_ARG = -1
MG_ERR_CUDA = -2
MG_ERR_TIMEOUT = -3
MG_ERR_NONFINITE = -4
MG_ERR_OOM = -5
MG_CYCLE_V, MG_CYCLE_F, MG_CYCLE_W = 0, 1, 2
MG_PREC_FP64, MG_PREC_MIXED = 0, 1


class mg_grid(C.Structure):
    _fields_ = [("ng", C.c_int), ("box_mpch", C.c_double), ("a", C.c_double), ("omega_m", C.c_double)]


class mg_dgp_params(C.Structure):
    _fields_ = [("rc_h0", C.c_double)]


class mg_kmo_params(C.Structure):
    _fields_ = [("n", C.c_int), ("k0", C.c_double), ("beta_kmo", C.c_double), ("lambda_", C.c_double),
                ("phibar_prime_over_h0", C.c_double), ("A_bar", C.c_double)]


class mg_opts(C.Structure):
    _fields_ = [("pre", C.c_int), ("post", C.c_int), ("max_cycles", C.c_int), ("cycle", C.c_int),
                ("precision", C.c_int), ("rtol", C.c_double), ("atol", C.c_double),
                ("warm_start", C.c_int), ("coarse_sweeps", C.c_int), ("use_graph", C.c_int),
                ("inner_cycles", C.c_int)]


class mg_stats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("status", C.c_int), ("eps_ref", C.c_double),
                ("eps", C.c_double * 65), ("n_eps", C.c_int), ("c_final", C.c_double),
                ("mean_shift", C.c_double), ("sqrt_clamps", C.c_longlong), ("ms", C.c_double),
                ("cell_updates", C.c_longlong), ("kernel_launches", C.c_longlong),
                ("fine_smooth_ms", C.c_double), ("fine_smooth_launches", C.c_longlong)]

    def eps_list(self):
        return list(self.eps[: self.n_eps])


class mg_instance(C.Structure):
    _fields_ = [("g", mg_grid), ("p", mg_dgp_params), ("delta", C.c_void_p), ("phi", C.c_void_p)]


class pm_state(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("mom", C.c_void_p), ("np", C.c_longlong), ("ng", C.c_int),
                ("box_mpch", C.c_double), ("omega_m", C.c_double), ("a", C.c_double), ("da", C.c_double),
                ("model", C.c_int), ("first", C.c_int), ("dgp", mg_dgp_params), ("phi_ws", C.c_void_p),
                ("kmo", mg_kmo_params), ("dphibar_da", C.c_double), ("e_a", C.c_double),
                ("e_mid", C.c_double)]


class mg_kmo_background_params(C.Structure):
    _fields_ = [("n", C.c_int), ("k0", C.c_double), ("beta_kmo", C.c_double), ("omega_m", C.c_double),
                ("h", C.c_double), ("t_cmb", C.c_double), ("n_eff", C.c_double), ("a_ini", C.c_double),
                ("phi_ini", C.c_double), ("dphi_ini", C.c_double), ("rtol", C.c_double), ("h0_tol", C.c_double)]


class dpm_config(C.Structure):
    _fields_ = [("ng", C.c_int), ("box_mpch", C.c_double), ("omega_m", C.c_double), ("a_start", C.c_double),
                ("a_end", C.c_double), ("nsteps", C.c_int), ("checkpoint_every", C.c_int), ("nbins", C.c_int),
                ("model", C.c_int), ("growth", C.c_double), ("vel", C.c_double)]


class mg_op_params(C.Structure):
    _fields_ = [("model", C.c_int), ("alpha", C.c_double), ("nkmo", C.c_int), ("gamma", C.c_double),
                ("bterm", C.c_double)]


_lib = None
_VP = C.c_void_p
_P = C.POINTER


def _declare(L):
    sig = {
        "mg_ctx_create": (C.c_int, [_P(C.c_void_p), C.c_int, _VP]),
        "mg_ctx_destroy": (None, [_VP]),
        "mg_last_error_string": (C.c_char_p, [_VP]),
        "mg_ctx_workspace_bytes": (C.c_longlong, [_VP]),
        "mg_ctx_set_profiling": (C.c_int, [_VP, C.c_int]),
        "mg_ctx_set_fp32_smoother": (C.c_int, [_VP, C.c_int]),
        "mg_ctx_set_fp32_smoother_shape": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int]),
        "mg_fp32_smoother_variants": (C.c_int, []),
        "mg_probe_alu_peaks": (C.c_int, [_VP, _P(C.c_double), _P(C.c_double)]),
        "mg_probe_fp64_math": (C.c_int, [_VP, C.c_int, _VP, _VP, C.c_longlong, C.c_double]),
        "mg_opts_default": (None, [_P(mg_opts)]),
        "mg_solve_dgp": (C.c_int, [_VP, C.c_int, _P(mg_instance), _P(mg_opts), _P(mg_stats)]),
        "mg_solve_kmouflage": (C.c_int, [_VP, _P(mg_grid), _P(mg_kmo_params), _P(mg_opts), _VP, _VP,
                                         _P(mg_stats)]),
        "mg_solve_kmouflage_linear": (C.c_int, [_VP, _P(mg_grid), _P(mg_kmo_params), _VP, _VP]),
        "pm_cic_deposit": (C.c_int, [_VP, C.c_int, _VP, C.c_longlong, _VP]),
        "pm_cic_index": (C.c_int, [_VP, C.c_int, _VP, C.c_longlong, _VP]),
        "pm_cic_deposit_noalloc": (C.c_int, [C.c_int, _VP, C.c_longlong, _VP, _VP]),
        "pm_step": (C.c_int, [_VP, _P(pm_state), _P(mg_opts), _P(mg_stats)]),
        "mg_kmo_background_defaults": (C.c_int, [_P(mg_kmo_background_params)]),
        "mg_kmo_background": (C.c_int, [_P(mg_kmo_background_params), C.c_double, C.c_int, _VP, _VP,
                                        _P(C.c_double)]),
        "pm_newton_potential": (C.c_int, [_VP, C.c_int, C.c_double, C.c_double, _VP, _VP]),
        "mg_solve_adjoint": (C.c_int, [_VP, _P(mg_grid), _P(mg_dgp_params), _P(mg_opts), _VP, _VP, _VP, _VP,
                                       _VP, _P(mg_stats)]),
        "dpm_run": (C.c_int, [_VP, _P(dpm_config), _P(mg_opts), _VP, _VP, C.c_double, _VP, _VP, _VP, _VP, _VP,
                              _P(mg_stats)]),
        "dpm_run_vjp": (C.c_int, [_VP, _P(dpm_config), _P(mg_opts), _VP, _VP, C.c_double, _VP, _VP, _VP, _VP,
                                  _P(mg_stats)]),
        "dpm_ic": (C.c_int, [_VP, _P(dpm_config), _VP, _VP, _VP, _VP]),
        "dpm_ic_adjoint": (C.c_int, [_VP, _P(dpm_config), _VP, _VP, _VP, _VP]),
        "dpm_deposit": (C.c_int, [_VP, C.c_int, _VP, C.c_longlong, _VP]),
        "dpm_deposit_adjoint": (C.c_int, [_VP, C.c_int, _VP, C.c_longlong, _VP, _VP]),
        "dpm_force": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP, C.c_longlong, _VP]),
        "dpm_force_adjoint": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP, C.c_longlong, _VP, _VP, _VP]),
        "dpm_power_spectrum": (C.c_int, [_VP, C.c_int, C.c_double, C.c_int, _VP, _VP, _VP]),
        "dpm_power_spectrum_adjoint": (C.c_int, [_VP, C.c_int, C.c_double, C.c_int, _VP, _VP, _VP]),
        "mg_op_smooth": (C.c_int, [_VP, _P(mg_op_params), C.c_int, C.c_int, C.c_double, _VP, _VP, _VP,
                                   C.c_double, C.c_int, _VP]),
        "mg_op_smooth_corr": (C.c_int, [_VP, _P(mg_op_params), C.c_int, C.c_double, _VP, _VP, _VP, _VP,
                                        C.c_double, C.c_int, _VP]),
        "mg_op_resid_restrict": (C.c_int, [_VP, _P(mg_op_params), C.c_int, C.c_int, C.c_double, _VP, _VP, _VP,
                                           _VP, _VP, _P(C.c_double), _P(C.c_double)]),
        "mg_op_coarse_source": (C.c_int, [_VP, _P(mg_op_params), C.c_int, C.c_int, C.c_double, _VP, _VP, _VP,
                                          _VP, _P(C.c_double)]),
        "mg_op_prolong_add": (C.c_int, [_VP, C.c_int, C.c_int, _VP, _VP, _VP]),
        "mg_op_coarsest": (C.c_int, [_VP, _P(mg_op_params), C.c_int, C.c_double, _VP, _VP, _VP, C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return sorted(sig)


DECLARED = None


def lib():
    """The loaded library (raises ImportError if it is not built)."""
    global _lib, DECLARED
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libmgglam.so is not built (run __graft_entry__.build()); there is no CPU fallback")
        _lib = C.CDLL(LIB_PATH)
        DECLARED = _declare(_lib)
    return _lib


class MGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("mgglam error %d: %s" % (code, msg))
        self.code = code


def _ptr(x):
    """Raw data pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("array arguments must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array arguments must be C-contiguous")
        return x.ctypes.data
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(x))


def _check_dtype(x, kind):
    if x is None:
        return
    name = str(getattr(x, "dtype", ""))
    want = {"f64": ("float64", "torch.float64"), "f32": ("float32", "torch.float32"),
            "i32": ("int32", "torch.int32")}[kind]
    if name not in want:
        raise TypeError("expected %s array, got %s" % (kind, name))


def opts(**kw) -> mg_opts:
    o = mg_opts()
    lib().mg_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Context:
    """An mg_ctx on one device; `stream` is a torch.cuda.Stream, a raw
    cudaStream_t integer or None."""

    def __init__(self, device: int = 0, stream=None):
        raw = getattr(stream, "cuda_stream", stream)
        h = C.c_void_p()
        rc = lib().mg_ctx_create(C.byref(h), int(device), raw)
        if rc != 0:
            raise MGError(rc, "mg_ctx_create failed (device %d)" % device)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().mg_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return lib().mg_last_error_string(self.h).decode()

    def workspace_bytes(self) -> int:
        return lib().mg_ctx_workspace_bytes(self.h)

    def set_profiling(self, on: bool):
        return self._rc(lib().mg_ctx_set_profiling(self.h, int(bool(on))))

    def set_fp32_smoother(self, choice: int):
        """-1 gathering kernel, 0 autotuned, k >= 1 streaming variant k."""
        return self._rc(lib().mg_ctx_set_fp32_smoother(self.h, int(choice)))

    def set_fp32_smoother_shape(self, n: int, bx: int, zc: int = 1):
        """Pin the gathering FP32 half-sweep's shape on n^3 levels (bx = 0: unpin)."""
        return self._rc(lib().mg_ctx_set_fp32_smoother_shape(self.h, int(n), int(bx), int(zc)))

    def probe_alu_peaks(self):
        """(FP64, FP32) FMA throughput in TFLOP/s measured on this device."""
        a, b = C.c_double(), C.c_double()
        self._rc(lib().mg_probe_alu_peaks(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def probe_fp64_math(self, fn: int, x, y, alpha: float = 1.0):
        """y = f(x) on device float64 tensors with the FP64 kernels' own
        arithmetic: fn 0 square root, 1 reciprocal, 2 nDGP N(Sigma = x)."""
        assert x.is_cuda and y.is_cuda and x.dtype == y.dtype and x.numel() == y.numel()
        self._rc(lib().mg_probe_fp64_math(self.h, int(fn), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                           x.numel(), float(alpha)))

    def _rc(self, rc, allow_warn=True):
        if rc < 0 or (rc > 0 and not allow_warn):
            raise MGError(rc, self.last_error())
        return rc


def mg_ctx_create(device=0, stream=None) -> Context:
    return Context(device, stream)


def mg_ctx_destroy(ctx: Context):
    ctx.close()


def mg_solve_dgp(ctx: Context, instances, o: mg_opts = None):
    """instances: list of dicts {ng, box_mpch, a, omega_m, rc_h0, delta, phi}.
    Returns (rc, [mg_stats])."""
    n = len(instances)
    arr = (mg_instance * n)()
    for q, d in enumerate(instances):
        _check_dtype(d["delta"], "f64")
        _check_dtype(d["phi"], "f64")
        arr[q].g = mg_grid(int(d["ng"]), float(d.get("box_mpch", d["ng"])), float(d["a"]), float(d["omega_m"]))
        arr[q].p = mg_dgp_params(float(d["rc_h0"]))
        arr[q].delta = _ptr(d["delta"])
        arr[q].phi = _ptr(d["phi"])
    st = (mg_stats * n)()
    rc = lib().mg_solve_dgp(ctx.h, n, arr, C.byref(o or opts()), st)
    ctx._rc(rc)
    return rc, list(st)


def mg_solve_kmouflage(ctx: Context, ng, box_mpch, a, omega_m, n, k0, beta_kmo, lam, phibar_prime_over_h0, A_bar,
                       delta, phi, o: mg_opts = None):
    _check_dtype(delta, "f64")
    _check_dtype(phi, "f64")
    g = mg_grid(int(ng), float(box_mpch), float(a), float(omega_m))
    p = mg_kmo_params(int(n), float(k0), float(beta_kmo), float(lam), float(phibar_prime_over_h0), float(A_bar))
    st = mg_stats()
    rc = lib().mg_solve_kmouflage(ctx.h, C.byref(g), C.byref(p), C.byref(o or opts()), _ptr(delta), _ptr(phi),
                                  C.byref(st))
    ctx._rc(rc)
    return rc, st


def mg_solve_kmouflage_linear(ctx: Context, ng, box_mpch, a, omega_m, n, k0, beta_kmo, lam, phibar_prime_over_h0,
                              A_bar, delta, phi):
    _check_dtype(delta, "f64")
    _check_dtype(phi, "f64")
    g = mg_grid(int(ng), float(box_mpch), float(a), float(omega_m))
    p = mg_kmo_params(int(n), float(k0), float(beta_kmo), float(lam), float(phibar_prime_over_h0), float(A_bar))
    ctx._rc(lib().mg_solve_kmouflage_linear(ctx.h, C.byref(g), C.byref(p), _ptr(delta), _ptr(phi)))


def pm_cic_deposit(ctx: Context, ng, pos, delta_out):
    _check_dtype(pos, "f32")
    _check_dtype(delta_out, "f64")
    npart = int(pos.shape[0])
    return ctx._rc(lib().pm_cic_deposit(ctx.h, int(ng), _ptr(pos), npart, _ptr(delta_out)))


def pm_cic_index(ctx: Context, ng, pos, idx_out):
    _check_dtype(pos, "f32")
    _check_dtype(idx_out, "i32")
    return ctx._rc(lib().pm_cic_index(ctx.h, int(ng), _ptr(pos), int(pos.shape[0]), _ptr(idx_out)))


def pm_newton_potential(ctx: Context, ng, a, omega_m, delta, phi_out):
    _check_dtype(delta, "f64")
    _check_dtype(phi_out, "f64")
    return ctx._rc(lib().pm_newton_potential(ctx.h, int(ng), float(a), float(omega_m), _ptr(delta),
                                             _ptr(phi_out)))


def make_pm_state(pos, mom, ng, box_mpch, omega_m, a, da, model=1, rc_h0=1.0, first=True, phi_ws=None, kmo=None,
                  hubble=None):
    """A pm_state over caller arrays (kept alive by the caller).  kmo (model
    2): dict(n, k0, beta, lam, phibar_prime_over_h0, A_bar, dphibar_da).
    hubble: (H/H0 at a, H/H0 at a + da/2), or None for LCDM's."""
    _check_dtype(pos, "f32")
    _check_dtype(mom, "f32")
    _check_dtype(phi_ws, "f64")
    k = kmo or dict(n=2, k0=0.0, beta=0.0, lam=1.0, phibar_prime_over_h0=0.0, A_bar=1.0, dphibar_da=0.0)
    kp = mg_kmo_params(int(k["n"]), float(k["k0"]), float(k["beta"]), float(k["lam"]),
                       float(k["phibar_prime_over_h0"]), float(k["A_bar"]))
    return pm_state(_ptr(pos), _ptr(mom), int(pos.shape[0]), int(ng), float(box_mpch), float(omega_m), float(a),
                    float(da), int(model), int(bool(first)), mg_dgp_params(float(rc_h0)), _ptr(phi_ws), kp,
                    float(k["dphibar_da"]), *(float(e) for e in (hubble or (0.0, 0.0))))


def kmo_background_params(**kw):
    """mg_kmo_background_params with the library defaults, overridden by kw
    (n, k0, beta_kmo, omega_m, h, t_cmb, n_eff, a_ini, phi_ini, dphi_ini,
    rtol, h0_tol)."""
    p = mg_kmo_background_params()
    lib().mg_kmo_background_defaults(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError("unknown background parameter %r" % k)
        setattr(p, k, v)
    return p


def fp32_smoother_variants() -> int:
    return int(lib().mg_fp32_smoother_variants())


def mg_kmo_background(p: mg_kmo_background_params, a, lam=0.0):
    """Kmouflage background at the scale factors a (host code in the
    library): returns (rc, lambda, table (len(a), 5) of [H/H0, phibar,
    dphibar/da, A(phibar), phibar'/H0]).  lam > 0 skips the shooting."""
    a = np.ascontiguousarray(np.atleast_1d(np.asarray(a, dtype=np.float64)))
    out = np.empty((a.size, 5))
    lam_out = C.c_double(0.0)
    rc = lib().mg_kmo_background(C.byref(p), float(lam), int(a.size), a.ctypes.data, out.ctypes.data,
                                 C.byref(lam_out))
    if rc < 0:
        raise MGError(rc, "mg_kmo_background: bad argument" if rc == MG_ERR_ARG else
                      "mg_kmo_background: the Friedmann equation lost its root or the integration failed")
    return rc, lam_out.value, out


def pm_step(ctx: Context, state: pm_state, o: mg_opts = None):
    st = mg_stats()
    rc = lib().pm_step(ctx.h, C.byref(state), C.byref(o or opts()), C.byref(st))
    ctx._rc(rc)
    return rc, st


def mg_solve_adjoint(ctx: Context, ng, box_mpch, a, omega_m, rc_h0, phi, delta, dL_dphi, dL_ddelta_out,
                     o: mg_opts = None):
    g = mg_grid(int(ng), float(box_mpch), float(a), float(omega_m))
    p = mg_dgp_params(float(rc_h0))
    drc = C.c_double(0.0)
    st = mg_stats()
    rc = lib().mg_solve_adjoint(ctx.h, C.byref(g), C.byref(p), C.byref(o or opts()), _ptr(phi), _ptr(delta),
                                _ptr(dL_dphi), _ptr(dL_ddelta_out), C.cast(C.pointer(drc), C.c_void_p),
                                C.byref(st))
    ctx._rc(rc)
    return rc, drc.value, st


# ------------------------------------------------- differentiable PM run

def make_dpm_config(ng, box_mpch, omega_m, a_start, a_end, nsteps, checkpoint_every=4, nbins=32, model=1,
                    growth=1.0, vel=0.0) -> dpm_config:
    return dpm_config(int(ng), float(box_mpch), float(omega_m), float(a_start), float(a_end), int(nsteps),
                      int(checkpoint_every), int(nbins), int(model), float(growth), float(vel))


def _host_f64(x, n):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
    if a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def dpm_run(ctx: Context, cfg: dpm_config, amp, noise, rc_h0, target=None, dnoise_out=None, want_drc=True,
            o: mg_opts = None):
    """Forward run (and the reverse pass when dnoise_out is given).
    Returns (P (nbins,), loss or None, dL/dR_c or None, stats)."""
    _check_dtype(amp, "f64")
    _check_dtype(noise, "f64")
    _check_dtype(dnoise_out, "f64")
    pk = np.zeros(cfg.nbins)
    tgt = None if target is None else _host_f64(target, cfg.nbins)
    loss = C.c_double(0.0)
    drc = C.c_double(0.0)
    st = mg_stats()
    rc = lib().dpm_run(ctx.h, C.byref(cfg), C.byref(o or opts()), _ptr(amp), _ptr(noise), float(rc_h0),
                       None if tgt is None else tgt.ctypes.data, pk.ctypes.data,
                       None if tgt is None else C.cast(C.pointer(loss), C.c_void_p), _ptr(dnoise_out),
                       C.cast(C.pointer(drc), C.c_void_p) if (dnoise_out is not None and want_drc) else None,
                       C.byref(st))
    ctx._rc(rc)
    return (pk, None if tgt is None else loss.value,
            drc.value if (dnoise_out is not None and want_drc) else None, st)


def dpm_run_vjp(ctx: Context, cfg: dpm_config, amp, noise, rc_h0, dpk, dnoise_out, want_drc=True,
                o: mg_opts = None):
    """Forward run and the reverse pass seeded with dL/dP = dpk (nbins).
    Returns (P (nbins,), dL/dR_c or None, stats); dL/dw goes to dnoise_out."""
    _check_dtype(amp, "f64")
    _check_dtype(noise, "f64")
    _check_dtype(dnoise_out, "f64")
    pk = np.zeros(cfg.nbins)
    g = _host_f64(dpk, cfg.nbins)
    drc = C.c_double(0.0)
    st = mg_stats()
    rc = lib().dpm_run_vjp(ctx.h, C.byref(cfg), C.byref(o or opts()), _ptr(amp), _ptr(noise), float(rc_h0),
                           g.ctypes.data, pk.ctypes.data, _ptr(dnoise_out),
                           C.cast(C.pointer(drc), C.c_void_p) if want_drc else None, C.byref(st))
    ctx._rc(rc)
    return pk, (drc.value if want_drc else None), st


def dpm_ic(ctx: Context, cfg: dpm_config, amp, noise, pos_out, mom_out):
    for x in (amp, noise, pos_out, mom_out):
        _check_dtype(x, "f64")
    ctx._rc(lib().dpm_ic(ctx.h, C.byref(cfg), _ptr(amp), _ptr(noise), _ptr(pos_out), _ptr(mom_out)))


def dpm_ic_adjoint(ctx: Context, cfg: dpm_config, amp, dpos, dmom, dnoise_out):
    for x in (amp, dpos, dmom, dnoise_out):
        _check_dtype(x, "f64")
    ctx._rc(lib().dpm_ic_adjoint(ctx.h, C.byref(cfg), _ptr(amp), _ptr(dpos), _ptr(dmom), _ptr(dnoise_out)))


def dpm_deposit(ctx: Context, ng, pos, delta_out):
    _check_dtype(pos, "f64")
    _check_dtype(delta_out, "f64")
    ctx._rc(lib().dpm_deposit(ctx.h, int(ng), _ptr(pos), pos.shape[0], _ptr(delta_out)))


def dpm_deposit_adjoint(ctx: Context, ng, pos, ddelta, dpos_out):
    for x in (pos, ddelta, dpos_out):
        _check_dtype(x, "f64")
    ctx._rc(lib().dpm_deposit_adjoint(ctx.h, int(ng), _ptr(pos), pos.shape[0], _ptr(ddelta), _ptr(dpos_out)))


def dpm_force(ctx: Context, ng, phin, phi, pos, force_out):
    for x in (phin, phi, pos, force_out):
        _check_dtype(x, "f64")
    ctx._rc(lib().dpm_force(ctx.h, int(ng), _ptr(phin), _ptr(phi), _ptr(pos), pos.shape[0], _ptr(force_out)))


def dpm_force_adjoint(ctx: Context, ng, phin, phi, pos, dforce, dpos_out, dphin_out):
    for x in (phin, phi, pos, dforce, dpos_out, dphin_out):
        _check_dtype(x, "f64")
    ctx._rc(lib().dpm_force_adjoint(ctx.h, int(ng), _ptr(phin), _ptr(phi), _ptr(pos), pos.shape[0],
                                    _ptr(dforce), _ptr(dpos_out), _ptr(dphin_out)))


def dpm_power_spectrum(ctx: Context, ng, box_mpch, nbins, delta):
    _check_dtype(delta, "f64")
    pk, cnt = np.zeros(nbins), np.zeros(nbins)
    ctx._rc(lib().dpm_power_spectrum(ctx.h, int(ng), float(box_mpch), int(nbins), _ptr(delta), pk.ctypes.data,
                                     cnt.ctypes.data))
    return pk, cnt


def dpm_power_spectrum_adjoint(ctx: Context, ng, box_mpch, nbins, delta, dpk, ddelta_out):
    _check_dtype(delta, "f64")
    _check_dtype(ddelta_out, "f64")
    d = _host_f64(dpk, nbins)
    ctx._rc(lib().dpm_power_spectrum_adjoint(ctx.h, int(ng), float(box_mpch), int(nbins), _ptr(delta),
                                             d.ctypes.data, _ptr(ddelta_out)))


# ---------------------------------------------------------------- kernel level

def op_params(model=0, alpha=0.0, nkmo=2, gamma=0.0, bterm=0.0):
    return mg_op_params(int(model), float(alpha), int(nkmo), float(gamma), float(bterm))


def mg_op_smooth(ctx, op, precision, n, h, u_in, s, f, c, colour, u_out):
    return ctx._rc(lib().mg_op_smooth(ctx.h, C.byref(op), precision, n, h, _ptr(u_in), _ptr(s), _ptr(f), c,
                                      colour, _ptr(u_out)))


def mg_op_smooth_corr(ctx, op, n, h, e_in, base, s, f, c, colour, e_out):
    return ctx._rc(lib().mg_op_smooth_corr(ctx.h, C.byref(op), n, h, _ptr(e_in), _ptr(base), _ptr(s), _ptr(f), c,
                                           colour, _ptr(e_out)))


def mg_op_resid_restrict(ctx, op, precision, n, h, u, s, f, Ru, Rd):
    c = C.c_double()
    e = C.c_double()
    ctx._rc(lib().mg_op_resid_restrict(ctx.h, C.byref(op), precision, n, h, _ptr(u), _ptr(s), _ptr(f), _ptr(Ru),
                                       _ptr(Rd), C.byref(c), C.byref(e)))
    return c.value, e.value


def mg_op_coarse_source(ctx, op, precision, n, h, Ru, Rd, s, f_out):
    c = C.c_double()
    ctx._rc(lib().mg_op_coarse_source(ctx.h, C.byref(op), precision, n, h, _ptr(Ru), _ptr(Rd), _ptr(s),
                                      _ptr(f_out), C.byref(c)))
    return c.value


def mg_op_prolong_add(ctx, precision, n, u_fine, uc, urc):
    return ctx._rc(lib().mg_op_prolong_add(ctx.h, precision, n, _ptr(u_fine), _ptr(uc), _ptr(urc)))


def mg_op_coarsest(ctx, op, n, h, u, s, f, sweeps):
    return ctx._rc(lib().mg_op_coarsest(ctx.h, C.byref(op), n, h, _ptr(u), _ptr(s), _ptr(f), sweeps))


# ---------------------------------------------------------------- autograd

def autograd_solve():
    """torch.autograd.Function over the nDGP solve: forward calls
    mg_solve_dgp, backward calls mg_solve_adjoint (gradients with respect to
    delta and to the scalar H0 r_c).  Usage:
        phi = autograd_solve().apply(delta, rc, ctx, a, omega_m, box_mpch, opts)
    with delta a CUDA FP64 tensor (ng^3) and rc a 0-d FP64 tensor."""
    import torch

    class MGSolveFn(torch.autograd.Function):
        @staticmethod
        def forward(fctx, delta, rc, mgctx, a, omega_m, box_mpch, o):
            phi = torch.zeros_like(delta)
            ng = int(delta.shape[0])
            mg_solve_dgp(mgctx, [dict(ng=ng, box_mpch=box_mpch, a=a, omega_m=omega_m, rc_h0=float(rc),
                                      delta=delta.contiguous(), phi=phi)], o)
            fctx.save_for_backward(delta, phi)
            fctx.args = (mgctx, a, omega_m, box_mpch, float(rc), o)
            return phi

        @staticmethod
        def backward(fctx, gphi):
            delta, phi = fctx.saved_tensors
            mgctx, a, omega_m, box_mpch, rc, o = fctx.args
            out = torch.empty_like(delta)
            _, drc, _ = mg_solve_adjoint(mgctx, int(delta.shape[0]), box_mpch, a, omega_m, rc, phi,
                                         delta.contiguous(), gphi.contiguous(), out, o)
            return out, torch.tensor(drc, dtype=torch.float64), None, None, None, None, None

    return MGSolveFn


def autograd_pm():
    """torch.autograd.Function over the differentiable particle-mesh run:
    forward gives the binned power spectrum P (nbins, FP64, on the noise
    tensor's device) from the white noise and R_c by dpm_run; backward calls
    dpm_run_vjp with the incoming dL/dP, so any loss of the caller's on P
    differentiates with respect to the noise and R_c.  Usage:
        pk = autograd_pm().apply(noise, rc, ctx, cfg, amp, opts)
    with noise a CUDA FP64 tensor (ng^3), rc a 0-d FP64 tensor and amp the
    rfft-grid amplitudes of dpm_run."""
    import torch

    class PMRunFn(torch.autograd.Function):
        @staticmethod
        def forward(fctx, noise, rc, mgctx, cfg, amp, o):
            noise = noise.contiguous()
            pk, _, _, _ = dpm_run(mgctx, cfg, amp, noise, float(rc), o=o)
            fctx.save_for_backward(noise)
            fctx.args = (mgctx, cfg, amp, float(rc), o, rc.device if torch.is_tensor(rc) else None)
            return torch.from_numpy(pk).to(noise.device)

        @staticmethod
        def backward(fctx, gpk):
            (noise,) = fctx.saved_tensors
            mgctx, cfg, amp, rc, o, rdev = fctx.args
            dn = torch.empty_like(noise)
            _, drc, _ = dpm_run_vjp(mgctx, cfg, amp, noise, rc, gpk.detach().double().cpu().numpy(), dn, o=o)
            grc = torch.tensor(drc, dtype=torch.float64, device=rdev) if rdev is not None else None
            return dn, grc, None, None, None, None

    return PMRunFn
