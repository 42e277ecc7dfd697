"""Python binding of ``libbridge.so``: the GB300 forward model and adjoint of
the differentiable fuzzy-cosmic-web field-level inference (arXiv 2506.03969).

This module only marshals arguments: every step of the forward model, its
adjoint and the leapfrog integrator runs in the library's CUDA kernels.  There
is no CPU fallback; if the library is missing or no GB300 is present the calls
raise.

The C functions keep their names (``bridge_create``, ``bridge_forward``,
``bridge_logpost_grad``, ``bridge_logpost_vjp``, ``bridge_logpost_grad_host``,
``bridge_leapfrog``, ``bridge_debug_field``...); ``Context`` wraps them for
torch tensors.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbridge.so")

BRIDGE_OK, BRIDGE_EINVAL, BRIDGE_ENOMEM, BRIDGE_ECUDA, BRIDGE_ENONFINITE, BRIDGE_ETIMEOUT, BRIDGE_ENODEVICE = range(7)
BRIDGE_FP32, BRIDGE_FP64 = 0, 1
BRIDGE_LEAPFROG, BRIDGE_TWO_STAGE, BRIDGE_FOURTH_ORDER = 0, 1, 2
FIELD_DELTA0, FIELD_PSI, FIELD_DELTA, FIELD_TIDAL, FIELD_HESSIAN, FIELD_LAMBDA, FIELD_LNNBAR = range(7)
MAX_REGIONS = 16


class BridgeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"bridge status {status}: {msg}")
        self.status = status


class bridge_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("batch", ctypes.c_int32), ("box", ctypes.c_double),
                ("pk_amp", ctypes.c_double), ("pk_ns", ctypes.c_double), ("pk_kc", ctypes.c_double),
                ("pk_pow", ctypes.c_double), ("growth_d", ctypes.c_double), ("d2_over_d2", ctypes.c_double),
                ("r_s", ctypes.c_double), ("lambda_th_phi", ctypes.c_double), ("lambda_th_delta", ctypes.c_double),
                ("sharpness", ctypes.c_double), ("n_regions", ctypes.c_int32), ("rho_floor", ctypes.c_double),
                ("precision", ctypes.c_int32), ("recompute_alpt", ctypes.c_int32), ("rsd_f", ctypes.c_double),
                ("rsd_los", ctypes.c_int32), ("deterministic", ctypes.c_int32)]


_D16 = ctypes.c_double * MAX_REGIONS


class bridge_profile_row(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class bridge_bias(ctypes.Structure):
    _fields_ = [("a", _D16), ("alpha", _D16), ("rho", _D16), ("eps", _D16), ("rhop", _D16), ("epsp", _D16),
                ("beta", _D16), ("prior_mask", ctypes.c_uint32), ("mu_alpha", ctypes.c_double),
                ("sigma_alpha", ctypes.c_double), ("mu_beta", ctypes.c_double), ("sigma_beta", ctypes.c_double),
                ("free_mask", ctypes.c_uint32), ("tie_classes", ctypes.c_int32)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libbridge.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2506_03969_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, cp, dp, i32p = ctypes.c_void_p, ctypes.POINTER(bridge_config), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
    bp = ctypes.POINTER(bridge_bias)
    L.bridge_validate_config.argtypes = [cp]; L.bridge_validate_config.restype = ctypes.c_int
    L.bridge_workspace_bytes.argtypes = [cp]; L.bridge_workspace_bytes.restype = ctypes.c_size_t
    L.bridge_pk_amplitude.argtypes = [ctypes.c_double] * 5; L.bridge_pk_amplitude.restype = ctypes.c_double
    L.bridge_create.argtypes = [cp, vp, ctypes.POINTER(vp)]; L.bridge_create.restype = ctypes.c_int
    L.bridge_destroy.argtypes = [vp]; L.bridge_destroy.restype = None
    L.bridge_forward.argtypes = [vp, vp, i32p, bp, vp, dp]; L.bridge_forward.restype = ctypes.c_int
    L.bridge_logpost_grad.argtypes = [vp, vp, i32p, bp, dp, vp, dp]; L.bridge_logpost_grad.restype = ctypes.c_int
    L.bridge_logpost_vjp.argtypes = [vp, vp, i32p, bp, dp, vp, dp]; L.bridge_logpost_vjp.restype = ctypes.c_int
    L.bridge_logpost_grad_host.argtypes = [vp, vp, i32p, bp, dp, vp, dp]
    L.bridge_logpost_grad_host.restype = ctypes.c_int
    L.bridge_leapfrog.argtypes = [vp, vp, vp, i32p, bp, ctypes.c_int32, ctypes.c_double, dp, dp]
    L.bridge_leapfrog.restype = ctypes.c_int
    L.bridge_integrate.argtypes = [vp, vp, vp, i32p, bp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, dp, dp]
    L.bridge_integrate.restype = ctypes.c_int
    L.bridge_leapfrog_steps.argtypes = [vp, vp, vp, vp, i32p, bp, ctypes.c_int32, ctypes.c_double, dp]
    L.bridge_leapfrog_steps.restype = ctypes.c_int
    L.bridge_dot.argtypes = [vp, vp, vp, dp]; L.bridge_dot.restype = ctypes.c_int
    L.bridge_integrate_joint.argtypes = [vp, vp, vp, dp, dp, i32p, bp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                         dp, dp]
    L.bridge_integrate_joint.restype = ctypes.c_int
    L.bridge_debug_field.argtypes = [vp, vp, i32p, bp, ctypes.c_int32, vp]; L.bridge_debug_field.restype = ctypes.c_int
    L.bridge_last_launch_count.argtypes = [vp]; L.bridge_last_launch_count.restype = ctypes.c_int64
    L.bridge_profile_enable.argtypes = [vp, ctypes.c_int]; L.bridge_profile_enable.restype = ctypes.c_int
    L.bridge_profile_read.argtypes = [vp, ctypes.POINTER(bridge_profile_row), ctypes.c_int]
    L.bridge_profile_read.restype = ctypes.c_int
    L.bridge_autotune.argtypes = [vp, vp, i32p, bp, i32p]; L.bridge_autotune.restype = ctypes.c_int
    L.bridge_fft_roundtrip.argtypes = [vp, vp, vp]; L.bridge_fft_roundtrip.restype = ctypes.c_int
    L.bridge_wiener_init.argtypes = [vp, i32p, vp]; L.bridge_wiener_init.restype = ctypes.c_int
    L.bridge_delta0_noalloc.argtypes = [cp, vp, vp, vp]; L.bridge_delta0_noalloc.restype = ctypes.c_int
    L.bridge_last_error.argtypes = [vp]; L.bridge_last_error.restype = ctypes.c_char_p
    L.bridge_status_string.argtypes = [ctypes.c_int]; L.bridge_status_string.restype = ctypes.c_char_p
    _lib = L
    return L


# ---------------------------------------------------------------------------
# host-only helpers
# ---------------------------------------------------------------------------
def bridge_pk_amplitude(sigma: float, radius: float, ns: float, kc: float, pw: float) -> float:
    return float(lib().bridge_pk_amplitude(sigma, radius, ns, kc, pw))


def make_config(n: int, box: float, batch: int = 1, sigma8: float = 0.8, pk_ns: float = 0.96, pk_kc: float = 0.02,
                pk_pow: float = 1.5, pk_amp: Optional[float] = None, growth_d: float = 1.0,
                d2_over_d2: float = -3.0 / 7.0, r_s: float = 4.0, lambda_th_phi: float = 0.0,
                lambda_th_delta: float = 0.0, sharpness: float = 20.0, n_regions: int = 4,
                rho_floor: float = 1e-6, precision: int = BRIDGE_FP32, recompute_alpt: bool = False,
                rsd_f: float = 0.0, rsd_los: int = 0, deterministic: bool = False) -> bridge_config:
    """A bridge_config; the P(k) amplitude is fixed by sigma(8 Mpc/h) = sigma8 unless given."""
    if pk_amp is None:
        pk_amp = bridge_pk_amplitude(sigma8, 8.0, pk_ns, pk_kc, pk_pow)
    return bridge_config(n, batch, box, pk_amp, pk_ns, pk_kc, pk_pow, growth_d, d2_over_d2, r_s, lambda_th_phi,
                         lambda_th_delta, sharpness, n_regions, rho_floor, precision, int(bool(recompute_alpt)),
                         float(rsd_f), int(rsd_los), int(bool(deterministic)))


def config_from(cfg, precision: int = BRIDGE_FP32, batch: Optional[int] = None,
                recompute_alpt: bool = False, deterministic: bool = False) -> bridge_config:
    """bridge_config from any object with the workload attributes (n, box, sigma8, ...)."""
    return make_config(cfg.n, cfg.box, batch=cfg.batch if batch is None else batch, sigma8=cfg.sigma8,
                       pk_ns=cfg.pk_ns, pk_kc=cfg.pk_kc, pk_pow=cfg.pk_pow, growth_d=cfg.growth_d,
                       d2_over_d2=cfg.d2_over_d2, r_s=cfg.r_s, lambda_th_phi=cfg.lambda_th_phi,
                       lambda_th_delta=cfg.lambda_th_delta, sharpness=cfg.sharpness, n_regions=cfg.n_regions,
                       rho_floor=cfg.rho_floor, precision=precision, recompute_alpt=recompute_alpt,
                       rsd_f=getattr(cfg, "rsd_f", 0.0), rsd_los=getattr(cfg, "rsd_los", 0),
                       deterministic=deterministic)


def all_free(n_regions: int) -> int:
    """free_mask selecting every alpha_r and beta_r entry of an untied table."""
    return (1 << (2 * n_regions)) - 1


def bias_array(biases: Sequence) -> ctypes.Array:
    """Array of bridge_bias from objects with a, alpha, rho, eps, rhop, epsp, beta lists and prior
    fields; free_mask / tie_classes default to every alpha_r and beta_r untied."""
    arr = (bridge_bias * len(biases))()
    for i, b in enumerate(biases):
        s = arr[i]
        for name in ("a", "alpha", "rho", "eps", "rhop", "epsp", "beta"):
            vals = list(getattr(b, name))
            dst = getattr(s, name)
            for r, v in enumerate(vals):
                dst[r] = float(v)
        s.prior_mask = int(getattr(b, "prior_mask", 0))
        s.mu_alpha, s.sigma_alpha = float(b.mu_alpha), float(b.sigma_alpha)
        s.mu_beta, s.sigma_beta = float(b.mu_beta), float(b.sigma_beta)
        fm = getattr(b, "free_mask", None)
        s.free_mask = all_free(len(list(b.alpha))) if fm is None else int(fm)
        s.tie_classes = int(getattr(b, "tie_classes", 0))
    return arr


def n_free(biases: Sequence) -> int:
    """Number of free bias parameters per chain (popcount of free_mask)."""
    return bin(int(bias_array(biases[:1])[0].free_mask)).count("1")


# ---------------------------------------------------------------------------
# context
# ---------------------------------------------------------------------------
def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


class Context:
    """One library context (workspace on the current CUDA device, bound to a stream)."""

    def __init__(self, cfg: bridge_config, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise BridgeError(BRIDGE_ENODEVICE, "no CUDA device")
        self.torch = torch
        self.cfg = cfg
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.dtype = torch.float64 if cfg.precision == BRIDGE_FP64 else torch.float32
        self.n, self.batch, self.n_regions = cfg.n, cfg.batch, cfg.n_regions
        h = ctypes.c_void_p()
        st = lib().bridge_create(ctypes.byref(cfg), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != BRIDGE_OK:
            raise BridgeError(st, lib().bridge_status_string(st).decode() + ": " + lib().bridge_last_error(None).decode())
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().bridge_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != BRIDGE_OK:
            raise BridgeError(st, lib().bridge_last_error(self.handle).decode())

    def _field(self, t, name):
        torch = self.torch
        if t.device.type != "cuda" or t.dtype != self.dtype or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor of dtype {self.dtype}")
        if t.numel() != self.batch * self.n ** 3:
            raise ValueError(f"{name} must hold batch * n^3 elements")
        return t

    def _counts(self, c):
        torch = self.torch
        if c.device.type != "cuda" or c.dtype != torch.int32 or not c.is_contiguous() or c.numel() != self.batch * self.n ** 3:
            raise ValueError("counts must be a contiguous CUDA int32 tensor of batch * n^3 elements")
        return c

    def launches(self) -> int:
        return int(lib().bridge_last_launch_count(self.handle))

    def bridge_profile_enable(self, on: bool = True):
        self._check(lib().bridge_profile_enable(self.handle, int(bool(on))))

    def bridge_profile_read(self):
        """Per kernel class: {name: (launches, total_ms, algorithmic_bytes)} (CUDA events on the context stream)."""
        rows = (bridge_profile_row * 64)()
        n = lib().bridge_profile_read(self.handle, rows, 64)
        if n < 0:
            self._check(-n)
        return {rows[i].name.decode(): (int(rows[i].launches), float(rows[i].total_ms), float(rows[i].bytes))
                for i in range(n)}

    def bridge_forward(self, nu, counts, biases, want_ln_nbar: bool = False):
        torch = self.torch
        self._field(nu, "nu"); self._counts(counts)
        out = torch.empty_like(nu) if want_ln_nbar else None
        lp = (ctypes.c_double * self.batch)()
        self._check(lib().bridge_forward(self.handle, ctypes.c_void_p(_ptr(nu)), ctypes.c_void_p(_ptr(counts)),
                                         bias_array(biases), ctypes.c_void_p(_ptr(out)), lp))
        return np.array(lp[:]), out

    def bridge_logpost_grad(self, nu, counts, biases, grad_out=None, want_bias_grad: bool = True):
        """(log posterior [B], d/d nu, d/d free bias parameters [B][popcount(free_mask)] or None)."""
        torch = self.torch
        self._field(nu, "nu"); self._counts(counts)
        g = grad_out if grad_out is not None else torch.empty_like(nu)
        lp = (ctypes.c_double * self.batch)()
        nf = n_free(biases)
        gb = (ctypes.c_double * (self.batch * nf))() if want_bias_grad and nf else None
        self._check(lib().bridge_logpost_grad(self.handle, ctypes.c_void_p(_ptr(nu)), ctypes.c_void_p(_ptr(counts)),
                                              bias_array(biases), lp, ctypes.c_void_p(_ptr(g)), gb))
        gbias = np.array(gb[:]).reshape(self.batch, nf) if gb is not None else None
        return np.array(lp[:]), g, gbias

    def bridge_logpost_vjp(self, nu, counts, biases, cotangent=None, grad_out=None, want_bias_grad: bool = False):
        """Backward pass: cotangent[b] * d log post_b / d nu (forward model re-evaluated from nu,
        ALPT included).  Returns (grad, bias gradient or None)."""
        torch = self.torch
        self._field(nu, "nu"); self._counts(counts)
        g = grad_out if grad_out is not None else torch.empty_like(nu)
        cot = None
        if cotangent is not None:
            cv = np.asarray(cotangent, dtype=np.float64).reshape(-1)
            if cv.size != self.batch:
                raise ValueError("cotangent must hold one value per chain")
            cot = (ctypes.c_double * self.batch)(*cv.tolist())
        nf = n_free(biases)
        gb = (ctypes.c_double * (self.batch * nf))() if want_bias_grad and nf else None
        self._check(lib().bridge_logpost_vjp(self.handle, ctypes.c_void_p(_ptr(nu)), ctypes.c_void_p(_ptr(counts)),
                                             bias_array(biases), cot, ctypes.c_void_p(_ptr(g)), gb))
        return g, (np.array(gb[:]).reshape(self.batch, nf) if gb is not None else None)

    def bridge_logpost_grad_host(self, nu_host, counts_host, biases, grad_host, want_bias_grad: bool = False):
        """Host (ideally pinned) torch CPU tensors in and out; copies are part of the call.
        Returns the log posterior [B], and with want_bias_grad also the free bias gradient."""
        lp = (ctypes.c_double * self.batch)()
        nf = n_free(biases)
        gb = (ctypes.c_double * (self.batch * nf))() if want_bias_grad and nf > 0 else None
        self._check(lib().bridge_logpost_grad_host(self.handle, ctypes.c_void_p(nu_host.data_ptr()),
                                                   ctypes.c_void_p(counts_host.data_ptr()), bias_array(biases), lp,
                                                   ctypes.c_void_p(grad_host.data_ptr()), gb))
        if not want_bias_grad:
            return np.array(lp[:])
        return np.array(lp[:]), (np.array(gb[:]).reshape(self.batch, nf) if gb is not None else None)

    def bridge_leapfrog(self, nu, p, counts, biases, n_steps: int, eps: float):
        """Leapfrog trajectory in place; returns (H0 [B], H1 [B]).  A chain whose H0 or H1 is not
        finite comes back with its start state (the library restores it) and its non-finite
        entries in the returned arrays; other errors raise."""
        self._field(nu, "nu"); self._field(p, "p"); self._counts(counts)
        h0 = (ctypes.c_double * self.batch)()
        h1 = (ctypes.c_double * self.batch)()
        st = lib().bridge_leapfrog(self.handle, ctypes.c_void_p(_ptr(nu)), ctypes.c_void_p(_ptr(p)),
                                   ctypes.c_void_p(_ptr(counts)), bias_array(biases), int(n_steps), float(eps), h0, h1)
        if st != BRIDGE_ENONFINITE:
            self._check(st)
        return np.array(h0[:]), np.array(h1[:])

    def bridge_integrate(self, nu, p, counts, biases, scheme: int, n_steps: int, eps: float):
        """Trajectory of a splitting integrator (BRIDGE_LEAPFROG, BRIDGE_TWO_STAGE,
        BRIDGE_FOURTH_ORDER) in place; returns (H0 [B], H1 [B]) as bridge_leapfrog does."""
        self._field(nu, "nu"); self._field(p, "p"); self._counts(counts)
        h0 = (ctypes.c_double * self.batch)()
        h1 = (ctypes.c_double * self.batch)()
        st = lib().bridge_integrate(self.handle, ctypes.c_void_p(_ptr(nu)), ctypes.c_void_p(_ptr(p)),
                                    ctypes.c_void_p(_ptr(counts)), bias_array(biases), int(scheme), int(n_steps),
                                    float(eps), h0, h1)
        if st != BRIDGE_ENONFINITE:
            self._check(st)
        return np.array(h0[:]), np.array(h1[:])

    def bridge_integrate_joint(self, nu, p, theta, p_theta, counts, biases, scheme: int, n_steps: int, eps: float):
        """Joint trajectory of (nu, theta = ln b) in place: nu, p on the device; theta, p_theta numpy
        float64 arrays [B][n_free] updated in place.  Returns (H0 [B], H1 [B]); chains whose H is
        not finite come back with their start state (see bridge_integrate_joint)."""
        self._field(nu, "nu"); self._field(p, "p"); self._counts(counts)
        nf = n_free(biases)
        for a, name in ((theta, "theta"), (p_theta, "p_theta")):
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and
                    a.size == self.batch * nf):
                raise ValueError(f"{name} must be a contiguous float64 array of batch * n_free values")
        h0 = (ctypes.c_double * self.batch)()
        h1 = (ctypes.c_double * self.batch)()
        dp = ctypes.POINTER(ctypes.c_double)
        st = lib().bridge_integrate_joint(self.handle, ctypes.c_void_p(_ptr(nu)), ctypes.c_void_p(_ptr(p)),
                                          theta.ctypes.data_as(dp), p_theta.ctypes.data_as(dp),
                                          ctypes.c_void_p(_ptr(counts)), bias_array(biases), int(scheme),
                                          int(n_steps), float(eps), h0, h1)
        if st != BRIDGE_ENONFINITE:
            self._check(st)
        return np.array(h0[:]), np.array(h1[:])

    def bridge_leapfrog_steps(self, nu, p, grad, counts, biases, n_steps: int, eps: float):
        """n leapfrog steps in place from (nu, p) with grad = gradient at nu (updated to the new nu);
        returns the log posterior [B] at the new nu (non-finite values are returned, not raised)."""
        self._field(nu, "nu"); self._field(p, "p"); self._field(grad, "grad"); self._counts(counts)
        lp = (ctypes.c_double * self.batch)()
        st = lib().bridge_leapfrog_steps(self.handle, ctypes.c_void_p(_ptr(nu)), ctypes.c_void_p(_ptr(p)),
                                         ctypes.c_void_p(_ptr(grad)), ctypes.c_void_p(_ptr(counts)), bias_array(biases),
                                         int(n_steps), float(eps), lp)
        self._check(st)
        return np.array(lp[:])

    def bridge_dot(self, a, b):
        """Per-chain sum a_i b_i in FP64 (host array [B])."""
        self._field(a, "a"); self._field(b, "b")
        out = (ctypes.c_double * self.batch)()
        self._check(lib().bridge_dot(self.handle, ctypes.c_void_p(_ptr(a)), ctypes.c_void_p(_ptr(b)), out))
        return np.array(out[:])

    def bridge_autotune(self, nu, counts, biases):
        """Pick launch shapes for this context by timing evaluations of this problem.
        Returns [ALPT node, ALPT-adjoint node, gather node CTAs per SM, web-adjoint blocks per chain]
        (0 = built-in choice)."""
        self._field(nu, "nu"); self._counts(counts)
        ch = (ctypes.c_int32 * 4)()
        self._check(lib().bridge_autotune(self.handle, ctypes.c_void_p(_ptr(nu)), ctypes.c_void_p(_ptr(counts)),
                                          bias_array(biases), ctypes.cast(ch, ctypes.c_void_p)))
        return [int(v) for v in ch]

    def bridge_wiener_init(self, counts, out=None):
        """Chain starting point nu^(0): the tracer contrast Wiener-filtered to white noise."""
        self._counts(counts)
        out = out if out is not None else self.torch.empty(counts.shape, dtype=self.dtype, device=counts.device)
        self._field(out, "out")
        self._check(lib().bridge_wiener_init(self.handle, ctypes.c_void_p(_ptr(counts)), ctypes.c_void_p(_ptr(out))))
        return out

    def bridge_fft_roundtrip(self, x, out=None):
        """IDFT(DFT(x)) through the library's FFT pass kernels (no operator)."""
        self._field(x, "x")
        out = out if out is not None else self.torch.empty_like(x)
        self._field(out, "out")
        self._check(lib().bridge_fft_roundtrip(self.handle, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(out))))
        return out

    def bridge_debug_field(self, nu, counts, biases, which: int):
        torch = self.torch
        self._field(nu, "nu"); self._counts(counts)
        comps = {FIELD_PSI: 3, FIELD_TIDAL: 6, FIELD_HESSIAN: 6, FIELD_LAMBDA: 3}.get(which, 1)
        out = torch.empty((self.batch, comps) + (self.n,) * 3, dtype=self.dtype, device=nu.device)
        self._check(lib().bridge_debug_field(self.handle, ctypes.c_void_p(_ptr(nu)), ctypes.c_void_p(_ptr(counts)),
                                             bias_array(biases), int(which), ctypes.c_void_p(_ptr(out))))
        return out


def bridge_delta0_noalloc(cfg: bridge_config, nu, delta0, stream=None):
    """delta0 = IDFT[sqrt(P/dx^3) DFT(nu)] (App. A) into the caller's `delta0`, with no device
    allocation and no context (scratch is a 4 MiB static array in the library; see bridge.h).
    nu, delta0: contiguous CUDA tensors of batch * n^3 elements (float32, or float64 for FP64).
    Asynchronous on `stream` (default: torch's current stream)."""
    import torch
    dt = torch.float64 if cfg.precision == BRIDGE_FP64 else torch.float32
    for t, name in ((nu, "nu"), (delta0, "delta0")):
        if t.device.type != "cuda" or t.dtype != dt or not t.is_contiguous() or t.numel() != cfg.batch * cfg.n ** 3:
            raise ValueError(f"{name} must be a contiguous CUDA {dt} tensor of batch * n^3 elements")
    s = stream if stream is not None else torch.cuda.current_stream(nu.device)
    st = lib().bridge_delta0_noalloc(ctypes.byref(cfg), ctypes.c_void_p(_ptr(nu)), ctypes.c_void_p(_ptr(delta0)),
                                     ctypes.c_void_p(s.cuda_stream))
    if st != BRIDGE_OK:
        raise BridgeError(st, lib().bridge_status_string(st).decode() + ": " + lib().bridge_last_error(None).decode())
    return delta0


def _make_autograd():
    import torch

    class LogPosterior(torch.autograd.Function):
        """log posterior(nu) with the hand-written adjoint as backward.

        forward(ctx_obj, nu, counts, biases) -> tensor [B] (float64) runs the
        forward model only (bridge_forward).  backward runs bridge_logpost_vjp,
        which evaluates the forward model again from the saved nu -- the ALPT
        displacement recomputed, not stored between the two passes -- and then
        the adjoint, scaled by the incoming gradient of each chain."""

        @staticmethod
        def forward(fctx, bctx: Context, nu, counts, biases):
            x = nu.detach().contiguous()
            lp, _ = bctx.bridge_forward(x, counts, biases)
            fctx.bctx, fctx.biases = bctx, biases
            fctx.save_for_backward(x, counts)
            return torch.tensor(lp, dtype=torch.float64, device=nu.device)

        @staticmethod
        def backward(fctx, grad_out):
            x, counts = fctx.saved_tensors
            cot = grad_out.detach().to(torch.float64).reshape(-1).cpu().numpy()
            g, _ = fctx.bctx.bridge_logpost_vjp(x, counts, fctx.biases, cotangent=cot)
            return None, g.reshape(x.shape), None, None

    return LogPosterior


_LP = None


def log_posterior(bctx: Context, nu, counts, biases):
    """Differentiable log posterior: torch autograd gets the library's adjoint gradient."""
    global _LP
    if _LP is None:
        _LP = _make_autograd()
    return _LP.apply(bctx, nu, counts, biases)
