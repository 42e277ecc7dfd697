"""Linear power spectrum and sigma(R) normalisation (oracle; test infrastructure only).

P(k) = A k^ns / (1 + (k/kc)^2)^pow is the analytic linear spectrum used by the
workloads (the paper fixes cosmology without printing P(k), Sect. 2.1).  The
amplitude A is set so that the rms of the linear field smoothed with a
spherical top hat of radius R = 8 Mpc/h equals sigma8:

    sigma^2(R) = 1/(2 pi^2) * int_0^inf k^2 P(k) W(kR)^2 dk,
    W(x) = 3 (sin x - x cos x) / x^3.

Pins (tests): sigma^2 closed forms for pure power laws n = -2 and n = -1; the roll-off factor
exactly 2^-pow at k = kc and the asymptotic slopes ns (k << kc) and ns - 2 pow (k >> kc).
"""
from __future__ import annotations

import math
import warnings

import numpy as np
from scipy import integrate


def power_spectrum(k, amp: float, ns: float, kc: float, pw: float):
    """P(k) for numpy arrays or floats; P(0) = 0."""
    k = np.asarray(k, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        p = amp * np.power(k, ns) / np.power(1.0 + (k / kc) ** 2, pw)
    return np.where(k > 0, p, 0.0)


def tophat_window(x):
    x = np.asarray(x, dtype=np.float64)
    small = np.abs(x) < 1e-3
    xs = np.where(small, 1.0, x)
    w = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs ** 3
    # series 1 - x^2/10 + x^4/280 near zero
    return np.where(small, 1.0 - x ** 2 / 10.0 + x ** 4 / 280.0, w)


def sigma2(radius: float, amp: float, ns: float, kc: float, pw: float) -> float:
    """sigma^2(R) by adaptive quadrature in ln k (scipy QUADPACK)."""
    def integrand(lnk):
        k = math.exp(lnk)
        return k ** 3 * float(power_spectrum(k, amp, ns, kc, pw)) * float(tophat_window(k * radius)) ** 2

    total = 0.0
    # split the range so the oscillating tail is resolved
    edges = np.linspace(math.log(1e-8), math.log(1e3 / radius), 64)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        for a, b in zip(edges[:-1], edges[1:]):
            v, _ = integrate.quad(integrand, a, b, limit=200, epsabs=0.0, epsrel=1e-12)
            total += v
    return total / (2.0 * math.pi ** 2)


def amplitude_for_sigma(target: float, radius: float, ns: float, kc: float, pw: float) -> float:
    """A such that sigma(R) = target (sigma^2 is linear in A)."""
    return target ** 2 / sigma2(radius, 1.0, ns, kc, pw)
