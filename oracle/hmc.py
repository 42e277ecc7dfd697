"""Hamiltonian integrators for HMC (oracle; test infrastructure only).

Sect. 2.2: Hamiltonian trajectories with potential U(nu) = -log posterior and
kinetic energy 1/2 |p|^2 (identity mass matrix).  The paper names second- and
fourth-order integrators and the Blanes et al. (2014) variant; each is a
splitting of exp(eps (A + B)) into kicks p <- p + c eps grad log post and drifts
nu <- nu + d eps p, with coefficients

  leapfrog (Stormer-Verlet)      kicks 1/2, 1/2            drifts 1
  two-stage (Blanes, Casas and   kicks b, 1 - 2b, b        drifts 1/2, 1/2
    Sanz-Serna 2014)             b = 0.211781 (their choice for HMC)
  fourth order (Yoshida 1990,    three leapfrog sub-steps of w1, w0, w1 times eps,
    symmetric triple jump)       w1 = 1 / (2 - 2^(1/3)), w0 = 1 - 2 w1

One step applies the kicks and drifts alternately, starting and ending with a
kick; the gradient is evaluated after every drift.
"""
from __future__ import annotations

import math

import numpy as np

from . import model

BCSS_B = 0.211781


def scheme_coefficients(scheme: str, b: float = BCSS_B):
    """(kicks, drifts) of one step, in units of eps: len(kicks) = len(drifts) + 1."""
    if scheme == "leapfrog":
        return [0.5, 0.5], [1.0]
    if scheme == "bcss2":
        return [b, 1.0 - 2.0 * b, b], [0.5, 0.5]
    if scheme == "yoshida4":
        w1 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
        w0 = 1.0 - 2.0 * w1
        # leapfrog(w1) leapfrog(w0) leapfrog(w1), adjacent half kicks written separately
        return [w1 / 2, w1 / 2 + w0 / 2, w0 / 2 + w1 / 2, w1 / 2], [w1, w0, w1]
    raise ValueError(scheme)


def integrate(nu0, p0, counts, cfg, bias, n_steps: int, eps: float, scheme: str = "leapfrog", grad_fn=None,
              b: float = BCSS_B):
    """Returns (nu, p, H0, H1) with H = -log post + 1/2 |p|^2, all float64."""
    if grad_fn is None:
        def grad_fn(x):
            lp, g, _, _ = model.logpost_and_grad(x, counts, cfg, bias)
            return lp, g
    kicks, drifts = scheme_coefficients(scheme, b)
    nu = np.array(nu0, dtype=np.float64)
    p = np.array(p0, dtype=np.float64)
    lp, g = grad_fn(nu)
    h0 = -lp + 0.5 * float((p ** 2).sum())
    for _ in range(n_steps):
        for j, d in enumerate(drifts):
            p = p + kicks[j] * eps * g
            nu = nu + d * eps * p
            lp, g = grad_fn(nu)
        p = p + kicks[-1] * eps * g
    h1 = -lp + 0.5 * float((p ** 2).sum())
    return nu, p, h0, h1


def leapfrog(nu0, p0, counts, cfg, bias, n_steps: int, eps: float, grad_fn=None):
    """The Stormer-Verlet integrator: p <- p + eps/2 grad; nu <- nu + eps p; p <- p + eps/2 grad."""
    return integrate(nu0, p0, counts, cfg, bias, n_steps, eps, "leapfrog", grad_fn)
