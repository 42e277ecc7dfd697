"""Leapfrog integrator for HMC (oracle; test infrastructure only).

Sect. 2.2: Hamiltonian trajectories with potential U(nu) = -log posterior and
kinetic energy 1/2 |p|^2 (identity mass matrix).  One leapfrog step:
p <- p + eps/2 grad log post; nu <- nu + eps p; p <- p + eps/2 grad log post.
"""
from __future__ import annotations

import numpy as np

from . import model


def leapfrog(nu0, p0, counts, cfg, bias, n_steps: int, eps: float, grad_fn=None):
    """Returns (nu, p, H0, H1) with H = -log post + 1/2 |p|^2, all float64."""
    if grad_fn is None:
        def grad_fn(x):
            lp, g, _, _ = model.logpost_and_grad(x, counts, cfg, bias)
            return lp, g
    nu = np.array(nu0, dtype=np.float64)
    p = np.array(p0, dtype=np.float64)
    lp, g = grad_fn(nu)
    h0 = -lp + 0.5 * float((p ** 2).sum())
    for _ in range(n_steps):
        p = p + 0.5 * eps * g
        nu = nu + eps * p
        lp, g = grad_fn(nu)
        p = p + 0.5 * eps * g
    h1 = -lp + 0.5 * float((p ** 2).sum())
    return nu, p, h0, h1
