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

Joint sampling (Sect. 2.1, 2.2): the free bias parameters move together with nu,
in log space theta = ln b, with the target log post(nu, e^theta) + sum theta
(the Jacobian of b = e^theta) and unit-mass momenta p_theta.
"""
from __future__ import annotations

import math

import numpy as np

import torch

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


def free_entries(bias):
    """(kind, region) of each free parameter in bit order of bias.free_mask (untied tables):
    kind 0 = alpha, 1 = beta."""
    nr = len(bias.alpha)
    mask = (1 << (2 * nr)) - 1 if bias.free_mask is None else bias.free_mask
    return [(q // nr, q % nr) for q in range(2 * nr) if (mask >> q) & 1]


def joint_logpost_and_grad(nu_np, theta_np, counts_np, cfg, bias):
    """log post(nu, b = e^theta) + sum theta and its gradients with respect to nu and theta
    (autograd of the oracle's log posterior with the free table entries replaced by e^theta)."""
    nu = torch.tensor(np.asarray(nu_np), dtype=model.DT, requires_grad=True)
    th = torch.tensor(np.asarray(theta_np), dtype=model.DT, requires_grad=True)
    t = model.bias_tables(bias)
    a, b = list(t["alpha"]), list(t["beta"])
    for k, (kind, r) in enumerate(free_entries(bias)):
        if kind == 0:
            a[r] = torch.exp(th[k])
        else:
            b[r] = torch.exp(th[k])
    t["alpha"], t["beta"] = torch.stack(a), torch.stack(b)
    lp = model.log_posterior(nu, torch.tensor(np.asarray(counts_np)), cfg, bias, t) + th.sum()
    g_nu, g_th = torch.autograd.grad(lp, (nu, th))
    return float(lp.detach()), g_nu.numpy(), g_th.numpy()


def integrate_joint(nu0, p0, theta0, ptheta0, counts, cfg, bias, n_steps: int, eps: float, scheme: str = "leapfrog"):
    """Joint trajectory; returns (nu, p, theta, p_theta, H0, H1) with
    H = -(log post + sum theta) + 1/2 |p|^2 + 1/2 |p_theta|^2."""
    kicks, drifts = scheme_coefficients(scheme)
    nu, p = np.array(nu0, dtype=np.float64), np.array(p0, dtype=np.float64)
    th, pt = np.array(theta0, dtype=np.float64), np.array(ptheta0, dtype=np.float64)
    lp, g, gt = joint_logpost_and_grad(nu, th, counts, cfg, bias)
    h0 = -lp + 0.5 * float((p ** 2).sum()) + 0.5 * float((pt ** 2).sum())
    for _ in range(n_steps):
        for j, d in enumerate(drifts):
            p = p + kicks[j] * eps * g
            pt = pt + kicks[j] * eps * gt
            nu = nu + d * eps * p
            th = th + d * eps * pt
            lp, g, gt = joint_logpost_and_grad(nu, th, counts, cfg, bias)
        p = p + kicks[-1] * eps * g
        pt = pt + kicks[-1] * eps * gt
    h1 = -lp + 0.5 * float((p ** 2).sum()) + 0.5 * float((pt ** 2).sum())
    return nu, p, th, pt, h0, h1
