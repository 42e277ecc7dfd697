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


def nuts_step(nu0, p0, counts, cfg, bias, eps: float, rng, max_depth: int = 10, grad_fn=None, delta_max: float = 1000.0,
              with_accept: bool = False):
    """One No-U-Turn transition (Hoffman & Gelman 2014, efficient NUTS with a slice variable) from
    nu0 with momentum p0.  Uniform draws from rng, in the order: slice level; then per doubling
    the direction, the subtree's proposal choices (taken only when the subtree has an admissible
    point) and the doubling's own proposal choice (taken only when the subtree did not stop).
    Returns (sample, depth, leapfrog steps), and with with_accept also the acceptance statistic
    of the last doubling's subtree: the mean over its states of min(1, exp(E - E0)), E the log
    joint density (their step-size adaptation statistic)."""
    if grad_fn is None:
        def grad_fn(x):
            lp, g, _, _ = model.logpost_and_grad(x, counts, cfg, bias)
            return lp, g
    steps = [0]

    def leap(state, v):
        x, r, lp, g = state
        r = r + 0.5 * v * eps * g
        x = x + v * eps * r
        lp, g = grad_fn(x)
        r = r + 0.5 * v * eps * g
        steps[0] += 1
        return (x, r, lp, g)

    def joint(state):
        return state[2] - 0.5 * float((state[1] ** 2).sum())

    def turning(minus, plus):
        d = plus[0] - minus[0]
        return float((d * minus[1]).sum()) < 0.0 or float((d * plus[1]).sum()) < 0.0

    acc = [0.0, 0]   # acceptance statistic of the subtree being built: sum, count

    def build(state, log_u, v, j):
        if j == 0:
            t = leap(state, v)
            e = joint(t)
            if not np.isfinite(e):
                e = -np.inf
            acc[0] += 0.0 if e == -np.inf else min(1.0, math.exp(min(0.0, e - e0)))
            acc[1] += 1
            return t, t, t, int(log_u <= e), bool(log_u < e + delta_max)
        minus, plus, prop, n1, ok = build(state, log_u, v, j - 1)
        if ok:
            if v < 0:
                minus, _, prop2, n2, ok2 = build(minus, log_u, v, j - 1)
            else:
                _, plus, prop2, n2, ok2 = build(plus, log_u, v, j - 1)
            if n1 + n2 > 0 and rng.random() < n2 / (n1 + n2):
                prop = prop2
            ok = ok2 and not turning(minus, plus)
            n1 += n2
        return minus, plus, prop, n1, ok

    lp0, g0 = grad_fn(np.asarray(nu0, dtype=np.float64))
    s0 = (np.asarray(nu0, dtype=np.float64), np.asarray(p0, dtype=np.float64), lp0, g0)
    e0 = joint(s0)
    log_u = e0 + math.log(rng.random())
    minus = plus = sample = s0
    n, depth, ok = 1, 0, True
    while ok and depth < max_depth:
        v = -1 if rng.random() < 0.5 else 1
        acc[0], acc[1] = 0.0, 0
        if v < 0:
            minus, _, prop, n2, ok2 = build(minus, log_u, v, depth)
        else:
            _, plus, prop, n2, ok2 = build(plus, log_u, v, depth)
        if ok2 and rng.random() < min(1.0, n2 / n):
            sample = prop
        n += n2
        ok = ok2 and not turning(minus, plus)
        depth += 1
    if with_accept:
        return sample[0], depth, steps[0], acc[0] / acc[1]
    return sample[0], depth, steps[0]


class DualAveraging:
    """Step-size adaptation of Hoffman & Gelman (2014, Sect. 3.2, dual averaging after Nesterov
    2009): after transition m (1-based) with acceptance statistic a_m,
        Hbar_m = (1 - 1/(m + t0)) Hbar_{m-1} + (delta - a_m) / (m + t0),
        log eps_m = mu - sqrt(m) / gamma * Hbar_m,  mu = log(10 eps_0),
        log epsbar_m = m^-kappa log eps_m + (1 - m^-kappa) log epsbar_{m-1},  epsbar_0 = 1,
    eps_m is used for the next transition and epsbar after the adaptation phase.  Defaults are
    theirs: delta = 0.8 (the paper does not state its target), gamma = 0.05, t0 = 10,
    kappa = 0.75."""

    def __init__(self, eps0: float, delta: float = 0.8, gamma: float = 0.05, t0: float = 10.0,
                 kappa: float = 0.75):
        self.mu = math.log(10.0 * eps0)
        self.delta, self.gamma, self.t0, self.kappa = delta, gamma, t0, kappa
        self.m, self.hbar, self.log_epsbar = 0, 0.0, 0.0
        self.eps = eps0

    def update(self, accept_stat: float) -> float:
        self.m += 1
        m = self.m
        w = 1.0 / (m + self.t0)
        self.hbar = (1.0 - w) * self.hbar + w * (self.delta - accept_stat)
        log_eps = self.mu - math.sqrt(m) / self.gamma * self.hbar
        eta = m ** (-self.kappa)
        self.log_epsbar = eta * log_eps + (1.0 - eta) * self.log_epsbar
        self.eps = math.exp(log_eps)
        return self.eps

    @property
    def final_eps(self) -> float:
        return math.exp(self.log_epsbar)
