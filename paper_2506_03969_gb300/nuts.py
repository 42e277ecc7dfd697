"""No-U-Turn sampler driven from the host over the library's leapfrog steps.

The paper samples its posterior with NUTS (Sect. 2.2: trajectories grown until
they turn back, tree depth up to 10).  This module is the sampler's control flow
only -- tree doubling, slice test, U-turn test, proposal choice -- in the form of
Hoffman & Gelman (2014, "efficient NUTS" with a slice variable).  Every field
operation runs in the library: one gradient evaluation per leapfrog step
(``bridge_leapfrog_steps``), FP64 dot products for the kinetic energy and the
U-turn criterion (``bridge_dot``); states are copied on the device.

Random draws (slice level, directions, proposal choices) come from the caller's
``numpy.random.Generator`` in the order the algorithm consumes them, so a run is
reproducible from its seed; the momentum is drawn by the caller.  One chain per
context (batch 1): each chain grows its own tree.

Step-size adaptation (``StepSizeAdaptation``) is their dual-averaging scheme
(Sect. 3.2 of the same paper), fed with each transition's acceptance statistic.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

DELTA_MAX = 1000.0   # a step whose energy exceeds the slice level by this much ends the trajectory


@dataclasses.dataclass
class _State:
    nu: object
    p: object
    g: object
    lp: float

    def clone(self) -> "_State":
        return _State(self.nu.clone(), self.p.clone(), self.g.clone(), self.lp)


@dataclasses.dataclass
class NutsResult:
    nu: object            # the sample (device tensor)
    logpost: float        # log posterior at the sample
    grad: object          # gradient at the sample (device tensor)
    depth: int            # tree depth reached
    n_leapfrog: int       # leapfrog steps taken (gradient evaluations)
    diverged: bool
    accept_stat: float    # mean of min(1, exp(E - E0)) over the last doubling's states


class NUTS:
    """One NUTS transition per call of ``step`` on a batch-1 ``Context``."""

    def __init__(self, ctx, counts, biases, eps: float, max_depth: int = 10):
        if ctx.batch != 1:
            raise ValueError("NUTS drives one chain per context (batch 1)")
        self.ctx, self.counts, self.biases = ctx, counts, biases
        self.eps, self.max_depth = float(eps), int(max_depth)
        self.n_leapfrog = 0
        self.diverged = False
        self._acc_sum, self._acc_n, self._e0 = 0.0, 0, 0.0

    def _dot(self, a, b) -> float:
        return float(self.ctx.bridge_dot(a, b)[0])

    def _leapfrog(self, s: _State, direction: int) -> _State:
        t = s.clone()
        lp = self.ctx.bridge_leapfrog_steps(t.nu, t.p, t.g, self.counts, self.biases, 1, direction * self.eps)
        t.lp = float(lp[0])
        self.n_leapfrog += 1
        return t

    def _energy(self, s: _State) -> float:
        """log post - 1/2 |p|^2 (the log of the joint density)."""
        return s.lp - 0.5 * self._dot(s.p, s.p)

    def _no_uturn(self, minus: _State, plus: _State) -> bool:
        # (nu+ - nu-) . p- >= 0 and (nu+ - nu-) . p+ >= 0
        d_m = self._dot(plus.nu, minus.p) - self._dot(minus.nu, minus.p)
        d_p = self._dot(plus.nu, plus.p) - self._dot(minus.nu, plus.p)
        return d_m >= 0.0 and d_p >= 0.0

    def _build(self, s: _State, log_u: float, direction: int, depth: int, rng):
        """Subtree of 2^depth steps from s; returns (minus, plus, proposal, n_ok, keep_going)."""
        if depth == 0:
            t = self._leapfrog(s, direction)
            e = self._energy(t)
            if not math.isfinite(e):
                e = -math.inf
            self._acc_sum += 0.0 if e == -math.inf else math.exp(min(0.0, e - self._e0))
            self._acc_n += 1
            n_ok = 1 if log_u <= e else 0
            ok = log_u < e + DELTA_MAX
            if not ok:
                self.diverged = True
            return t, t, t, n_ok, ok
        minus, plus, prop, n_ok, ok = self._build(s, log_u, direction, depth - 1, rng)
        if ok:
            if direction < 0:
                minus, _, prop2, n2, ok2 = self._build(minus, log_u, direction, depth - 1, rng)
            else:
                _, plus, prop2, n2, ok2 = self._build(plus, log_u, direction, depth - 1, rng)
            if n_ok + n2 > 0 and rng.random() < n2 / (n_ok + n2):
                prop = prop2
            ok = ok2 and self._no_uturn(minus, plus)
            n_ok += n2
        return minus, plus, prop, n_ok, ok

    def step(self, nu, p, grad, logpost: float, rng: np.random.Generator) -> NutsResult:
        """One transition from nu (with its gradient and log posterior) and momentum p (both device
        tensors, not modified); returns the new sample."""
        self.n_leapfrog = 0
        self.diverged = False
        s0 = _State(nu.clone(), p.clone(), grad.clone(), float(logpost))
        self._e0 = self._energy(s0)
        log_u = self._e0 + math.log(rng.random())
        minus, plus, sample = s0, s0, s0
        n, depth, ok = 1, 0, True
        while ok and depth < self.max_depth:
            direction = -1 if rng.random() < 0.5 else 1
            self._acc_sum, self._acc_n = 0.0, 0
            if direction < 0:
                minus, _, prop, n2, ok2 = self._build(minus, log_u, direction, depth, rng)
            else:
                _, plus, prop, n2, ok2 = self._build(plus, log_u, direction, depth, rng)
            if ok2 and rng.random() < min(1.0, n2 / n):
                sample = prop
            n += n2
            ok = ok2 and self._no_uturn(minus, plus)
            depth += 1
        return NutsResult(sample.nu, sample.lp, sample.g, depth, self.n_leapfrog, self.diverged,
                          self._acc_sum / max(self._acc_n, 1))


class StepSizeAdaptation:
    """Dual averaging of the log step size towards a target acceptance statistic (Hoffman &
    Gelman 2014, Sect. 3.2): with w = 1/(m + t0) after transition m,
    H <- (1 - w) H + w (target - a_m); log eps = log(10 eps0) - sqrt(m) H / gamma; the running
    average log eps_bar <- m^-kappa log eps + (1 - m^-kappa) log eps_bar is the step to keep once
    adaptation ends.  Defaults as theirs (target 0.8, gamma 0.05, t0 10, kappa 0.75)."""

    def __init__(self, eps0: float, target: float = 0.8, gamma: float = 0.05, t0: float = 10.0,
                 kappa: float = 0.75):
        self.anchor = math.log(10.0 * float(eps0))
        self.target, self.gamma, self.t0, self.kappa = target, gamma, t0, kappa
        self.count, self.h, self.log_avg = 0, 0.0, 0.0
        self.eps = float(eps0)

    def update(self, accept_stat: float) -> float:
        """Record one transition's acceptance statistic; returns the step for the next one."""
        self.count += 1
        w = 1.0 / (self.count + self.t0)
        self.h += w * ((self.target - accept_stat) - self.h)
        log_eps = self.anchor - math.sqrt(self.count) * self.h / self.gamma
        weight = self.count ** -self.kappa
        self.log_avg += weight * (log_eps - self.log_avg)
        self.eps = math.exp(log_eps)
        return self.eps

    @property
    def adapted_eps(self) -> float:
        """The averaged step to use after adaptation."""
        return math.exp(self.log_avg)
