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


class NUTS:
    """One NUTS transition per call of ``step`` on a batch-1 ``Context``."""

    def __init__(self, ctx, counts, biases, eps: float, max_depth: int = 10):
        if ctx.batch != 1:
            raise ValueError("NUTS drives one chain per context (batch 1)")
        self.ctx, self.counts, self.biases = ctx, counts, biases
        self.eps, self.max_depth = float(eps), int(max_depth)
        self.n_leapfrog = 0
        self.diverged = False

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
        log_u = self._energy(s0) + math.log(rng.random())
        minus, plus, sample = s0, s0, s0
        n, depth, ok = 1, 0, True
        while ok and depth < self.max_depth:
            direction = -1 if rng.random() < 0.5 else 1
            if direction < 0:
                minus, _, prop, n2, ok2 = self._build(minus, log_u, direction, depth, rng)
            else:
                _, plus, prop, n2, ok2 = self._build(plus, log_u, direction, depth, rng)
            if ok2 and rng.random() < min(1.0, n2 / n):
                sample = prop
            n += n2
            ok = ok2 and self._no_uturn(minus, plus)
            depth += 1
        return NutsResult(sample.nu, sample.lp, sample.g, depth, self.n_leapfrog, self.diverged)
