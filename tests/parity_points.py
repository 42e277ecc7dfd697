"""Inputs for the GPU parity tests, built with the FP64 oracle (test infrastructure).

Two properties of the model make its exact gradient ill-conditioned at some
inputs, whatever the implementation:

* Spherical collapse (Sect. 2.3, reading G4): d theta_SC / d delta0 =
  -D (1 - 2/3 D delta0)^(-1/2) diverges as D delta0 -> 3/2.  A cell 1e-5 below
  the threshold has a derivative of about -270 whose relative change under an
  FP32-sized change of delta0 (1e-7) is 1e-2.  Random fields at 128^3 and above
  always have such cells.
* Near-empty cells that hold tracers (Sect. 2.6): d log P / d rho = alpha n / rho
  for a CIC mass rho ~ 1e-4 follows the relative change of rho, i.e. the last
  bits of the displacement.

``condition`` moves a white-noise input by the oracle's inverse of App. A so
that every cell keeps a stated gap from the collapse threshold, and optionally
clears the counts of near-empty cells; the result is a point where the FP64
gradient moves by less than the FP32 bounds under an FP32 rounding of the
input, so that a GPU/oracle difference above the bound is an error of the
GPU path, not of the point.  Near-empty cells with tracers occur even in a mock
drawn from the model itself (at 256^3 a few hundred of the 16.8M cells), and
there they dominate the gradient: the data-consistent points clear them too.
Every input stays synthetic and seeded; nothing here reads the CUDA path.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from oracle import model


def f32(x) -> np.ndarray:
    """The FP32 rounding of x, as float64: the exact input both sides see."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def off_collapse(nu: np.ndarray, cfg, gap: float):
    """nu (float64, FP32-representable on return) moved so that |D delta0 - 3/2| >= gap in every
    cell: cells closer than the gap get D delta0 = 3/2 -/+ 2 gap on their own side, and nu is
    mapped back through the inverse of App. A with its mean kept.  Returns (nu, moved cells)."""
    D = cfg.growth_d
    if D == 0.0:
        return f32(nu), 0
    g = model.Grid(cfg.n, cfg.box)
    moved_total = 0
    x = f32(nu)
    for _ in range(3):   # the FP32 rounding of the moved input can bring a cell back; repeat
        d0 = model.delta0_from_nu(torch.tensor(x), cfg, g)
        y = D * d0
        near = (y - 1.5).abs() < gap
        m = int(near.sum())
        if m == 0:
            return x, moved_total
        moved_total += m
        ynew = torch.where(y < 1.5, torch.full_like(y, 1.5 - 2 * gap), torch.full_like(y, 1.5 + 2 * gap))
        d0 = torch.where(near, ynew / D, d0)
        x = f32(model.nu_from_delta0(d0, cfg, nu_mean=float(np.mean(x)), g=g).numpy())
    raise AssertionError("could not keep every cell off the collapse threshold")


def clear_near_empty(nu: np.ndarray, counts: np.ndarray, cfg, bias, mass: float = 1e-2,
                     keep_below: float = 0.0) -> np.ndarray:
    """Counts with the tracers removed from cells whose CIC mass rho = 1 + delta lies in
    (keep_below, mass) at nu (the oracle's forward model).  keep_below > 0 keeps the counts of
    cells deep on the density floor, where the likelihood term does not depend on nu."""
    f = model.forward_fields(nu, counts, cfg, bias)
    rho = 1.0 + f["delta"]
    out = counts.copy()
    out[(rho < mass) & (rho > keep_below)] = 0
    return out


def condition(nu: np.ndarray, counts: np.ndarray, cfg, bias, gap: float = 1e-3, clear_empty: bool = False):
    """Both treatments: (nu, counts, moved cells, cleared cells)."""
    x, moved = off_collapse(nu, cfg, gap)
    c = counts
    if clear_empty:
        c = clear_near_empty(x, counts, cfg, bias)
    return x, c, moved, int((c != counts).sum())


def bias_abs_terms(nu: np.ndarray, counts: np.ndarray, cfg, bias):
    """Per bias entry r, the sums over cells of the absolute contributions to d log P / d alpha_r
    and d log P / d beta_r (Sect. 2.5, 2.6), plus the prior's.

    The gradient with respect to alpha_r is sum_i w_ri ln u_i dL/dlnf_i (u = max(1 + delta,
    floor); alpha enters f only as u^alpha) and that with respect to beta_r is sum_i w_ri
    dL/dbeta_i.  At the data-generating field those sums nearly cancel, so the ratio of the
    absolute sum to the sum -- the cancellation factor -- multiplies the per-term rounding of any
    finite-precision evaluation.  Returns (abs_alpha, abs_beta, sum_alpha, sum_beta); the
    sums are the gradient itself."""
    with torch.no_grad():
        fw = model.forward(torch.tensor(nu, dtype=model.DT), cfg, model.bias_tables(bias),
                           counts=torch.tensor(counts), keep=True)
    w = fw["weights"]
    lnu = torch.log(torch.clamp(1.0 + fw["delta"], min=cfg.rho_floor))
    lnf = fw["lnf"].clone().requires_grad_(True)
    beta_i = fw["beta"].clone().requires_grad_(True)
    n_tr = float(np.asarray(counts).sum())
    ln_nbar = math.log(n_tr) + lnf - torch.logsumexp(lnf.reshape(-1), 0)
    ll = model.nb_logpmf_ln(torch.tensor(counts, dtype=model.DT), ln_nbar, beta_i).sum()
    g_lnf, g_beta = torch.autograd.grad(ll, (lnf, beta_i))
    t_a = (w * (lnu * g_lnf)[None]).reshape(w.shape[0], -1)
    t_b = (w * g_beta[None]).reshape(w.shape[0], -1)
    abs_a, abs_b, sum_a, sum_b = t_a.abs().sum(1), t_b.abs().sum(1), t_a.sum(1), t_b.sum(1)
    tables = model.bias_tables(bias, requires_grad=True)
    lp_prior = model.log_prior_bias(tables, bias)
    if lp_prior.requires_grad:
        pa, pb = torch.autograd.grad(lp_prior, (tables["alpha"], tables["beta"]))
        abs_a, abs_b = abs_a + pa.abs(), abs_b + pb.abs()
        sum_a, sum_b = sum_a + pa, sum_b + pb
    return abs_a.numpy(), abs_b.numpy(), sum_a.numpy(), sum_b.numpy()
