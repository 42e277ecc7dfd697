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
