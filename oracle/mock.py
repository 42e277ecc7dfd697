"""Mock tracer counts from the forward model (oracle; test infrastructure only).

Sect. 3 generates the data with the same forward model as the inference
(self-specified setting) and the gamma-Poisson hierarchy of Sect. 2.6:
lambda_i ~ Gamma(shape beta_i, scale nbar_i/beta_i), n*_i ~ Poisson(lambda_i).
The total N_tr = mean * N^3 fixes the normalisation for mock generation.
"""
from __future__ import annotations

import numpy as np
import torch

from . import model


def mock_counts(nu_true, cfg, bias, seed: int) -> np.ndarray:
    with torch.no_grad():
        nu = torch.tensor(np.asarray(nu_true), dtype=model.DT)
        fw = model.forward(nu, cfg, model.bias_tables(bias), n_tracers=cfg.mean_tracers * cfg.n ** 3)
        nbar = torch.exp(fw["ln_nbar"]).numpy()
        beta = fw["beta"].numpy()
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = rng.gamma(shape=beta, scale=nbar / beta)
    return rng.poisson(lam).astype(np.int32)
