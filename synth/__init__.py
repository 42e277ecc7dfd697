"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the FP64 oracle.

This module holds *data* only: mesh/box geometry, power-spectrum family
parameters, the bias tables printed in the paper, and seeded random draws
(white noise, momenta, finite-difference directions, per-chain parameter
perturbations, count fields for timing runs).  It contains none of the
method's arithmetic (no FFT, no ALPT, no bias, no likelihood): whatever the
method computes is computed independently by ``oracle/`` and by the CUDA
library.

Random numbers come from numpy's PCG64 generator with explicit seeds, so the
same seed gives the same input on every machine.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

# ----------------------------------------------------------------------------
# Paper tables (Sect. 3, Tables 2 and 3).  Region order within a web is
# voids, sheets, filaments, knots (V, S, F, K), i.e. the number of eigenvalues
# above threshold 0, 1, 2, 3 (Sect. 2.8, Eq. hard_cweb).
# ----------------------------------------------------------------------------
#: Table 2, TEST1: power-law exponent alpha and NB dispersion beta per Phi-web class.
TABLE2_TEST1_ALPHA = (1.10, 1.03, 1.15, 1.23)
TABLE2_TEST1_BETA = (10.10, 13.70, 12.10, 14.40)
#: Table 2, TEST2.
TABLE2_TEST2_ALPHA = (1.05, 1.11, 1.23, 1.30)
TABLE2_TEST2_BETA = (7.10, 8.70, 8.10, 9.40)
#: Table 3, TEST3: (alpha, beta, epsilon, rho) for Phi-web class j (outer) and
#: delta-web class k (inner); row index = 4*j + k.
TABLE3_TEST3 = (
    (1.29, 5.80, 1.02, 0.22), (1.05, 14.30, 1.06, 0.26), (1.14, 11.87, 0.97, 0.16), (1.34, 10.60, 1.00, 0.20),
    (1.04, 10.74, 1.00, 0.20), (1.06, 11.57, 0.97, 0.17), (1.11, 12.59, 0.98, 0.18), (1.05, 13.67, 1.06, 0.26),
    (0.94, 5.71, 1.02, 0.22), (1.13, 13.42, 0.93, 0.13), (1.27, 7.75, 0.96, 0.16), (1.20, 11.21, 1.01, 0.21),
    (1.18, 8.36, 0.99, 0.19), (1.01, 11.24, 0.96, 0.16), (1.07, 10.99, 0.94, 0.14), (1.17, 9.71, 1.08, 0.28),
)
#: Sect. 3 (validation set-up): log-normal prior hyper-parameters of alpha and beta.
PRIOR_MU_ALPHA, PRIOR_SIGMA_ALPHA = 0.27, 0.30
PRIOR_MU_BETA, PRIOR_SIGMA_BETA = 2.12, 0.20
#: Sect. 2.8: eigenvalue threshold used in the paper's runs.
PAPER_LAMBDA_TH = 0.05
#: Sect. 2.3: ALPT blend radius r_s [Mpc/h].
PAPER_RS = 4.0


@dataclasses.dataclass
class Bias:
    """Per-region bias table (regions r = 0..n_regions-1).

    Eq. local_bias parameters a (amplitude), alpha, rho, eps (first cut-off),
    rhop, epsp (second cut-off) and the NB dispersion beta (Sect. 2.6), plus the
    log-normal prior hyper-parameters (Eq. lognormal), the set of regions the
    prior applies to, and the free (sampled) parameters: bit q of ``free_mask``
    selects parameter q of alpha_0..alpha_{P-1}, beta_0..beta_{P-1}, with P =
    n_regions, or P = 4 Phi-web classes when ``tie_classes`` is set (16-region
    tables, whose four delta-web entries per Phi class then move together;
    ``None`` means every entry, untied).
    """
    a: List[float]
    alpha: List[float]
    rho: List[float]
    eps: List[float]
    rhop: List[float]
    epsp: List[float]
    beta: List[float]
    prior_mask: int = 0
    mu_alpha: float = PRIOR_MU_ALPHA
    sigma_alpha: float = PRIOR_SIGMA_ALPHA
    mu_beta: float = PRIOR_MU_BETA
    sigma_beta: float = PRIOR_SIGMA_BETA
    free_mask: Optional[int] = None
    tie_classes: int = 0

    @property
    def n_regions(self) -> int:
        return len(self.alpha)

    def copy(self) -> "Bias":
        return dataclasses.replace(self, **{f: list(getattr(self, f)) for f in
                                            ("a", "alpha", "rho", "eps", "rhop", "epsp", "beta")})


@dataclasses.dataclass
class Config:
    """One workload: mesh, box, linear power spectrum family and web settings.

    P(k) = A k^ns / (1 + (k/kc)^2)^pk_pow, with A fixed by sigma(R=8 Mpc/h) = sigma8.
    """
    name: str
    n: int
    box: float
    n_regions: int = 4
    sigma8: float = 0.8
    pk_ns: float = 0.96
    pk_kc: float = 0.02
    pk_pow: float = 1.5
    growth_d: float = 1.0
    d2_over_d2: float = -3.0 / 7.0
    r_s: float = PAPER_RS
    lambda_th_phi: float = 0.0
    lambda_th_delta: float = 0.0
    sharpness: float = 20.0
    rho_floor: float = 1e-6
    mean_tracers: float = 0.5
    batch: int = 1
    seed_truth: int = 1001
    seed_counts: int = 2001
    seed_eval: int = 3001
    seed_dirs: int = 4001
    seed_momentum: int = 5001
    seed_perturb: int = 6001
    nb_beta: Optional[float] = None  # global beta override (configs that fix one beta)
    rsd_f: float = 0.0               # redshift-space displacement with linear velocity f (0: real space)
    rsd_los: int = 0                 # line of sight: 0 plane-parallel along z, 1 radial from the box centre

    @property
    def dx(self) -> float:
        return self.box / self.n


def bias_phi_web(alpha=TABLE2_TEST1_ALPHA, beta=None, global_beta: Optional[float] = 5.0) -> Bias:
    """4-class (Phi-web) table: alpha from Table 2 TEST1, (eps, rho) from the
    diagonal of Table 3, beta global (config value) or per class."""
    diag = [TABLE3_TEST3[5 * j] for j in range(4)]
    if beta is None:
        beta = [global_beta] * 4 if global_beta is not None else list(TABLE2_TEST1_BETA)
    return Bias(a=[1.0] * 4, alpha=list(alpha), rho=[d[3] for d in diag], eps=[d[2] for d in diag],
                rhop=[0.0] * 4, epsp=[1.0] * 4, beta=list(beta), prior_mask=0xF, free_mask=0xFF)


def bias_hierarchical(global_beta: Optional[float] = None) -> Bias:
    """16-region (Phi x delta web) table from Table 3 (TEST3); rho' = 0, eps' = 1
    as in Sect. 3 so the second cut-off factor is one.  Free parameters: alpha_j
    and beta_j of the four Phi-web classes, each shared by its four delta-web
    sub-classes (8 free parameters, Table 2)."""
    t = TABLE3_TEST3
    beta = [r[1] for r in t] if global_beta is None else [global_beta] * 16
    return Bias(a=[1.0] * 16, alpha=[r[0] for r in t], rho=[r[3] for r in t], eps=[r[2] for r in t],
                rhop=[0.0] * 16, epsp=[1.0] * 16, beta=beta, prior_mask=0xFFFF, free_mask=0xFF, tie_classes=1)


def config(i: int) -> Config:
    """The five workloads: 0: 32^3 L=300 4-class; 1: 128^3 L=1000 hierarchical;
    2: 256^3 L=1000 hierarchical (HMC trajectory); 3: 16 x 128^3 batched;
    4: 512^3 L=2000 hierarchical, beta=2, mean 0.05."""
    if i == 0:
        return Config("32^3 L=300 Phi-web", 32, 300.0, n_regions=4, nb_beta=5.0,
                      seed_truth=1001, seed_counts=2001, seed_eval=3001, seed_dirs=4001)
    if i == 1:
        return Config("128^3 L=1000 Phi x delta web", 128, 1000.0, n_regions=16,
                      seed_truth=1002, seed_counts=2002, seed_eval=3002, seed_dirs=4002)
    if i == 2:
        return Config("256^3 L=1000 Phi x delta web", 256, 1000.0, n_regions=16,
                      seed_truth=1003, seed_counts=2003, seed_eval=3003, seed_momentum=5003)
    if i == 3:
        return Config("16 x 128^3 L=1000 Phi x delta web", 128, 1000.0, n_regions=16, batch=16,
                      seed_truth=1004, seed_counts=2004, seed_eval=3004, seed_perturb=6004)
    if i == 4:
        return Config("512^3 L=2000 Phi x delta web", 512, 2000.0, n_regions=16, nb_beta=2.0,
                      mean_tracers=0.05, seed_truth=1005, seed_counts=2005, seed_eval=3005)
    raise ValueError(i)


def default_bias(cfg: Config) -> Bias:
    if cfg.n_regions == 4:
        return bias_phi_web(global_beta=cfg.nb_beta if cfg.nb_beta is not None else 5.0)
    return bias_hierarchical(global_beta=cfg.nb_beta)


# ----------------------------------------------------------------------------
# Seeded draws.
# ----------------------------------------------------------------------------
def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def white_noise(n: int, seed: int, batch: Optional[int] = None) -> np.ndarray:
    """i.i.d. standard normal field(s), float64, C order [x][y][z] (Appendix A)."""
    shape = (n, n, n) if batch is None else (batch, n, n, n)
    return _rng(seed).standard_normal(shape)


def momentum(n: int, seed: int, batch: Optional[int] = None) -> np.ndarray:
    """HMC momenta, i.i.d. standard normal (identity mass matrix)."""
    return white_noise(n, seed, batch)


def directions(n: int, seed: int, count: int) -> np.ndarray:
    """Unit-norm random directions in R^{n^3} for finite-difference checks."""
    d = _rng(seed).standard_normal((count, n, n, n))
    d /= np.sqrt((d ** 2).sum(axis=(1, 2, 3), keepdims=True))
    return d


def eval_point(n: int, seed_truth: int, seed_eval: int, scale: float = 0.3,
               batch: Optional[int] = None) -> np.ndarray:
    """An evaluation point near the truth: nu_true + scale * fresh noise."""
    return white_noise(n, seed_truth, batch) + scale * white_noise(n, seed_eval, batch)


def perturbed_biases(base: Bias, batch: int, seed: int, rel: float = 0.05) -> List[Bias]:
    """Per-chain tables with alpha and beta scaled by independent factors in (1-rel, 1+rel)."""
    rng = _rng(seed)
    out = []
    for _ in range(batch):
        b = base.copy()
        fa = rng.uniform(1 - rel, 1 + rel, size=b.n_regions)
        fb = rng.uniform(1 - rel, 1 + rel, size=b.n_regions)
        b.alpha = [float(v * f) for v, f in zip(b.alpha, fa)]
        b.beta = [float(v * f) for v, f in zip(b.beta, fb)]
        out.append(b)
    return out


def timing_counts(n: int, seed: int, mean: float, beta: float = 5.0, sigma_ln: float = 1.0,
                  batch: Optional[int] = None) -> np.ndarray:
    """Count field for timing runs at sizes where a CPU mock is too slow.

    Counts are negative-binomial draws (numpy's sampler) whose per-cell mean is
    log-normal with unit log-variance, normalised to ``mean`` tracers per cell:
    heavy at zero with a clustered-like tail.  Only the count histogram affects
    the work of any kernel (the likelihood's per-cell sum runs over m < n*).
    """
    rng = _rng(seed)
    shape = (n, n, n) if batch is None else (batch, n, n, n)
    g = rng.standard_normal(shape)
    m = mean * np.exp(sigma_ln * g - 0.5 * sigma_ln ** 2)
    p = beta / (beta + m)
    return rng.negative_binomial(beta, p).astype(np.int32)
