"""FP64 forward model and log posterior, written step by step from the paper.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Conventions (readings of the paper where it is silent; each one is listed with
its reason in the design notes):
  * Mesh: N^3 cells of side dx = L/N, fields in C order [x][y][z].
    Forward DFT unnormalised (``torch.fft.rfftn``), inverse with 1/N^3.
    Wavenumbers k_j = 2 pi m_j / L with m_j the signed integer frequency.
  * Any operator with an odd power of k_j sets k_j = 0 on the Nyquist plane of
    axis j; even powers keep k_j^2.  1/k^2 is 0 at k = 0.  Every operator then
    maps real fields to real fields and has an exact transpose.
  * White noise -> linear field (App. A): delta0_hat = sqrt(P(k)/dx^3) DFT(nu).
    App. A's printed prefactor is dimensionally inconsistent; this choice makes
    <|delta0_hat|^2> dx^3/N^3 = P(k).
  * ALPT (Sect. 2.3): Psi = K o Psi_2LPT + (1-K) o Psi_SC, K(k) = exp(-k^2 r_s^2/2),
    2LPT: Psi1 = -D grad phi1 with lap phi1 = delta0; Psi2 = D2 grad phi2 with
    lap phi2 = S2 = sum_{i<j}(phi1_ii phi1_jj - phi1_ij^2), D2 = (D2/D^2) D^2.
    Spherical collapse: Psi_SC curl-free with divergence
    3[(1 - 2/3 D delta0)^(1/2) - 1] for D delta0 < 3/2, else -3.
  * Redshift space (Sect. 2.9), b_v = 1 and the linear velocity v/(aH) =
    f Psi_1 (config rsd_f = f; 0 = real space), before the mass assignment:
    plane-parallel along z (rsd_los = 0): Psi_z += f Psi_1,z; radial from
    the centre of the volume (rsd_los = 1): Psi += f (Psi_1 . r) r / |r|^2
    with r the particle's real-space position relative to the centre.
  * CIC: the particle of cell q sits at q + Psi/dx (cell units); trilinear
    weights, periodic; delta = rho - 1 (one particle per cell).
  * Phi-web: tidal tensor T_jk = d_j d_k Phi with lap Phi = delta (Sect. 2.8);
    delta-web: Hessian H_jk = d_j d_k delta (App. B).  Eigenvalues sorted in
    descending order lambda1 >= lambda2 >= lambda3 (App. B ordering, which is
    the one under which Sect. 2.8's w1 > w2 > w3 holds).
  * Fuzzy memberships (Eq. sigmoid, Eq. soft_cweb_p): w_n = sigma(s(lambda_n - th)),
    pK = w3, pF = w2 - w3, pS = w1 - w2, pV = 1 - w1.  Hierarchical (Sect. 2.7):
    p_{4j+k} = pPhi_j * pdelta_k.
  * Bias (Eq. local_bias with per-voxel parameters b_i = sum_r b^(r) p_i^(r)):
    ln f = ln a + alpha ln u - (u/rho)^eps - (rho'/u)^eps', u = max(1+delta, floor).
    Normalisation: nbar = N_tr f / sum f with N_tr = sum n*.
  * Likelihood (Sect. 2.6): NB with shape beta, scale nbar/beta, per cell.
  * Prior: -1/2 sum nu^2 (constant dropped) + log-normal (Eq. lognormal) on
    alpha_r and beta_r for regions r in the prior mask.
"""
from __future__ import annotations

import math
from typing import Dict, Optional

import numpy as np
import torch

from . import cosmo

DT = torch.float64
CDT = torch.complex128
_AMP_CACHE: Dict[tuple, float] = {}


def amplitude(cfg) -> float:
    key = (cfg.sigma8, cfg.pk_ns, cfg.pk_kc, cfg.pk_pow)
    if key not in _AMP_CACHE:
        _AMP_CACHE[key] = cosmo.amplitude_for_sigma(cfg.sigma8, 8.0, cfg.pk_ns, cfg.pk_kc, cfg.pk_pow)
    return _AMP_CACHE[key]


# ----------------------------------------------------------------------------
# Wavenumbers and spectral operators
# ----------------------------------------------------------------------------
class Grid:
    """k-space grid in the r2c layout (N, N, N/2+1)."""

    def __init__(self, n: int, box: float):
        self.n, self.box, self.dx = n, box, box / n
        kf = 2.0 * math.pi / box
        m = np.fft.fftfreq(n, d=1.0 / n)               # 0..n/2-1, -n/2..-1
        mz = np.arange(n // 2 + 1, dtype=np.float64)   # 0..n/2
        kx = torch.tensor(kf * m, dtype=DT).view(n, 1, 1)
        ky = torch.tensor(kf * m, dtype=DT).view(1, n, 1)
        kz = torch.tensor(kf * mz, dtype=DT).view(1, 1, n // 2 + 1)
        nyq = n // 2
        odd = np.where(np.arange(n) == nyq, 0.0, kf * m)
        oddz = np.where(np.arange(n // 2 + 1) == nyq, 0.0, kf * mz)
        self.k = [kx, ky, kz]                         # for even powers
        self.k_odd = [torch.tensor(odd, dtype=DT).view(n, 1, 1),
                      torch.tensor(odd, dtype=DT).view(1, n, 1),
                      torch.tensor(oddz, dtype=DT).view(1, 1, n // 2 + 1)]
        k2 = kx ** 2 + ky ** 2 + kz ** 2
        self.k2 = k2
        self.kmag = torch.sqrt(k2)
        inv = torch.zeros_like(k2)
        nz = k2 > 0
        inv[nz] = 1.0 / k2[nz]
        self.inv_k2 = inv

    # operators on spectra -------------------------------------------------
    def grad_mult(self, j):
        """Multiplier of d/dx_j: i k_j (odd power: Nyquist zeroed)."""
        return 1j * self.k_odd[j]

    def hess_mult(self, j, k):
        """Multiplier of d^2/dx_j dx_k: -k_j^2 on the diagonal, -k_j k_k off it."""
        if j == k:
            return -(self.k[j] ** 2)
        return -(self.k_odd[j] * self.k_odd[k])

    def rfft(self, f):
        return torch.fft.rfftn(f)

    def irfft(self, fh):
        return torch.fft.irfftn(fh, s=(self.n, self.n, self.n))


SYM_PAIRS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))   # stored order xx xy xz yy yz zz


# ----------------------------------------------------------------------------
# M_delta (App. A)
# ----------------------------------------------------------------------------
def delta0_from_nu(nu: torch.Tensor, cfg, g: Optional[Grid] = None) -> torch.Tensor:
    g = g or Grid(cfg.n, cfg.box)
    amp = amplitude(cfg)
    pk = torch.tensor(cosmo.power_spectrum(g.kmag.numpy(), amp, cfg.pk_ns, cfg.pk_kc, cfg.pk_pow), dtype=DT)
    return g.irfft(torch.sqrt(pk / g.dx ** 3) * g.rfft(nu))


def delta0_at_cells(nu_np, cfg, cells) -> np.ndarray:
    """delta0 of App. A at selected cells (flat C-order indices), with the inverse DFT written out
    cell by cell: delta0(x) = N^-3 sum_k c(kz) Re[delta0_hat(k) exp(2 pi i k.x / N)] over the half
    spectrum, c = 1 on the kz = 0 and kz = N/2 planes and 2 elsewhere (Hermitian symmetry).
    For meshes whose full oracle forward model is too large for a test."""
    n = cfg.n
    g = Grid(n, cfg.box)
    amp = amplitude(cfg)
    pk = torch.tensor(cosmo.power_spectrum(g.kmag.numpy(), amp, cfg.pk_ns, cfg.pk_kc, cfg.pk_pow), dtype=DT)
    d0h = (torch.sqrt(pk / g.dx ** 3) * g.rfft(torch.tensor(np.asarray(nu_np), dtype=DT))).numpy()
    c = np.full(n // 2 + 1, 2.0)
    c[0] = c[n // 2] = 1.0
    mx = np.arange(n)
    mz = np.arange(n // 2 + 1)
    out = []
    for q in np.asarray(cells).ravel():
        x, y, z = int(q) // (n * n), (int(q) // n) % n, int(q) % n
        ez = c * np.exp(2j * math.pi * mz * z / n)
        ey = np.exp(2j * math.pi * mx * y / n)
        ex = np.exp(2j * math.pi * mx * x / n)
        v = ex @ ((d0h @ ez) @ ey)        # sums over kz, then ky, then kx
        out.append(float(np.real(v)) / n ** 3)
    return np.array(out)


def nu_from_delta0(delta0: torch.Tensor, cfg, nu_mean: float = 0.0, g: Optional[Grid] = None) -> torch.Tensor:
    """Inverse of the white-noise map of App. A on the modes k != 0:
    DFT(nu)(k) = DFT(delta0)(k) / sqrt(P(k)/dx^3).  P(0) = 0 leaves the k = 0 mode of nu
    undetermined; it is set so that mean(nu) = nu_mean."""
    g = g or Grid(cfg.n, cfg.box)
    amp = amplitude(cfg)
    pk = torch.tensor(cosmo.power_spectrum(g.kmag.numpy(), amp, cfg.pk_ns, cfg.pk_kc, cfg.pk_pow), dtype=DT)
    scale = torch.sqrt(pk / g.dx ** 3)
    inv = torch.zeros_like(scale)
    nz = scale > 0
    inv[nz] = 1.0 / scale[nz]
    nh = g.rfft(delta0) * inv
    nh[0, 0, 0] = nu_mean * cfg.n ** 3
    return g.irfft(nh)


def wiener_init(counts_np, cfg) -> np.ndarray:
    """Starting point of a chain (Sect. 2.2): the observed tracer contrast
    delta*_tr = n* N^3 / N_tr - 1 Wiener-filtered (Zaroubi et al. 1995) back to a linear
    field and mapped to white noise.  Signal: the evolved linear field D delta0 with power
    D^2 P(k) (the spectrum assumed known); noise: white Poisson shot noise of power
    P_N = L^3 / N_tr; no peculiar motions.  Per mode k != 0:
        delta0^(0)_hat = D P / (D^2 P + P_N) DFT(delta*_tr),
    and nu^(0) is the inverse of App. A applied to delta0^(0) (mean zero)."""
    g = Grid(cfg.n, cfg.box)
    n = torch.tensor(np.asarray(counts_np), dtype=DT)
    ntr = float(n.sum())
    d = n * (cfg.n ** 3 / ntr) - 1.0
    amp = amplitude(cfg)
    pk = torch.tensor(cosmo.power_spectrum(g.kmag.numpy(), amp, cfg.pk_ns, cfg.pk_kc, cfg.pk_pow), dtype=DT)
    D = cfg.growth_d
    pn = cfg.box ** 3 / ntr
    filt = D * pk / (D * D * pk + pn)
    d0 = g.irfft(filt * g.rfft(d))
    return nu_from_delta0(d0, cfg, nu_mean=0.0, g=g).numpy()


# ----------------------------------------------------------------------------
# M_Psi: ALPT (Sect. 2.3) + CIC
# ----------------------------------------------------------------------------
def theta_sc(delta0: torch.Tensor, growth: float) -> torch.Tensor:
    """Divergence of the spherical-collapse displacement."""
    x = growth * delta0
    arg = torch.clamp(1.0 - (2.0 / 3.0) * x, min=1e-12)
    return torch.where(x < 1.5, 3.0 * (torch.sqrt(arg) - 1.0), torch.full_like(x, -3.0))


def alpt_displacement(delta0: torch.Tensor, cfg, g: Optional[Grid] = None, parts: bool = False):
    """Psi in cell units, shape (3, N, N, N)."""
    g = g or Grid(cfg.n, cfg.box)
    D = cfg.growth_d
    D2 = cfg.d2_over_d2 * D * D
    d0h = g.rfft(delta0)
    phi1_h = -d0h * g.inv_k2                         # lap phi1 = delta0
    phi = {(j, k): g.irfft(g.hess_mult(j, k) * phi1_h) for (j, k) in SYM_PAIRS}
    s2 = (phi[0, 0] * phi[1, 1] + phi[0, 0] * phi[2, 2] + phi[1, 1] * phi[2, 2]
          - phi[0, 1] ** 2 - phi[0, 2] ** 2 - phi[1, 2] ** 2)
    phi2_h = -g.rfft(s2) * g.inv_k2                  # lap phi2 = S2
    tsc = theta_sc(delta0, D)
    phisc_h = -g.rfft(tsc) * g.inv_k2                # lap phi_sc = theta_sc
    kern = torch.exp(-0.5 * g.k2 * cfg.r_s ** 2)
    psi = []
    for j in range(3):
        gj = g.grad_mult(j)
        lpt = -D * gj * phi1_h + D2 * gj * phi2_h
        sc = gj * phisc_h
        psi.append(g.irfft(kern * lpt + (1.0 - kern) * sc) / g.dx)
    f_rsd = getattr(cfg, "rsd_f", 0.0)
    radial = bool(f_rsd) and getattr(cfg, "rsd_los", 0) == 1
    if f_rsd and not radial:
        # redshift space (Sect. 2.9, Eq. of delta(s)) with b_v = 1, plane-parallel line of sight
        # along z and the linear-theory velocity v / (aH) = f Psi_1: s_z = r_z + f Psi_1,z, where
        # Psi_1 = -D grad phi1 is the first-order (Zel'dovich) displacement
        psi[2] = psi[2] + f_rsd * g.irfft(-D * g.grad_mult(2) * phi1_h) / g.dx
    psi = torch.stack(psi)
    if radial:
        psi1 = torch.stack([g.irfft(-D * g.grad_mult(j) * phi1_h) / g.dx for j in range(3)])
        psi = radial_rsd(psi, psi1, f_rsd, g.n)
    if parts:
        return psi, dict(phi=phi, s2=s2, theta_sc=tsc)
    return psi


def radial_rsd(psi: torch.Tensor, psi1: torch.Tensor, f: float, n: int) -> torch.Tensor:
    """Redshift-space displacement with the observer at the centre of the volume (Sect. 2.9, Eq. of
    delta(s), b_v = 1): s = r + (v . r) r / (aH r^2) with v/(aH) = f Psi_1, the linear-theory
    velocity.  Cell units: the particle of cell q sits at q + Psi in real space, the observer at
    the centre c = n/2 of the cube [0, n)^3, r = q + Psi - c (not wrapped), so
        Psi_s = Psi + f (Psi_1 . r) r / |r|^2;
    a particle exactly at the observer is not moved."""
    q = torch.stack(torch.meshgrid(*(torch.arange(n, dtype=psi.dtype),) * 3, indexing="ij"))
    r = q + psi - 0.5 * n
    r2 = (r * r).sum(0)
    a = torch.where(r2 > 0, (psi1 * r).sum(0) / torch.where(r2 > 0, r2, torch.ones_like(r2)), torch.zeros_like(r2))
    return psi + f * a * r


def cic_delta(psi_cells: torch.Tensor) -> torch.Tensor:
    """Cloud-in-cell density contrast of particles at q + psi (cell units)."""
    n = psi_cells.shape[-1]
    idx = torch.arange(n, dtype=DT)
    q = torch.stack(torch.meshgrid(idx, idx, idx, indexing="ij"))
    pos = q + psi_cells
    i0 = torch.floor(pos)
    f = pos - i0
    i0 = i0.to(torch.int64)
    rho = torch.zeros(n ** 3, dtype=DT)
    for a in (0, 1):
        wx = f[0] if a else 1.0 - f[0]
        ix = (i0[0] + a) % n
        for b in (0, 1):
            wy = f[1] if b else 1.0 - f[1]
            iy = (i0[1] + b) % n
            for c in (0, 1):
                wz = f[2] if c else 1.0 - f[2]
                iz = (i0[2] + c) % n
                flat = (ix * n + iy) * n + iz
                rho = rho.index_add(0, flat.reshape(-1), (wx * wy * wz).reshape(-1))
    return rho.view(n, n, n) - 1.0


# ----------------------------------------------------------------------------
# Cosmic web (Sect. 2.8, App. B)
# ----------------------------------------------------------------------------
def tidal_tensor(delta: torch.Tensor, g: Grid):
    phi_h = -g.rfft(delta) * g.inv_k2                # lap Phi = delta
    return torch.stack([g.irfft(g.hess_mult(j, k) * phi_h) for (j, k) in SYM_PAIRS])


def density_hessian(delta: torch.Tensor, g: Grid):
    dh = g.rfft(delta)
    return torch.stack([g.irfft(g.hess_mult(j, k) * dh) for (j, k) in SYM_PAIRS])


def sym_matrix(comps: torch.Tensor) -> torch.Tensor:
    """(6, ...) stored components -> (..., 3, 3) symmetric matrices."""
    xx, xy, xz, yy, yz, zz = comps
    r0 = torch.stack([xx, xy, xz], -1)
    r1 = torch.stack([xy, yy, yz], -1)
    r2 = torch.stack([xz, yz, zz], -1)
    return torch.stack([r0, r1, r2], -2)


def eigenvalues_desc(comps: torch.Tensor) -> torch.Tensor:
    """(3, ...) eigenvalues lambda1 >= lambda2 >= lambda3 (library eigvalsh)."""
    lam = torch.linalg.eigvalsh(sym_matrix(comps))   # ascending
    return torch.flip(lam, dims=(-1,)).movedim(-1, 0)


def memberships(lam: torch.Tensor, s: float, th: float) -> torch.Tensor:
    """(4, ...) fuzzy memberships in order V, S, F, K (Eq. soft_cweb_p)."""
    w = torch.sigmoid(s * (lam - th))
    w1, w2, w3 = w[0], w[1], w[2]
    return torch.stack([1.0 - w1, w1 - w2, w2 - w3, w3])


def hard_classes(lam: torch.Tensor, th: float) -> torch.Tensor:
    """Eq. hard_cweb: number of eigenvalues above threshold (0=V .. 3=K)."""
    return (lam > th).sum(dim=0)


def region_weights(p_phi: torch.Tensor, p_delta: Optional[torch.Tensor]) -> torch.Tensor:
    if p_delta is None:
        return p_phi
    return (p_phi[:, None] * p_delta[None, :]).reshape(16, *p_phi.shape[1:])


# ----------------------------------------------------------------------------
# Bias and likelihood (Sect. 2.5, 2.6)
# ----------------------------------------------------------------------------
def _table(bias, name, requires=None):
    v = getattr(bias, name)
    if isinstance(v, torch.Tensor):
        return v
    return torch.tensor(v, dtype=DT)


def interp(table: torch.Tensor, weights: torch.Tensor) -> torch.Tensor:
    return torch.einsum("r,r...->...", table, weights)


def log_f(delta, weights, tables, rho_floor):
    u = torch.clamp(1.0 + delta, min=rho_floor)
    lnu = torch.log(u)
    a = interp(tables["a"], weights)
    al = interp(tables["alpha"], weights)
    rho = interp(tables["rho"], weights)
    eps = interp(tables["eps"], weights)
    rhop = interp(tables["rhop"], weights)
    epsp = interp(tables["epsp"], weights)
    on = rhop > 0
    base2 = torch.where(on, rhop / u, torch.ones_like(u))
    cut2 = torch.where(on, torch.pow(base2, epsp), torch.zeros_like(u))
    return torch.log(a) + al * lnu - torch.pow(u / rho, eps) - cut2


def nb_logpmf(n: torch.Tensor, nbar: torch.Tensor, beta: torch.Tensor) -> torch.Tensor:
    """Negative-binomial log pmf with shape beta and scale nbar/beta (gamma-Poisson)."""
    return (torch.lgamma(n + beta) - torch.lgamma(beta) - torch.lgamma(n + 1.0)
            + beta * torch.log(beta / (beta + nbar)) + n * torch.log(nbar / (beta + nbar)))


def nb_logpmf_ln(n: torch.Tensor, ln_nbar: torch.Tensor, beta: torch.Tensor) -> torch.Tensor:
    """The same log pmf with the mean given by its logarithm (Sect. 2.6, Eq. log_likelihood in
    log space): n (ln nbar - ln(beta + nbar)) - beta log1p(nbar / beta), so that a mean that
    underflows to 0 (the cut-offs of Eq. local_bias in empty cells) gives the limit log P(0) = 0
    instead of 0 * log 0."""
    nbar = torch.exp(ln_nbar)
    return (torch.lgamma(n + beta) - torch.lgamma(beta) - torch.lgamma(n + 1.0)
            - beta * torch.log1p(nbar / beta) + n * (ln_nbar - torch.log(beta + nbar)))


def lognormal_logpdf(b: torch.Tensor, mu: float, sigma: float) -> torch.Tensor:
    lb = torch.log(b)
    return -lb - math.log(sigma * math.sqrt(2.0 * math.pi)) - (lb - mu) ** 2 / (2.0 * sigma ** 2)


# ----------------------------------------------------------------------------
# Composition
# ----------------------------------------------------------------------------
def bias_tables(bias, requires_grad=False):
    t = {k: torch.tensor(getattr(bias, k), dtype=DT) for k in ("a", "alpha", "rho", "eps", "rhop", "epsp", "beta")}
    if requires_grad:
        t["alpha"].requires_grad_(True)
        t["beta"].requires_grad_(True)
    return t


def forward(nu: torch.Tensor, cfg, tables, counts: Optional[torch.Tensor] = None,
            n_tracers: Optional[float] = None, keep: bool = False, psi_shift: Optional[torch.Tensor] = None):
    """Forward model; returns dict with ln_nbar, beta_i (and intermediates if keep).
    psi_shift: an optional displacement (cells) added to Psi before the mass assignment, for
    measuring how the results depend on the particle positions (conditioning studies)."""
    g = Grid(cfg.n, cfg.box)
    d0 = delta0_from_nu(nu, cfg, g)
    psi = alpt_displacement(d0, cfg, g)
    if psi_shift is not None:
        psi = psi + psi_shift
    delta = cic_delta(psi)
    T = tidal_tensor(delta, g)
    lam_phi = eigenvalues_desc(T)
    p_phi = memberships(lam_phi, cfg.sharpness, cfg.lambda_th_phi)
    H = lam_delta = p_delta = None
    if cfg.n_regions == 16:
        H = density_hessian(delta, g)
        lam_delta = eigenvalues_desc(H)
        p_delta = memberships(lam_delta, cfg.sharpness, cfg.lambda_th_delta)
    wts = region_weights(p_phi, p_delta)
    lnf = log_f(delta, wts, tables, cfg.rho_floor)
    beta_i = interp(tables["beta"], wts)
    if n_tracers is None:
        n_tracers = float(counts.sum()) if counts is not None else cfg.mean_tracers * cfg.n ** 3
    ln_nbar = math.log(n_tracers) + lnf - torch.logsumexp(lnf.reshape(-1), 0)
    out = dict(ln_nbar=ln_nbar, beta=beta_i)
    if keep:
        out.update(delta0=d0, psi=psi, delta=delta, T=T, H=H, lam_phi=lam_phi, lam_delta=lam_delta,
                   p_phi=p_phi, p_delta=p_delta, weights=wts, lnf=lnf)
    return out


def log_prior_bias(tables, bias) -> torch.Tensor:
    lp = torch.zeros((), dtype=DT)
    for r in range(len(bias.alpha)):
        if (bias.prior_mask >> r) & 1:
            lp = lp + lognormal_logpdf(tables["alpha"][r], bias.mu_alpha, bias.sigma_alpha)
            lp = lp + lognormal_logpdf(tables["beta"][r], bias.mu_beta, bias.sigma_beta)
    return lp


def log_posterior(nu: torch.Tensor, counts: torch.Tensor, cfg, bias, tables=None, keep=False, psi_shift=None):
    tables = tables if tables is not None else bias_tables(bias)
    fw = forward(nu, cfg, tables, counts=counts, keep=keep, psi_shift=psi_shift)
    n = counts.to(DT)
    loglik = nb_logpmf_ln(n, fw["ln_nbar"], fw["beta"]).sum()
    lp = -0.5 * (nu ** 2).sum() + loglik + log_prior_bias(tables, bias)
    if keep:
        fw["loglik"] = loglik
        return lp, fw
    return lp


def logpost_and_grad(nu_np, counts_np, cfg, bias, psi_shift=None):
    """(log posterior, d/d nu, d/d alpha_r, d/d beta_r) by autograd, float64 (psi_shift: see forward)."""
    nu = torch.tensor(np.asarray(nu_np), dtype=DT, requires_grad=True)
    counts = torch.tensor(np.asarray(counts_np))
    tables = bias_tables(bias, requires_grad=True)
    shift = None if psi_shift is None else torch.tensor(np.asarray(psi_shift), dtype=DT)
    lp = log_posterior(nu, counts, cfg, bias, tables, psi_shift=shift)
    g_nu, g_a, g_b = torch.autograd.grad(lp, (nu, tables["alpha"], tables["beta"]))
    return float(lp.detach()), g_nu.numpy(), g_a.numpy(), g_b.numpy()


def logpost_value(nu_np, counts_np, cfg, bias) -> float:
    with torch.no_grad():
        nu = torch.tensor(np.asarray(nu_np), dtype=DT)
        counts = torch.tensor(np.asarray(counts_np))
        return float(log_posterior(nu, counts, cfg, bias))


def forward_fields(nu_np, counts_np, cfg, bias) -> Dict[str, np.ndarray]:
    """All intermediate fields as numpy float64 arrays (for parity tests)."""
    with torch.no_grad():
        nu = torch.tensor(np.asarray(nu_np), dtype=DT)
        counts = torch.tensor(np.asarray(counts_np))
        lp, fw = log_posterior(nu, counts, cfg, bias, keep=True)
    out = {k: v.numpy() for k, v in fw.items() if isinstance(v, torch.Tensor) and v.dim() > 0}
    out["logpost"] = float(lp)
    out["loglik"] = float(fw["loglik"])
    return out
