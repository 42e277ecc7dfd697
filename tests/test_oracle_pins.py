"""Pins for the FP64 oracle: closed forms, limits, library distributions, brute force.

Each test names what fixes the expected value (the paper's tables, a textbook
integral, a library distribution, a brute-force sum, a finite difference)
rather than re-typing the oracle's own formula.
"""
import json
import math
import os

import numpy as np
import pytest
import torch
from scipy import stats

import synth
from oracle import cosmo, hmc, mock, model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_cfg(n=8, box=80.0, n_regions=16, **kw):
    cfg = synth.Config("pin", n, box, n_regions=n_regions, **kw)
    return cfg


# ---------------------------------------------------------------------------
# paper tables (Tables 1-3, Sect. 2.3, 2.8, 3)
# ---------------------------------------------------------------------------
def test_tables_match_paper_fixture():
    g = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))
    assert list(synth.TABLE2_TEST1_ALPHA) == g["table2_test1"]["alpha"]
    assert list(synth.TABLE2_TEST1_BETA) == g["table2_test1"]["beta"]
    assert list(synth.TABLE2_TEST2_ALPHA) == g["table2_test2"]["alpha"]
    assert list(synth.TABLE2_TEST2_BETA) == g["table2_test2"]["beta"]
    assert [list(r) for r in synth.TABLE3_TEST3] == g["table3_test3"]["rows"]
    p = g["prior"]
    assert (synth.PRIOR_MU_ALPHA, synth.PRIOR_SIGMA_ALPHA, synth.PRIOR_MU_BETA, synth.PRIOR_SIGMA_BETA) == \
        (p["mu_alpha"], p["sigma_alpha"], p["mu_beta"], p["sigma_beta"])
    assert synth.PAPER_LAMBDA_TH == g["lambda_th"]["value"]
    assert synth.PAPER_RS == g["r_s"]["value"]
    # Table 1 geometry: k_nyq = pi / dL printed to two decimals.
    t1 = g["table1_geometry"]
    for dl, L, kn, kna in zip(t1["dL"], t1["L"], t1["k_nyq"], t1["k_nyq_aniso"]):
        assert L == t1["N"] * dl
        grid = model.Grid(t1["N"], float(L))
        knyq = float(grid.k[2].max())
        assert abs(knyq - kn) < 0.006
        # the printed anisotropic values are sqrt(3) x the *rounded* k_nyq (TEST2: 1.10)
        assert abs(math.sqrt(3) * kn - kna) < 0.012


# ---------------------------------------------------------------------------
# power spectrum normalisation: closed forms of int x^(n+2) W(x)^2 dx
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ns,closed", [
    (-2.0, lambda A, R: 3.0 * A / (10.0 * math.pi * R)),          # 9 * pi/15 / (2 pi^2 R)
    (-1.0, lambda A, R: 9.0 * A / (8.0 * math.pi ** 2 * R ** 2)),  # 9/4 / (2 pi^2 R^2)
])
def test_sigma2_power_law_closed_form(ns, closed):
    A, R = 2.5, 8.0
    got = cosmo.sigma2(R, A, ns, 1.0, 0.0)   # pk_pow = 0: pure power law
    tol = 1e-7 if ns == -2.0 else 1e-4       # n = -1 has a 1/k^2 tail beyond the cut
    assert abs(got / closed(A, R) - 1) < tol


def test_amplitude_gives_sigma8():
    A = cosmo.amplitude_for_sigma(0.8, 8.0, 0.96, 0.02, 1.5)
    assert abs(math.sqrt(cosmo.sigma2(8.0, A, 0.96, 0.02, 1.5)) - 0.8) < 1e-10
    assert cosmo.power_spectrum(0.0, A, 0.96, 0.02, 1.5) == 0.0


def test_power_spectrum_rolloff_closed_forms():
    """P(k) = A k^ns / (1 + (k/kc)^2)^pow at pow != 0: at k = kc the roll-off factor is exactly
    2^-pow; far above kc the logarithmic slope tends to ns - 2 pow, far below it to ns.  A
    roll-off written as (1 + k/kc)^2 (4^-pow at kc) or with the exponent's sign flipped
    (2^+pow) fails the first check."""
    A, ns, kc, pw = 3.7, 0.96, 0.02, 1.5
    assert abs(float(cosmo.power_spectrum(kc, A, ns, kc, pw)) / (A * kc ** ns * 2.0 ** -pw) - 1) < 1e-14
    assert abs(float(cosmo.power_spectrum(2 * kc, A, 0.0, kc, 2.0)) - A / 25.0) < 1e-14 * A   # (1 + 4)^-2
    def slope(k1, k2):
        p1, p2 = (float(cosmo.power_spectrum(k, A, ns, kc, pw)) for k in (k1, k2))
        return math.log(p2 / p1) / math.log(k2 / k1)
    assert abs(slope(1e4 * kc, 2e4 * kc) - (ns - 2 * pw)) < 1e-7
    assert abs(slope(1e-5 * kc, 2e-5 * kc) - ns) < 1e-8


def test_wiener_init_matches_dense_real_space_filter():
    """Sect. 2.2 initialisation against the textbook Wiener filter written with dense matrices
    in real space on a 4^3 mesh: signal covariance S of D delta0 (columns of the brute-force-
    pinned white-noise map applied to unit vectors, S = D^2 A A^T), noise N = (N^3 / N_tr) I
    (Poisson variance of n* N^3 / N_tr per cell), estimate s = S (S + N)^-1 delta*_tr; then
    delta0 = s / D and nu = A^+ delta0 (least-squares solve).  Independent of the Fourier-space
    form of the filter and of its shot-noise power L^3 / N_tr."""
    n = 4
    cfg = small_cfg(n=n, box=60.0, n_regions=4, growth_d=0.8)
    counts = np.random.default_rng(41).poisson(3.0, (n, n, n)).astype(np.int32)
    got = model.wiener_init(counts, cfg).ravel()
    m = n ** 3
    A = np.zeros((m, m))
    for i in range(m):
        e = np.zeros(m)
        e[i] = 1.0
        A[:, i] = model.delta0_from_nu(torch.tensor(e.reshape(n, n, n)), cfg).numpy().ravel()
    D = cfg.growth_d
    S = D * D * A @ A.T
    ntr = counts.sum()
    d = counts.ravel() * (m / ntr) - 1.0
    s = S @ np.linalg.solve(S + (m / ntr) * np.eye(m), d)
    nu = np.linalg.lstsq(A, s / D, rcond=1e-12)[0]
    np.testing.assert_allclose(got, nu - nu.mean(), rtol=1e-8, atol=1e-10)
    assert abs(got.mean()) < 1e-12


def test_delta0_at_cells_matches_the_full_inverse_transform():
    """The inverse DFT written out cell by cell equals the library inverse FFT of the same
    spectrum (itself pinned by the brute-force DFT above), including cells on the Nyquist
    planes of every axis."""
    cfg = small_cfg(n=16, box=160.0, n_regions=4)
    nu = synth.white_noise(16, 23)
    full = model.delta0_from_nu(torch.tensor(nu), cfg).numpy().ravel()
    cells = np.array([0, 5, 8 * 256 + 8 * 16 + 8, 15 * 256 + 3 * 16 + 8, 4095])
    np.testing.assert_allclose(model.delta0_at_cells(nu, cfg, cells), full[cells], rtol=1e-11, atol=1e-13)


def test_nu_from_delta0_inverts_the_white_noise_map():
    """The inverse of App. A on k != 0 (Wiener initialisation and test-input construction):
    round trips through the brute-force-pinned forward map, with the k = 0 mode of nu set by
    its mean (P(0) = 0 leaves it free)."""
    cfg = small_cfg(n=16, box=160.0, n_regions=4)
    nu = torch.tensor(synth.white_noise(16, 21))
    d0 = model.delta0_from_nu(nu, cfg)
    back = model.nu_from_delta0(d0, cfg, nu_mean=float(nu.mean()))
    assert float((back - nu).abs().max()) < 1e-10
    d = torch.tensor(synth.white_noise(16, 22))
    d0b = model.delta0_from_nu(model.nu_from_delta0(d, cfg), cfg)
    assert float((d0b - (d - d.mean())).abs().max()) < 1e-10


# ---------------------------------------------------------------------------
# DFT conventions and spectral operators: brute-force matrix DFT on 4^3
# ---------------------------------------------------------------------------
def _brute_operator(f, box, mult_fn):
    """Apply a k-space multiplier by explicit sums over all N^3 modes (no FFT library)."""
    n = f.shape[0]
    kf = 2 * math.pi / box
    m = np.array([j if j < n // 2 else j - n for j in range(n)], dtype=float)
    x = np.arange(n)
    E = np.exp(-2j * math.pi * np.outer(m, x) / n)         # E[m, x]
    fh = np.einsum("ax,by,cz,xyz->abc", E, E, E, f)
    M = np.zeros((n, n, n), dtype=complex)
    for a in range(n):
        for b in range(n):
            for c in range(n):
                M[a, b, c] = mult_fn(kf * m[a], kf * m[b], kf * m[c], (a == n // 2, b == n // 2, c == n // 2))
    Einv = np.conj(E)
    return np.einsum("ax,by,cz,abc->xyz", Einv, Einv, Einv, M * fh).real / n ** 3


def test_spectral_gradient_and_hessian_brute_force():
    rng = np.random.default_rng(0)
    n, box = 4, 10.0
    f = rng.standard_normal((n, n, n))
    g = model.Grid(n, box)
    ft = torch.tensor(f)
    for j in range(3):
        got = g.irfft(g.grad_mult(j) * g.rfft(ft)).numpy()

        def mult(kx, ky, kz, nyq, j=j):
            k = (kx, ky, kz)[j]
            return 0.0 if nyq[j] else 1j * k
        np.testing.assert_allclose(got, _brute_operator(f, box, mult), atol=1e-12)
    for (j, k) in model.SYM_PAIRS:
        got = g.irfft(g.hess_mult(j, k) * g.rfft(ft)).numpy()

        def mult(kx, ky, kz, nyq, j=j, k=k):
            kk = (kx, ky, kz)
            if j == k:
                return -kk[j] ** 2
            return 0.0 if (nyq[j] or nyq[k]) else -kk[j] * kk[k]
        np.testing.assert_allclose(got, _brute_operator(f, box, mult), atol=1e-12)


def test_white_noise_impulse_response_brute_force():
    """App. A: delta0 = IDFT(sqrt(P/dx^3) DFT(nu)); for nu = unit impulse DFT(nu) = 1."""
    cfg = small_cfg(n=4, box=40.0)
    n = cfg.n
    nu = np.zeros((n, n, n))
    nu[0, 0, 0] = 1.0
    got = model.delta0_from_nu(torch.tensor(nu), cfg).numpy()
    A = model.amplitude(cfg)
    dx = cfg.box / n

    def mult(kx, ky, kz, nyq):
        k = math.sqrt(kx * kx + ky * ky + kz * kz)
        return math.sqrt(float(cosmo.power_spectrum(k, A, cfg.pk_ns, cfg.pk_kc, cfg.pk_pow)) / dx ** 3)
    np.testing.assert_allclose(got, _brute_operator(nu, cfg.box, mult), rtol=1e-12, atol=1e-14)


def test_white_noise_power_statistics():
    """<|delta0_hat|^2> dx^3 / N^3 = P(k) (chi^2 over seeds and modes)."""
    cfg = small_cfg(n=16, box=200.0)
    g = model.Grid(cfg.n, cfg.box)
    A = model.amplitude(cfg)
    pk = cosmo.power_spectrum(g.kmag.numpy(), A, cfg.pk_ns, cfg.pk_kc, cfg.pk_pow)
    ratios = []
    for s in range(64):
        d0 = model.delta0_from_nu(torch.tensor(synth.white_noise(cfg.n, 100 + s)), cfg, g)
        ph = np.abs(torch.fft.rfftn(d0).numpy()) ** 2 * g.dx ** 3 / cfg.n ** 3
        m = pk > 0
        ratios.append((ph[m] / pk[m]))
    r = np.concatenate(ratios)
    # each ratio is chi^2_2/2 (or chi^2_1 on self-conjugate planes), mean 1
    assert abs(r.mean() - 1.0) < 5 * r.std() / math.sqrt(r.size)


# ---------------------------------------------------------------------------
# ALPT: plane waves (Zel'dovich, 2LPT), spherical collapse, blend limits
# ---------------------------------------------------------------------------
def _mesh(n):
    i = np.arange(n)
    return np.meshgrid(i, i, i, indexing="ij")


def test_zeldovich_single_plane_wave():
    cfg = small_cfg(n=16, box=100.0, r_s=0.0, growth_d=0.7)
    n, dx = cfg.n, cfg.box / cfg.n
    X, Y, Z = _mesh(n)
    k = 2 * math.pi * 3 / cfg.box
    A = 0.4
    d0 = A * np.cos(k * X * dx)
    psi, parts = model.alpt_displacement(torch.tensor(d0), cfg, parts=True)
    np.testing.assert_allclose(parts["s2"].numpy(), 0.0, atol=1e-13)
    expect = -cfg.growth_d * A * np.sin(k * X * dx) / k / dx
    np.testing.assert_allclose(psi[0].numpy(), expect, atol=1e-12)
    np.testing.assert_allclose(psi[1:].numpy(), 0.0, atol=1e-12)


def test_2lpt_two_orthogonal_waves():
    cfg = small_cfg(n=16, box=100.0, r_s=0.0, growth_d=1.0)
    n, dx = cfg.n, cfg.box / cfg.n
    X, Y, Z = _mesh(n)
    k1, k2 = 2 * math.pi * 2 / cfg.box, 2 * math.pi * 3 / cfg.box
    A1, A2 = 0.3, 0.2
    x, y = X * dx, Y * dx
    d0 = A1 * np.cos(k1 * x) + A2 * np.cos(k2 * y)
    psi = model.alpt_displacement(torch.tensor(d0), cfg).numpy() * dx
    D2 = -3.0 / 7.0
    ex = -A1 * np.sin(k1 * x) / k1 + D2 * A1 * A2 * k1 * np.sin(k1 * x) * np.cos(k2 * y) / (k1 ** 2 + k2 ** 2)
    ey = -A2 * np.sin(k2 * y) / k2 + D2 * A1 * A2 * k2 * np.cos(k1 * x) * np.sin(k2 * y) / (k1 ** 2 + k2 ** 2)
    np.testing.assert_allclose(psi[0], ex, atol=1e-12)
    np.testing.assert_allclose(psi[1], ey, atol=1e-12)
    np.testing.assert_allclose(psi[2], 0.0, atol=1e-12)


def test_rsd_plane_parallel_closed_forms():
    """Sect. 2.9 with b_v = 1, line of sight z, linear velocity v/(aH) = f Psi_1.  Two orthogonal
    waves along x and z (r_s = 0, pure 2LPT): the z displacement becomes (1 + f) times its
    Zel'dovich part plus the unchanged second-order part (so using the whole 2LPT Psi_z instead
    of Psi_1,z fails), and the x displacement does not change; a wave along x alone is not moved
    at all."""
    f = 0.8
    cfg = small_cfg(n=16, box=100.0, r_s=0.0, growth_d=1.0, rsd_f=f)
    n, dx = cfg.n, cfg.box / cfg.n
    X, Y, Z = _mesh(n)
    k1, k3 = 2 * math.pi * 2 / cfg.box, 2 * math.pi * 3 / cfg.box
    A1, A3 = 0.3, 0.2
    x, z = X * dx, Z * dx
    d0 = A1 * np.cos(k1 * x) + A3 * np.cos(k3 * z)
    psi = model.alpt_displacement(torch.tensor(d0), cfg).numpy() * dx
    D2 = -3.0 / 7.0
    ex = -A1 * np.sin(k1 * x) / k1 + D2 * A1 * A3 * k1 * np.sin(k1 * x) * np.cos(k3 * z) / (k1 ** 2 + k3 ** 2)
    ez = -(1 + f) * A3 * np.sin(k3 * z) / k3 + D2 * A1 * A3 * k3 * np.cos(k1 * x) * np.sin(k3 * z) / (k1 ** 2 + k3 ** 2)
    np.testing.assert_allclose(psi[0], ex, atol=1e-12)
    np.testing.assert_allclose(psi[1], 0.0, atol=1e-12)
    np.testing.assert_allclose(psi[2], ez, atol=1e-12)
    dx_only = A1 * np.cos(k1 * x)
    off = small_cfg(n=16, box=100.0, r_s=0.0, growth_d=1.0)
    np.testing.assert_allclose(model.alpt_displacement(torch.tensor(dx_only), cfg).numpy(),
                               model.alpt_displacement(torch.tensor(dx_only), off).numpy(), atol=1e-14)


def test_rsd_radial_equals_plane_parallel_on_the_axis():
    """Radial line of sight (observer at the centre c = n/2 of the volume, Sect. 2.9): for a plane
    wave along z the displacement is along z everywhere, so on the line x = y = c through the
    observer the line of sight is z itself and the radial redshift-space displacement equals the
    plane-parallel one; off that line it gains x and y components."""
    f, n, box = 0.8, 16, 100.0
    dx = box / n
    X, Y, Z = _mesh(n)
    d0 = torch.tensor(0.2 * np.cos(2 * math.pi * 3 / box * Z * dx))
    pp = model.alpt_displacement(d0, small_cfg(n=n, box=box, r_s=0.0, growth_d=1.0, rsd_f=f)).numpy()
    rad = model.alpt_displacement(d0, small_cfg(n=n, box=box, r_s=0.0, growth_d=1.0, rsd_f=f, rsd_los=1)).numpy()
    axis = (X == n // 2) & (Y == n // 2)
    np.testing.assert_allclose(rad[:, axis], pp[:, axis], atol=1e-12)
    assert np.abs(rad[0][~axis]).max() > 1e-2 and np.abs(rad[1][~axis]).max() > 1e-2


def test_rsd_radial_closed_form_two_waves():
    """Two orthogonal waves along x and z, pure 2LPT (r_s = 0): the real-space displacement Psi is
    the closed form of the 2LPT pin and the linear one Psi_1 its Zel'dovich part.  Each particle
    sits at r = q + Psi - c relative to the observer (c = n/2; the Eulerian, not the Lagrangian,
    position) and moves by f (Psi_1 . r) r / |r|^2 -- the linear velocity, not the full 2LPT
    displacement, projected on its own line of sight."""
    f, n, box = 0.8, 16, 100.0
    cfg = small_cfg(n=n, box=box, r_s=0.0, growth_d=1.0, rsd_f=f, rsd_los=1)
    dx = box / n
    X, Y, Z = _mesh(n)
    k1, k3 = 2 * math.pi * 2 / box, 2 * math.pi * 3 / box
    A1, A3 = 0.3, 0.2
    x, z = X * dx, Z * dx
    d0 = A1 * np.cos(k1 * x) + A3 * np.cos(k3 * z)
    D2 = -3.0 / 7.0
    z1x, z1z = -A1 * np.sin(k1 * x) / k1 / dx, -A3 * np.sin(k3 * z) / k3 / dx    # Zel'dovich, cells
    psi = np.stack([z1x + D2 * A1 * A3 * k1 * np.sin(k1 * x) * np.cos(k3 * z) / (k1 ** 2 + k3 ** 2) / dx,
                    np.zeros_like(x),
                    z1z + D2 * A1 * A3 * k3 * np.cos(k1 * x) * np.sin(k3 * z) / (k1 ** 2 + k3 ** 2) / dx])
    r = np.stack([X, Y, Z]) + psi - n / 2
    r2 = (r * r).sum(0)
    centre = r2 < 1e-20   # the particle at the observer (Psi vanishes there): not moved
    proj = np.where(centre, 0.0, (z1x * r[0] + z1z * r[2]) / np.where(centre, 1.0, r2))
    expect = psi + f * proj * r
    got = model.alpt_displacement(torch.tensor(d0), cfg).numpy()
    np.testing.assert_allclose(got, expect, atol=1e-11)


def test_rsd_radial_is_linear_in_f_and_conserves_mass():
    """The radial shift is linear in f (Psi(2f) - Psi(0) = 2 (Psi(f) - Psi(0))) for a random field
    with the ALPT blend on, and the CIC mass of the redshift-space positions is N^3."""
    d0 = model.delta0_from_nu(torch.tensor(synth.white_noise(16, 31)), small_cfg(n=16, box=160.0, growth_d=1.0))
    p = [model.alpt_displacement(d0, small_cfg(n=16, box=160.0, growth_d=1.0, rsd_f=f, rsd_los=1)).numpy()
         for f in (0.0, 0.5, 1.0)]
    np.testing.assert_allclose(p[2] - p[0], 2 * (p[1] - p[0]), atol=1e-12)
    assert np.abs(p[1] - p[0]).max() > 1e-2
    rho = model.cic_delta(torch.tensor(p[1])) + 1.0
    assert abs(float(rho.sum()) - 16 ** 3) < 1e-9


def test_rsd_only_moves_the_line_of_sight_component():
    """A random field with the ALPT blend on: RSD leaves Psi_x, Psi_y unchanged and adds to Psi_z a
    term linear in f (Psi_z(2f) - Psi_z(0) = 2 (Psi_z(f) - Psi_z(0))), which is curl-free with
    divergence -f D d^2 phi1 / dz^2 in k space (brute force on the spectrum)."""
    base = small_cfg(n=16, box=160.0, growth_d=1.0)
    d0 = model.delta0_from_nu(torch.tensor(synth.white_noise(16, 31)), base)
    p0 = model.alpt_displacement(d0, base).numpy()
    p1 = model.alpt_displacement(d0, small_cfg(n=16, box=160.0, growth_d=1.0, rsd_f=0.5)).numpy()
    p2 = model.alpt_displacement(d0, small_cfg(n=16, box=160.0, growth_d=1.0, rsd_f=1.0)).numpy()
    np.testing.assert_allclose(p1[:2], p0[:2], atol=1e-14)
    np.testing.assert_allclose(p2[2] - p0[2], 2 * (p1[2] - p0[2]), atol=1e-12)
    # the added z displacement: -f D d/dz of phi1 with lap phi1 = delta0 -> in k space
    # i kz (f D) delta0_hat / k^2 (cell units), Nyquist plane of kz zeroed
    g = model.Grid(16, 160.0)
    add_h = torch.fft.rfftn(torch.tensor(p2[2] - p0[2])) * g.dx
    d0h = torch.fft.rfftn(d0)
    expect = 1j * g.k_odd[2] * 1.0 * d0h * g.inv_k2
    assert float((add_h - expect).abs().max()) < 1e-10 * float(expect.abs().max())


def test_spherical_collapse_pointwise():
    x = torch.tensor([0.0, 1e-4, -1e-4, 0.3, 1.5, 2.0, -1.5], dtype=torch.float64)
    t = model.theta_sc(x, 1.0).numpy()
    assert t[0] == 0.0
    # Taylor: 3[(1-2x/3)^(1/2)-1] = -x - x^2/6 - x^3/18 + O(x^4)
    for v, got in zip(x.numpy()[1:3], t[1:3]):
        assert abs(got - (-v - v * v / 6 - v ** 3 / 18)) < 1e-15
    assert t[4] == -3.0 and t[5] == -3.0            # collapsed: divergence -3
    assert abs(t[6] - 3 * (math.sqrt(2.0) - 1)) < 1e-14
    assert abs(t[3] - 3 * (math.sqrt(0.8) - 1)) < 1e-14


def _divergence_hat(psi_cells, g):
    return sum(g.grad_mult(j) * g.rfft(psi_cells[j] * g.dx) for j in range(3))


def test_blend_limits_sc_divergence():
    """r_s -> infinity: Psi is the curl-free field with divergence theta_SC (off Nyquist, k != 0)."""
    cfg = small_cfg(n=16, box=100.0, r_s=1e6)
    g = model.Grid(cfg.n, cfg.box)
    d0 = model.delta0_from_nu(torch.tensor(synth.white_noise(cfg.n, 5)), cfg, g)
    psi = model.alpt_displacement(d0, cfg, g)
    div = _divergence_hat(psi, g).numpy()
    th = g.rfft(model.theta_sc(d0, cfg.growth_d)).numpy()
    n = cfg.n
    mask = np.ones_like(div, dtype=bool)
    mask[n // 2, :, :] = mask[:, n // 2, :] = mask[:, :, n // 2] = False
    mask[0, 0, 0] = False
    np.testing.assert_allclose(div[mask], th[mask], rtol=1e-10, atol=1e-10 * np.abs(th).max())
    # curl-free: d_x Psi_y == d_y Psi_x
    cxy = (g.grad_mult(0) * g.rfft(psi[1]) - g.grad_mult(1) * g.rfft(psi[0])).numpy()
    assert np.abs(cxy).max() < 1e-10 * np.abs(div).max()


def test_blend_is_kernel_weighted_mix():
    """Psi(r_s) = K(k) Psi(r_s=0) + (1-K(k)) Psi(r_s=inf), K a radial Gaussian."""
    base = dict(n=16, box=100.0)
    d0 = model.delta0_from_nu(torch.tensor(synth.white_noise(16, 9)), small_cfg(**base))
    g = model.Grid(16, 100.0)
    lpt = model.alpt_displacement(d0, small_cfg(r_s=0.0, **base), g)
    sc = model.alpt_displacement(d0, small_cfg(r_s=1e6, **base), g)
    mid = model.alpt_displacement(d0, small_cfg(r_s=6.0, **base), g)
    for j in range(3):
        a, b, c = (g.rfft(v[j]).numpy() for v in (lpt, sc, mid))
        sel = np.abs(a - b) > 1e-6 * np.abs(a).max()
        kern = ((c - b) / (a - b))[sel]
        np.testing.assert_allclose(kern.imag, 0.0, atol=1e-9)
        kk = np.broadcast_to(g.k2.numpy(), a.shape)[sel]
        np.testing.assert_allclose(kern.real, np.exp(-0.5 * kk * 36.0), rtol=1e-8, atol=1e-12)


# ---------------------------------------------------------------------------
# CIC
# ---------------------------------------------------------------------------
def test_cic_invariants():
    n = 8
    zero = torch.zeros(3, n, n, n, dtype=torch.float64)
    assert torch.all(model.cic_delta(zero) == 0)
    rng = np.random.default_rng(1)
    psi = torch.tensor(rng.normal(0, 1.5, (3, n, n, n)))
    d = model.cic_delta(psi)
    assert abs(float(d.sum())) < 1e-10                  # mass conservation
    assert float(d.min()) >= -1.0
    # integer displacement forming a permutation of cells: delta == 0
    perm = rng.permutation(n ** 3)
    X, Y, Z = _mesh(n)
    tgt = np.stack(np.unravel_index(perm, (n, n, n))).reshape(3, n, n, n)
    psi_int = torch.tensor((tgt - np.stack([X, Y, Z])).astype(float) + n * rng.integers(-1, 2, (3, n, n, n)))
    assert torch.all(model.cic_delta(psi_int).abs() < 1e-12)


def test_cic_single_particle_split():
    n = 8
    psi = torch.zeros(3, n, n, n, dtype=torch.float64)
    psi[:, 7, 2, 3] = torch.tensor([0.5, 0.25, -0.125])
    rho = (model.cic_delta(psi) + 1.0).numpy()
    exp = np.ones((n, n, n))
    exp[7, 2, 3] -= 1.0
    for a, wa in ((7, 0.5), (0, 0.5)):                  # periodic wrap in x
        for b, wb in ((2, 0.75), (3, 0.25)):
            for c, wc in ((2, 0.125), (3, 0.875)):
                exp[a, b, c] += wa * wb * wc
    np.testing.assert_allclose(rho, exp, atol=1e-15)


# ---------------------------------------------------------------------------
# tidal tensor, Hessian and eigenvalues
# ---------------------------------------------------------------------------
def test_plane_wave_tidal_tensor_and_eigenvalues():
    n, box = 16, 64.0
    g = model.Grid(n, box)
    X, Y, Z = _mesh(n)
    dx = box / n
    kv = 2 * math.pi / box * np.array([2.0, 2.0, 0.0])
    A = 0.7
    delta = A * np.cos((kv[0] * X + kv[1] * Y + kv[2] * Z) * dx)
    T = model.tidal_tensor(torch.tensor(delta), g).numpy()
    H = model.density_hessian(torch.tensor(delta), g).numpy()
    khat = kv / np.linalg.norm(kv)
    for c, (j, k) in enumerate(model.SYM_PAIRS):
        np.testing.assert_allclose(T[c], khat[j] * khat[k] * delta, atol=1e-12)
        np.testing.assert_allclose(H[c], -kv[j] * kv[k] * delta, atol=1e-12)
    lam = model.eigenvalues_desc(torch.tensor(T)).numpy()
    exp = np.sort(np.stack([delta, 0 * delta, 0 * delta]), axis=0)[::-1]
    np.testing.assert_allclose(lam, exp, atol=1e-12)
    # trace of T is delta (Poisson equation), trace of H is lap delta
    np.testing.assert_allclose(T[0] + T[3] + T[5], delta - delta.mean(), atol=1e-12)


def test_eigenvalues_rotated_diagonal():
    rng = np.random.default_rng(2)
    m = 200
    d = rng.normal(size=(m, 3))
    Q, _ = np.linalg.qr(rng.normal(size=(m, 3, 3)))
    M = Q @ (d[:, :, None] * np.eye(3)) @ np.transpose(Q, (0, 2, 1))
    comps = torch.tensor(np.stack([M[:, 0, 0], M[:, 0, 1], M[:, 0, 2], M[:, 1, 1], M[:, 1, 2], M[:, 2, 2]]))
    lam = model.eigenvalues_desc(comps).numpy()
    np.testing.assert_allclose(lam, -np.sort(-d, axis=1).T, atol=1e-12)


# ---------------------------------------------------------------------------
# fuzzy web
# ---------------------------------------------------------------------------
def test_memberships_partition_and_hard_limit():
    rng = np.random.default_rng(3)
    lam = np.sort(rng.normal(size=(3, 4000)), axis=0)[::-1].copy()
    lam_t = torch.tensor(lam)
    p = model.memberships(lam_t, 20.0, 0.05).numpy()
    np.testing.assert_allclose(p.sum(0), 1.0, atol=1e-14)
    assert p.min() >= 0
    # s -> infinity reproduces Eq. hard_cweb: W = number of eigenvalues above threshold
    ph = model.memberships(lam_t, 1e4, 0.05).numpy()
    W = model.hard_classes(lam_t, 0.05).numpy()
    ok = np.all(np.abs(lam - 0.05) > 1e-2, axis=0)
    assert ok.sum() > 3000
    np.testing.assert_allclose(ph[:, ok], np.eye(4)[W[ok]].T, atol=1e-12)


def test_region_index_order_hierarchical():
    """p_{4j+k} = pPhi_j * pdelta_k: with one-hot webs the region is 4*W_phi + W_delta."""
    rng = np.random.default_rng(4)
    lp = torch.tensor(np.sort(rng.normal(size=(3, 500)), axis=0)[::-1].copy())
    ld = torch.tensor(np.sort(rng.normal(size=(3, 500)), axis=0)[::-1].copy())
    w = model.region_weights(model.memberships(lp, 1e5, 0.0), model.memberships(ld, 1e5, 0.0)).numpy()
    reg = 4 * model.hard_classes(lp, 0.0).numpy() + model.hard_classes(ld, 0.0).numpy()
    ok = (np.abs(lp.numpy()).min(0) > 1e-3) & (np.abs(ld.numpy()).min(0) > 1e-3)
    np.testing.assert_allclose(w[:, ok], np.eye(16)[reg[ok]].T, atol=1e-12)


# ---------------------------------------------------------------------------
# bias, normalisation, likelihood, prior
# ---------------------------------------------------------------------------
def _uniform_bias(nr, **over):
    b = dict(a=[1.0] * nr, alpha=[1.0] * nr, rho=[1e30] * nr, eps=[1.0] * nr,
             rhop=[0.0] * nr, epsp=[1.0] * nr, beta=[5.0] * nr)
    b.update({k: [v] * nr for k, v in over.items()})
    return synth.Bias(**b)


def test_linear_bias_special_case_closed_form():
    """alpha = 1, no cut-offs: nbar = N_tr (1+delta)/N^3 (CIC conserves mass)."""
    cfg = small_cfg(n=8, box=80.0, n_regions=16)
    nu = torch.tensor(synth.white_noise(8, 11))
    b = _uniform_bias(16)
    fw = model.forward(nu, cfg, model.bias_tables(b), n_tracers=123.0, keep=True)
    u = 1.0 + fw["delta"].numpy()
    assume = u.min() > cfg.rho_floor
    assert assume
    np.testing.assert_allclose(np.exp(fw["ln_nbar"].numpy()), 123.0 * u / 8 ** 3, rtol=1e-12)


def test_cutoff_special_cases():
    cfg = small_cfg(n=8, box=80.0, n_regions=4)
    nu = torch.tensor(synth.white_noise(8, 12))
    # alpha = 0, rho = 1, eps = 1: f = exp(-u)
    fw = model.forward(nu, cfg, model.bias_tables(_uniform_bias(4, alpha=0.0, rho=1.0)), n_tracers=50.0, keep=True)
    u = np.maximum(1.0 + fw["delta"].numpy(), cfg.rho_floor)
    np.testing.assert_allclose(np.exp(fw["ln_nbar"].numpy()), 50.0 * np.exp(-u) / np.exp(-u).sum(), rtol=1e-12)
    # second cut-off alone (alpha = 0, rho' = 0.5, eps' = 2): f = exp(-(0.5/u)^2)
    fw = model.forward(nu, cfg, model.bias_tables(_uniform_bias(4, alpha=0.0, rhop=0.5, epsp=2.0)),
                       n_tracers=50.0, keep=True)
    f = np.exp(-(0.5 / u) ** 2)
    np.testing.assert_allclose(np.exp(fw["ln_nbar"].numpy()), 50.0 * f / f.sum(), rtol=1e-12)
    # rho' = 0 gives the factor one (Sect. 3 reading by continuity)
    a = model.forward(nu, cfg, model.bias_tables(_uniform_bias(4, rhop=0.0)), n_tracers=50.0)["ln_nbar"]
    b = model.forward(nu, cfg, model.bias_tables(_uniform_bias(4, rhop=1e-300)), n_tracers=50.0)["ln_nbar"]
    np.testing.assert_allclose(a.numpy(), b.numpy(), rtol=1e-12)


def test_first_cutoff_closed_form_away_from_unity():
    """Eq. local_bias first cut-off at rho = 0.5, eps = 2 (alpha = 0, a = 1): f = exp(-4 u^2).
    At rho = eps = 1 the forms (u/rho)^eps, u^eps/rho and u/rho^eps coincide; here they give
    exp(-4 u^2), exp(-2 u^2) and exp(-4 u), so a misplaced exponent fails."""
    cfg = small_cfg(n=8, box=80.0, n_regions=4)
    nu = torch.tensor(synth.white_noise(8, 17))
    fw = model.forward(nu, cfg, model.bias_tables(_uniform_bias(4, alpha=0.0, rho=0.5, eps=2.0)),
                       n_tracers=64.0, keep=True)
    u = np.maximum(1.0 + fw["delta"].numpy(), cfg.rho_floor)
    f = np.exp(-4.0 * u * u)
    np.testing.assert_allclose(np.exp(fw["ln_nbar"].numpy()), 64.0 * f / f.sum(), rtol=1e-12)


def test_parameters_are_interpolated_before_the_bias_law():
    """Sect. 2.8: each voxel uses b_i = sum_r b^(r) p_i^(r) inside Eq. local_bias (parameters
    mixed, not the per-region laws).  Two distinct parameter sets -- region 0 (voids) and the
    other three regions sharing one -- make the mix a single membership p_V = 1 - w1, computed
    here from the eigenvalues of the oracle's tidal tensor by numpy's eigvalsh at finite
    sharpness s = 20.  Checked voxel by voxel: rho and eps mixed inside -(u/rho)^eps (alpha = 0,
    a = 1), and the NB dispersion beta mixed linearly."""
    cfg = small_cfg(n=8, box=80.0, n_regions=4)
    nu = torch.tensor(synth.white_noise(8, 12))
    b = _uniform_bias(4, alpha=0.0)
    b.rho, b.eps, b.beta = [0.5, 2.0, 2.0, 2.0], [1.0, 3.0, 3.0, 3.0], [5.0, 9.0, 9.0, 9.0]
    fw = model.forward(nu, cfg, model.bias_tables(b), n_tracers=40.0, keep=True)
    T = fw["T"].numpy().reshape(6, -1)
    mats = np.stack([np.array([[t[0], t[1], t[2]], [t[1], t[3], t[4]], [t[2], t[4], t[5]]]) for t in T.T])
    lam1 = np.linalg.eigvalsh(mats)[:, -1]
    pv = 1.0 / (1.0 + np.exp(cfg.sharpness * (lam1 - cfg.lambda_th_phi)))
    assert 20 < np.count_nonzero((pv > 0.1) & (pv < 0.9))      # the mix is exercised
    u = np.maximum(1.0 + fw["delta"].numpy().ravel(), cfg.rho_floor)
    rho_i = 0.5 * pv + 2.0 * (1.0 - pv)
    eps_i = 1.0 * pv + 3.0 * (1.0 - pv)
    lnf = -(u / rho_i) ** eps_i
    ln_nbar = math.log(40.0) + lnf - np.log(np.exp(lnf).sum())
    np.testing.assert_allclose(fw["ln_nbar"].numpy().ravel(), ln_nbar, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(fw["beta"].numpy().ravel(), 5.0 * pv + 9.0 * (1.0 - pv), rtol=1e-12)


def test_hard_web_picks_class_parameters():
    """s -> infinity: each voxel uses the parameters of its hard class (row 4*W_phi + W_delta)."""
    cfg = small_cfg(n=8, box=80.0, n_regions=16, sharpness=1e6)
    nu = torch.tensor(synth.white_noise(8, 13))
    rng = np.random.default_rng(5)
    b = _uniform_bias(16, alpha=0.0)
    b.alpha = list(rng.uniform(0.5, 1.5, 16))
    fw = model.forward(nu, cfg, model.bias_tables(b), n_tracers=10.0, keep=True)
    reg = (4 * model.hard_classes(fw["lam_phi"], 0.0) + model.hard_classes(fw["lam_delta"], 0.0)).numpy()
    ok = (np.abs(fw["lam_phi"].numpy()).min(0) > 1e-4) & (np.abs(fw["lam_delta"].numpy()).min(0) > 1e-4)
    u = np.maximum(1.0 + fw["delta"].numpy(), cfg.rho_floor)   # empty cells sit on the floor
    np.testing.assert_allclose(fw["lnf"].numpy()[ok], (np.array(b.alpha)[reg] * np.log(u))[ok], rtol=1e-9, atol=1e-12)


def test_normalisation_sum():
    cfg = synth.config(0)
    cfg.n, cfg.box = 16, 150.0
    bias = synth.default_bias(cfg)
    nu = torch.tensor(synth.white_noise(16, 14))
    fw = model.forward(nu, cfg, model.bias_tables(bias), n_tracers=777.0)
    assert abs(float(torch.exp(fw["ln_nbar"]).sum()) - 777.0) < 1e-9


def test_nb_matches_scipy_and_poisson_limit():
    rng = np.random.default_rng(6)
    n = rng.integers(0, 40, 500).astype(float)
    nbar = rng.uniform(0.01, 20.0, 500)
    beta = rng.uniform(0.5, 30.0, 500)
    got = model.nb_logpmf(torch.tensor(n), torch.tensor(nbar), torch.tensor(beta)).numpy()
    np.testing.assert_allclose(got, stats.nbinom.logpmf(n, beta, beta / (beta + nbar)), rtol=1e-10, atol=1e-10)
    got_p = model.nb_logpmf(torch.tensor(n), torch.tensor(nbar), torch.tensor(np.full(500, 1e8))).numpy()
    np.testing.assert_allclose(got_p, stats.poisson.logpmf(n, nbar), rtol=1e-6, atol=1e-6)



def test_nb_log_space_form_matches_and_handles_underflow():
    """The log-space form equals the library NB where the mean is representable, and reaches the
    exact limit log P(n=0) = 0 (with zero derivative) when the mean underflows to 0."""
    rng = np.random.default_rng(7)
    n = rng.integers(0, 12, 300).astype(float)
    nbar = np.exp(rng.uniform(-6, 3, 300))
    beta = rng.uniform(0.5, 8.0, 300)
    got = model.nb_logpmf_ln(torch.tensor(n), torch.tensor(np.log(nbar)), torch.tensor(beta)).numpy()
    ref = stats.nbinom.logpmf(n, beta, beta / (beta + nbar))
    assert np.max(np.abs(got - ref)) < 1e-10
    ln_nbar = torch.tensor([-2.0e6, -800.0], dtype=torch.float64, requires_grad=True)
    lp = model.nb_logpmf_ln(torch.zeros(2, dtype=torch.float64), ln_nbar, torch.tensor([1.5, 4.0], dtype=torch.float64))
    lp.sum().backward()
    assert torch.all(torch.isfinite(lp)) and float(lp.abs().max()) == 0.0
    assert float(ln_nbar.grad.abs().max()) < 1e-300

def test_lognormal_prior_matches_scipy():
    b = np.array([0.3, 1.0, 1.3, 8.0, 11.0])
    for mu, s in ((0.27, 0.30), (2.12, 0.20)):
        got = model.lognormal_logpdf(torch.tensor(b), mu, s).numpy()
        np.testing.assert_allclose(got, stats.lognorm.logpdf(b, s=s, scale=math.exp(mu)), rtol=1e-12)


def test_prior_mask_selects_regions():
    """Eq. lognormal applies to alpha_r and beta_r of the regions whose bit is set in the prior
    mask, and to no other entry: bits 1 and 3 give exactly the four scipy log-densities of
    alpha_1, alpha_3, beta_1, beta_3."""
    b = synth.bias_phi_web(global_beta=None)
    b.prior_mask = 0b1010
    tables = model.bias_tables(b)
    got = float(model.log_prior_bias(tables, b))
    a, be = np.array(b.alpha), np.array(b.beta)
    ref = (stats.lognorm.logpdf(a[[1, 3]], s=b.sigma_alpha, scale=math.exp(b.mu_alpha)).sum()
           + stats.lognorm.logpdf(be[[1, 3]], s=b.sigma_beta, scale=math.exp(b.mu_beta)).sum())
    assert abs(got - ref) < 1e-12 * abs(ref)
    b.prior_mask = 0
    assert float(model.log_prior_bias(model.bias_tables(b), b)) == 0.0


def test_mock_gamma_poisson_moments():
    """Sect. 2.6: gamma-Poisson counts have mean nbar and variance nbar + nbar^2/beta."""
    cfg = small_cfg(n=32, box=64.0, n_regions=4, mean_tracers=2.0)
    b = _uniform_bias(4, alpha=0.0, beta=3.0)        # flat f: nbar = mean everywhere
    nu = synth.white_noise(32, 15)
    c = mock.mock_counts(nu, cfg, b, 99).astype(float)
    m, v = c.mean(), c.var()
    se_m = math.sqrt((2.0 + 4.0 / 3.0) / c.size)
    assert abs(m - 2.0) < 5 * se_m
    assert abs(v - (2.0 + 4.0 / 3.0)) < 0.05 * (2.0 + 4.0 / 3.0)


def test_flat_likelihood_gradient_is_minus_nu():
    """With f independent of nu the likelihood is flat and d log post/d nu = -nu (Eq. posterior)."""
    cfg = small_cfg(n=8, box=80.0, n_regions=4)
    b = _uniform_bias(4, alpha=0.0)
    nu = synth.white_noise(8, 16)
    counts = np.random.default_rng(7).poisson(0.5, (8, 8, 8)).astype(np.int32)
    _, g, _, _ = model.logpost_and_grad(nu, counts, cfg, b)
    np.testing.assert_allclose(g, -nu, atol=1e-12)


# ---------------------------------------------------------------------------
# gradients: autograd vs central finite differences
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n_regions,rsd_f,rsd_los", [(4, 0.0, 0), (16, 0.0, 0), (16, 0.8, 1)])
def test_gradient_matches_central_fd(n_regions, rsd_f, rsd_los):
    cfg = small_cfg(n=8, box=60.0, n_regions=n_regions, rsd_f=rsd_f, rsd_los=rsd_los)
    bias = synth.default_bias(cfg)
    nu_t = synth.white_noise(8, 21)
    counts = mock.mock_counts(nu_t, cfg, bias, 22)
    nu = nu_t + 0.3 * synth.white_noise(8, 23)
    lp, g, ga, gb = model.logpost_and_grad(nu, counts, cfg, bias)
    dirs = synth.directions(8, 24, 8)
    h = 1e-5
    errs = []
    for d in dirs:
        fp = model.logpost_value(nu + h * d, counts, cfg, bias)
        fm = model.logpost_value(nu - h * d, counts, cfg, bias)
        fd = (fp - fm) / (2 * h)
        errs.append(abs(fd - float((g * d).sum())) / max(abs(fd), 1e-3))
    # a CIC cell crossing inside [-h, h] can spoil one direction; the median must be tight
    assert np.median(errs) < 1e-7 and np.sort(errs)[-2] < 1e-5
    # bias-table gradients
    for r in (0, n_regions - 1):
        for name, gg in (("alpha", ga), ("beta", gb)):
            bp, bm = bias.copy(), bias.copy()
            getattr(bp, name)[r] += 1e-6
            getattr(bm, name)[r] -= 1e-6
            fd = (model.logpost_value(nu, counts, cfg, bp) - model.logpost_value(nu, counts, cfg, bm)) / 2e-6
            assert abs(fd - gg[r]) < 1e-5 * max(1.0, abs(fd))


# ---------------------------------------------------------------------------
# HMC (Sect. 2.2)
# ---------------------------------------------------------------------------
def test_leapfrog_prior_only_is_exact_linear_map():
    """Prior only: H = 1/2 nu^2 + 1/2 p^2 per coordinate; leapfrog is a fixed 2x2 map."""
    rng = np.random.default_rng(8)
    nu0, p0 = rng.normal(size=(8, 8, 8)), rng.normal(size=(8, 8, 8))
    eps, steps = 0.1, 7

    def prior_only(x):
        return -0.5 * float((x ** 2).sum()), -x
    nu, p, h0, h1 = hmc.leapfrog(nu0, p0, None, None, None, steps, eps, grad_fn=prior_only)
    M = np.array([[1 - eps ** 2 / 2, eps], [-eps + eps ** 3 / 4, 1 - eps ** 2 / 2]])
    Mk = np.linalg.matrix_power(M, steps)
    np.testing.assert_allclose(nu, Mk[0, 0] * nu0 + Mk[0, 1] * p0, atol=1e-13)
    np.testing.assert_allclose(p, Mk[1, 0] * nu0 + Mk[1, 1] * p0, atol=1e-13)


def test_leapfrog_reversible_and_second_order():
    cfg = small_cfg(n=8, box=60.0, n_regions=4)
    bias = synth.default_bias(cfg)
    nu_t = synth.white_noise(8, 31)
    counts = mock.mock_counts(nu_t, cfg, bias, 32)
    nu0 = nu_t + 0.2 * synth.white_noise(8, 33)
    p0 = synth.momentum(8, 34)
    nu1, p1, h0, h1 = hmc.leapfrog(nu0, p0, counts, cfg, bias, 5, 0.02)
    nu2, p2, _, _ = hmc.leapfrog(nu1, -p1, counts, cfg, bias, 5, 0.02)
    np.testing.assert_allclose(nu2, nu0, atol=1e-10)
    np.testing.assert_allclose(-p2, p0, atol=1e-10)
    # |dH| scales as eps^2 over a fixed trajectory length
    dh = []
    for eps, steps in ((0.02, 4), (0.01, 8)):
        _, _, a, b = hmc.leapfrog(nu0, p0, counts, cfg, bias, steps, eps)
        dh.append(abs(b - a))
    assert 2.5 < dh[0] / dh[1] < 6.0


# ---------------------------------------------------------------------------
# higher-order integrators (Sect. 2.2): exact harmonic-oscillator flow
# ---------------------------------------------------------------------------
def _oscillator(x0, p0, t):
    """Exact flow of H = (x^2 + p^2)/2: a rotation by t."""
    c, s = math.cos(t), math.sin(t)
    return c * x0 + s * p0, -s * x0 + c * p0


@pytest.mark.parametrize("scheme,order", [("leapfrog", 2), ("bcss2", 2), ("yoshida4", 4)])
def test_integrators_converge_to_the_exact_flow_at_their_order(scheme, order):
    """For the prior-only Hamiltonian (U = |nu|^2/2, unit oscillators) every integrator
    approaches the exact rotation with global error O(eps^order) at fixed time, and is
    reversible (negating p returns to the start)."""
    grad = lambda x: (-0.5 * float((x ** 2).sum()), -x)
    x0, p0 = np.array([1.0, -0.3]), np.array([0.2, 0.7])
    T = 1.3
    errs = []
    for n in (20, 40, 80):
        x, p, _, _ = hmc.integrate(x0, p0, None, None, None, n, T / n, scheme, grad_fn=grad)
        xe, pe = _oscillator(x0, p0, T)
        errs.append(math.hypot(*(x - xe)) + math.hypot(*(p - pe)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - order) < 0.15 for r in rates), rates
    x, p, _, _ = hmc.integrate(x0, p0, None, None, None, 7, 0.1, scheme, grad_fn=grad)
    xb, pb, _, _ = hmc.integrate(x, -p, None, None, None, 7, 0.1, scheme, grad_fn=grad)
    assert np.allclose(xb, x0, atol=1e-13) and np.allclose(-pb, p0, atol=1e-13)


def test_integrator_coefficients():
    """Consistency (kicks and drifts each sum to one step) and Yoshida's fourth-order condition
    2 w1^3 + w0^3 = 0 for the triple jump."""
    for scheme in ("leapfrog", "bcss2", "yoshida4"):
        k, d = hmc.scheme_coefficients(scheme)
        assert abs(sum(k) - 1) < 1e-15 and abs(sum(d) - 1) < 1e-15 and len(k) == len(d) + 1
        assert np.allclose(k, k[::-1]) and np.allclose(d, d[::-1])       # symmetric: time-reversible
    _, d = hmc.scheme_coefficients("yoshida4")
    assert abs(2 * d[0] ** 3 + d[1] ** 3) < 1e-14


def test_two_stage_energy_error_below_leapfrog_at_equal_cost():
    """Blanes et al. (2014): for Gaussian targets the two-stage splitting (two gradients per step)
    has a smaller energy error than leapfrog with half the step (same gradient count)."""
    grad = lambda x: (-0.5 * float((x ** 2).sum()), -x)
    rng = np.random.default_rng(3)
    x0, p0 = rng.standard_normal(64), rng.standard_normal(64)
    _, _, h0, h1 = hmc.integrate(x0, p0, None, None, None, 10, 0.4, "bcss2", grad_fn=grad)
    _, _, g0, g1 = hmc.integrate(x0, p0, None, None, None, 20, 0.2, "leapfrog", grad_fn=grad)
    assert abs(h1 - h0) < abs(g1 - g0)


# ---------------------------------------------------------------------------
# joint sampling of (nu, ln b) (Sect. 2.1, 2.2)
# ---------------------------------------------------------------------------
def _joint_case():
    cfg = small_cfg(n=8, box=80.0, n_regions=4, mean_tracers=2.0)
    bias = synth.bias_phi_web(global_beta=None)
    bias.free_mask = 0xFF
    nu = synth.white_noise(8, 51)
    counts = mock.mock_counts(nu, cfg, bias, 52)
    theta = np.log(np.concatenate([bias.alpha, bias.beta]))
    return cfg, bias, nu, counts, theta


def test_joint_theta_gradient_matches_central_fd():
    """d/d theta of log post(nu, e^theta) + sum theta against central differences in theta (the
    Jacobian term and the chain rule b d/db both enter)."""
    cfg, bias, nu, counts, theta = _joint_case()
    _, _, gt = hmc.joint_logpost_and_grad(nu, theta, counts, cfg, bias)
    h = 1e-6
    for k in range(theta.size):
        e = np.zeros_like(theta)
        e[k] = h
        fp = hmc.joint_logpost_and_grad(nu, theta + e, counts, cfg, bias)[0]
        fm = hmc.joint_logpost_and_grad(nu, theta - e, counts, cfg, bias)[0]
        assert abs((fp - fm) / (2 * h) - gt[k]) <= 1e-6 * max(1.0, abs(gt[k])), k


def test_joint_integrator_reversible_and_second_order():
    cfg, bias, nu, counts, theta = _joint_case()
    rng = np.random.default_rng(53)
    p0, pt0 = rng.standard_normal(nu.shape), rng.standard_normal(theta.shape)
    x, p, th, pt, h0, h1 = hmc.integrate_joint(nu, p0, theta, pt0, counts, cfg, bias, 4, 0.02)
    xb, pb, thb, ptb, _, _ = hmc.integrate_joint(x, -p, th, -pt, counts, cfg, bias, 4, 0.02)
    assert np.abs(xb - nu).max() < 1e-9 and np.abs(thb - theta).max() < 1e-9
    assert np.abs(pb + p0).max() < 1e-9 and np.abs(ptb + pt0).max() < 1e-9
    dh = [abs(hmc.integrate_joint(nu, p0, theta, pt0, counts, cfg, bias, n, 0.08 / n)[5] - h0) for n in (2, 4)]
    assert 3.0 < dh[0] / dh[1] < 5.0      # energy error O(eps^2) at fixed trajectory length


def test_nuts_leaves_a_gaussian_invariant():
    """The oracle's NUTS transition on a standard normal target (prior only): after many
    transitions from a fixed start the samples have mean 0 and variance 1 (detailed balance of
    the slice / doubling construction); trajectories stop by U-turns well before the depth cap."""
    grad = lambda x: (-0.5 * float((x ** 2).sum()), -x)
    rng = np.random.default_rng(61)
    x = np.full(3, 2.0)
    xs, depths = [], []
    for _ in range(3000):
        x, depth, _ = hmc.nuts_step(x, rng.standard_normal(3), None, None, None, 0.3, rng, max_depth=8, grad_fn=grad)
        xs.append(x.copy())
        depths.append(depth)
    xs = np.array(xs[200:])
    se = 3.0 / math.sqrt(len(xs))
    assert np.all(np.abs(xs.mean(0)) < 4 * se) and np.all(np.abs(xs.var(0) - 1.0) < 0.12)
    assert max(depths) < 8


def test_nuts_acceptance_statistic_one_step_closed_form():
    """With max_depth = 1 the only subtree is one leapfrog step, so the acceptance statistic is
    min(1, exp(-dH)) of that step; for the standard normal target the step and its energy error
    follow by hand: x1 = x + v eps (p - v eps x / 2), p1 = p - v eps (x + x1) / 2."""
    grad = lambda x: (-0.5 * float((x ** 2).sum()), -x)
    for seed, eps in ((3, 0.4), (4, 1.3), (5, 1.9)):
        x0 = np.array([0.7, -1.2])
        p0 = np.array([0.3, 0.9])
        rng = np.random.default_rng(seed)
        _, depth, steps, stat = hmc.nuts_step(x0, p0, None, None, None, eps, rng, max_depth=1, grad_fn=grad,
                                              with_accept=True)
        r2 = np.random.default_rng(seed)
        r2.random()
        v = -1.0 if r2.random() < 0.5 else 1.0
        x1 = x0 + v * eps * (p0 - 0.5 * v * eps * x0)
        p1 = p0 - 0.5 * v * eps * (x0 + x1)
        dH = 0.5 * float((x1 ** 2 + p1 ** 2).sum()) - 0.5 * float((x0 ** 2 + p0 ** 2).sum())
        assert depth == 1 and steps == 1
        assert abs(stat - min(1.0, math.exp(-dH))) < 1e-14, (stat, dH)


def test_dual_averaging_fixed_point_and_direction():
    """Dual averaging (Hoffman & Gelman 2014, Sect. 3.2): an acceptance statistic equal to the
    target leaves the step at its anchor 10 eps0 for good; statistics above the target grow the
    step, below it shrink it."""
    da = hmc.DualAveraging(0.05)
    for _ in range(20):
        e = da.update(0.8)
        assert abs(e - 0.5) < 1e-14
    assert abs(da.final_eps - 0.5) < 1e-14
    up, down = hmc.DualAveraging(0.05), hmc.DualAveraging(0.05)
    eu = [up.update(0.99) for _ in range(5)]
    ed = [down.update(0.3) for _ in range(5)]
    assert all(a > 0.5 for a in eu) and all(b < 0.5 for b in ed)
    assert eu[-1] > eu[0] and ed[-1] < ed[0]


def test_nuts_step_size_adaptation_reaches_the_target():
    """NUTS with dual averaging on a 50-dimensional standard normal from a far too small step:
    after 150 adaptation transitions the averaged step gives a mean acceptance statistic near the
    target 0.8 over 150 further transitions, and the step lands in the range where leapfrog on a
    unit Gaussian accepts that often (about 0.5-1.5)."""
    grad = lambda x: (-0.5 * float((x ** 2).sum()), -x)
    rng = np.random.default_rng(71)
    x = rng.standard_normal(50)
    da = hmc.DualAveraging(0.01)
    eps = 0.01
    for _ in range(150):
        x, _, _, a = hmc.nuts_step(x, rng.standard_normal(50), None, None, None, eps, rng, max_depth=8,
                                   grad_fn=grad, with_accept=True)
        eps = da.update(a)
    eps = da.final_eps
    stats = []
    for _ in range(150):
        x, _, _, a = hmc.nuts_step(x, rng.standard_normal(50), None, None, None, eps, rng, max_depth=8,
                                   grad_fn=grad, with_accept=True)
        stats.append(a)
    print(f"adapted eps {eps:.3f}, mean acceptance {np.mean(stats):.3f}")
    assert 0.5 < eps < 1.5 and 0.7 < np.mean(stats) < 0.9


def test_displacement_shift_hook_moves_particles():
    """The conditioning hook adds a displacement (cells) before the mass assignment: a uniform
    shift by one cell along x rolls the density by one cell (CIC permutation invariance), and a
    zero shift changes nothing."""
    cfg = small_cfg(n=8, box=80.0, n_regions=4)
    nu = torch.tensor(synth.white_noise(8, 71))
    t = model.bias_tables(synth.bias_phi_web())
    d = model.forward(nu, cfg, t, n_tracers=10.0, keep=True)["delta"]
    shift = torch.zeros(3, 8, 8, 8, dtype=model.DT)
    assert torch.equal(model.forward(nu, cfg, t, n_tracers=10.0, keep=True, psi_shift=shift)["delta"], d)
    shift[0] = 1.0
    d1 = model.forward(nu, cfg, t, n_tracers=10.0, keep=True, psi_shift=shift)["delta"]
    assert float((d1 - torch.roll(d, 1, dims=0)).abs().max()) < 1e-12
